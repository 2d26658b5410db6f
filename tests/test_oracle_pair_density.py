"""Pins for the oracle's pair densities (Eq. ism, Eq. pak).

* real-space brute force: the Bloch functions of Eq. pak are evaluated
  point by point at the true k+q (no umklapp bookkeeping) and the matrix
  element <psi_{a,k+q}| e^{i(q+G).r} |psi_{b,k}> is integrated over the cell;
* orthogonality: at q = 0, G = 0 the matrix element is <psi_a|psi_b> = 0 for
  an empty band a and an occupied band b;
* plane-wave states: for V = 0, M is a Kronecker delta in the plane waves;
* the "grid" (modulo FFT grid) and "free" index conventions agree when the
  grid is free of aliasing.
"""
import numpy as np

from conftest import workload
from oracle import lattice, pair_density as pd
from synth import Bands, fcc_cell


def _psi_on_points(bands, k_index, band, r_cart):
    npw = int(bands.npw[k_index])
    m = bands.miller[k_index, :npw].astype(np.float64)
    kg = (m + bands.kfrac[k_index][None, :]) @ bands.cell.recip        # k' + G (Cartesian)
    c = bands.coef[k_index, band, :npw]
    return np.exp(1j * r_cart @ kg.T) @ c


def test_real_space_brute_force(micro):
    wl = micro
    b = wl.bands
    q = wl.q[0]
    G = lattice.eps_sphere(b.cell.lat, q, wl.ecut_eps[0])
    M = pd.pair_density(b, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    # uniform grid on the cell, fine enough to integrate the product exactly
    n = 16
    f = np.stack(np.meshgrid(*[np.arange(n) / n] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    r = f @ b.cell.lat
    nk = b.kfrac.shape[0]
    kq = (b.kfrac + q[None, :])                       # true k+q, not reduced to the mesh
    rng = np.random.default_rng(5)
    for _ in range(6):
        k = int(rng.integers(nk))
        a = int(rng.integers(wl.nemp))
        o = int(rng.integers(wl.nocc))
        ig = int(rng.integers(len(G)))
        # the state labelled k+q is the mesh state k' (same function, Eq. pak is periodic in k)
        kp = int(np.argmin(np.linalg.norm(np.mod(b.kfrac - kq[k][None, :] + 0.5, 1.0) - 0.5, axis=1)))
        psi_a = _psi_on_points(b, kp, wl.nocc + a, r)
        psi_b = _psi_on_points(b, k, o, r)
        qg = (q + G[ig]) @ b.cell.recip
        val = np.mean(np.conj(psi_a) * np.exp(1j * r @ qg) * psi_b)
        col = (k * wl.nemp + a) * wl.nocc + o
        assert abs(val - M[ig, col]) < 1e-12, (val, M[ig, col])


def test_orthogonality_q0(small):
    wl = small
    b = wl.bands
    M = pd.pair_density(b, wl.nocc, wl.nemp, np.zeros(3), np.zeros((1, 3), dtype=np.int64), fft=wl.fft)
    assert np.abs(M).max() < 1e-13


def _plane_wave_bands(kmesh, a, ecut):
    from synth.epm import kmesh_frac, psi_sphere
    cell = fcc_cell(a)
    kf = kmesh_frac(kmesh)
    spheres = [psi_sphere(cell.recip, k, ecut) for k in kf]
    npw = np.array([len(s) for s in spheres], dtype=np.int32)
    nb = int(npw.min())
    pmax = int(npw.max())
    miller = np.zeros((len(kf), pmax, 3), dtype=np.int32)
    coef = np.zeros((len(kf), nb, pmax), dtype=np.complex128)
    energy = np.zeros((len(kf), nb))
    for i, s in enumerate(spheres):
        miller[i, :len(s)] = s
        kin = 0.5 * np.sum(((s + kf[i]) @ cell.recip) ** 2, axis=1)
        order = np.argsort(kin, kind="stable")[:nb]
        coef[i, np.arange(nb), order] = 1.0
        energy[i] = kin[order]
    return Bands(cell=cell, kmesh=tuple(kmesh), kfrac=kf, npw=npw, miller=miller,
                 coef=coef, energy=energy, ecut_psi=ecut)


def test_plane_wave_kronecker():
    b = _plane_wave_bands((2, 2, 2), 10.2, 3.0)
    nb = b.coef.shape[1]
    nocc, nemp = nb // 2, nb - nb // 2
    q = np.array([0.5, 0.0, 0.0])
    G = lattice.eps_sphere(b.cell.lat, q, 1.2)
    M = pd.pair_density(b, nocc, nemp, q, G, fft=(12, 12, 12))
    assert set(np.unique(np.round(np.abs(M), 12))) <= {0.0, 1.0}
    # the nonzero element: plane wave of band a at k' equals k + q + G + G_b
    kp, g0 = lattice.umklapp(b.kmesh, q)
    for k in range(b.kfrac.shape[0]):
        for a in range(nemp):
            ga = b.miller[kp[k], np.argmax(np.abs(b.coef[kp[k], nocc + a]))]
            for o in range(nocc):
                gb = b.miller[k, np.argmax(np.abs(b.coef[k, o]))]
                col = (k * nemp + a) * nocc + o
                want = np.all(G == (ga - gb - g0[k])[None, :], axis=1).astype(float)
                assert np.array_equal(np.abs(M[:, col]).round(12), want)


def test_grid_and_free_agree(micro):
    wl = micro
    b = wl.bands
    q = wl.q[0]
    G = lattice.eps_sphere(b.cell.lat, q, wl.ecut_eps[0])
    Mg = pd.pair_density(b, wl.nocc, wl.nemp, q, G, fft=wl.fft, wrap=True)
    Mf = pd.pair_density(b, wl.nocc, wl.nemp, q, G, wrap=False)
    assert np.abs(Mg - Mf).max() < 1e-14


def test_completeness_free_variant():
    """With the complete set of bands at k' (Gamma only, q = 0, all N_pw eigenvectors), the
    squared pair densities of an occupied band b summed over every band a equal the weight of
    C_b that the shift by G keeps inside the sphere:  sum_a |M^G_ab|^2 = sum_{G1: G1+G in sphere}
    |C_b[G1]|^2  (Parseval in the orthonormal eigenbasis of H_Gamma)."""
    from dataclasses import replace
    from synth.epm import make_bands, psi_sphere
    cell = fcc_cell(10.2)
    ecut = 2.0
    npw = len(psi_sphere(cell.recip, np.zeros(3), ecut))
    pot = {"kind": "shells", "nshell": 6, "vmin": 0.1, "vmax": 0.3}
    full = make_bands(cell, (1, 1, 1), ecut, npw, pot, seed=7, workers=1)
    ob = 2                                               # the occupied band b
    # band 0 = b (the "occupied" slot), bands 1..npw = all eigenvectors (the "empty" slots)
    coef = np.concatenate([full.coef[:, ob:ob + 1], full.coef], axis=1)
    energy = np.concatenate([full.energy[:, ob:ob + 1], full.energy], axis=1)
    b2 = replace(full, coef=coef, energy=energy)
    G = lattice.eps_sphere(cell.lat, np.zeros(3), 0.6)
    M = pd.pair_density(b2, 1, npw, np.zeros(3), G, wrap=False)          # [NG, npw]
    lhs = np.sum(np.abs(M) ** 2, axis=1)
    m = full.miller[0, :npw].astype(np.int64)
    inside = {tuple(r) for r in m}
    cb = full.coef[0, ob, :npw]
    rhs = np.array([sum(abs(cb[i]) ** 2 for i in range(npw) if tuple(m[i] + g) in inside) for g in G])
    assert len(G) > 4 and np.all(rhs < 1.0 + 1e-12)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12)
