"""Pins for the oracle's chi0 (Eq. chi) and W (Eq. epsGG, Eq. Wq).

* free-electron gas: plane-wave states with energy occupations and the plain
  X of Eq. Xakqbk reproduce the Lindhard function chi_L(Q, i nu) per volume;
  the reference is a one-dimensional integral checked against the textbook
  static closed form (tests/golden/lindhard_static.json);
* Hermiticity and negative semidefiniteness on the imaginary axis;
* frequency symmetry on the real axis: retarded chi(-w) = chi(w)^*,
  time-ordered chi(-w) = chi(w);
* the (1 - T T) cRPA factor: T = 1 everywhere removes all polarization;
* W: chi = 0 gives W = v exactly; eps^-1 eps = 1; W - v is negative
  semidefinite on the imaginary axis.
"""
import json
import os
from dataclasses import replace

import numpy as np
from scipy.integrate import quad

from conftest import workload
from oracle import chi0 as C, dyson, lattice, pair_density as pd, tetra
from synth import Bands, sc_cell
from synth.epm import kmesh_frac, psi_sphere

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lindhard_imag(Q, nu, kf):
    """chi_L(Q, i nu) per volume, spin included, as a 1D integral over |p|."""
    def integrand(p):
        a = p * Q + 0.5 * Q * Q
        b = p * Q - 0.5 * Q * Q
        return p * np.log((nu * nu + a * a) / (nu * nu + b * b))
    val, _ = quad(integrand, 0.0, kf, limit=200, epsabs=0, epsrel=1e-12)
    return -val / (2.0 * np.pi ** 2 * Q)


def test_lindhard_reference_matches_textbook_static_form():
    g = json.load(open(os.path.join(GOLDEN, "lindhard_static.json")))
    kf = 1.0
    for x, F in zip(g["x"], g["F"]):
        Q = 2.0 * kf * x
        static = -(kf / np.pi ** 2) * F
        assert abs(lindhard_imag(Q, 1e-9, kf) - static) < 1e-6 * abs(static)


def _pw_bands(a, kmesh, ecut):
    cell = sc_cell(a)
    kf = kmesh_frac(kmesh)
    spheres = [psi_sphere(cell.recip, k, ecut) for k in kf]
    nb = min(len(s) for s in spheres)
    pmax = max(len(s) for s in spheres)
    nk = len(kf)
    miller = np.zeros((nk, pmax, 3), dtype=np.int32)
    coef = np.zeros((nk, 2 * nb, pmax), dtype=np.complex128)
    energy = np.zeros((nk, 2 * nb))
    for i, s in enumerate(spheres):
        miller[i, :len(s)] = s
        kin = 0.5 * np.sum(((s + kf[i]) @ cell.recip) ** 2, axis=1)
        order = np.argsort(kin, kind="stable")[:nb]
        for rep in range(2):          # the band list twice: every (a, b) pair appears
            coef[i, rep * nb + np.arange(nb), order] = 1.0
            energy[i, rep * nb:(rep + 1) * nb] = kin[order]
    npw = np.array([len(s) for s in spheres], dtype=np.int32)
    return Bands(cell=cell, kmesh=tuple(kmesh), kfrac=kf, npw=npw, miller=miller,
                 coef=coef, energy=energy, ecut_psi=ecut), nb


def _free_electron_chi00(n, kf, nu, m_q):
    a = 4.0
    bands, nb = _pw_bands(a, (n, n, n), ecut=0.5 * (kf + 2.6) ** 2)
    q = np.array([m_q / n, 0.0, 0.0])
    G = np.zeros((1, 3), dtype=np.int64)
    M = pd.pair_density(bands, nb, nb, q, G, fft=(16, 16, 16))
    kp, _ = lattice.umklapp(bands.kmesh, q)
    Q = np.linalg.norm(q @ bands.cell.recip)
    ef = 0.5 * kf * kf
    e_o = bands.energy[:, :nb]
    e_a = bands.energy[kp, nb:]
    # the plane-wave set at every k reaches above every allowed final state
    assert e_o.max(axis=1).min() > 0.5 * (kf + Q) ** 2
    z1, z2 = tetra.poles(nu, "imag", 0.0, "time")
    X = tetra.lorentz_x(e_o, e_a, z1, z2)                            # [k, a, o, f]
    occ = (e_o < ef)[:, None, :, None] & (e_a >= ef)[:, :, None, None]
    w = (2.0 / n ** 3) * (X * occ)
    w = w.reshape(-1, len(nu)).T
    chi = C.chi0(M, w)[:, 0, 0]
    return chi / bands.cell.omega, np.array([lindhard_imag(Q, v, kf) for v in nu])


def test_free_electron_lindhard():
    nu = np.array([0.2, 0.5])
    errs = []
    for n in (6, 12):
        chi, ref = _free_electron_chi00(n, 0.8, nu, n // 3)
        errs.append(np.max(np.abs(chi - ref) / np.abs(ref)))
    assert errs[1] < 0.03, errs
    assert errs[1] < errs[0], errs


def test_hermitian_negative_semidefinite_imag_axis(micro):
    wl = micro
    b = wl.bands
    q = wl.q[0]
    kp, _ = lattice.umklapp(b.kmesh, q)
    gap = (b.energy[kp, wl.nocc:][:, :, None] - b.energy[:, :wl.nocc][:, None, :]).min()
    assert gap > 0
    G = lattice.eps_sphere(b.cell.lat, q, wl.ecut_eps[0])
    M = pd.pair_density(b, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    chi = C.chi0(M, C.pair_weights(wl, q))
    assert np.abs(chi - np.conj(np.transpose(chi, (0, 2, 1)))).max() < 1e-14 * np.abs(chi).max()
    for c in chi:
        ev = np.linalg.eigvalsh(c)
        assert ev.max() < 1e-12 * np.abs(ev).max()
        assert ev.min() < 0


def _chi_pm(wl, ordering):
    b = wl.bands
    q = wl.q[0]
    freq = np.array([0.1, 0.35, -0.1, -0.35])
    wl2 = replace(wl, freq=freq, ordering=ordering, axis="real", delta=0.02)
    G = lattice.eps_sphere(b.cell.lat, q, wl.ecut_eps[0])
    M = pd.pair_density(b, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    return C.chi0(M, C.pair_weights(wl2, q))


def test_frequency_symmetry(micro):
    ret = _chi_pm(micro, "retarded")
    assert np.abs(ret[2:] - np.conj(ret[:2])).max() < 1e-13 * np.abs(ret).max()
    tord = _chi_pm(micro, "time")
    assert np.abs(tord[2:] - tord[:2]).max() < 1e-13 * np.abs(tord).max()
    assert np.abs(ret[:2] - tord[:2]).max() > 1e-6 * np.abs(ret).max()   # the two readings differ


def test_crpa_full_projection_removes_polarization(micro):
    wl = replace(micro, T=np.ones_like(micro.bands.energy))
    w = C.pair_weights(wl, wl.q[0])
    assert np.abs(w).max() == 0.0


def test_screened_interaction(micro):
    wl = micro
    b = wl.bands
    q = wl.q[0]
    G = lattice.eps_sphere(b.cell.lat, q, wl.ecut_eps[0])
    vs = dyson.coulomb_sqrt(b.cell.lat, q, G)
    # chi = 0  ->  W = v exactly
    W0 = dyson.screened(np.zeros((1, len(G), len(G)), dtype=np.complex128), vs)
    assert np.array_equal(W0[0], np.diag(vs * vs).astype(np.complex128))
    M = pd.pair_density(b, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    chi = C.chi0(M, C.pair_weights(wl, q))
    eps = dyson.epsilon(chi, vs)
    W = dyson.screened(chi, vs)
    for f in range(len(wl.freq)):
        einv = W[f] / (vs[:, None] * vs[None, :])
        assert np.abs(einv @ eps[f] - np.eye(len(G))).max() < 1e-12
        ev = np.linalg.eigvalsh(W[f] - np.diag(vs * vs))
        assert ev.max() < 1e-12 * np.abs(ev).max()
    # tail: 4 pi / (Omega |q+G|^2) on the shell between the two cut-offs
    T = lattice.tail_sphere(b.cell.lat, q, wl.ecut_eps[0], b.ecut_psi)
    qg = (T + q[None, :]) @ b.cell.recip
    assert np.allclose(dyson.tail(b.cell.lat, q, T), 4 * np.pi / (b.cell.omega * np.sum(qg * qg, axis=1)), rtol=1e-14)
