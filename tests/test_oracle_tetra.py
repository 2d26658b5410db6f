"""Pins for the oracle's frequency weights (Eq. Xakqbk, Eq. tetrahedron).

* divided differences against 50-digit arithmetic (mpmath), including
  clustered and repeated nodes;
* the tetrahedron integral against brute-force quadrature over the simplex;
* confluent limit: equal nodes give 1/(4 (z - d)); flat bands give back the
  Lorentzian X of Eq. Xakqbk exactly (pins the 1/6 and the 24 tetrahedra);
* continuity across the delta_a degeneracy switch;
* geometry: 6 tetrahedra per sub-cell on the shortest diagonal, each mesh
  point in 24 tetrahedra, volumes 1/6 of a sub-cell.
"""
import numpy as np
import pytest

from oracle import tetra
from oracle.lattice import umklapp


def _dd_exact(nodes, z):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    xs = sorted(mp.mpf(float(v)) for v in nodes)
    zz = mp.mpc(z.real, z.imag)

    def f(x):
        return (zz - x) ** 3 * mp.log(zz - x)
    n = len(xs)
    tab = [[None] * n for _ in range(n)]
    for i in range(n):
        tab[i][i] = f(xs[i])
    for ln in range(1, n):
        for i in range(n - ln):
            j = i + ln
            if xs[j] == xs[i]:
                tab[i][j] = mp.diff(f, xs[i], ln) / mp.factorial(ln)
            else:
                tab[i][j] = (tab[i + 1][j] - tab[i][j - 1]) / (xs[j] - xs[i])
    return complex(tab[0][n - 1])


def test_divided_difference_vs_50_digits():
    rng = np.random.default_rng(11)
    worst = 0.0
    for trial in range(160):
        kind = trial % 4
        if kind == 0:
            nodes = rng.uniform(0, 1, 5)
        elif kind == 1:
            nodes = 0.5 + rng.uniform(-1, 1, 5) * 10 ** rng.uniform(-9, -1)
        elif kind == 2:
            a, b = rng.uniform(0, 1, 2)
            nodes = np.array([a, a + 1e-6 * rng.standard_normal(), b, b + 1e-4 * rng.standard_normal(), a])
        else:
            nodes = rng.uniform(0, 0.05, 5)
            nodes[4] = nodes[int(rng.integers(4))]
        z = complex(rng.uniform(-1, 2), rng.choice([1, -1]) * 10 ** rng.uniform(-3, 0.5))
        v = tetra.divided_difference(nodes[None, :], np.array([z]))[0]
        e = _dd_exact(nodes, z)
        worst = max(worst, abs(v - e) / abs(e))
    assert worst < 2e-12


def test_equal_nodes_confluent():
    z = np.array([0.3 + 0.01j, -0.2 + 1.5j])
    d = 0.17
    v = tetra.divided_difference(np.full((2, 5), d), z)
    assert np.allclose(v, 1.0 / (4.0 * (z - d)), rtol=1e-14, atol=0)


def _simplex_quadrature(n):
    """Gauss-Legendre points on the unit 3-simplex via the collapsed (Duffy) map."""
    t, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    U, V, W = np.meshgrid(t, t, t, indexing="ij")
    WU, WV, WW = np.meshgrid(w, w, w, indexing="ij")
    l1 = U
    l2 = (1 - U) * V
    l3 = (1 - U) * (1 - V) * W
    l4 = 1 - l1 - l2 - l3
    jac = (1 - U) ** 2 * (1 - V)
    lam = np.stack([l1, l2, l3, l4], axis=-1).reshape(-1, 4)
    return lam, (WU * WV * WW * jac).reshape(-1)


def test_tetrahedron_integral_brute_force():
    lam, wq = _simplex_quadrature(48)
    assert abs(wq.sum() - 1.0 / 6.0) < 1e-14
    rng = np.random.default_rng(3)
    for _ in range(8):
        d = rng.uniform(0.1, 0.6, 4)
        z = complex(rng.uniform(0.0, 0.7), rng.choice([1, -1]) * rng.uniform(0.15, 0.5))
        D = lam @ d
        for j in range(4):
            brute = 6.0 * np.sum(wq * lam[:, j] / (z - D))
            nodes = np.array([d[0], d[1], d[2], d[3], d[j]])
            val = tetra.divided_difference(nodes[None, :], np.array([z]))[0]
            assert abs(val - brute) < 1e-9 * abs(brute), (val, brute)


def test_flat_bands_give_lorentzian(micro):
    wl = micro
    e = wl.bands.energy.copy()
    e[:] = e.mean(axis=0)[None, :]          # no dispersion: every tetrahedron has equal nodes
    kp, _ = umklapp(wl.bands.kmesh, wl.q[0])
    tets = tetra.tetrahedra(wl.bands.kmesh, wl.bands.cell.recip)
    z1, z2 = tetra.poles(wl.freq, "real", 0.01, "time")
    x = tetra.vertex_weights(e[:, :wl.nocc], e[kp, wl.nocc:], tets, z1, z2, 1e-8, 1e-8)
    ref = tetra.lorentz_x(e[:, :wl.nocc], e[kp, wl.nocc:], z1, z2)
    assert np.allclose(x, ref, rtol=1e-13, atol=0)


def test_degeneracy_switch_is_continuous():
    da = 1e-8
    z = np.array([0.4 + 0.002j, 1.3j, -0.2 + 0.05j])
    base = np.array([0.21, 0.33, 0.21, 0.52, 0.33])
    vals = []
    for sep in (da * 0.999, da * 1.001):
        nodes = base.copy()
        nodes[2] = 0.21 + sep
        vals.append(tetra.divided_difference(nodes[None, :], z, delta_a=da, delta_r=0.0))
    assert np.all(np.abs(vals[0] - vals[1]) <= 1e-9 * np.abs(vals[1]))


def test_large_broadening_tends_to_lorentzian(micro):
    wl = micro
    kp, _ = umklapp(wl.bands.kmesh, wl.q[0])
    tets = tetra.tetrahedra(wl.bands.kmesh, wl.bands.cell.recip)
    e = wl.bands.energy
    d = e[kp, wl.nocc:][:, :, None] - e[:, :wl.nocc][:, None, :]
    spread = np.ptp(d)
    errs = []
    for scale in (1e2, 1e3):
        z1, z2 = tetra.poles([0.0], "real", scale * spread, "time")
        x = tetra.vertex_weights(e[:, :wl.nocc], e[kp, wl.nocc:], tets, z1, z2, 1e-8, 1e-8)
        ref = tetra.lorentz_x(e[:, :wl.nocc], e[kp, wl.nocc:], z1, z2)
        errs.append(np.max(np.abs(x - ref) / np.abs(ref)))
    # the deviation is first order in spread / delta
    assert errs[0] < 2.0 / 1e2 and errs[1] < 2.0 / 1e3
    assert 5.0 < errs[0] / errs[1] < 20.0


def test_tetrahedra_geometry(micro):
    b = micro.bands
    tets = tetra.tetrahedra(b.kmesh, b.cell.recip)
    nk = b.kfrac.shape[0]
    assert tets.shape == (6 * nk, 4)
    assert np.all(np.bincount(tets.ravel(), minlength=nk) == 24)
    # fcc with this reciprocal basis: the shortest main diagonal is (1,1,1)
    lens = [np.linalg.norm(np.array(s) @ b.cell.recip) for s in [(1, 1, 1), (-1, 1, 1), (1, -1, 1), (1, 1, -1)]]
    assert np.argmin(lens) == 0
    # every tetrahedron of the first sub-cell spans volume 1/6 of it (unwrapped offsets)
    n = np.array(b.kmesh)
    idx = np.array([[k // (n[1] * n[2]), (k // n[2]) % n[1], k % n[2]] for k in range(nk)])
    vols = []
    for t in tets[:6]:
        p = idx[t].astype(float)
        p = np.where(p - p[0] > n / 2, p - n, p)
        p = np.where(p - p[0] < -n / 2, p + n, p)
        vols.append(abs(np.linalg.det(p[1:] - p[0])) / 6.0)
    assert np.allclose(vols, 1.0 / 6.0)


def test_large_nu_asymptote(micro):
    """At z = +-i nu with nu far above the transition energies, each divided difference over five
    nodes tends to 1/(4 (z - c)), c the mean of its nodes (the Taylor series of f_z about c starts
    with f''''(c)/4! and h_1 of the centred nodes vanishes).  The two poles then give -c / (2 nu^2),
    so nu^2 x(k) -> -(1/12) sum over the 24 tetrahedra t around k of (sum_v D_v + D_k) / 5, with an
    error of order (D / nu)^2; for flat bands this is the -2 D of the Lorentzian X."""
    b = micro.bands
    q = micro.q[0]
    kp, _ = umklapp(b.kmesh, q)
    e_occ = b.energy[:, :micro.nocc]
    e_emp = b.energy[kp, micro.nocc:micro.nocc + micro.nemp]
    tets = tetra.tetrahedra(b.kmesh, b.cell.recip)
    nu = 1.0e3
    z1, z2 = tetra.poles(np.array([nu]), "imag", 0.0, "time")
    x = tetra.vertex_weights(e_occ, e_emp, tets, z1, z2, 1e-8, 1e-8)[..., 0]      # [k, a, o]
    D = e_emp[:, :, None] - e_occ[:, None, :]                                     # [k, a, o]
    want = np.zeros_like(D)
    for k in range(D.shape[0]):
        around = tets[np.any(tets == k, axis=1)]
        assert len(around) == 24
        for t in around:
            want[k] += (D[t].sum(axis=0) + D[k]) / 5.0
    want *= -1.0 / 12.0
    assert np.abs(x.imag).max() < 1e-12 * np.abs(x.real).max()
    assert np.allclose(nu ** 2 * x.real, want, rtol=1e-5, atol=0)


def test_mesh_convergence_against_dense_k_sum():
    """On an n^3 mesh the Brillouin-zone mean of the vertex weights tends to the zone average of
    1/(z1 - D(k)) + 1/(z2 - D(k)), the function the tetrahedra integrate, for a smooth periodic
    transition energy D(k) = D0 + t (3 - sum_i cos 2 pi k_i).  Linear interpolation of D makes the
    error second order in the mesh spacing: it falls about fourfold from n = 6 to n = 12, and the
    Richardson combination (4 S_12 - S_6) / 3 lands far closer than S_12.  The reference is a
    dense periodic sum (spectrally accurate for this analytic integrand).  This pins the mesh
    decomposition, the 24-tetrahedra sum and the weights' normalisation together."""
    from synth.epm import fcc_cell, kmesh_frac
    recip = fcc_cell(10.2).recip

    def D(kf):
        return 0.5 + 0.05 * (3.0 - np.cos(2 * np.pi * kf[:, 0]) - np.cos(2 * np.pi * kf[:, 1])
                             - np.cos(2 * np.pi * kf[:, 2]))
    z1, z2 = tetra.poles([0.55, 0.7], "real", 0.05, "time")
    d = D(kmesh_frac((96, 96, 96)))[:, None]
    ref = np.mean(1.0 / (z1[None, :] - d) + 1.0 / (z2[None, :] - d), axis=0)
    S = {}
    for n in (6, 12):
        tets = tetra.tetrahedra((n, n, n), recip)
        x = tetra.vertex_weights(np.zeros((n ** 3, 1)), D(kmesh_frac((n, n, n)))[:, None], tets, z1, z2,
                                 1e-8, 1e-8)
        S[n] = x[:, 0, 0, :].mean(axis=0)
    e6, e12 = np.abs(S[6] - ref), np.abs(S[12] - ref)
    assert np.all((3.5 < e6 / e12) & (e6 / e12 < 4.5))
    assert np.all(np.abs((4.0 * S[12] - S[6]) / 3.0 - ref) < 0.15 * e12)
