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
  semidefinite on the imaginary axis;
* sign of the broadening: with the time-ordered X of Eq. Xakqbk every
  diagonal element has Im chi_GG(w) <= 0 on the real axis (each pole term has
  a negative imaginary part); the retarded form is odd in that sign;
* f-sum rule at large imaginary frequency: nu^2 chi_GG'(i nu) tends to
  -(4/N_k) times the double commutator sum_o <o|[X, [H, Y]]|o> with
  X = e^{-i(q+G').r}, Y = e^{i(q+G).r} (exact in the space of the computed
  bands), and, with a complete band set, ||nu^2 chi_GG / Omega -> -n_e |q+G|^2||
  (n_e = 2 N_occ / Omega): pins the 2 / N_k prefactor and the spin factor;
* the cRPA factor's band and k indices (1 - T_{a,k+q} T_{o,k}).
"""
import json
import os
from dataclasses import replace

import numpy as np
from scipy.integrate import quad

from conftest import workload
from oracle import chi0 as C, dyson, lattice, pair_density as pd, tetra
from synth import Bands, fcc_cell, make_bands, sc_cell
from synth.configs import Workload, _mid_gap_cutoff
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
    # the plane-wave set at every k reaches above every allowed final state
    assert bands.energy[:, :nb].max(axis=1).min() > 0.5 * (kf + Q) ** 2
    # plain X of Eq. Xakqbk at the mesh points, energy occupations at the Fermi level
    wl = Workload(name="free", bands=bands, fft=(16, 16, 16), nocc=nb, nemp=nb, q=q[None, :],
                  ecut_eps=np.array([1.0]), axis="imag", freq=np.asarray(nu, dtype=np.float64), delta=0.0)
    w = C.pair_weights(wl, q, kind="lorentz", fermi=ef)
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


def test_im_chi_nonpositive_on_the_real_axis(small):
    """Eq. Xakqbk: 1/(w - D + i d) and -1/(w + D - i d) both have a negative imaginary part for
    d > 0, and the tetrahedron weights integrate X against non-negative barycentric weights, so
    every diagonal element Im chi_GG(w) = sum_b Im w_b |M^G_b|^2 is <= 0, at every real w.  For
    the retarded form the second pole term changes sign: Im chi_GG(-w) = -Im chi_GG(w)."""
    wl = small
    q = wl.q[0]
    G = lattice.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    M = pd.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    freq = np.array([-0.6, -0.25, 0.0, 0.15, 0.3, 0.45, 0.8])
    for kind in ("tetra", "lorentz"):
        wt = replace(wl, axis="real", delta=0.02, ordering="time", freq=freq)
        chi = C.chi0(M, C.pair_weights(wt, q, kind=kind))
        im = np.einsum("fgg->fg", chi).imag
        scale = np.abs(im).max()
        assert scale > 0
        assert im.max() <= 1e-14 * scale, (kind, im.max() / scale)
        # a resonance inside the transition range makes Im chi clearly negative there
        assert im[freq == 0.3].min() < -1e-3 * scale
    wr = replace(wl, axis="real", delta=0.02, ordering="retarded", freq=np.array([0.3, -0.3]))
    chi = C.chi0(M, C.pair_weights(wr, q))
    im = np.einsum("fgg->fg", chi).imag
    assert im[0].max() <= 1e-14 * np.abs(im).max()
    assert np.abs(im[0] + im[1]).max() <= 1e-12 * np.abs(im).max()


def test_fsum_double_commutator_in_the_band_space(micro):
    """f-sum rule (large imaginary frequency limit of Eq. chi with the plain X of Eq. Xakqbk,
    band-index occupations, q = 0 on a 2x2x2 mesh).  For i nu with d = 0,
    X = -2 D / (nu^2 + D^2), so nu^2 chi_GG' -> -(2/N_k) sum 2 D M^G M^G'^*.  Summed with
    chi_{-G',-G} this is -(4/N_k) sum_k sum_o <o|[X, [H, Y]]|o> (X = e^{-iG'.r}, Y = e^{iG.r},
    H, X, Y taken in the space spanned by the computed bands, where the identity is exact: the
    occupied-occupied terms of the spectral sum cancel).  The right side is formed here from
    the band energies and the coefficient vectors by matrix commutators, without pair
    densities or weights; a wrong 2/N_k, spin factor or pole sign fails it."""
    wl = micro
    b = wl.bands
    q = np.zeros(3)
    Gs = np.array([(1, 0, 0), (0, 1, -1), (1, 1, -1), (0, 0, 2), (-1, 2, 0)])
    L = np.concatenate([Gs, -Gs])
    n = len(L)
    M = pd.pair_density(b, wl.nocc, wl.nemp, q, L, fft=wl.fft, wrap=False)
    nk = b.kfrac.shape[0]
    assert nk == 8

    def nu2chi(nu):
        wi = replace(wl, freq=np.array([nu]), axis="imag", delta=0.0, q=q[None, :])
        return nu * nu * C.chi0(M, C.pair_weights(wi, q, kind="lorentz"))[0]
    nu = 400.0
    lim = (4.0 * nu2chi(2.0 * nu) - nu2chi(nu)) / 3.0      # Richardson in 1/nu^2
    neg = [int(np.nonzero((L == -g).all(axis=1))[0][0]) for g in L]
    sym = lim + lim[np.ix_(neg, neg)].T
    nb = wl.nocc + wl.nemp
    rhs = np.zeros((n, n), dtype=np.complex128)
    for k in range(nk):
        npw = int(b.npw[k])
        m = b.miller[k, :npw].astype(np.int64)
        ck = b.coef[k, :nb, :npw]
        pos = {tuple(r): i for i, r in enumerate(m)}
        ybar = []
        for g in L:
            Y = np.zeros((npw, npw))
            for j, r in enumerate(m):
                i = pos.get(tuple(r + g))
                if i is not None:
                    Y[i, j] = 1.0
            ybar.append(ck.conj() @ Y @ ck.T)           # <n| e^{iG.r} |m> in the band space
        H = np.diag(b.energy[k, :nb])
        for i in range(n):
            for j in range(n):
                X, Y = ybar[j].conj().T, ybar[i]
                HY = H @ Y - Y @ H
                cm = X @ HY - HY @ X
                rhs[i, j] += np.trace(cm[:wl.nocc, :wl.nocc])
    rhs *= -4.0 / nk
    assert np.abs(sym - rhs).max() <= 1e-9 * np.abs(rhs).max()


def test_fsum_physical_limit_complete_band_set():
    """With every band of the plane-wave set (Gamma only, N_k = 1), the double commutator is
    |G|^2 per occupied state up to the basis edge, so nu^2 chi_GG(i nu) / Omega tends to
    -n_e |G|^2 with n_e = 2 N_occ / Omega (spin included), the textbook f-sum rule; the
    remaining basis-edge error shrinks as the basis grows."""
    cell = fcc_cell(10.2)
    nocc = 4
    Gs = np.array([(1, 0, 0), (1, 1, -1), (0, 0, 2)])
    g2 = np.sum((Gs @ cell.recip) ** 2, axis=1)
    ne = 2.0 * nocc / cell.omega
    errs = []
    for target in (300, 600):
        ec = _mid_gap_cutoff(cell.recip, (0.0, 0.0, 0.0), target, exclude_zero=False)
        npw = len(psi_sphere(cell.recip, np.zeros(3), ec))
        b = make_bands(cell, (1, 1, 1), ec, npw, dict(kind="shells", nshell=6, vmin=0.1, vmax=0.3), seed=5,
                       workers=1)
        wl = Workload(name="gamma", bands=b, fft=(32, 32, 32), nocc=nocc, nemp=npw - nocc, q=np.zeros((1, 3)),
                      ecut_eps=np.array([1.0]), axis="imag", freq=np.array([1.0]), delta=0.0)
        M = pd.pair_density(b, nocc, npw - nocc, np.zeros(3), Gs, fft=(32, 32, 32), wrap=False)

        def nu2chi(nu):
            w = C.pair_weights(replace(wl, freq=np.array([nu])), np.zeros(3), kind="lorentz")
            return nu * nu * np.diag(C.chi0(M, w)[0]).real
        nu = 2000.0
        lim = (4.0 * nu2chi(2.0 * nu) - nu2chi(nu)) / 3.0
        errs.append(np.abs(lim / cell.omega / (-ne * g2) - 1.0).max())
    assert errs[1] < 0.01, errs
    assert errs[1] < errs[0], errs


def test_crpa_factor_indices(small):
    """Eq. chi's factor (1 - T_{a,k+q} T_{o,k}): T on the empty band at k' = k + q and on the
    occupied band at k.  Make T = 1 on every empty band of one mesh point k1 and on every
    occupied band of k2 = k1 - q: exactly the pairs of k = k2 lose their weight, every other
    weight is unchanged.  (T at k for both bands, or at k + q for both, or the two swapped,
    removes other pairs or none.)"""
    wl = replace(small, axis="imag", delta=0.0, freq=np.array([0.05, 0.4]))
    q = wl.q[0]
    b = wl.bands
    nk = b.kfrac.shape[0]
    kp, _ = lattice.umklapp(b.kmesh, q)
    k2 = 5
    k1 = int(kp[k2])
    assert k1 != k2 and kp[k1] != k2
    T = np.zeros_like(b.energy)
    T[k1, wl.nocc:wl.nocc + wl.nemp] = 1.0
    T[k2, :wl.nocc] = 1.0
    w0 = C.pair_weights(wl, q)
    w1 = C.pair_weights(replace(wl, T=T), q)
    npk = wl.nocc * wl.nemp
    cols = np.arange(k2 * npk, (k2 + 1) * npk)
    rest = np.setdiff1d(np.arange(nk * npk), cols)
    assert np.abs(w0[:, cols]).min() > 0
    assert np.all(w1[:, cols] == 0)
    assert np.array_equal(w1[:, rest], w0[:, rest])


def test_crpa_weights_from_the_wannier_construction(small):
    """Eq. tak with the projected-Gaussian stand-in: 0 <= T <= 1, the weights of a k point sum to the
    number of Wannier functions, and when the orbitals span the whole window (as many orbitals as
    window bands) T is 1 there, so the constrained chi0 is the full chi0 less the chi0 of the
    window-to-window transitions alone."""
    from synth.wannier import gaussian_wannier
    wl = replace(small, axis="imag", delta=0.0, freq=np.array([0.05, 0.4]))
    b = wl.bands
    first, nwin = wl.nocc - 2, 4                  # two occupied and two empty bands
    centers = np.array([(0.1, 0.2, 0.0), (0.5, 0.4, 0.3)])
    _, T = gaussian_wannier(b, nwin, centers, 1.6, first=first, with_T=True)
    assert T.min() >= -1e-14 and T.max() <= 1 + 1e-12
    assert np.allclose(T.sum(axis=1), 2.0, atol=1e-10)
    centers4 = np.array([(0.1, 0.2, 0.0), (0.5, 0.4, 0.3), (0.7, 0.1, 0.6), (0.3, 0.8, 0.9)])
    _, T4 = gaussian_wannier(b, nwin, centers4, 1.6, first=first, with_T=True)
    assert np.allclose(T4[:, first:first + nwin], 1.0, atol=1e-10)
    q = wl.q[0]
    w_full = C.pair_weights(wl, q)
    w_crpa = C.pair_weights(replace(wl, T=T4), q)
    # pairs (a, o) with both bands in the window: a < first + nwin (empty index a + nocc), o >= first
    nk = b.kfrac.shape[0]
    a = np.arange(wl.nemp)[:, None] + wl.nocc
    o = np.arange(wl.nocc)[None, :]
    inside = ((a < first + nwin) & (o >= first)).reshape(-1)
    mask = np.tile(inside, nk)
    assert np.abs(w_crpa[:, mask]).max() <= 1e-9 * np.abs(w_full).max()      # T = 1 up to rounding
    assert np.array_equal(w_crpa[:, ~mask], w_full[:, ~mask])
