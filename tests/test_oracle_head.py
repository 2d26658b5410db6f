"""Pins for the oracle's q -> 0 limit (Sec. 2.3, Eq. eps00, Eq. momentum) and optical spectra
(Eqs. epsilonM, eels, optical-conductivity, reflectance).

* Eq. momentum against the band dispersion: dE_a/dk = p_aa (Hellmann-Feynman), by central
  differences of directly diagonalised Hamiltonians at an off-mesh k;
* the k.p limit of the pair densities against Hamiltonians diagonalised at k and k + q (q small,
  off the mesh, Richardson in q): |M^0_ao|^2 / q^2 -> |u_ao|^2 and M^G_ao conj(M^0_ao) / q ->
  M^G_ao(k, k) conj(u_ao), u = qhat.p / (E_a - E_o): the head and wings of chi;
* the optical prefactors: the f-sum of Re sigma for a Lorentz oscillator (integral of Re sigma over
  w > 0 is w_p^2 / 8) and the normal-incidence reflectivity ((n-1)/(n+1))^2 for a real index n.
"""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import head as OH


@pytest.fixture(scope="module")
def model():
    from synth import make_workload
    wl = make_workload("micro", cache=False)            # uncached: the potential's shells are in meta
    return wl


def _ham(b, m, kf):
    """H at the fractional k kf in the plane-wave set m (Miller [n, 3]): kinetic + shell potential."""
    m = m.astype(np.float64)
    kin = 0.5 * np.sum(((m + kf) @ b.cell.recip) ** 2, axis=1)
    d = m[:, None, :] - m[None, :, :]
    g2 = np.sum((d @ b.cell.recip) ** 2, axis=-1)
    H = np.zeros((len(m), len(m)))
    for s, v in zip(b.meta["shells"], b.meta["v_shell"]):
        H[np.abs(g2 - s) < 1e-7 * max(1.0, s)] = v
    H[np.diag_indices(len(m))] += kin
    return H


def _bands_at(b, m, kf, nb):
    e, v = np.linalg.eigh(_ham(b, m, kf))
    return e[:nb], v[:, :nb].T.astype(np.complex128)


def _one_k(b, m, kf, nb):
    """A Bands-like object holding one k point with the plane-wave set m (for OH.momentum)."""
    from dataclasses import replace
    e, c = _bands_at(b, m, kf, nb)
    return replace(b, kfrac=np.asarray(kf)[None, :], npw=np.array([len(m)]), miller=m[None].astype(np.int32),
                   coef=c[None], energy=e[None]), e, c


def test_momentum_is_the_band_velocity(model):
    b = model.bands
    kf = np.array([0.13, 0.27, 0.41])
    m = b.miller[0, :b.npw[0]].astype(np.int64)
    nb = 6
    one, e0, _ = _one_k(b, m, kf, nb)
    p = OH.momentum(one, 0, np.arange(nb), np.arange(nb))
    Binv = np.linalg.inv(b.cell.recip)
    h = 1e-4
    for mu in range(3):
        dk = np.zeros(3)
        dk[mu] = h                                         # Cartesian step, in fractional units:
        df = dk @ Binv
        ep, _ = _bands_at(b, m, kf + df, nb)
        em, _ = _bands_at(b, m, kf - df, nb)
        grad = (ep - em) / (2 * h)
        assert np.abs(grad - p[np.arange(nb), np.arange(nb), mu].real).max() < 1e-6
        assert np.abs(p[np.arange(nb), np.arange(nb), mu].imag).max() < 1e-12


def test_kp_limit_of_the_pair_densities(model):
    b = model.bands
    kf = np.array([0.13, 0.27, 0.41])
    m = b.miller[0, :b.npw[0]].astype(np.int64)
    nocc, nb = 4, 8
    qhat = np.array([0.3, -0.5, 0.8])
    qhat /= np.linalg.norm(qhat)
    one, e0, c0 = _one_k(b, m, kf, nb)
    occ, emp = np.arange(nocc), np.arange(nocc, nb)
    u = (OH.momentum(one, 0, emp, occ) @ qhat) / (e0[emp][:, None] - e0[occ][None, :])
    G = np.array([1, 0, -1])
    pos = {tuple(r): i for i, r in enumerate(m)}
    sh = np.array([pos.get(tuple(r + G), -1) for r in m])      # index of G1 + G
    ok = sh >= 0

    def mg(ca, co):                                          # M^G = sum_G1 conj(C_a[G1 + G]) C_o[G1]
        out = np.zeros((len(emp), len(occ)), dtype=np.complex128)
        out += (ca[:, sh[ok]].conj()) @ co[:, ok].T
        return out
    MG0 = mg(c0[emp], c0[occ])

    def ratios(dq):
        _, cq = _bands_at(b, m, kf + (dq * qhat) @ np.linalg.inv(b.cell.recip), nb)
        M0 = cq[emp].conj() @ c0[occ].T                      # same G set: e^{iq.r} keeps G
        MG = mg(cq[emp], c0[occ])
        return np.abs(M0) ** 2 / dq ** 2, MG * M0.conj() / dq
    a1, w1 = ratios(2e-4)
    a2, w2 = ratios(1e-4)
    head = 2 * a2 - a1                                       # Richardson, error O(q) -> O(q^2)
    wing = 2 * w2 - w1
    assert np.abs(head - np.abs(u) ** 2).max() < 1e-6 * np.abs(u).max() ** 2
    assert np.abs(wing - MG0 * u.conj()).max() < 1e-6 * np.abs(MG0 * u.conj()).max()


def test_optical_prefactors():
    wp, w0, gam = 0.6, 0.3, 0.02

    def einv(w):
        return 1.0 / (1.0 + wp * wp / (w0 * w0 - w * w - 1j * gam * w))
    val, _ = quad(lambda w: OH.macroscopic(np.array([w]), np.array([einv(w)]))[2][0], 0.0, 50.0,
                  limit=500, points=[w0])
    assert abs(val - wp * wp / 8.0) < 2e-3 * wp * wp / 8.0
    n = 2.3
    eps_m, loss, sigma, refl = OH.macroscopic(np.array([0.1]), np.array([1.0 / n ** 2 + 0j]))
    assert abs(refl[0] - ((n - 1) / (n + 1)) ** 2) < 1e-14
    assert abs(eps_m[0] - n * n) < 1e-12 and loss[0] == 0.0
