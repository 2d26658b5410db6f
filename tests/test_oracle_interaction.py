"""Pins for the oracle's screened direct and exchange integrals (Sec. 2.4, Eqs. matrix_U, matrix_V,
matrix_J, matrix_X).

* bare integrals by a second route: the Wannier functions are built on the real-space grid of
  the Born-von Karman supercell of the k mesh (phi_i0 = N_k^-1/2 sum_k psi~_ik), their densities
  |phi_i0|^2 and pair products phi_i0^* phi_jR are Fourier transformed on that grid, and the
  Coulomb energies (4 pi / V) sum_Q n_a(Q) n_b(Q)^* / |Q|^2 are summed over the same Q = q + G;
  the oracle's k-summed coefficient convolutions, phases e^{-iq.R}, e^{-ik.R} and 4 pi/(Omega N_q)
  must give the same numbers;
* the Wannier functions are normalised and their densities integrate to one (the reading that
  makes rho_iq(G) a density's Fourier component);
* screened = bare when W = v (chi = 0): the epsilon sphere and the tail make up the whole
  wave-function sphere.
"""
import numpy as np
import pytest

from conftest import workload
from oracle import interaction as OI, lattice as OL
from synth.wannier import gaussian_wannier

R_LIST = np.array([(0, 0, 0), (1, 0, 0), (0, 1, -1)])


@pytest.fixture(scope="module")
def wan():
    # a 3x3x3 mesh: on a 2-point axis R and -R would be the same supercell vector, and phase or
    # orbital-order mistakes would cancel
    wl = workload("small")
    coef_w = gaussian_wannier(wl.bands, 4, np.array([(0.1, 0.2, 0.0), (0.5, 0.4, 0.3)]), sigma=1.6)
    return wl, coef_w


def _oracle_bare(wl, coef_w):
    b = wl.bands
    nk = b.kfrac.shape[0]
    nw = coef_w.shape[1]
    U = np.zeros((len(R_LIST), nw, nw), dtype=np.complex128)
    J = np.zeros_like(U)
    for q in b.kfrac:
        G = OL.eps_sphere(b.cell.lat, q, b.ecut_psi)                  # 0 < 1/2|q+G|^2 <= E_psi
        M = OI.wannier_pair_density(b, coef_w, q, G, wrap=False)
        rd, rx = OI.densities(M, b.kfrac, nw, R_LIST)
        u, j = OI.q_term_bare(rd, rx, OI.coulomb(b.cell.lat, q, G), q, R_LIST, nk)
        U += u
        J += j
    return U, J


def _real_space(wl, coef_w, nc=20):
    """Wannier functions phi_j0 on the supercell grid (nc points per cell axis)."""
    b = wl.bands
    n = np.array(b.kmesh)
    L = n * nc
    nk = int(np.prod(n))
    V = nk * b.cell.omega
    nw = coef_w.shape[1]
    phi = np.zeros((nw,) + tuple(L), dtype=np.complex128)
    for k in range(nk):
        npw = int(b.npw[k])
        m = np.rint(n[None, :] * (b.miller[k, :npw] + b.kfrac[k][None, :])).astype(np.int64)   # supercell units
        assert np.all(np.abs(m) < L // 2)
        for j in range(nw):
            F = np.zeros(tuple(L), dtype=np.complex128)
            idx = np.mod(m, L[None, :])
            F[idx[:, 0], idx[:, 1], idx[:, 2]] = coef_w[k, j, :npw]
            phi[j] += np.fft.ifftn(F) * np.prod(L)            # sum_G C e^{i(k+G).r}
    phi /= np.sqrt(nk) * np.sqrt(V)
    return phi, L, V


def test_bare_integrals_against_real_space_supercell(wan):
    wl, coef_w = wan
    b = wl.bands
    U, J = _oracle_bare(wl, coef_w)
    phi, L, V = _real_space(wl, coef_w)
    nw = phi.shape[0]
    dv = V / np.prod(L)
    # normalisation: int |phi_j0|^2 = 1 and <phi_i0|phi_j0> = delta_ij
    ov = np.einsum("ixyz,jxyz->ij", phi.conj(), phi) * dv
    assert np.abs(ov - np.eye(nw)).max() < 1e-10
    # Q = q + G on the supercell reciprocal lattice, 0 < 1/2|Q|^2 <= E_psi
    m = np.stack(np.meshgrid(*[np.fft.fftfreq(int(l), 1.0 / int(l)) for l in L], indexing="ij"), axis=-1)
    Q = (m / np.array(b.kmesh)[None, None, None, :]) @ b.cell.recip
    Q2 = np.sum(Q * Q, axis=-1)
    sel = (0.5 * Q2 <= b.ecut_psi) & (Q2 > 1e-12)
    kern = np.where(sel, 4.0 * np.pi / np.where(sel, Q2, 1.0), 0.0) / V

    def ft(f):                                                    # int f(r) e^{iQ.r} dr
        return np.fft.ifftn(f) * np.prod(L) * dv

    nc = L // np.array(b.kmesh)
    n0 = [ft(np.abs(phi[i]) ** 2) for i in range(nw)]
    for r, R in enumerate(R_LIST):
        shifted = np.roll(phi, tuple(int(R[a] * nc[a]) for a in range(3)), axis=(1, 2, 3))   # phi_jR(r) = phi_j0(r - R)
        for i in range(nw):
            for j in range(nw):
        # U_{i0jR}: densities of phi_i0 and phi_jR;  J_{i0jR}: pair product phi_i0^* phi_jR
                nj = ft(np.abs(shifted[j]) ** 2)
                u = np.sum(kern * n0[i] * nj.conj())
                p = ft(phi[i].conj() * shifted[j])
                jj = np.sum(kern * p * p.conj())
                assert abs(U[r, i, j] - u) <= 1e-9 * abs(u), (r, i, j, U[r, i, j], u)
                assert abs(J[r, i, j] - jj) <= 1e-9 * abs(U[0, 0, 0]), (r, i, j, J[r, i, j], jj)
    # onsite direct integrals are real and positive, the largest of all
    assert np.all(U[0].diagonal().real > 0) and np.abs(U[0].diagonal().imag).max() < 1e-12 * U[0, 0, 0].real


def test_screened_equals_bare_without_polarization(wan):
    """Eq. matrix_U with eps^-1 = 1 (W = v on the epsilon sphere) plus the tail is Eq. matrix_V."""
    wl, coef_w = wan
    b = wl.bands
    nk = b.kfrac.shape[0]
    nw = coef_w.shape[1]
    Ub, Jb = _oracle_bare(wl, coef_w)
    U = np.zeros((1, len(R_LIST), nw, nw), dtype=np.complex128)
    J = np.zeros_like(U)
    cut = wl.ecut_eps[0]
    for q in b.kfrac:
        G = OL.eps_sphere(b.cell.lat, q, cut)
        T = OL.tail_sphere(b.cell.lat, q, cut, b.ecut_psi)
        rd, rx = OI.densities(OI.wannier_pair_density(b, coef_w, q, G), b.kfrac, nw, R_LIST)
        rdt, rxt = OI.densities(OI.wannier_pair_density(b, coef_w, q, T), b.kfrac, nw, R_LIST)
        W = np.diag(OI.coulomb(b.cell.lat, q, G)).astype(np.complex128)[None]
        u, j = OI.q_term(rd, rx, W, rdt, rxt, OI.coulomb(b.cell.lat, q, T), q, R_LIST, nk)
        U += u
        J += j
    assert np.abs(U[0] - Ub).max() <= 1e-12 * np.abs(Ub).max()
    assert np.abs(J[0] - Jb).max() <= 1e-12 * np.abs(Jb).max()
