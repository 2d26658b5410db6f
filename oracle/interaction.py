"""Screened direct and exchange integrals U_{i0jR}(w), J_{i0jR}(w) and their bare forms (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 2.4, Eq. matrix_U:
    U_{i0jR}(w) = 4pi/(Omega N_q) sum_q sum_{G,G' in eps sphere} e^{-i q.R} rho_iq(G) eps^-1_GG'(q,w) rho_jq(G')^*
                + 4pi/(Omega N_q) sum_q sum_{G in tail}       e^{-i q.R} rho_iq(G) rho_jq(G)^*
  with rho_iq(G) = (1/(|q+G| N_k)) sum_k <phi~_{i,k+q}| e^{i(q+G).r} |phi~_{i,k}>.
Eq. matrix_J (no phase factor; R enters the density):
    J_{i0jR}(w) = 4pi/(Omega N_q) sum_q [ sum_{G,G'} rho_ijRq(G) eps^-1_GG' rho_ijRq(G')^* + sum_tail |rho_ijRq(G)|^2 ]
  with rho_ijRq(G) = (1/(N_k |q+G|)) sum_k e^{-i k.R} <phi~_{i,k+q}| e^{i(q+G).r} |phi~_{j,k}>.
Eq. matrix_V / matrix_X: the bare integrals, eps^-1 replaced by the identity.

Readings taken here:
  * the Bloch orbitals phi~_ik are normalised on the crystal like the Bloch functions (Eq. pak),
    so (1/N_k) sum_k <phi~_{k+q}|e^{iQ.r}|phi~_k> is the Fourier component at Q = q+G of the
    Wannier function's density (it tends to 1 as Q -> 0);
  * in the definition of rho_iq(G) both orbitals are i (the density of Wannier function i;
    the printed ket index j is read as i);
  * with v^1/2_G = sqrt(4pi/Omega)/|q+G| the first term is rho^_i W rho^_j^H with W of Eq. Wq and
    rho^ = rho |q+G|, and the tail term uses W's bare diagonal 4pi/(Omega |q+G|^2);
  * the bare exchange integral sums over the whole wave-function sphere, like the bare direct
    one (it is Eq. matrix_J with eps^-1 -> identity, whose tail term extends to N_G^psi; the
    printed upper limit N_G^eps of Eq. matrix_X is read as N_G^psi);
  * q = 0, G = 0 is left out (the same convention as the epsilon sphere of this path).

The pair densities <phi~_{a,k+q}|e^{i(q+G).r}|phi~_{o,k}> are the direct G-space convolution of
pair_density.py applied to the Wannier coefficient vectors.
"""
import numpy as np

from .lattice import reciprocal, volume
from .pair_density import pair_density


def wannier_pair_density(bands, coef_w, q_frac, gsphere, fft=None, wrap=False):
    """M[G, (k * nw + a) * nw + o] = <phi~_{a,k+q}| e^{i(q+G).r} |phi~_{o,k}> for all orbital pairs."""
    from dataclasses import replace
    nw = coef_w.shape[1]
    wb = replace(bands, coef=np.concatenate([coef_w, coef_w], axis=1), energy=np.zeros((coef_w.shape[0], 2 * nw)))
    return pair_density(wb, nw, nw, q_frac, gsphere, fft=fft, wrap=wrap)


def densities(M, kfrac, nw, R_list):
    """(rho_d [nw, NG], rho_x [nR, nw, nw, NG]) without the 1/|q+G| factor:
    rho_d[i] = (1/N_k) sum_k M(k; i, i),  rho_x[R, i, j] = (1/N_k) sum_k e^{-2 pi i k.R} M(k; i, j)."""
    ng = M.shape[0]
    nk = kfrac.shape[0]
    Mk = M.reshape(ng, nk, nw, nw)                                 # [G, k, a, o]
    rho_d = np.einsum("gkii->ig", Mk) / nk
    ph = np.exp(-2j * np.pi * (np.asarray(R_list, dtype=np.float64) @ kfrac.T))   # [nR, k]
    rho_x = np.einsum("rk,gkij->rijg", ph, Mk) / nk
    return rho_d, rho_x


def q_term(rho_d, rho_x, W, rho_d_t, rho_x_t, vt, q_frac, R_list, nq):
    """This q's contribution to U and J [F, nR, nw, nw]: W [F, NG, NG] on the epsilon sphere, rho on
    the sphere and on the tail (vt: 4pi/(Omega |q+G|^2) of the tail)."""
    ph = np.exp(-2j * np.pi * (np.asarray(R_list, dtype=np.float64) @ np.asarray(q_frac)))   # e^{-iq.R}
    nf = W.shape[0]
    nR, nw = rho_x.shape[0], rho_x.shape[1]
    U = np.zeros((nf, nR, nw, nw), dtype=np.complex128)
    J = np.zeros_like(U)
    tail_d = (rho_d_t * vt[None, :]) @ rho_d_t.conj().T                       # [i, j]
    tail_x = np.einsum("rijg,g,rijg->rij", rho_x_t, vt, rho_x_t.conj())
    for f in range(nf):
        ud = rho_d @ W[f] @ rho_d.conj().T
        for r in range(nR):
            U[f, r] = ph[r] * (ud + tail_d)
            x = rho_x[r].reshape(nw * nw, -1)
            J[f, r] = np.einsum("ag,gh,ah->a", x, W[f], x.conj()).reshape(nw, nw) + tail_x[r]
    return U / nq, J / nq


def q_term_bare(rho_d, rho_x, v, q_frac, R_list, nq):
    """Eq. matrix_V / matrix_X term of one q: rho over the whole wave-function sphere, v = 4pi/(Omega|q+G|^2)."""
    ph = np.exp(-2j * np.pi * (np.asarray(R_list, dtype=np.float64) @ np.asarray(q_frac)))
    U = ph[:, None, None] * ((rho_d * v[None, :]) @ rho_d.conj().T)[None]
    J = np.einsum("rijg,g,rijg->rij", rho_x, v, rho_x.conj())
    return U / nq, J / nq


def coulomb(lat, q_frac, miller):
    """4 pi / (Omega |q+G|^2) of the given Miller list."""
    b = reciprocal(lat)
    qg = (np.asarray(miller, dtype=np.float64) + np.asarray(q_frac)[None, :]) @ b
    return 4.0 * np.pi / volume(lat) / np.sum(qg * qg, axis=1)
