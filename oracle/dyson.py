"""Symmetric dielectric matrix and screened interaction (oracle).

Eq. epsGG:  eps_GG' = delta_GG' - (4 pi / Omega) chi_GG' / (|q+G| |q+G'|).
Eq. Wq:     W_GG' = (4 pi / Omega) eps^-1_GG' / (|q+G| |q+G'|) inside the
            epsilon sphere, and 4 pi / (Omega |q+G|^2) on the diagonal for
            E_cut^eps < 1/2|q+G|^2 <= E_cut^psi (returned as a separate tail).
Written with v^{1/2}_G = sqrt(4 pi / Omega) / |q+G| this is
W = v^{1/2} (1 - v^{1/2} chi v^{1/2})^{-1} v^{1/2}.  The inverse is a
library LU solve (numpy.linalg.solve against the identity).
"""
import numpy as np

from .lattice import reciprocal, volume


def coulomb_sqrt(lat, q_frac, miller):
    b = reciprocal(lat)
    qg = (np.asarray(miller, dtype=np.float64) + np.asarray(q_frac)[None, :]) @ b
    return np.sqrt(4.0 * np.pi / volume(lat)) / np.linalg.norm(qg, axis=1)


def epsilon(chi, vs):
    ng = chi.shape[-1]
    return np.eye(ng)[None] - vs[None, :, None] * chi * vs[None, None, :]


def screened(chi, vs):
    eps = epsilon(chi, vs)
    ng = chi.shape[-1]
    out = np.empty_like(eps)
    for f in range(eps.shape[0]):
        out[f] = np.linalg.solve(eps[f], np.eye(ng, dtype=np.complex128))
    return vs[None, :, None] * out * vs[None, None, :]


def tail(lat, q_frac, tail_miller):
    return coulomb_sqrt(lat, q_frac, tail_miller) ** 2
