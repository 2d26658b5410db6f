"""Polarization chi_GG'(q, w) as a dense sum (oracle).

Eq. chi:  chi_GG'(q,w) = (2/N_k) sum_k sum_{a unocc} sum_{b occ}
              (1 - T_{a,k+q} T_{b,k}) M^G_ab M^{G'}_ab^* X_ab(w).
The factor 2 is the spin sum; T = 0 is the usual RPA (Eq. tak).  The pair
weight w_b(w) = (2/N_k)(1 - T T) x carries everything but the matrix
elements, so chi(w) = M diag(w(w)) M^H with M[G, b] (pair order of
pair_density.py).

Occupations: band-index occupations by default (the n_occ lowest bands of
each k are occupied, the next n_emp empty).  With `fermi` given, a metal:
  * Lorentzian weights: a pair counts only when its occupied state lies below
    the Fermi energy and its empty state at k+q on or above it (energy
    occupations, as in the free-electron gas), a factor on the pair weight;
  * tetrahedron weights: each tetrahedron is clipped to its part where band o
    (at k) lies below the Fermi energy and band a (at k+q) above it, both
    interpolated linearly (Fermi-surface clipping; tetra.metal_vertex_weights).
A metal's band list holds its partly filled bands in both ranges (the first
n_occ entries are the bands that may be occupied, the next n_emp those that
may be empty), so a pair (a, o) of one band with itself is an intraband term.
"""
import numpy as np

from .lattice import umklapp
from .tetra import poles, tetrahedra, vertex_weights, metal_vertex_weights, lorentz_x


def pair_weights(wl, q_frac, k_list=None, kind="tetra", fermi=None):
    """w[f, b] for the pairs of k_list (default all), Eq. chi prefactors x X."""
    b = wl.bands
    nk = b.kfrac.shape[0]
    kp, _ = umklapp(b.kmesh, q_frac)
    e_occ = b.energy[:, :wl.nocc]
    e_emp = b.energy[kp, wl.nocc:wl.nocc + wl.nemp]
    z1, z2 = poles(wl.freq, wl.axis, wl.delta, wl.ordering)
    ks = np.arange(nk) if k_list is None else np.asarray(k_list)
    if kind == "tetra" and fermi is not None:
        tets = tetrahedra(b.kmesh, b.cell.recip)
        x = metal_vertex_weights(e_occ, e_emp, tets, z1, z2, wl.delta_a, wl.delta_r, fermi, k_list=ks)
    elif kind == "tetra":
        tets = tetrahedra(b.kmesh, b.cell.recip)
        x = vertex_weights(e_occ, e_emp, tets, z1, z2, wl.delta_a, wl.delta_r, k_list=ks)
    elif kind == "lorentz":
        x = lorentz_x(e_occ[ks], e_emp[ks], z1, z2)
    else:
        raise ValueError(kind)
    if wl.T is not None:
        # empty band a at k' = k+q, occupied band o at k
        tt = 1.0 - wl.T[kp][:, wl.nocc:wl.nocc + wl.nemp][:, :, None] * wl.T[:, :wl.nocc][:, None, :]
        x = x * tt[ks][..., None]
    if fermi is not None and kind == "lorentz":
        sel = (e_occ < fermi)[:, None, :] & (e_emp >= fermi)[:, :, None]     # [k, a, o]
        x = x * sel[ks][..., None]
    w = (2.0 / nk) * x                                    # [k, a, o, f]
    return np.ascontiguousarray(w.reshape(-1, w.shape[-1]).T)   # [f, b]


def chi0(M, w):
    """chi[f] = M diag(w[f]) M^H (Eq. chi), M [NG, K], w [F, K] -> [F, NG, NG]."""
    M = np.asarray(M, dtype=np.complex128)
    out = np.empty((w.shape[0], M.shape[0], M.shape[0]), dtype=np.complex128)
    for f in range(w.shape[0]):
        out[f] = (M * w[f][None, :]) @ M.conj().T
    return out
