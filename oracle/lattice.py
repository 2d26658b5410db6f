"""Lattice bookkeeping for the oracle (test infrastructure only).

Sec. 2.3 (after Eq. epsGG): the polarization matrix is restricted to the
G vectors with 1/2|q+G|^2 <= E_cut^eps.  At q = 0 the G = 0 component is
left out of the sphere (its Coulomb factor 4 pi / |q+G|^2 diverges; the
analytic head of Eq. eps00 is not part of this path).
Eq. Wq: beyond that sphere, up to 1/2|q+G|^2 <= E_cut^psi, W is diagonal.
Both lists are returned in lexicographic (m1, m2, m3) Miller order.
"""
import numpy as np


def reciprocal(lat):
    lat = np.asarray(lat, dtype=np.float64)
    return 2.0 * np.pi * np.linalg.inv(lat).T


def volume(lat):
    return float(abs(np.linalg.det(np.asarray(lat, dtype=np.float64))))


def _box(lat, gmax, shift):
    a_len = np.linalg.norm(np.asarray(lat, dtype=np.float64), axis=1)
    nmax = np.floor(gmax * a_len / (2.0 * np.pi) + np.abs(shift) + 1).astype(int)
    out = []
    for m1 in range(-nmax[0], nmax[0] + 1):
        for m2 in range(-nmax[1], nmax[1] + 1):
            for m3 in range(-nmax[2], nmax[2] + 1):
                out.append((m1, m2, m3))
    return np.array(out, dtype=np.int64)


def half_q_plus_g_sq(lat, q_frac, miller):
    b = reciprocal(lat)
    qg = (np.asarray(miller, dtype=np.float64) + np.asarray(q_frac)[None, :]) @ b
    return 0.5 * np.sum(qg * qg, axis=1)


def eps_sphere(lat, q_frac, ecut_eps):
    """Miller list of the epsilon sphere for q (Sec. 2.3), lexicographic order."""
    q = np.asarray(q_frac, dtype=np.float64)
    g = _box(lat, np.sqrt(2.0 * ecut_eps), q)
    e = half_q_plus_g_sq(lat, q, g)
    keep = (e <= ecut_eps) & (e > 1e-14)
    return g[keep]


def tail_sphere(lat, q_frac, ecut_eps, ecut_psi):
    """Miller list with E_cut^eps < 1/2|q+G|^2 <= E_cut^psi (Eq. Wq, second case)."""
    q = np.asarray(q_frac, dtype=np.float64)
    g = _box(lat, np.sqrt(2.0 * ecut_psi), q)
    e = half_q_plus_g_sq(lat, q, g)
    keep = (e > ecut_eps) & (e <= ecut_psi)
    return g[keep]


def kmesh_index(kmesh, i):
    n1, n2, n3 = kmesh
    return (i[0] % n1) * n2 * n3 + (i[1] % n2) * n3 + (i[2] % n3)


def umklapp(kmesh, q_frac):
    """For every mesh point k: (index of k', G0) with k + q = k' + G0, k' in [0,1)^3."""
    n = np.asarray(kmesh, dtype=np.int64)
    qi = np.rint(np.asarray(q_frac) * n).astype(np.int64)
    if np.max(np.abs(qi / n - np.asarray(q_frac))) > 1e-9:
        raise ValueError("q is not a vector of the k mesh")
    nk = int(np.prod(n))
    kp = np.zeros(nk, dtype=np.int64)
    g0 = np.zeros((nk, 3), dtype=np.int64)
    for k in range(nk):
        i = np.array([k // (n[1] * n[2]), (k // n[2]) % n[1], k % n[2]])
        j = i + qi
        g0[k] = np.floor_divide(j, n)
        kp[k] = kmesh_index(kmesh, j - g0[k] * n)
    return kp, g0
