"""Intraband (Drude) plasma frequency of the usual RPA (oracle), Sec. 2.3, Eq. plasma.

TEST INFRASTRUCTURE ONLY (see the package header).

Eq. plasma is a Fermi-surface integral of the diagonal momentum matrix elements (Eq. momentum):
    (w_pl^2)^{mu nu} = (4 pi / Omega) (2 / N_k) sum_k sum_a (1 - T_ak^2) p^mu_aa(k) p^nu_aa(k) delta(E_ak - E_F),
    p_aa(k) = sum_G |C_a(k+G)|^2 (k + G).
Reading: the printed equation has neither the 4 pi / Omega nor the spin factor and names the
result w_pl; the term it feeds into Eq. eps00 is w_pl^2 / (w (w + i d)), which is the Drude form
when w_pl^2 = 4 pi n_eff (atomic units) with the spin sum included; that is what is computed here
(and it gives 4 pi n for free electrons, the pin).

The delta function is integrated with the same tetrahedra as the frequency weights (6 per sub-cell,
24 around each mesh point, quantities linear in each): by the Hermite-Genocchi formula the vertex-j
integral (1/V_t) int_t lambda_j delta(E_F - D(k)) dk is the fourth divided difference
g[d1, d2, d3, d4, d_j] of g(x) = (x - E_F)^3_+ (whose fourth derivative is 6 delta(x - E_F)), and the
mesh-point weight is (1/6) sum over its 24 tetrahedra, so that (1/N_k) sum_k x_k f_k is the zone
average of f delta(E_F - E).  The divided difference of the truncated cubic is evaluated as the cubic
B-spline on the five nodes (Curry and Schoenberg) by the Cox-de Boor recursion, which has no
cancellation when nodes cluster.
"""
import numpy as np

from .lattice import reciprocal, volume
from .tetra import tetrahedra


def _bspline(t, x, i, k):
    """Normalised B-spline M_k(t; x_i..x_{i+k}) (integral one), by the Cox-de Boor recursion:
    M_1 = 1/(x_{i+1} - x_i) on [x_i, x_{i+1}), and
    M_k = k / ((k-1)(x_{i+k} - x_i)) [(t - x_i) M_{k-1}(x_i..) + (x_{i+k} - t) M_{k-1}(x_{i+1}..)];
    every term is non-negative, so clustered knots cost no accuracy."""
    a, b = x[..., i], x[..., i + k]
    w = b - a
    if k == 1:
        return np.where((t >= a) & (t < b) & (w > 0), 1.0 / np.where(w > 0, w, 1.0), 0.0)
    left = _bspline(t, x, i, k - 1)
    right = _bspline(t, x, i + 1, k - 1)
    val = k / ((k - 1) * np.where(w > 0, w, 1.0)) * ((t - a) * left + (b - t) * right)
    return np.where(w > 0, val, 0.0)


def _trunc_cubic_dd(nodes, ef):
    """g[x0..x4] for g(x) = (x - ef)^3_+ , nodes [..., 5]: by Curry and Schoenberg this divided
    difference is M_4(ef; sorted nodes) / 4, the cubic B-spline on the five nodes."""
    x = np.sort(np.asarray(nodes, dtype=np.float64), axis=-1)
    return _bspline(np.asarray(ef, dtype=np.float64), x, 0, 4) / 4.0


def delta_weights(energy, kmesh, recip, ef):
    """x[k, a]: (1/N_k) sum_k x[k, a] f(k) is the zone average of f delta(E_F - E_a(k))."""
    nk, nb = energy.shape
    tets = tetrahedra(kmesh, recip)
    x = np.zeros((nk, nb))
    d = energy[tets]                                            # [T, 4, nb]
    for j in range(4):
        nodes = np.stack([d[:, 0], d[:, 1], d[:, 2], d[:, 3], d[:, j]], axis=-1)   # [T, nb, 5]
        np.add.at(x, tets[:, j], _trunc_cubic_dd(nodes, ef) / 6.0)
    return x


def diagonal_momentum(bands, nband):
    """p[k, a, mu] = sum_G |C_a(k+G)|^2 (k + G)_mu (Cartesian)."""
    nk = bands.kfrac.shape[0]
    out = np.zeros((nk, nband, 3))
    b = reciprocal(bands.cell.lat)
    for k in range(nk):
        n = int(bands.npw[k])
        kg = (bands.miller[k, :n].astype(np.float64) + bands.kfrac[k]) @ b
        out[k] = (np.abs(bands.coef[k, :nband, :n]) ** 2) @ kg
    return out


def plasma_tensor(bands, ef, nband, T=None):
    """(w_pl^2)^{mu nu} [3, 3] of Eq. plasma over the lowest nband bands (T [nk, nband] or None)."""
    e = bands.energy[:, :nband]
    x = delta_weights(e, bands.kmesh, reciprocal(bands.cell.lat), ef)
    if T is not None:
        x = x * (1.0 - np.asarray(T)[:, :nband] ** 2)
    p = diagonal_momentum(bands, nband)
    nk = e.shape[0]
    return (4.0 * np.pi / volume(bands.cell.lat)) * (2.0 / nk) * np.einsum("ka,kam,kan->mn", x, p, p)
