"""Pair densities M^G_ab(k+q, k) by direct G-space convolution (oracle).

Eq. ism: M^G_ab(k+q,k) = <psi_{a,k+q}| e^{i(q+G).r} |psi_{b,k}>, with the
Bloch functions of Eq. pak normalised on the crystal volume.  Writing
k + q = k' + G0 (k' on the mesh) and inserting the plane-wave expansions,
the integral leaves one Kronecker delta, so

    M^G_ab = sum_{G1 in sphere(k)}  conj(C_a(k')[G1 + G + G0]) * C_b(k)[G1],

a coefficient outside the sphere of k' being zero.  The paper evaluates this
with FFTs; the oracle writes the sum out.  Two index conventions:
  * wrap=True  ("grid"): G1+G+G0 is reduced modulo the FFT grid per axis,
    which is exactly the circular convolution an FFT product computes;
  * wrap=False ("free"): no reduction (the plain definition).
They agree whenever the grid is free of aliasing.

Pair ordering (column index of M): b = (k * n_emp + a) * n_occ + o, where
a = alpha - n_occ runs over the empty bands at k+q and o over the occupied
bands at k (0-based).
"""
import numpy as np

from .lattice import umklapp


def _grid_table(miller_k, npw, fft):
    """Position of each wrapped Miller index of a sphere on the FFT grid (-1: absent)."""
    m = np.asarray(miller_k[:npw], dtype=np.int64)
    n = np.asarray(fft, dtype=np.int64)
    table = -np.ones(tuple(n), dtype=np.int64)
    w = np.mod(m, n[None, :])
    if len(np.unique(w, axis=0)) != npw:
        raise ValueError("wave-function sphere does not fit the FFT grid")
    table[w[:, 0], w[:, 1], w[:, 2]] = np.arange(npw)
    return table


def pair_density(bands, nocc, nemp, q_frac, gsphere, fft=None, k_list=None, wrap=True):
    """M[G, b] for b over the pairs of the k points in k_list (default: all)."""
    kp_of, g0_of = umklapp(bands.kmesh, q_frac)
    nk = bands.kfrac.shape[0]
    ks = list(range(nk)) if k_list is None else list(k_list)
    G = np.asarray(gsphere, dtype=np.int64)
    ng = G.shape[0]
    out = np.zeros((ng, len(ks) * nemp * nocc), dtype=np.complex128)
    for ik, k in enumerate(ks):
        kp, g0 = kp_of[k], g0_of[k]
        npw_k, npw_kp = int(bands.npw[k]), int(bands.npw[kp])
        m1 = np.asarray(bands.miller[k, :npw_k], dtype=np.int64)
        c_occ = bands.coef[k, :nocc, :npw_k]                   # [nocc, npw_k]
        c_emp = bands.coef[kp, nocc:nocc + nemp, :npw_kp]      # [nemp, npw_kp]
        if wrap:
            table = _grid_table(bands.miller[kp], npw_kp, fft)
        else:
            table = {tuple(r): i for i, r in enumerate(np.asarray(bands.miller[kp, :npw_kp], dtype=np.int64))}
        for ig in range(ng):
            tgt = m1 + (G[ig] + g0)[None, :]                   # G1 + G + G0
            if wrap:
                w = np.mod(tgt, np.asarray(fft, dtype=np.int64)[None, :])
                idx = table[w[:, 0], w[:, 1], w[:, 2]]
            else:
                idx = np.array([table.get(tuple(r), -1) for r in tgt], dtype=np.int64)
            valid = idx >= 0
            shifted = np.zeros((nemp, npw_k), dtype=np.complex128)
            shifted[:, valid] = c_emp[:, idx[valid]]
            # M[a, o] = sum_G1 conj(C_a(k')[G1+G+G0]) C_o(k)[G1]
            mblock = np.conj(shifted) @ c_occ.T                 # [nemp, nocc]
            base = ik * nemp * nocc
            out[ig, base:base + nemp * nocc] = mblock.reshape(-1)
    return out
