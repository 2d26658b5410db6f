"""Localized orbitals standing in for maximally localized Wannier functions (setup only).

The interaction step of the method takes Wannier functions from a separate program (the paper's
`wannier` stage, which precedes calc_int).  Here they are made from seeded s-type Gaussians: at each
k point the Gaussian g_i centred at tau_i, Bloch-summed,
    g_ik(G) = exp(-|k+G|^2 s^2 / 2 - i (k+G).tau_i),
is projected on the lowest `nwin` bands, A[a, i] = <psi_ak | g_ik>, and the projections are made
orthonormal (Loewdin, U^k = A (A^H A)^{-1/2}).  The cRPA weight of band a at k (Eq. tak) is
T_ak = sum_i |U^k_ai|^2.  The Bloch orbital of Wannier function i at k has
plane-wave coefficients C~_ik = sum_a U^k_ai C_ak in the band set's own plane-wave order, normalised
to one like the bands.  Nothing here is a step of the screened-interaction method itself.
"""
import numpy as np


def gaussian_wannier(bands, nwin, centers_frac, sigma, first=0, with_T=False):
    """Coefficients [nk][nw][npw_max] (complex128, zero padded) of the projected Gaussians at the
    fractional centres centers_frac [nw][3] (width sigma, bohr) in the window of the nwin bands from
    band `first` on.  With with_T also the cRPA weights T [nk][nband] of Eq. tak,
    T_ak = sum_i |U^k_ai|^2 (zero outside the window)."""
    cell = bands.cell
    tau = np.asarray(centers_frac, dtype=np.float64) @ cell.lat          # Cartesian centres
    nw = tau.shape[0]
    if nw > nwin:
        raise ValueError("more orbitals than bands in the window")
    nk, nband, pmax = bands.coef.shape
    out = np.zeros((nk, nw, pmax), dtype=np.complex128)
    T = np.zeros((nk, nband))
    for k in range(nk):
        n = int(bands.npw[k])
        kg = (bands.miller[k, :n].astype(np.float64) + bands.kfrac[k]) @ cell.recip
        g = np.exp(-0.5 * sigma * sigma * np.sum(kg * kg, axis=1))[None, :] * np.exp(-1j * (tau @ kg.T))
        C = bands.coef[k, first:first + nwin, :n]                          # [nwin, n]
        A = C.conj() @ g.T                                                 # [nwin, nw]
        s, V = np.linalg.eigh(A.conj().T @ A)
        if s.min() <= 1e-10 * s.max():
            raise ValueError("the Gaussians have no independent projection on the band window")
        U = A @ (V * (1.0 / np.sqrt(s))[None, :]) @ V.conj().T              # Loewdin
        out[k, :, :n] = U.T @ C
        T[k, first:first + nwin] = np.sum(np.abs(U) ** 2, axis=1)
    return (out, T) if with_T else out
