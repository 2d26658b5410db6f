"""q -> 0 limit of chi0 and epsilon for an insulator, and the optical spectra (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 2.3, Eq. eps00 (Eq. eps00-cRPA without the intraband term, which vanishes for a gapped
system): lim_{q->0} eps_00 = 1 - (4 pi / Omega) lim chi_00 / q^2, with the long-wavelength limit of
the pair densities taken analytically (Hybertsen and Louie, as the paper cites for insulators).
With the momentum matrix of Eq. momentum (local potential: exact),
    p_ao(k) = <psi_ak| -i nabla |psi_ok> = sum_G C_a(k+G)^* (k+G) C_o(k+G),
first-order k.p gives for a != o  M^0_ao(k+q, k) = <psi_{a,k+q}| e^{iq.r} |psi_ok> -> q.p_ao / (E_ak - E_ok).
So, along the unit direction qhat, with u_b = qhat.p_b / D_b for the pair b = (k, a, o):
    head = lim chi_00 / q^2   = sum_b w_b |u_b|^2
    wing = lim chi_G0 / |q|   = sum_b w_b M^G_b conj(u_b),   lim chi_0G / |q| = sum_b w_b u_b conj(M^G_b)
(w_b the pair weights at q = 0 and M^G_b the pair densities at q = 0, G != 0).  That is Eq. chi
for an extended set of rows in which the G = 0 row is u: chi_ext = M_ext diag(w) M_ext^H.

Reading: the paper writes the head with d^2 chi_00/dq^2; it is read as the q^2 coefficient
lim chi_00 / q^2 (the factor that v_0 = 4 pi / (Omega q^2) multiplies), not twice it.

Macroscopic quantities (Eqs. epsilonM, eels, optical-conductivity, reflectance), from the head
element of the inverse of the extended epsilon:
    eps_M = 1 / eps^-1_00,  L = -Im eps^-1_00,  Re sigma = (w / 4 pi) Im eps_M,
    R = |(1 - sqrt(eps^-1_00)) / (1 + sqrt(eps^-1_00))|^2.
Reading: the printed reflectance has no square; the normal-incidence reflectivity is the squared
modulus of that amplitude ratio (which equals |(sqrt(eps_M) - 1)/(sqrt(eps_M) + 1)|^2), taken here.
"""
import numpy as np

from .lattice import reciprocal, volume


def momentum(bands, k, bands_a, bands_o):
    """p[a, o, mu] = sum_G conj(C_a(k+G)) (k+G)_mu C_o(k+G) (Cartesian), Eq. momentum."""
    n = int(bands.npw[k])
    kg = (bands.miller[k, :n].astype(np.float64) + bands.kfrac[k]) @ reciprocal(bands.cell.lat)
    Ca = bands.coef[k, bands_a, :n]
    Co = bands.coef[k, bands_o, :n]
    return np.stack([(Ca.conj() * kg[None, :, m]) @ Co.T for m in range(3)], axis=-1)


def head_row(wl, qhat, k_list=None):
    """u[b] = qhat.p_b / (E_ak - E_ok) for the pairs b = (k, a, o) at q = 0 (pair order of Eq. chi)."""
    b = wl.bands
    qhat = np.asarray(qhat, dtype=np.float64)
    qhat = qhat / np.linalg.norm(qhat)
    ks = range(b.kfrac.shape[0]) if k_list is None else k_list
    out = []
    for k in ks:
        emp = np.arange(wl.nocc, wl.nocc + wl.nemp)
        occ = np.arange(wl.nocc)
        p = momentum(b, k, emp, occ) @ qhat                           # [a, o]
        d = b.energy[k, emp][:, None] - b.energy[k, occ][None, :]
        out.append((p / d).reshape(-1))
    return np.concatenate(out)


def extended_rows(u, M):
    """M_ext: the head row u (the long-wavelength limit of M^{G=0} / |q|) above the rows of M."""
    return np.concatenate([u[None, :], M], axis=0)


def coulomb_sqrt_ext(lat, miller):
    """v^1/2 of the extended rows at q -> 0: sqrt(4 pi/Omega) for the head (the 1/|q| it carries is
    taken out with the q of u), sqrt(4 pi/Omega)/|G| for the rest."""
    b = reciprocal(lat)
    g = np.linalg.norm(np.asarray(miller, dtype=np.float64) @ b, axis=1)
    s = np.sqrt(4.0 * np.pi / volume(lat))
    return np.concatenate([[s], s / g])


def macroscopic(freq, einv00):
    """(eps_M, L, Re sigma, R) per frequency from eps^-1_00 (real frequencies)."""
    einv00 = np.asarray(einv00, dtype=np.complex128)
    eps_m = 1.0 / einv00
    loss = -einv00.imag
    sigma = np.asarray(freq) / (4.0 * np.pi) * eps_m.imag
    s = np.sqrt(einv00)
    refl = np.abs((1.0 - s) / (1.0 + s)) ** 2
    return eps_m, loss, sigma, refl
