"""Pins for the oracle's Fermi-surface integral and plasma frequency (Sec. 2.3, Eq. plasma).

* one tetrahedron: the delta-function weights of its four corners sum to the derivative of the
  occupied fraction of its volume, the textbook piecewise closed form (E - d1)^3 / prod(d_i - d1)
  below the second corner energy, and its mirror image above the third;
* free electrons (plane-wave bands of a simple-cubic cell): the density of states at E_F tends to
  Omega sqrt(2 E_F) / (2 pi^2) per spin, and w_pl^2 to 4 pi n (n = k_F^3 / (3 pi^2), spin included),
  the Drude value, with the error shrinking as the mesh grows.
"""
import numpy as np

from oracle import plasma as OPL
from synth import Bands, sc_cell
from synth.epm import kmesh_frac, psi_sphere


def test_single_tetrahedron_corner_weights():
    rng = np.random.default_rng(4)
    for _ in range(50):
        d = np.sort(rng.uniform(-1.0, 1.0, 4))
        for E, lo in ((d[0] + 0.7 * (d[1] - d[0]), True), (d[2] + 0.4 * (d[3] - d[2]), False)):
            w = sum(OPL._trunc_cubic_dd(np.append(d, d[j])[None, :], E)[0] for j in range(4))
            if lo:
                ref = 3 * (E - d[0]) ** 2 / ((d[1] - d[0]) * (d[2] - d[0]) * (d[3] - d[0]))
            else:
                ref = 3 * (d[3] - E) ** 2 / ((d[3] - d[0]) * (d[3] - d[1]) * (d[3] - d[2]))
            assert abs(w - ref) <= 1e-10 * abs(ref)


def _free_bands(n, a, ecut):
    cell = sc_cell(a)
    kf = kmesh_frac((n, n, n))
    spheres = [psi_sphere(cell.recip, k, ecut) for k in kf]
    nb = min(len(s) for s in spheres)
    pmax = max(len(s) for s in spheres)
    nk = len(kf)
    miller = np.zeros((nk, pmax, 3), dtype=np.int32)
    coef = np.zeros((nk, nb, pmax), dtype=np.complex128)
    energy = np.zeros((nk, nb))
    for i, s in enumerate(spheres):
        miller[i, :len(s)] = s
        kin = 0.5 * np.sum(((s + kf[i]) @ cell.recip) ** 2, axis=1)
        order = np.argsort(kin, kind="stable")[:nb]
        coef[i, np.arange(nb), order] = 1.0
        energy[i] = kin[order]
    return Bands(cell=cell, kmesh=(n, n, n), kfrac=kf, npw=np.array([len(s) for s in spheres], dtype=np.int32),
                 miller=miller, coef=coef, energy=energy, ecut_psi=ecut), nb


def test_free_electron_dos_and_plasma_frequency():
    a, kf = 4.0, 1.1
    ef = 0.5 * kf * kf
    n_e = kf ** 3 / (3 * np.pi ** 2)
    errs_w, errs_g, errs_o = [], [], []
    for n in (6, 14):
        b, nb = _free_bands(n, a, ecut=0.5 * (kf + 2.2) ** 2)
        assert b.energy[:, -1].min() > ef + 0.5           # every band that crosses E_F is in the set
        x = OPL.delta_weights(b.energy, b.kmesh, b.cell.recip, ef)
        g = x.sum() / b.kfrac.shape[0]
        errs_g.append(abs(g / (b.cell.omega * np.sqrt(2 * ef) / (2 * np.pi ** 2)) - 1))
        w2 = OPL.plasma_tensor(b, ef, nb)
        errs_w.append(np.abs(np.diag(w2) / (4 * np.pi * n_e) - 1).max())
        errs_o.append(np.abs(w2 - np.diag(np.diag(w2))).max() / w2[0, 0])     # isotropic in the limit
    # the sorted band index of crossing plane waves is interpolated linearly: first-order convergence
    assert errs_g[1] < 0.03 and errs_w[1] < 0.03 and errs_o[1] < 0.02, (errs_g, errs_w, errs_o)
    assert errs_g[1] < errs_g[0] and errs_w[1] < errs_w[0] and errs_o[1] < errs_o[0], (errs_g, errs_w, errs_o)
