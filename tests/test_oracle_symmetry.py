"""Pin for the oracle's rotation of q-point matrices (Sec. 3.1, Eq. symeps): with the plain
Lorentzian X of Eq. Xakqbk at the mesh points (a k sum that the cube's rotations map onto itself),
chi0 computed directly at the image q = q* S - G_s equals chi0 at q* with its G indices rotated,
for every rotation that maps the mesh onto itself; the tetrahedron weights, whose six-tetrahedra
split of a sub-cell singles out one main diagonal, agree only to integration error.  The band
counts put both ends of the band list in gaps at every k (6 + 6 bands of the 4^3 fcc cell): a
list that ends inside a degenerate multiplet at some k is not mapped onto itself by the rotations."""
from dataclasses import replace

import numpy as np

from conftest import workload
from oracle import chi0 as C, lattice as L, pair_density as PD, symmetry as SY
from synth.epm import cubic_rotations


def _chi(wl, q, cut, kind):
    G = L.eps_sphere(wl.cell.lat, q, cut)
    M = PD.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    return G, C.chi0(M, C.pair_weights(wl, q, kind=kind))


def test_rotated_chi0_equals_direct_chi0():
    wl = workload("tiny", nocc=6, nemp=6)
    assert (wl.bands.energy[:, 6] - wl.bands.energy[:, 5]).min() > 1e-2     # the occupied set ends in a gap
    wl = replace(wl, freq=wl.freq[[0, 4]])
    qs = np.array([0.25, 0.0, 0.0])
    cut = wl.ecut_eps[0]
    Gs, chi_s = _chi(wl, qs, cut, "lorentz")
    _, chi_s_t = _chi(wl, qs, cut, "tetra")
    n = np.array(wl.bands.kmesh)
    seen = 0
    for S in cubic_rotations(wl.cell.recip):
        img = qs @ S
        q = np.mod(img, 1.0)
        q[np.abs(q - 1.0) < 1e-12] = 0.0
        if np.allclose(q, qs) or seen >= 3:
            continue
        g_s = np.rint(img - q).astype(np.int64)
        assert np.allclose(q * n, np.rint(q * n))
        G, chi = _chi(wl, q, cut, "lorentz")
        perm = SY.image_index(Gs, G, S, g_s)
        rot = SY.rotate(chi_s, perm)
        assert np.abs(rot - chi).max() <= 1e-12 * np.abs(chi).max()
        _, chi_t = _chi(wl, q, cut, "tetra")
        rot_t = SY.rotate(chi_s_t, perm)
        assert np.abs(rot_t - chi_t).max() <= 5e-2 * np.abs(chi_t).max()
        seen += 1
    assert seen == 3
