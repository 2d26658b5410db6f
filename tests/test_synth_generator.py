"""Pins of the synthetic band generator (it prepares the inputs; it is not the method).

Each k point's coefficients must be eigenvectors of the model Hamiltonian of Eq. pak's plane-wave
basis, H_k[G, G'] = 1/2 |k + G|^2 delta_GG' + V(G - G'), on the sphere 1/2 |k + G|^2 <= E_cut^psi,
with V constant on the reciprocal-lattice shells the generator drew.  The pair-density pins rely
on the other properties checked here: orthonormal coefficients per k, ascending energies, and
zero padding beyond each k's plane-wave count.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def micro_fresh():
    from synth import make_workload
    return make_workload("micro", cache=False)     # uncached: the potential's shells are in meta


def _hamiltonian(b, k):
    """H_k built from its definition: kinetic diagonal plus the shell potential V(G - G')."""
    n = int(b.npw[k])
    m = b.miller[k, :n].astype(np.float64)
    kin = 0.5 * np.sum(((m + b.kfrac[k]) @ b.cell.recip) ** 2, axis=1)
    shells = np.asarray(b.meta["shells"], dtype=np.float64)
    vals = np.asarray(b.meta["v_shell"], dtype=np.float64)
    d = m[:, None, :] - m[None, :, :]
    g2 = np.sum((d @ b.cell.recip) ** 2, axis=-1)
    H = np.zeros((n, n), dtype=np.complex128)
    for s, v in zip(shells, vals):
        H[np.abs(g2 - s) < 1e-7 * max(1.0, s)] = v
    H[np.diag_indices(n)] += kin
    return H


def test_eigenpairs_of_the_model_hamiltonian(micro_fresh):
    b = micro_fresh.bands
    nband = b.energy.shape[1]
    for k in range(b.kfrac.shape[0]):
        n = int(b.npw[k])
        H = _hamiltonian(b, k)
        assert np.array_equal(H, H.conj().T)
        C = b.coef[k, :, :n]                       # [nband][npw]: row alpha holds C_alpha(k)[G]
        R = H @ C.T - C.T * b.energy[k][None, :]
        assert np.abs(R).max() <= 1e-10
        # the lowest nband eigenvalues of H, in ascending order
        assert np.allclose(b.energy[k], np.linalg.eigvalsh(H)[:nband], rtol=0, atol=1e-10)
        assert np.all(np.diff(b.energy[k]) >= 0)


def test_orthonormal_coefficients_and_zero_padding(micro_fresh):
    b = micro_fresh.bands
    nband = b.energy.shape[1]
    for k in range(b.kfrac.shape[0]):
        n = int(b.npw[k])
        C = b.coef[k, :, :n]
        assert np.allclose(C.conj() @ C.T, np.eye(nband), rtol=0, atol=1e-12)
        assert not np.any(b.coef[k, :, n:])
        assert not np.any(b.miller[k, n:])


def test_plane_wave_set_is_the_psi_sphere(micro_fresh):
    """The Miller set of each k is exactly {G : 1/2 |k + G|^2 <= E_cut^psi}, by brute force over a
    box that surely contains the sphere."""
    b = micro_fresh.bands
    r = np.arange(-8, 9)
    box = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    for k in range(b.kfrac.shape[0]):
        e = 0.5 * np.sum(((box + b.kfrac[k]) @ b.cell.recip) ** 2, axis=1)
        want = {tuple(g) for g in box[e <= b.ecut_psi]}
        got = {tuple(g) for g in b.miller[k, :int(b.npw[k])]}
        assert got == want
        assert np.abs(box[e <= b.ecut_psi]).max() < 8     # the box was large enough


def test_rotated_band_sets_match_direct_diagonalisation():
    """Band sets filled by rotating one eigenvector set per orbit of the cube's 48 rotations
    (the shell potential depends on |G| alone): at every mesh point the energies equal those of
    a direct diagonalisation, the Miller sets are the same spheres, and the rotated vectors are
    orthonormal eigenvectors of H_k rebuilt from its definition."""
    from synth import fcc_cell, make_bands
    from synth.configs import _mid_gap_cutoff_mesh
    cell = fcc_cell(10.2)
    pot = dict(kind="shells", nshell=6, vmin=0.1, vmax=0.3)
    ec = _mid_gap_cutoff_mesh(cell.recip, (4, 4, 4), 300)
    direct = make_bands(cell, (4, 4, 4), ec, 16, pot, seed=3, workers=1)
    rot = make_bands(cell, (4, 4, 4), ec, 16, pot, seed=3, workers=1, symmetry=True)
    assert rot.meta["irreducible_k"] == 8
    assert np.abs(direct.energy - rot.energy).max() < 1e-10
    assert np.array_equal(direct.npw, rot.npw) and np.array_equal(direct.miller, rot.miller)
    for k in range(rot.kfrac.shape[0]):
        n = int(rot.npw[k])
        H = _hamiltonian(rot, k)
        C = rot.coef[k, :, :n]
        assert np.abs(H @ C.T - C.T * rot.energy[k][None, :]).max() < 1e-10
        assert np.abs(C.conj() @ C.T - np.eye(C.shape[0])).max() < 1e-12


def test_psi_cutoff_off_every_mesh_sphere():
    """The wave-function cut-off lies in a gap of 1/2|k+G|^2 over every mesh point, so that no
    sphere membership depends on the rounding of a value equal to the cut-off."""
    from synth import fcc_cell
    from synth.configs import _mid_gap_cutoff_mesh
    from synth.epm import _miller_box, kmesh_frac
    cell = fcc_cell(10.2)
    for mesh, target in (((4, 4, 4), 300), ((3, 3, 3), 110)):
        ec = _mid_gap_cutoff_mesh(cell.recip, mesh, target)
        g = _miller_box(cell.recip, np.sqrt(2.0 * ec), (1.0, 1.0, 1.0))
        for k in kmesh_frac(mesh):
            e = 0.5 * np.sum(((g + k) @ cell.recip) ** 2, axis=1)
            assert np.abs(e - ec).min() > 1e-6 * ec
