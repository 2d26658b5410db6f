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
