"""The largest sphere of the workloads (NG about 4000, the large simple-cubic cell): the three
contraction tiers at NG = 4000 on seeded inputs, and the FP64 Dyson solve at NG about 4000, each
against the oracle.  These are the edge of the tile grids (20 x 125 tiles of the BF16x3 kernel,
63 x 63 of the FP64 one) and of the shared-memory pivot arrays of the Dyson kernels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402
from oracle import chi0 as OC, dyson as OD, lattice as OL  # noqa: E402
from synth import sc_cell  # noqa: E402
from synth.configs import _mid_gap_cutoff  # noqa: E402


def _rel_fro(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.fixture(scope="module")
def big_cell():
    """Context of the a = 20 bohr simple-cubic cell with a 2^3 mesh and an epsilon cut-off of about
    4000 sphere points at q = (1/2, 0, 0); the bands are minimal stand-ins (the solve needs only the
    sphere and the state of a loaded context)."""
    cell = sc_cell(20.0)
    q = np.array([0.5, 0.0, 0.0])
    ecut_eps = _mid_gap_cutoff(cell.recip, q, 4000, exclude_zero=True)
    ecut_psi = 1.5 * ecut_eps
    kmesh = (2, 2, 2)
    ctx = rp.Context(cell.lat, kmesh, (16, 16, 16), ecut_psi, ecut_eps)
    nk, npw, nband = 8, 4, 2
    miller = np.zeros((nk, npw, 3), dtype=np.int32)
    miller[:, :, 0] = np.arange(npw)[None, :] - 1
    coef = np.zeros((nk, nband, npw), dtype=np.complex128)
    coef[:, 0, 0] = 1.0
    coef[:, 1, 1] = 1.0
    energy = np.tile(np.array([-0.5, 0.5]), (nk, 1))
    ctx.load_bands(1, np.full(nk, npw, dtype=np.int32), miller, coef, energy)
    return cell, q, ctx


@pytest.mark.parametrize("precision,tol", [(rp.RP_FP64_NATIVE, 1e-12), (rp.RP_TF32X3, 2e-6),
                                           (rp.RP_BF16X3, 1e-4)])
def test_contraction_ng_4000(big_cell, precision, tol):
    _, _, ctx = big_cell
    rng = np.random.default_rng(4000)
    ng, K, nf = 4000, 1500, 1
    M = rng.standard_normal((ng, K)) + 1j * rng.standard_normal((ng, K))
    w = rng.standard_normal((nf, K)) + 1j * rng.standard_normal((nf, K))
    ref = OC.chi0(M, w)
    got = ctx.rp_contract_chi0(M, w, precision=precision)
    assert np.all(_rel_fro(got, ref) < tol)


def test_dyson_ng_about_4000(big_cell):
    cell, q, ctx = big_cell
    G, T = ctx.rp_sphere_size(q)
    ng = len(G)
    assert 3500 < ng <= 4096
    G_ref = OL.eps_sphere(cell.lat, q, _mid_gap_cutoff(cell.recip, q, 4000, exclude_zero=True))
    assert np.array_equal(G, G_ref)
    rng = np.random.default_rng(7)
    nf = 2
    B = (rng.standard_normal((nf, ng, 64)) + 1j * rng.standard_normal((nf, ng, 64))) * 0.05
    chi = -np.einsum("fik,fjk->fij", B, B.conj())          # negative semidefinite, like chi0 at i nu
    W, tail = ctx.rp_solve_w(q, chi)
    vs = OD.coulomb_sqrt(cell.lat, q, G)
    W_ref = OD.screened(chi, vs)
    assert np.all(_rel_fro(W, W_ref) < 1e-11)
    assert np.allclose(tail, OD.tail(cell.lat, q, T), rtol=1e-14, atol=0)
    # the Hermitian positive definite sweep (eps >= 1 here) at the same size
    ctx.rp_set_dyson_hermitian(True)
    Wh, _ = ctx.rp_solve_w(q, chi)
    ctx.rp_set_dyson_hermitian(False)
    assert np.all(_rel_fro(Wh, W_ref) < 1e-11)
