"""Interaction step (Sec. 2.4) on the GPU through the C ABI against the oracle: the q terms of the
screened direct and exchange integrals (Eq. matrix_U, Eq. matrix_J) accumulated over three q points
(Gamma among them) for a seeded W of the Eq. Wq form, and the bare integrals (Eq. matrix_V,
Eq. matrix_X).  Wannier functions: projected Gaussians on the tiny workload's occupied bands.
FP64 throughout: 1e-11 of the largest integral."""
import numpy as np
import pytest

from conftest import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402
from oracle import dyson as OD, interaction as OI, lattice as OL  # noqa: E402
from synth.wannier import gaussian_wannier  # noqa: E402

R_LIST = np.array([(0, 0, 0), (1, 0, 0), (0, 1, -1), (2, -1, 1)])
QS = [np.zeros(3), np.array([0.25, 0.0, 0.0]), np.array([0.25, 0.5, 0.75])]


def _seeded_w(lat, q, G, nf, seed):
    """W = v^1/2 (1 + X) v^1/2 with X a small seeded Hermitian matrix per frequency."""
    rng = np.random.default_rng(seed)
    vs = OD.coulomb_sqrt(lat, q, G)
    out = np.empty((nf, len(G), len(G)), dtype=np.complex128)
    for f in range(nf):
        X = 0.05 * (rng.standard_normal((len(G),) * 2) + 1j * rng.standard_normal((len(G),) * 2))
        out[f] = (np.eye(len(G)) + X + X.conj().T) * vs[:, None] * vs[None, :]
    return out


@pytest.mark.parametrize("on_device", [False, True])
def test_interaction_terms_against_oracle(on_device):
    wl = workload("tiny")
    b = wl.bands
    coef_w = gaussian_wannier(b, wl.nocc, np.array([(0.1, 0.2, 0.0), (0.5, 0.4, 0.3)]), sigma=1.6)
    nw = coef_w.shape[1]
    nk = b.kfrac.shape[0]
    ctx = rp.context_for(wl)
    ctx.rp_load_wannier(coef_w)
    cut = wl.ecut_eps[0]
    nf = 2
    Uo = np.zeros((nf, len(R_LIST), nw, nw), dtype=np.complex128)
    Jo = np.zeros_like(Uo)
    Ubo = np.zeros((1, len(R_LIST), nw, nw), dtype=np.complex128)
    Jbo = np.zeros_like(Ubo)
    U = J = Ub = Jb = None
    for iq, q in enumerate(QS):
        G = OL.eps_sphere(b.cell.lat, q, cut)
        T = OL.tail_sphere(b.cell.lat, q, cut, b.ecut_psi)
        P = OL.eps_sphere(b.cell.lat, q, b.ecut_psi)
        W = _seeded_w(b.cell.lat, q, G, nf, 40 + iq)
        rd, rx = OI.densities(OI.wannier_pair_density(b, coef_w, q, G), b.kfrac, nw, R_LIST)
        rdt, rxt = OI.densities(OI.wannier_pair_density(b, coef_w, q, T), b.kfrac, nw, R_LIST)
        u, j = OI.q_term(rd, rx, W, rdt, rxt, OI.coulomb(b.cell.lat, q, T), q, R_LIST, nk)
        Uo += u
        Jo += j
        rdp, rxp = OI.densities(OI.wannier_pair_density(b, coef_w, q, P), b.kfrac, nw, R_LIST)
        u, j = OI.q_term_bare(rdp, rxp, OI.coulomb(b.cell.lat, q, P), q, R_LIST, nk)
        Ubo[0] += u
        Jbo[0] += j
        Wg = torch.from_numpy(W).cuda() if on_device else W
        U, J = ctx.rp_interaction(q, R_LIST, W=Wg, U=U, J=J, accumulate=iq > 0)
        if on_device and Ub is None:
            Ub = torch.zeros((1, len(R_LIST), nw, nw), dtype=torch.complex128, device="cuda")
            Jb = torch.zeros_like(Ub)
        Ub, Jb = ctx.rp_interaction(q, R_LIST, U=Ub, J=Jb, accumulate=iq > 0)
    if on_device:
        torch.cuda.synchronize()
        U, J, Ub, Jb = (x.cpu().numpy() for x in (U, J, Ub, Jb))
    scale = np.abs(Uo).max()
    assert np.abs(U - Uo).max() <= 1e-11 * scale
    assert np.abs(J - Jo).max() <= 1e-11 * scale
    assert np.abs(Ub - Ubo).max() <= 1e-11 * np.abs(Ubo).max()
    assert np.abs(Jb - Jbo).max() <= 1e-11 * np.abs(Ubo).max()
    assert np.abs(Uo - Ubo).max() > 1e-3 * scale           # the screening changed the integrals


def test_interaction_needs_wannier_functions():
    wl = workload("micro")
    ctx = rp.context_for(wl)
    with pytest.raises(rp.RPError) as e:
        ctx._lib.nw = 1
        ctx.nw = 1
        ctx.rp_interaction(wl.q[0], [(0, 0, 0)])
    assert e.value.code == rp.RP_ERR_STATE
