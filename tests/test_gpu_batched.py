"""The batched workload (all 216 q of a 6^3 mesh, epsilon spheres of 300-900 G chosen per q, 24
imaginary frequencies, 16 + 64 bands) at full size, on six q: Gamma, the q with the largest sphere
and four seeded ones.  Per q, against the FP64 oracle: the pair densities of one k point element
by element and the tetrahedron weights of two k points at three frequencies; then the batched
BF16x3 build of the six against the per-q FP64 builds (the same sums), and the batched Dyson step
against the per-q one."""
import numpy as np
import pytest

from conftest import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402
from oracle import chi0 as OC, lattice as OL, pair_density as OP  # noqa: E402

FI = [0, 11, 23]


def _rel_fro(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.fixture(scope="module")
def batched():
    return workload("batched")


@pytest.fixture(scope="module")
def picks(batched):
    wl = batched
    cut_rank = np.argsort(wl.ecut_eps)
    rng = np.random.default_rng(216)
    seeded = [int(i) for i in rng.choice(np.arange(1, len(wl.q)), size=6, replace=False)]
    out = [0, int(cut_rank[-1])]
    for i in seeded:
        if i not in out and len(out) < 6:
            out.append(i)
    assert np.allclose(wl.q[0], 0.0)
    return out


def test_sampled_parity_on_six_q(batched, picks):
    from dataclasses import replace
    wl = batched
    b = wl.bands
    nb = wl.nocc + wl.nemp
    npk = wl.nocc * wl.nemp
    ngs = []
    for i in picks:
        q, cut = wl.q[i], float(wl.ecut_eps[i])
        ctx = rp.Context(b.cell.lat, b.kmesh, wl.fft, b.ecut_psi, cut)
        ctx.load_bands(wl.nocc, b.npw, b.miller, b.coef[:, :nb], b.energy[:, :nb])
        G = OL.eps_sphere(b.cell.lat, q, cut)
        ngs.append(len(G))
        ref = OP.pair_density(b, wl.nocc, wl.nemp, q, G, fft=wl.fft, k_list=[7])
        got = ctx.rp_pair_density(q, 7, 8)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        wref = OC.pair_weights(replace(wl, freq=wl.freq[FI]), q, k_list=[7, 150])
        w = ctx.rp_tetra_weights(q, rp.RP_AXIS_IMAG, rp.RP_TIME_ORDERED, wl.freq[FI], wl.delta)
        cols = np.concatenate([np.arange(k * npk, (k + 1) * npk) for k in (7, 150)])
        assert np.abs(w[:, cols] - wref).max() <= 1e-11 * np.abs(wref).max()
        ctx.close()
    # sphere sizes drawn from 300..900 and placed at the nearest gap of |q+G|^2 (a few G either way)
    assert min(ngs) >= 280 and max(ngs) <= 950 and len(set(ngs)) > 3


def test_batched_build_and_dyson_against_single_q(batched, picks):
    wl = batched
    ctx = rp.context_for(wl)
    qs = wl.q[picks]
    cuts = wl.ecut_eps[picks]
    freq = wl.freq[FI]
    outs = ctx.rp_build_chi0_batched(qs, rp.RP_AXIS_IMAG, rp.RP_TIME_ORDERED, freq, wl.delta, rp.RP_BF16X3,
                                     ecut_eps=cuts)
    Ws = ctx.rp_solve_w_batched(qs, outs, ecut_eps=cuts)
    ref = ctx.rp_build_chi0_batched(qs, rp.RP_AXIS_IMAG, rp.RP_TIME_ORDERED, freq, wl.delta, rp.RP_FP64_NATIVE,
                                    ecut_eps=cuts)
    for i, (chi, (W, tail), r) in enumerate(zip(outs, Ws, ref)):
        assert np.all(_rel_fro(chi, r) < 1e-4)
        one = rp.Context(wl.bands.cell.lat, wl.bands.kmesh, wl.fft, wl.bands.ecut_psi, float(cuts[i]))
        one.load_bands(wl.nocc, wl.bands.npw, wl.bands.miller, wl.bands.coef[:, :wl.nocc + wl.nemp],
                       wl.bands.energy[:, :wl.nocc + wl.nemp])
        W1, t1 = one.rp_solve_w(qs[i], chi)
        assert np.all(_rel_fro(W, W1) < 1e-13) and np.array_equal(tail, t1)
        one.close()
    # device buffers: the packed list-kernel solve over all six q against the host-buffer results
    dev = [torch.from_numpy(c).cuda() for c in outs]
    dW = ctx.rp_solve_w_batched(qs, dev, ecut_eps=cuts)
    ctx.rp_check_numeric()
    for (W, _), d in zip(Ws, dW):
        assert np.all(_rel_fro(d.cpu().numpy(), W) < 1e-13)
