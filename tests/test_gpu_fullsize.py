"""GPU path at the full medium size (NG = 402, 512 k, 40 + 160 bands, 20 real frequencies), in the
launch configuration the benchmark times, against the FP64 oracle on the outputs it can compute
in seconds, and through properties that hold at any size.

- pair densities of one k point (6400 pairs x 402 sphere points), element by element;
- tetrahedron weights of two sampled k points at three of the 20 frequencies (FP64 tier and the
  FP32 pass of the split tiers; the GPU computes all pairs and frequencies, as in the benchmark);
- the contraction at full NG on the oracle's own M and w of one k point (FP64, TF32x3, BF16x3);
- virtual shards: the sum of the FP64 contractions of two k halves equals the fused FP64 build
  (the linearity the k-block streaming and any k sharding over GPUs rely on);
- the BF16x3 build against the FP64 build on the same inputs (the benchmark's error figure).
"""
import numpy as np
import pytest

from conftest import workload

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402
from oracle import chi0 as OC, lattice as OL, pair_density as OP  # noqa: E402

# FP32 weight pass: |w32 - w64| <= 1e-4 max|w| per frequency (the split tiers' stated bound);
# BF16x3 contraction: relative Frobenius error 1e-4 per frequency
FP32_WEIGHT_TOL = 1e-4
BF16X3_TOL = 1e-4


@pytest.fixture(scope="module")
def medium():
    return workload("medium")


@pytest.fixture(scope="module")
def mctx(medium):
    return rp.context_for(medium)


FI = [0, 7, 19]          # sampled frequencies (lowest, middle, highest)
KS = [0, 300]            # sampled k points


@pytest.fixture(scope="module")
def oracle_sample(medium):
    """The oracle's M of k = 0 and weights of KS at the FI frequencies (computed once)."""
    from dataclasses import replace
    q = medium.q[0]
    G = OL.eps_sphere(medium.cell.lat, q, medium.ecut_eps[0])
    M0 = OP.pair_density(medium.bands, medium.nocc, medium.nemp, q, G, fft=medium.fft, k_list=[0])
    w = OC.pair_weights(replace(medium, freq=medium.freq[FI]), q, k_list=KS)
    return G, M0, w


def _rel_fro(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_pair_density_full_size_one_k(medium, mctx, oracle_sample):
    q = medium.q[0]
    G, ref, _ = oracle_sample
    got = mctx.rp_pair_density(q, 0, 1)
    assert got.shape == ref.shape == (len(G), medium.nocc * medium.nemp)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision,tol", [(rp.RP_FP64_NATIVE, 1e-11), (rp.RP_BF16X3, FP32_WEIGHT_TOL)])
def test_weights_full_size_sampled(medium, mctx, oracle_sample, precision, tol):
    q = medium.q[0]
    ks = KS
    ref = oracle_sample[2]
    npk = medium.nocc * medium.nemp
    w = torch.empty((len(medium.freq), medium.bands.kfrac.shape[0] * npk), dtype=torch.complex128, device="cuda")
    mctx.rp_tetra_weights(q, rp.RP_AXIS_REAL, rp.RP_TIME_ORDERED, medium.freq, medium.delta, medium.delta_a,
                          medium.delta_r, out=w, precision=precision)
    cols = np.concatenate([np.arange(k * npk, (k + 1) * npk) for k in ks])
    got = w[:, torch.from_numpy(cols).cuda()].cpu().numpy()[FI]
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - ref) <= tol * scale)


@pytest.mark.parametrize("precision,tol", [(rp.RP_FP64_NATIVE, 1e-12), (rp.RP_BF16X3, BF16X3_TOL),
                                           (rp.RP_TF32X3, 2e-6)])
def test_contraction_full_ng_on_oracle_inputs(medium, mctx, oracle_sample, precision, tol):
    _, M, w2 = oracle_sample
    w = np.ascontiguousarray(w2[:, :M.shape[1]])            # the k = 0 columns
    ref = OC.chi0(M, w)
    got = mctx.rp_contract_chi0(M, w, precision=precision)
    assert np.all(_rel_fro(got, ref) < tol)


def test_virtual_shards_sum_to_fused_build(medium, mctx):
    q = medium.q[0]
    fi = [0, 19]
    freq = medium.freq[fi]
    g, _ = mctx.rp_sphere_size(q)
    ng = len(g)
    nk = medium.bands.kfrac.shape[0]
    npk = medium.nocc * medium.nemp
    w = torch.empty((len(freq), nk * npk), dtype=torch.complex128, device="cuda")
    mctx.rp_tetra_weights(q, rp.RP_AXIS_REAL, rp.RP_TIME_ORDERED, freq, medium.delta, medium.delta_a,
                          medium.delta_r, out=w)
    chi_sum = torch.zeros((len(freq), ng, ng), dtype=torch.complex128, device="cuda")
    for k0, k1 in ((0, nk // 2), (nk // 2, nk)):
        M = torch.empty((ng, (k1 - k0) * npk), dtype=torch.complex128, device="cuda")
        mctx.rp_pair_density(q, k0, k1, out=M)
        ws = w[:, k0 * npk:k1 * npk].contiguous()
        chi_sum += mctx.rp_contract_chi0(M, ws)
        del M, ws
    fused = torch.empty_like(chi_sum)
    mctx.rp_build_chi0(q, rp.RP_AXIS_REAL, rp.RP_TIME_ORDERED, freq, medium.delta, rp.RP_FP64_NATIVE,
                       medium.delta_a, medium.delta_r, out=fused)
    torch.cuda.synchronize()
    assert np.all(_rel_fro(chi_sum.cpu().numpy(), fused.cpu().numpy()) < 1e-12)
    # the split tier on the same inputs, against the FP64 build
    split = torch.empty_like(chi_sum)
    mctx.rp_build_chi0(q, rp.RP_AXIS_REAL, rp.RP_TIME_ORDERED, freq, medium.delta, rp.RP_BF16X3,
                       medium.delta_a, medium.delta_r, out=split)
    torch.cuda.synchronize()
    e = _rel_fro(split.cpu().numpy(), fused.cpu().numpy())
    print("medium BF16x3 vs FP64 chi0 rel err", e)
    assert np.all(e < BF16X3_TOL)
