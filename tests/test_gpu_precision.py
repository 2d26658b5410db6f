"""GPU path at the full size of the precision workload (10^3 k mesh, 64 + 448 bands, about 4000
plane waves, NG about 1500, 30 real frequencies), in the launch configuration the benchmark times,
against the FP64 oracle on the outputs it computes in seconds to minutes:

- pair densities of one k point (28672 pairs x NG), element by element (FP64 tier);
- tetrahedron weights of two sampled k points at three of the 30 frequencies (FP64 tier and the
  FP32 pass of the split tiers; the GPU computes all pairs and frequencies, as in the benchmark);
- the contraction at full NG on the oracle's own M and w of one k point (FP64, BF16x3, TF32x3);
- the BF16x3 build against the FP64 build on a k subset (the benchmark's error figure), through
  rp_build_chi0_kset.
"""
import numpy as np
import pytest

from conftest import workload

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402
from oracle import chi0 as OC, lattice as OL, pair_density as OP  # noqa: E402

FP32_WEIGHT_TOL = 1e-4      # |w32 - w64| <= 1e-4 max|w| per frequency (split tiers' weight pass)
BF16X3_TOL = 1e-4           # relative Frobenius error per frequency
TF32X3_TOL = 2e-6
FI = [0, 14, 29]            # sampled frequencies (lowest, middle, highest)
KS = [0, 537]               # sampled k points


@pytest.fixture(scope="module")
def prec():
    return workload("precision")


@pytest.fixture(scope="module")
def pctx(prec):
    return rp.context_for(prec)


@pytest.fixture(scope="module")
def oracle_sample(prec):
    from dataclasses import replace
    q = prec.q[0]
    G = OL.eps_sphere(prec.cell.lat, q, prec.ecut_eps[0])
    M0 = OP.pair_density(prec.bands, prec.nocc, prec.nemp, q, G, fft=prec.fft, k_list=[0])
    w = OC.pair_weights(replace(prec, freq=prec.freq[FI]), q, k_list=KS)
    w0 = np.ascontiguousarray(w[:, :M0.shape[1]])            # the k = 0 columns
    return G, M0, w, OC.chi0(M0, w0)


def _rel_fro(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_workload_shape(prec, pctx):
    q = prec.q[0]
    g, _ = pctx.rp_sphere_size(q)
    assert prec.bands.kfrac.shape[0] == 1000 and prec.nocc == 64 and prec.nemp == 448
    assert 1400 <= len(g) <= 1600
    assert 3800 <= int(prec.bands.npw.min()) and int(prec.bands.npw.max()) <= 4300


def test_pair_density_full_size_one_k(prec, pctx, oracle_sample):
    q = prec.q[0]
    G, ref, _, _ = oracle_sample
    got = pctx.rp_pair_density(q, 0, 1)
    assert got.shape == ref.shape == (len(G), prec.nocc * prec.nemp)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision,tol", [(rp.RP_FP64_NATIVE, 1e-11), (rp.RP_BF16X3, FP32_WEIGHT_TOL)])
def test_weights_full_size_sampled(prec, pctx, oracle_sample, precision, tol):
    q = prec.q[0]
    ref = oracle_sample[2]
    npk = prec.nocc * prec.nemp
    w = torch.empty((len(prec.freq), prec.bands.kfrac.shape[0] * npk), dtype=torch.complex128, device="cuda")
    pctx.rp_tetra_weights(q, rp.RP_AXIS_REAL, rp.RP_TIME_ORDERED, prec.freq, prec.delta, prec.delta_a,
                          prec.delta_r, out=w, precision=precision)
    cols = torch.from_numpy(np.concatenate([np.arange(k * npk, (k + 1) * npk) for k in KS])).cuda()
    got = w[:, cols].cpu().numpy()[FI]
    del w
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - ref) <= tol * scale)


@pytest.mark.parametrize("precision,tol", [(rp.RP_FP64_NATIVE, 1e-12), (rp.RP_BF16X3, BF16X3_TOL),
                                           (rp.RP_TF32X3, TF32X3_TOL)])
def test_contraction_full_ng_on_oracle_inputs(pctx, oracle_sample, precision, tol):
    _, M, w2, ref = oracle_sample
    w = np.ascontiguousarray(w2[:, :M.shape[1]])            # the k = 0 columns
    got = pctx.rp_contract_chi0(M, w, precision=precision)
    err = _rel_fro(got, ref)
    print("precision-size contraction rel err", precision, err)
    assert np.all(err < tol)


def test_split_build_against_fp64_on_a_k_subset(prec, pctx):
    """The benchmark's error figure: the BF16x3 build and the FP64 build summed over the same four
    k points (full-mesh weights) at three frequencies; the FP64 subset build is itself the sum of
    the oracle-checked pieces above."""
    q = prec.q[0]
    ks = [0, 137, 537, 911]
    freq = prec.freq[FI]
    g, _ = pctx.rp_sphere_size(q)
    out = {}
    for p in (rp.RP_FP64_NATIVE, rp.RP_BF16X3):
        chi = torch.empty((len(freq), len(g), len(g)), dtype=torch.complex128, device="cuda")
        pctx.rp_build_chi0_kset(q, ks, rp.RP_AXIS_REAL, rp.RP_TIME_ORDERED, freq, prec.delta, p, prec.delta_a,
                                prec.delta_r, out=chi)
        out[p] = chi.cpu().numpy()
    pctx.rp_check_numeric()
    e = _rel_fro(out[rp.RP_BF16X3], out[rp.RP_FP64_NATIVE])
    print("precision k-subset BF16x3 vs FP64 chi0 rel err", e)
    assert np.all(e < BF16X3_TOL)
