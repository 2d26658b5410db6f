"""rp_contract_chi0_static: the BF16x3 contraction for callers that cannot allocate device memory
(its scratch is a fixed array inside the library).  Called twice in a row through the C ABI, its
output must match the allocating entry point rp_contract_chi0 within the split-precision
tolerance of the other tests; an over-size request is refused before anything runs.

This file sorts last so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest

from conftest import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402

BF16X3_TOL = 1e-4


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_static_scratch_contraction_matches_allocating_path():
    lib = rp.library()
    torch.cuda.set_device(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(3)
    ctx = rp.context_for(workload("micro"))
    for ng, K, nf in [(150, 5000, 2), (77, 1000, 3)]:
        M = torch.randn(ng, K, dtype=torch.complex128, device="cuda", generator=g)
        w = torch.randn(nf, K, dtype=torch.complex128, device="cuda", generator=g)
        ref = ctx.rp_contract_chi0(M, w, precision=rp.RP_BF16X3)
        outs = []
        for _ in range(2):                       # the shared array keeps the last call's contents
            out = torch.full((nf, ng, ng), float("nan"), dtype=torch.complex128, device="cuda")
            code = lib.rp_contract_chi0_static(ng, K, nf, ctypes.c_void_p(M.data_ptr()),
                                               ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                               stream)
            assert code == rp.RP_OK
            outs.append(out)
        # no device wait gave up in the last call (the status call allocates nothing either)
        assert lib.rp_contract_chi0_static_status(stream) == rp.RP_OK
        torch.cuda.synchronize()
        for out in outs:
            assert torch.isfinite(out).all()
            assert _rel(out, ref) < BF16X3_TOL
        # the FP64 flushes are atomic additions, so the summation order may differ between calls
        assert _rel(outs[0], outs[1]) < 1e-12


def test_static_scratch_rejects_oversize():
    lib = rp.library()
    M = torch.zeros(1, dtype=torch.complex128, device="cuda")
    # ng * kp2 beyond the 24 MiB bf16 half of the array
    code = lib.rp_contract_chi0_static(4096, 4096, 1, ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(M.data_ptr()),
                                       ctypes.c_void_p(M.data_ptr()), None)
    assert code == rp.RP_ERR_ARG
