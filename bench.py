#!/usr/bin/env python
"""chi0 / W benchmark: one step = the whole hot path for one q of a synthetic workload
(pair densities, tetrahedron weights, chi0 contraction, Dyson solve), timed on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload precision] [--precision bf16x3|tf32x3|fp64]
                  [--shard replica|k]
  python bench.py --impl reference ...     # the FP64 CPU oracle on the same workload (bounded sample)
  python bench.py --kernel contraction ... # the dominant kernel alone, at the workload's launch shape

Prints one JSON line (rank 0).  Metric: chi0 build TFLOP/s with the algorithmic count
8 NG^2 K N_w per q (K = N_k N_occ N_emp band pairs).  Multi-GPU: `--shard replica` (default) runs
independent replicas (weak scaling, no collective on the data path); `--shard k` shares the k points
of the one q out over the ranks, sums chi0 with one all-reduce and splits the Dyson step over the
frequencies (strong scaling).  With --gpus N > 1 and no torchrun environment the script starts its
own N ranks.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "chi0 build TFLOP/s & %tensor-pipe peak, split-precision vs FP64, at stated error"
STAGES = ["gather_inverse", "pair_forward", "tetra_weights", "contraction", "dyson", "operands"]
CONTRACT_SRC = os.path.join(ROOT, "paper_2001_02351_gb300", "csrc", "rp_contract_tc.cu")

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the BF16x3
# contraction kernel at each workload's launch shape, from one ncu capture of
# `python bench.py --kernel contraction --workload <w>`, valid for the kernel source whose
# sha256 starts with the given prefix (null traffic otherwise).
TRAFFIC = {("precision", "bf16x3"): (44_598_248_192, "bd172516418fe28f")}


def measured_traffic(workload, precision):
    """(bytes per launch, note) if a capture of the current kernel source exists, else (None, why)."""
    key = (workload, precision)
    if key not in TRAFFIC:
        return None, "no ncu capture of this kernel at this workload's launch shape"
    nbytes, prefix = TRAFFIC[key]
    src = hashlib.sha256(open(CONTRACT_SRC, "rb").read()).hexdigest()
    if not src.startswith(prefix):
        return None, "kernel changed since the ncu capture"
    return nbytes, "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at the bench's launch shape"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def falg(ng, K, nf):
    return 8.0 * ng * ng * K * nf


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm = [float(r[0]) for r in self.rows if len(r) >= 2 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 2 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 4 + i and r[4 + i].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def spawn_ranks(n):
    """Run this script as n ranks on this node (torch.distributed.run on 127.0.0.1) and relay them."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def max_over_ranks(x, device=None):
    """The largest x over the ranks of the default process group (x itself on one rank)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(flops_per_rank, seconds, ws):
    """Whole-job TFLOP/s of ws replicas that each did flops_per_rank in `seconds` (the slowest)."""
    return ws * flops_per_rank / seconds / 1e12


def k_shards(nk, ws):
    """Contiguous k ranges [k0, k1) of the ranks, as even as the mesh allows."""
    return [(r * nk // ws, (r + 1) * nk // ws) for r in range(ws)]


def f_shards(nf, ws):
    """Contiguous frequency ranges of the ranks for the Dyson step (empty for ranks beyond nf)."""
    return [(r * nf // ws, (r + 1) * nf // ws) for r in range(ws)]


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def blas_threads():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return cpu_cores()


def subset_k(nk, n=4, seed=2001_02351):
    """Seeded k points of the sampled references (distinct, sorted)."""
    rng = np.random.default_rng(seed)
    return sorted(int(k) for k in rng.choice(nk, size=min(n, nk), replace=False))


def hermitian_eps(wl):
    """eps = 1 - v^1/2 chi0 v^1/2 is Hermitian positive definite for the time-ordered chi0 of the
    imaginary axis: the Dyson step may take the lower-triangle sweep."""
    return wl.axis == "imag" and wl.ordering == "time"


def sample_emp(wl, pairs=8192):
    """Empty bands of a bounded oracle sample: the lowest ones, about `pairs` pairs per k point on a
    48^3 grid (fewer on larger grids: the oracle's cost per pair grows with the grid)."""
    scaled = pairs * 48 ** 3 // int(np.prod(wl.fft))
    return int(min(wl.nemp, max(8, scaled // wl.nocc)))


def oracle_sample(wl, k_list, f_idx, nemp=None):
    """Oracle chi0 contribution of the pairs of k_list (the lowest nemp empty bands) at frequencies
    f_idx: (seconds, algorithmic flops)."""
    from dataclasses import replace

    from oracle import chi0 as OC, lattice as OL, pair_density as OP
    q = wl.q[0]
    nemp = wl.nemp if nemp is None else nemp
    wl2 = replace(wl, freq=wl.freq[f_idx], nemp=nemp)
    t0 = time.perf_counter()
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    M = OP.pair_density(wl.bands, wl.nocc, nemp, q, G, fft=wl.fft, k_list=k_list)
    w = OC.pair_weights(wl2, q, k_list=k_list)
    OC.chi0(M, w)
    dt = time.perf_counter() - t0
    return dt, falg(len(G), len(k_list) * wl.nocc * nemp, len(f_idx))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from synth import make_workload
    wl = make_workload(args.workload)
    nf = len(wl.freq)
    nk = wl.bands.kfrac.shape[0]
    f_idx = [0, nf - 1]
    ks = subset_k(nk, max(args.steps, 1))
    ne = sample_emp(wl)
    times, flops = [], 0.0
    for s in range(args.steps):
        dt, fl = oracle_sample(wl, [ks[s % len(ks)]], f_idx, ne)
        times.append(dt)
        flops = fl
    t = float(np.mean(times))
    val = flops / t / 1e12
    sample = (f"one k point per step (k = {ks[:args.steps]} of {nk}) with the lowest {ne} of {wl.nemp} empty "
              f"bands, frequencies {f_idx} of {nf}: oracle pair densities, tetrahedron weights and chi0 partial sum")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "sample": sample},
           "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": blas_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def contraction_launch_shape(nk, nocc, nemp):
    """Pairs per contraction launch of rp_build_chi0: whole k points, about 64k pair columns."""
    kcols = nocc * nemp
    kb = max(1, min(nk, 65536 // kcols))
    return kb * kcols


def run_kernel(args):
    """The BF16x3 contraction alone, at the launch shape rp_build_chi0 uses for the workload
    (NG of its q, pairs per launch, all its frequencies), on seeded random operands: the command
    the kernel's ncu captures run."""
    import torch

    import paper_2001_02351_gb300 as rp
    from synth.configs import workload_shape
    sh = workload_shape(args.workload)
    spec, cell = sh["spec"], sh["cell"]
    torch.cuda.set_device(0)
    ctx = rp.Context(cell.lat, spec["kmesh"], spec["fft"], sh["ecut_psi"], float(sh["ecut_eps"][0]))
    g, _ = ctx.rp_sphere_size(sh["q"][0])
    ng, nf = len(g), len(spec["freq"])
    nk = int(np.prod(spec["kmesh"]))
    K = contraction_launch_shape(nk, spec["nocc"], spec["nemp"])
    gen = torch.Generator(device="cuda").manual_seed(7)
    M = torch.randn((ng, K), dtype=torch.complex128, device="cuda", generator=gen)
    w = torch.randn((nf, K), dtype=torch.complex128, device="cuda", generator=gen) * 1e-3
    chi = torch.empty((nf, ng, ng), dtype=torch.complex128, device="cuda")
    prec = {"fp64": rp.RP_FP64_NATIVE, "bf16x3": rp.RP_BF16X3, "tf32x3": rp.RP_TF32X3}[args.precision]
    ctx.rp_profile_enable(True)
    for _ in range(args.warmup + args.steps):
        ctx.rp_contract_chi0(M, w, precision=prec, out=chi)
    torch.cuda.synchronize()
    ms, nl = ctx.rp_profile_read()
    ctx.rp_check_numeric()
    per = ms[3] / max(1, nl[3])
    print(json.dumps({"kernel": "contraction", "workload": args.workload, "ng": ng, "pairs_per_launch": K, "nfreq": nf,
                      "launches": int(nl[3]), "ms_per_launch": per,
                      "tflops": falg(ng, K, nf) / (per * 1e-3) / 1e12}), flush=True)
    return 0


def run_interaction(args):
    """The interaction step (screened direct and exchange integrals of Wannier functions) for the q
    points of a workload's mesh, timed per q on the device with a seeded W = v^1/2 (1 + X) v^1/2 per
    q: the Wannier pair densities on the wave-function sphere, the density rows, one pass over W and
    the bilinear forms."""
    import torch
    import paper_2001_02351_gb300 as rp
    from synth import make_workload
    from synth.wannier import gaussian_wannier
    wl = make_workload(args.workload)
    torch.cuda.set_device(0)
    b = wl.bands
    nw = 3
    coef_w = gaussian_wannier(b, wl.nocc, np.array([(0.1, 0.2, 0.0), (0.5, 0.4, 0.3), (0.7, 0.1, 0.6)]), 1.6)
    ctx = rp.context_for(wl)
    ctx.rp_load_wannier(coef_w)
    R = np.array([(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 1)])
    nf = len(wl.freq)
    rng = np.random.default_rng(5)
    qs = b.kfrac[rng.choice(len(b.kfrac), size=min(8, len(b.kfrac)), replace=False)]
    Ws = []
    for q in qs:
        g, _ = ctx.rp_sphere_size(q)
        vs = np.sqrt(4 * np.pi / b.cell.omega) / np.linalg.norm((g + q) @ b.cell.recip, axis=1)
        X = 0.05 * (rng.standard_normal((len(g), len(g))) + 1j * rng.standard_normal((len(g), len(g))))
        W1 = (np.eye(len(g)) + X + X.conj().T) * vs[:, None] * vs[None, :]
        Ws.append(torch.from_numpy(np.repeat(W1[None], nf, axis=0)).cuda())
    U = J = None
    for i, q in enumerate(qs):                    # warm-up pass
        U, J = ctx.rp_interaction(q, R, W=Ws[i], U=U, J=J, accumulate=i > 0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i, q in enumerate(qs):
        U, J = ctx.rp_interaction(q, R, W=Ws[i], U=U, J=J, accumulate=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / len(qs)
    ng = [W.shape[1] for W in Ws]
    nb = nw + len(R) * nw * nw
    wbytes = np.mean([nf * n * n * 16 for n in ng])
    flop = np.mean([8.0 * nf * n * n * nb for n in ng])
    print(json.dumps({"kernel": "interaction", "workload": args.workload, "nq_timed": len(qs), "nw": nw, "nR": len(R),
                      "nfreq": nf, "ng_mean": float(np.mean(ng)), "ms_per_q": ms,
                      "W_read_GBps": wbytes / (ms * 1e-3) / 1e9, "W_rows_fp64_TFLOPs": flop / (ms * 1e-3) / 1e12,
                      "note": "per q: Wannier pair densities on the wave-function sphere, density rows, one pass over "
                              "W against nw + nR nw^2 rows, bilinear forms"}), flush=True)
    return 0


def run_batched(args):
    """Every q of the batched workload's mesh (uneven epsilon spheres) in one batched build and one
    batched Dyson call per step; the metric's count summed over the q points."""
    import torch
    import paper_2001_02351_gb300 as rp
    from synth import make_workload
    wl = make_workload(args.workload)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    prec = {"fp64": rp.RP_FP64_NATIVE, "bf16x3": rp.RP_BF16X3, "tf32x3": rp.RP_TF32X3}[args.precision]
    axis = rp.RP_AXIS_IMAG if wl.axis == "imag" else rp.RP_AXIS_REAL
    ctx = rp.context_for(wl)
    ctx.rp_set_dyson_hermitian(hermitian_eps(wl))
    qs, cuts = wl.q, wl.ecut_eps
    nf = len(wl.freq)
    nk = wl.bands.kfrac.shape[0]
    K = nk * wl.nocc * wl.nemp
    ngs = [len(ctx.rp_sphere_size(q, c)[0]) for q, c in zip(qs, cuts)]
    chis = [torch.empty((nf, n, n), dtype=torch.complex128, device=dev) for n in ngs]
    Ws = [torch.empty_like(c) for c in chis]
    F = sum(falg(n, K, nf) for n in ngs)

    def step():
        ctx.rp_build_chi0_batched(qs, axis, rp.RP_TIME_ORDERED, wl.freq, wl.delta, prec, ecut_eps=cuts, outs=chis)
        ctx.rp_solve_w_batched(qs, chis, ecut_eps=cuts, outs=Ws)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.rp_check_numeric()
    clocks = ClockSampler(0)
    ctx.rp_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks.start()
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    stage_ms, launches = ctx.rp_profile_read()
    ctx.rp_check_numeric()
    ms_step = e0.elapsed_time(e1) / args.steps
    pk = peaks()
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    t_con = stage_ms[3] / args.steps * 1e-3
    achieved = F / t_con / 1e12 if t_con > 0 else None
    res = {"metric": METRIC, "value": F / (ms_step * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"fp64": "f64", "bf16x3": "bf16x3", "tf32x3": "tf32x3"}[args.precision],
           "data": "synthetic (seeded empirical-pseudopotential bands)",
           "config": {"workload": args.workload, "nq": len(qs), "ng_min": min(ngs), "ng_max": max(ngs),
                      "pairs_K": K, "nfreq": nf, "nk": nk, "nocc": wl.nocc, "nemp": wl.nemp, "axis": wl.axis,
                      "precision": args.precision, "l2": "inputs larger than L2", "parallelism": "replicas x1",
                      "dyson": "hermitian sweep" if hermitian_eps(wl) else "pivoted Gauss-Jordan"},
           "stages_ms_per_step": {n: stage_ms[i] / args.steps for i, n in enumerate(STAGES)},
           "gpu_launches": int(launches.sum()),
           "roofline": {"bound": "tensor", "kernel": "chi0 contraction", "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak if achieved else None, "traffic": None,
                        "peak_source": "of measured: bf16 sustained",
                        "frac_of_formulation_ceiling": 3.0 * achieved / peak
                        if achieved and args.precision == "bf16x3" else None},
           "clocks": clk, "e2e": None, "cpu_baseline": None}
    print(json.dumps(res), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision")
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "bf16x3", "tf32x3"])
    ap.add_argument("--shard", default="replica", choices=["replica", "k"])
    ap.add_argument("--kernel", default=None, choices=[None, "contraction", "interaction"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return spawn_ranks(args.gpus)
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel == "contraction":
        return run_kernel(args)
    if args.kernel == "interaction":
        return run_interaction(args)
    if args.workload == "batched":
        return run_batched(args)

    import torch
    import paper_2001_02351_gb300 as rp
    from synth import make_workload

    ws, rank, local = dist_env()
    wl = make_workload(args.workload)      # before CUDA start-up: the band generator may fork
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    q = wl.q[0]
    prec = {"fp64": rp.RP_FP64_NATIVE, "bf16x3": rp.RP_BF16X3, "tf32x3": rp.RP_TF32X3}[args.precision]
    axis = rp.RP_AXIS_IMAG if wl.axis == "imag" else rp.RP_AXIS_REAL
    ordering = rp.RP_TIME_ORDERED if wl.ordering == "time" else rp.RP_RETARDED
    ctx = rp.context_for(wl)
    ctx.rp_set_dyson_hermitian(hermitian_eps(wl))
    G, tl = ctx.rp_sphere_size(q)
    ng, nf = len(G), len(wl.freq)
    nk = wl.bands.kfrac.shape[0]
    npk = wl.nocc * wl.nemp
    K = nk * npk
    F = falg(ng, K, nf)
    chi = torch.empty((nf, ng, ng), dtype=torch.complex128, device=dev)
    W = torch.empty_like(chi)
    tail = torch.zeros(max(1, len(tl)), dtype=torch.float64, device=dev)
    # tile width of the BF16x3 contraction for this NG and launch shape: the autotuner's choice,
    # cached per device and shape
    tile = None
    if prec == rp.RP_BF16X3:
        cache_dir = os.environ.get("RP_CACHE_DIR", os.path.join(os.path.expanduser("~"), ".cache", "respack_gb300"))
        tile, tile_ms = ctx.tuned_tile(ng, contraction_launch_shape(nk, wl.nocc, wl.nemp), nf,
                                       os.path.join(cache_dir, "contraction_tiles.json"))
    shard_k = args.shard == "k" and ws > 1
    k0, k1 = k_shards(nk, ws)[rank] if shard_k else (0, nk)
    f0, f1 = f_shards(nf, ws)[rank] if shard_k else (0, nf)
    my_k = list(range(k0, k1))

    def build(c, out):
        if shard_k:
            # this rank's k points, then the sum over ranks (the one exchange of the sharded path)
            c.rp_build_chi0_kset(q, my_k, axis, ordering, wl.freq, wl.delta, prec, wl.delta_a, wl.delta_r, out=out)
            import torch.distributed as dist
            dist.all_reduce(torch.view_as_real(out))
        else:
            c.rp_build_chi0(q, axis, ordering, wl.freq, wl.delta, prec, wl.delta_a, wl.delta_r, out=out)

    def step():
        build(ctx, chi)
        if f1 > f0:
            ctx.rp_solve_w(q, chi[f0:f1], out=W[f0:f1], tail=tail)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.rp_check_numeric()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(torch.cuda.current_device())
    ctx.rp_profile_enable(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms_total = e0.elapsed_time(e1)
    stage_ms, launches = ctx.rp_profile_read()
    ctx.rp_profile_enable(False)
    ctx.rp_check_numeric()
    ms_total = max_over_ranks(ms_total, dev)
    ms_step = ms_total / args.steps
    # replicas: every rank did the whole q; k shards: the ranks did one q together
    value = F / (ms_step * 1e-3) / 1e12 if shard_k else job_rate(F, ms_step * 1e-3, ws)

    # dominant kernel: the chi0 contraction (tensor pipe), timed inside a long step -> sustained peak
    pk = peaks()
    t_con = stage_ms[3] / args.steps * 1e-3
    F_rank = falg(ng, (k1 - k0) * npk, nf)
    if prec == rp.RP_FP64_NATIVE:
        peak = pk.get("bf16_tflops_sustained", 1700.0) * 1.25 / 2250.0
        peak_note = "of measured: bf16 sustained x nominal fp64/bf16 ratio 1.25/2250"
    elif prec == rp.RP_TF32X3:
        peak = pk.get("bf16_tflops_sustained", 1700.0) * 1.1 / 2.25
        peak_note = "of measured: bf16 sustained x nominal tf32/bf16 ratio 1.1/2.25"
    else:
        peak = pk.get("bf16_tflops_sustained", 1700.0)
        peak_note = "of measured: bf16 sustained (MEASURED_PEAKS.json)"
    # algorithmic flops of this rank's share of a step / summed device time of its contraction launches
    achieved = F_rank / t_con / 1e12 if t_con > 0 else None
    traffic, traffic_note = measured_traffic(args.workload, args.precision)
    nlaunch = int(launches[3]) // args.steps
    roof = {"bound": "tensor", "kernel": "k_contract_bf16x3" if prec == rp.RP_BF16X3 else "chi0 contraction",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic, "traffic_note": traffic_note, "launches_per_step": nlaunch,
            "ms_per_launch": float(stage_ms[3]) / max(1, int(launches[3])), "tile_bn": tile,
            "algorithmic_flop_per_launch": F_rank / max(1, nlaunch), "peak_source": peak_note}
    if prec == rp.RP_BF16X3 and achieved:
        # three bf16 products per real product, four real products per complex one: 12 bf16 MACs per
        # complex MAC of 8 algorithmic flops, so a third of the bf16 rate is this formulation's ceiling
        roof["formulation_ceiling"] = peak / 3.0
        roof["frac_of_formulation_ceiling"] = achieved / (peak / 3.0)
    # the sustained peak was measured at its own median SM clock: the fraction at this run's clock too
    peak_mhz = (pk.get("clocks_under_load") or {}).get("sm_mhz_median")
    if achieved and peak_mhz and clk.get("sm_mhz"):
        roof["frac_at_run_clock"] = achieved / (peak * clk["sm_mhz"] / peak_mhz)
        roof["clock_note"] = (f"peak scaled from its measured median {peak_mhz:.0f} MHz to this run's median "
                              f"{clk['sm_mhz']:.0f} MHz")

    res = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "strong" if shard_k else "weak",
           "vs_baseline": None, "dtype": {"fp64": "f64", "bf16x3": "bf16x3", "tf32x3": "tf32x3"}[args.precision],
           "data": "synthetic (seeded empirical-pseudopotential bands)",
           "config": {"workload": args.workload, "ng": ng, "pairs_K": K, "nfreq": nf, "nk": nk,
                      "nocc": wl.nocc, "nemp": wl.nemp, "npw_max": int(wl.bands.npw.max()), "fft": list(wl.fft),
                      "axis": wl.axis, "precision": args.precision,
                      "l2": "inputs larger than L2 (bands and per-step scratch > 129 MB)",
                      "dyson": "hermitian sweep" if hermitian_eps(wl) else "pivoted Gauss-Jordan",
                      "parallelism": f"k shards x{ws}" if shard_k else f"replicas x{ws}"},
           "stages_ms_per_step": {n: stage_ms[i] / args.steps for i, n in enumerate(STAGES)},
           "gpu_launches": int(launches.sum()), "roofline": roof, "clocks": clk}

    # the native-FP64 reference needs the FP64 plane kernels (residue masks of at most 32 points per
    # axis); on larger grids its pair stage takes the generic line passes, far too slow at these sizes
    fp64_ref = ctx.rp_transform_grid(q)[0][0] <= 32
    if prec != rp.RP_FP64_NATIVE and not args.no_fp64 and rank == 0 and not fp64_ref:
        res["fp64_reference"] = {"skipped": "transform grid above 32 points: the FP64 pair stage has no plane "
                                            "kernel there (the split tier is checked against the oracle in "
                                            "tests/test_gpu_large.py)"}
    if prec != rp.RP_FP64_NATIVE and not args.no_fp64 and rank == 0 and fp64_ref:
        # native FP64 and the timed tier on the same inputs: the sum over four seeded k points
        # (full-mesh weights) at three frequencies; W errors from the Dyson step applied to each
        # subset chi0 scaled by N_k / 4 (the subset's estimate of the whole sum, of the right size
        # and conditioning)
        ks = subset_k(nk)
        fi = [0, nf // 2, nf - 1]
        f3 = wl.freq[fi]
        sub = {}
        for p in (rp.RP_FP64_NATIVE, prec):
            c3 = torch.empty((len(fi), ng, ng), dtype=torch.complex128, device=dev)
            ctx.rp_profile_enable(True)
            ctx.rp_build_chi0_kset(q, ks, axis, ordering, f3, wl.delta, p, wl.delta_a, wl.delta_r, out=c3)
            torch.cuda.synchronize()
            ms_p, _ = ctx.rp_profile_read()
            ctx.rp_profile_enable(False)
            Wp, _ = ctx.rp_solve_w(q, c3 * (nk / len(ks)))
            torch.cuda.synchronize()
            sub[p] = (c3, Wp, ms_p)
        ctx.rp_check_numeric()

        def rel(a, b):
            return [float(torch.linalg.norm(a[i] - b[i]) / torch.linalg.norm(b[i])) for i in range(a.shape[0])]
        c64, W64, ms64 = sub[rp.RP_FP64_NATIVE]
        cs, Ws, _ = sub[prec]
        Fs = falg(ng, len(ks) * npk, len(fi))
        res["fp64_reference"] = {
            "k_points": ks, "freq_index": fi, "contraction_tflops": Fs / (ms64[3] * 1e-3) / 1e12,
            "contraction_ms": float(ms64[3]), "chi0_rel_err": rel(cs, c64), "W_rel_err": rel(Ws, W64),
            "note": "native FP64 GPU path on a k subset (its pieces are checked against the FP64 oracle in "
                    "the test-suite); W from the subset chi0 scaled by N_k/4"}

    if not args.no_e2e:
        # end to end through the C ABI with host buffers: bands H2D (pinned), chi0 / W back to the host
        b = wl.bands
        nb = wl.nocc + wl.nemp
        coef = torch.from_numpy(np.ascontiguousarray(b.coef[:, :nb])).pin_memory()
        energy = torch.from_numpy(np.ascontiguousarray(b.energy[:, :nb])).pin_memory()
        miller = torch.from_numpy(np.ascontiguousarray(b.miller)).pin_memory()
        npw = torch.from_numpy(np.ascontiguousarray(b.npw)).pin_memory()
        chi_h = torch.empty((nf, ng, ng), dtype=torch.complex128).pin_memory()
        W_h = torch.empty_like(chi_h).pin_memory()
        tail_h = np.zeros(max(1, len(tl)))
        # bands in; chi0 out of the build, back in for the Dyson step (a host-buffer call); W and tail out
        h2d = coef.numel() * 16 + energy.numel() * 8 + miller.numel() * 4 + npw.numel() * 4 + chi_h.numel() * 16
        d2h = chi_h.numel() * 16 + W_h.numel() * 16 + tail_h.size * 8
        ectx = rp.Context(b.cell.lat, b.kmesh, wl.fft, b.ecut_psi, float(wl.ecut_eps[0]))
        if tile:
            ectx.rp_set_contraction_tile(ng, tile)
        ectx.rp_set_dyson_hermitian(hermitian_eps(wl))
        del ctx                                            # one band set on the device at a time

        def e2e_step():
            ectx.rp_load_bands(wl.nocc, npw.numpy(), miller.numpy(), coef.numpy(), energy.numpy())
            if shard_k:
                chi_d = torch.empty((nf, ng, ng), dtype=torch.complex128, device=dev)
                build(ectx, chi_d)
                chi_h.copy_(chi_d)
            else:
                ectx.rp_build_chi0(q, axis, ordering, wl.freq, wl.delta, prec, wl.delta_a, wl.delta_r,
                                   out=chi_h.numpy())
            if f1 > f0:
                ectx.rp_solve_w(q, chi_h.numpy()[f0:f1], out=W_h.numpy()[f0:f1], tail=tail_h)
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        te = max_over_ranks((time.perf_counter() - t0) / args.steps, dev)
        e2e_val = F / te / 1e12 if shard_k else job_rate(F, te, ws)
        res["e2e"] = {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "ms_per_step": te * 1e3}
        ectx.close()

    if rank == 0 and not args.no_cpu:
        k_list, f_idx, ne = subset_k(nk, 1), [0, nf - 1], sample_emp(wl)
        dt, fl = oracle_sample(wl, k_list, f_idx, ne)
        res["cpu_baseline"] = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": blas_threads(), "kind": "oracle",
                               "sample": f"k-point {k_list} of {nk} with the lowest {ne} of {wl.nemp} empty bands, "
                                         f"frequencies {f_idx} of {nf}: oracle pair densities, tetrahedron weights "
                                         f"and chi0 partial sum ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
