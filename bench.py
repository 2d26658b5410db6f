#!/usr/bin/env python
"""chi0 / W benchmark: one step = the whole hot path for one q of a synthetic workload
(pair densities, tetrahedron weights, chi0 contraction, Dyson solve), timed on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload medium] [--precision fp64|bf16x3]
  python bench.py --impl reference ...     # the FP64 CPU oracle on the same workload (bounded sample)

Prints one JSON line (rank 0).  Metric: chi0 build TFLOP/s with the algorithmic count
8 NG^2 K N_w per q (K = N_k N_occ N_emp band pairs).  Multi-GPU runs are replicas (each rank
repeats the step on its own GPU): weak scaling, no collective on the data path.
"""
import argparse
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
# DRAM traffic of one contraction launch (ncu), valid only for the source it was measured on
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "contraction_medium_bf16x3.md")
CONTRACT_SRC = os.path.join(ROOT, "paper_2001_02351_gb300", "csrc", "rp_contract_tc.cu")


def measured_traffic(workload, precision):
    """(bytes per launch, note) from the committed ncu summary if it matches this run, else (None, why)."""
    import hashlib
    import re
    if workload != "medium" or precision != "bf16x3":
        return None, "no ncu capture for this workload"
    try:
        text = open(TRAFFIC_PROFILE).read()
        src = hashlib.sha256(open(CONTRACT_SRC, "rb").read()).hexdigest()
    except OSError:
        return None, "ncu summary missing"
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h:
        return None, "ncu summary without traffic"
    if not src.startswith(h.group(1)):
        return None, "kernel changed since the ncu capture"
    return int(m.group(1)), "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch of K = 64000 pairs"


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


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(wl, k_list, f_idx):
    """Oracle chi0 contribution of the pairs of k_list at frequencies f_idx: (seconds, algorithmic flops)."""
    from dataclasses import replace

    from oracle import chi0 as OC, lattice as OL, pair_density as OP
    q = wl.q[0]
    wl2 = replace(wl, freq=wl.freq[f_idx])
    t0 = time.perf_counter()
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    M = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft, k_list=k_list)
    w = OC.pair_weights(wl2, q, k_list=k_list)
    OC.chi0(M, w)
    dt = time.perf_counter() - t0
    return dt, falg(len(G), len(k_list) * wl.nocc * wl.nemp, len(f_idx))


def blas_threads():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return cpu_cores()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from synth import make_workload
    wl = make_workload(args.workload)
    nf = len(wl.freq)
    k_list, f_idx = [0], [0, nf - 1]
    for _ in range(args.warmup):
        pass   # the oracle has nothing to warm up; each step below is a full bounded sample
    times, flops = [], 0.0
    for s in range(args.steps):
        dt, fl = oracle_sample(wl, [s % wl.bands.kfrac.shape[0]], f_idx)
        times.append(dt)
        flops = fl
    t = float(np.mean(times))
    val = flops / t / 1e12
    sample = f"k-point(s) {k_list} of {wl.bands.kfrac.shape[0]}, frequencies {f_idx} of {nf}: M, weights, chi0 partial sum"
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "sample": sample},
           "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": blas_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="medium")
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "bf16x3", "tf32x3"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

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
    G, tl = ctx.rp_sphere_size(q)
    ng, nf = len(G), len(wl.freq)
    K = wl.bands.kfrac.shape[0] * wl.nocc * wl.nemp
    F = falg(ng, K, nf)
    chi = torch.empty((nf, ng, ng), dtype=torch.complex128, device=dev)
    W = torch.empty_like(chi)
    tail = torch.zeros(max(1, len(tl)), dtype=torch.float64, device=dev)

    def step():
        ctx.rp_build_chi0(q, axis, ordering, wl.freq, wl.delta, prec, wl.delta_a, wl.delta_r, out=chi)
        ctx.rp_solve_w(q, chi, out=W, tail=tail)

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
    ms_total = max_over_ranks(ms_total, dev)
    ms_step = ms_total / args.steps
    value = job_rate(F, ms_step * 1e-3, ws)

    # dominant kernel: the chi0 contraction (tensor pipe)
    pk = peaks()
    t_con = stage_ms[3] / args.steps * 1e-3
    if prec == rp.RP_FP64_NATIVE:
        # FP64 tensor peak = measured bf16 burst x nominal FP64/BF16 ratio (1.25 / 2250)
        peak = pk.get("bf16_tflops", 1900.0) * 1.25 / 2250.0
        peak_note = "measured bf16 burst x nominal fp64/bf16 ratio 1.25/2250"
    elif prec == rp.RP_TF32X3:
        # TF32 tensor peak = measured bf16 sustained x nominal TF32/BF16 ratio (1.1 / 2.25)
        peak = pk.get("bf16_tflops_sustained", 1700.0) * 1.1 / 2.25
        peak_note = "measured bf16 sustained x nominal tf32/bf16 ratio 1.1/2.25"
    else:
        peak = pk.get("bf16_tflops_sustained", 1700.0)
        peak_note = "measured bf16 sustained"
    # algorithmic flops of the timed steps / summed duration of the contraction kernel's launches
    achieved = F / t_con / 1e12 if t_con > 0 else None
    traffic, traffic_note = measured_traffic(args.workload, args.precision)
    roof = {"bound": "tensor", "kernel": "chi0 contraction", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_note": traffic_note, "launches_per_step": int(launches[3]) // args.steps,
            "ms_per_launch": float(stage_ms[3]) / max(1, int(launches[3])), "peak_source": peak_note}

    res = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"fp64": "f64", "bf16x3": "bf16x3", "tf32x3": "tf32x3"}[args.precision],
           "data": "synthetic (seeded empirical-pseudopotential bands)",
           "config": {"workload": args.workload, "ng": ng, "pairs_K": K, "nfreq": nf, "nk": int(wl.bands.kfrac.shape[0]),
                      "nocc": wl.nocc, "nemp": wl.nemp, "fft": list(wl.fft), "axis": wl.axis,
                      "precision": args.precision, "l2": "inputs larger than L2 (bands and per-step scratch > 129 MB)",
                      "parallelism": f"replicas x{ws}"},
           "stages_ms_per_step": {n: stage_ms[i] / args.steps for i, n in enumerate(STAGES)},
           "gpu_launches": int(launches.sum()), "roofline": roof, "clocks": clk}

    if prec != rp.RP_FP64_NATIVE and not args.no_fp64:
        # the same q with the native FP64 path on two of the frequencies: its contraction rate,
        # and the per-frequency error of the split-precision chi0 and W against it
        fi = [0, nf - 1]
        f2 = wl.freq[fi]
        chi64 = torch.empty((len(fi), ng, ng), dtype=torch.complex128, device=dev)
        ctx.rp_profile_enable(True)
        ctx.rp_build_chi0(q, axis, ordering, f2, wl.delta, rp.RP_FP64_NATIVE, wl.delta_a, wl.delta_r, out=chi64)
        W64, _ = ctx.rp_solve_w(q, chi64)
        torch.cuda.synchronize()
        ms64, _ = ctx.rp_profile_read()
        ctx.rp_profile_enable(False)
        W_split = W[fi]

        def rel(a, b):
            return [float(torch.linalg.norm(a[i] - b[i]) / torch.linalg.norm(b[i])) for i in range(a.shape[0])]
        res["fp64_reference"] = {
            "freq_index": fi, "contraction_tflops": falg(ng, K, len(fi)) / (ms64[3] * 1e-3) / 1e12,
            "contraction_ms": float(ms64[3]), "chi0_rel_err": rel(chi[fi], chi64), "W_rel_err": rel(W_split, W64),
            "note": "native FP64 GPU path (itself checked against the FP64 oracle in the test-suite)"}

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
        h2d = coef.numel() * 16 + energy.numel() * 8 + miller.numel() * 4 + npw.numel() * 4 + chi_h.numel() * 16
        d2h = chi_h.numel() * 16 + W_h.numel() * 16 + tail_h.size * 8
        ectx = rp.Context(b.cell.lat, b.kmesh, wl.fft, b.ecut_psi, float(wl.ecut_eps[0]))

        def e2e_step():
            ectx.rp_load_bands(wl.nocc, npw.numpy(), miller.numpy(), coef.numpy(), energy.numpy())
            ectx.rp_build_chi0(q, axis, ordering, wl.freq, wl.delta, prec, wl.delta_a, wl.delta_r, out=chi_h.numpy())
            ectx.rp_solve_w(q, chi_h.numpy(), out=W_h.numpy(), tail=tail_h)
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        te = max_over_ranks((time.perf_counter() - t0) / args.steps, dev)
        res["e2e"] = {"value": job_rate(F, te, ws), "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "ms_per_step": te * 1e3}
        ectx.close()

    if rank == 0 and not args.no_cpu:
        k_list, f_idx = [0], [0, nf - 1]
        dt, fl = oracle_sample(wl, k_list, f_idx)
        res["cpu_baseline"] = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": blas_threads(), "kind": "oracle",
                               "sample": f"k-point 0 of {K // (wl.nocc * wl.nemp)}, frequencies {f_idx} of {nf}: "
                                         f"oracle M, tetrahedron weights and chi0 partial sum ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
