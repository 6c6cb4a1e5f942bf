"""Benchmark of the MPS TE-PAI hot path on GB300.

Metric: two-site gate-updates per second at chi = 128 (every SVD update of an
MPS TE-PAI sample: Pauli-rotation gates plus the swaps that route the ring
bond). One step evolves a batch of independently sampled circuits, each for
a window of Trotter steps, from a shared random MPS whose bonds are at the
cap. Each step then measures every <Z_i> and forms the signed ensemble
reduction. All of this is one pass of the hot path. Successive steps use new
sample indices, so every step evolves new circuits.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TE-PAI MPS gate-updates/s at chi=128"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one ensemble_kernel
# launch of the default workload, divided by the two-site updates of that launch
# (7.897e12 B over 123751 updates), from one ncu capture of the current kernel.
DRAM_BYTES_PER_UPDATE = 6.381e7
UNIT = "updates/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--window", type=int, default=1, help="Trotter steps evolved per sample")
    ap.add_argument("--batch", type=int, default=0,
                    help="samples per step (0 = 16 per SM: the persistent CTAs' tail, where the last "
                         "samples straggle, stays below 10%% of a step)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tts", action="store_true", help="skip the ring-of-8 time-to-<Z> comparison")
    ap.add_argument("--n", type=int, default=64, help="ring size (profiling cases only)")
    ap.add_argument("--chi", type=int, default=128, help="bond cap (profiling cases only)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.device = device
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle leg
def _oracle_worker(args):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    window, offset = args
    import workloads as W
    from oracle import run as orun
    prob, par, init = W.bench_workload(1, window_steps=window, sample_offset=offset)
    t = time.perf_counter()
    r = orun.run(prob, par, init_tensors=init[0], floor_rel=4e-6, gap_rel=1e-4)
    dt = time.perf_counter() - t
    st = r["stats"][0]
    return st["gate_updates"] + st["swap_updates"], dt


def oracle_sample(window: int, offsets, procs: int):
    """The FP64 oracle, as it stands, on `procs` host processes (one BLAS thread
    each), one bench sample per process. Returns (updates, wall seconds)."""
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    t = time.perf_counter()
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(window, o) for o in offsets])
    wall = time.perf_counter() - t
    return sum(u for u, _ in res), wall


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- reference arm
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    procs = max(1, min(cpu_cores(), 16))
    window = 1
    batch = procs
    for w in range(a.warmup):
        oracle_sample(window, [10_000_000 + w * batch + i for i in range(batch)], procs)
    tot_u, tot_t = 0.0, 0.0
    for s in range(a.steps):
        u, t = oracle_sample(window, [20_000_000 + s * batch + i for i in range(batch)], procs)
        tot_u += u
        tot_t += t
    val = tot_u / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot_t / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "ring64_xxz_chi128_window", "n": 64, "chi_max": 128,
                       "window_steps": window, "batch": batch, "init": "shared random MPS at chi=128",
                       "l2": "host CPU run"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": f"{batch} samples x {window} Trotter step(s) per step, "
                                       f"one process (1 BLAS thread) per sample"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- time to <Z>, ring of 8
def tts_ring8(T, W, torch, local, subset=16):
    """Time-to-<Z_0> on the ring8_heisenberg_T1 workload (ring of 8, 1000 samples, N = 2000):
    mixed precision with batched persistent CTAs, against the plain FP64 form
    with one sample per launch (timed on `subset` samples, scaled to 1000).
    The error is max |mean_mixed - mean_fp64| on the same seeded circuits. The
    FP64 path equals the oracle to 1e-10 in the parity tests."""
    prob, par, _ = W.workload(W.RING8)
    ctx = T.tepai_create(local)
    try:
        mixed = W.Params(**{**par.__dict__, "precision": 1})
        T.tepai_run(ctx, prob, W.Params(**{**mixed.__dict__, "n_samples": 8}))   # context set-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        rm = T.tepai_run(ctx, prob, mixed)
        t_mixed = time.perf_counter() - t
        t = time.perf_counter()
        rf = T.tepai_run(ctx, prob, par)
        t_fp64_batched = time.perf_counter() - t
        t = time.perf_counter()
        for s in range(subset):
            T.tepai_run(ctx, prob, W.Params(**{**par.__dict__, "n_samples": 1, "sample_offset": s}))
        t_one = (time.perf_counter() - t) / subset * par.n_samples
        # the same ensemble drawn in the N -> infinity limit (no Trotter error)
        cont = W.Params(**{**mixed.__dict__, "variant": T.TEPAI_CONTINUOUS})
        t = time.perf_counter()
        rc = T.tepai_run(ctx, prob, cont)
        t_cont = time.perf_counter() - t
    finally:
        T.tepai_destroy(ctx)
    err = float(abs(rm["mean"] - rf["mean"]).max())
    return {"config": "ring8_heisenberg_T1 (N=2000, 1000 samples, chi_max=16, <Z_0> at 10 times)",
            "mixed_batched_s": t_mixed, "fp64_batched_s": t_fp64_batched,
            "fp64_one_sample_per_launch_s": t_one, "one_per_launch_subset": subset,
            "speedup_vs_fp64_one_per_launch": t_one / t_mixed,
            "max_abs_err_mixed_vs_fp64": err,
            "stderr_fp64": float(rf["stderr"].max()),
            "mixed_continuous_s": t_cont,
            "events_per_sample_finite_n": rm["stats"]["events"] / par.n_samples,
            "events_per_sample_continuous": rc["stats"]["events"] / par.n_samples,
            "sampler_phase_share_continuous": rc["stats"]["phase_cycles"]["sampler"]
            / max(1.0, float(sum(rc["stats"]["phase_cycles"].values()))),
            "sampler_phase_share_finite_n": rm["stats"]["phase_cycles"]["sampler"]
            / max(1.0, float(sum(rm["stats"]["phase_cycles"].values()))),
            "max_abs_diff_continuous_vs_finite_n": float(abs(rc["mean"] - rm["mean"]).max())}


# ---------------------------------------------------------------- our arm
def run_ours(a):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import workloads as W
    from paper_2604_13144_gb300 import tepai as T

    sms = torch.cuda.get_device_properties(local).multi_processor_count
    batch = a.batch or 16 * sms
    prob, par, init = W.bench_workload(batch, window_steps=a.window, chi=a.chi, n=a.n)
    stream = torch.cuda.current_stream()
    run = T.DeviceRun(prob, par, init, stream=stream)
    base = 1_000_000 * (rank + 1)

    def step(i):
        run.set_sample_offset(base + i * batch)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run.execute()
        e1.record(stream)
        st = run.stats()            # synchronises the stream
        if st["device_status"][0] != 0:
            raise RuntimeError(f"device check failed: {st['device_status']}")
        return e0.elapsed_time(e1), st

    for i in range(a.warmup):
        step(i)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    t0 = time.perf_counter()
    upd, flops, kms, events, sweeps, qrm = 0.0, 0.0, 0.0, 0.0, 0.0, 0.0
    jpairs, jrots = 0.0, 0.0
    phases, subphases = {}, {}
    grid = 1
    nconv, maxchi = 0, 0
    order_on = 0
    for i in range(a.steps):
        ms, st = step(a.warmup + i)
        order_on = st["sample_order"]
        kms += ms
        upd += st["gate_updates"] + st["swap_updates"]
        flops += st["alg_flops"]
        events += st["events"]
        sweeps += st["jacobi_sweeps"]
        qrm += st["qr_moves"]
        jpairs += st["jacobi_pairs"]
        jrots += st["jacobi_rotations"]
        grid = st["grid_ctas"]
        for k, v in st["phase_cycles"].items():
            phases[k] = phases.get(k, 0.0) + v
        for k, v in st["subphase_cycles"].items():
            subphases[k] = subphases.get(k, 0.0) + v
        nconv += st["n_not_converged"]
        maxchi = max(maxchi, st["max_chi"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = time.perf_counter() - t0
    clocks = clk.stop()
    if dist:
        t = torch.tensor([elapsed], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
        u = torch.tensor([upd], dtype=torch.float64, device="cuda")
        dist.all_reduce(u)
        upd_all = float(u.item())
    else:
        upd_all = upd
    value = upd_all / elapsed

    # end-to-end through the C-ABI with host buffers (planning, H2D, kernels, D2H)
    ctx = T.tepai_create(local, stream.cuda_stream)
    e2e_par = W.Params(**{**par.__dict__, "sample_offset": base + 500_000})
    T.tepai_run(ctx, prob, e2e_par, init)           # allocates the context workspace once
    torch.cuda.synchronize()
    e2e_u, t1 = 0.0, time.perf_counter()
    for i in range(max(1, a.e2e_steps)):
        e2e_par = W.Params(**{**par.__dict__, "sample_offset": base + 600_000 + i * batch})
        r = T.tepai_run(ctx, prob, e2e_par, init)
        e2e_u += r["stats"]["gate_updates"] + r["stats"]["swap_updates"]
    e2e_t = time.perf_counter() - t1
    T.tepai_destroy(ctx)
    M, nobs, n = par.n_snapshots, prob.n, prob.n
    L = 4 * n
    h2d = (sum(t.size for t in init[0]) * 16 + (n + 1) * 4 + L * 288 + M * 12 + nobs * 4 + n
           + 4 * n * 8)
    d2h = 5 * M * nobs * 8

    if rank != 0:
        return 0
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops / (kms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * elapsed / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"ring{n}_xxz_chi{par.chi_max}_window", "n": n, "chi_max": par.chi_max,
                   "cutoff": par.cutoff, "delta": "pi/1024", "N": par.n_steps, "T": par.T,
                   "window_steps": a.window, "batch": batch, "init": "shared random MPS at chi=128",
                   "precision": "mixed (FP32 tensors/SVD, FP64 bookkeeping)",
                   "parallelism": f"samples sharded over {world} GPU(s)",
                   "l2": "inputs larger than L2 (per-CTA MPS arenas, GBs)"},
        "e2e": {"value": e2e_u / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        # per step: the ensemble kernel and the reduction, plus the sample-cost
        # and ordering kernels when the call hands out samples costliest first
        "gpu_launches": (2 + 2 * order_on) * a.steps,
        "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": (DRAM_BYTES_PER_UPDATE * upd / a.steps
                                 if (n, par.chi_max) == (64, 128) else None),
                     "peak_note": "FP32 FMA: 152 SM x 128 lanes x 2 flop x 2070 MHz (derived)"},
        "stats": {"events_per_s": events / elapsed, "updates": upd, "alg_flops": flops,
                  "sweeps_per_svd": sweeps / max(upd, 1.0),
                  "qr_moves_per_update": qrm / max(upd, 1.0),
                  "jacobi_pairs_per_svd": jpairs / max(upd, 1.0),
                  "jacobi_rotated_frac": jrots / max(jpairs, 1.0),
                  "jacobi_cycles_per_pair": phases.get("jacobi", 0.0) / max(jpairs, 1.0),
                  "updates_per_event": upd / max(events, 1.0),
                  "phase_share": {k: round(v / max(sum(phases.values()), 1.0), 4) for k, v in phases.items()},
                  "subphase_share": {k: round(v / max(sum(phases.values()), 1.0), 4)
                                     for k, v in subphases.items()},
                  "cta_busy_frac": sum(phases.values()) / max(kms / 1e3 * SM_MAX_MHZ * 1e6 * grid, 1.0),
                  "kernel_ms": kms, "not_converged": nconv, "max_chi": maxchi, "grid_ctas": grid},
    }
    if not a.no_tts and world == 1:
        line["tts_ring8"] = tts_ring8(T, W, torch, local)
    if not a.no_cpu_baseline and world == 1:
        procs = max(1, min(cpu_cores(), 16))
        u, t = oracle_sample(1, [base + 900_000 + i for i in range(procs)], procs)
        line["cpu_baseline"] = {"value": u / t, "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": f"{procs} samples x 1 Trotter step of the same workload, "
                                          f"one process (1 BLAS thread) per sample"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
