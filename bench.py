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
UNIT = "updates/s"
SM_MAX_MHZ = 2070.0
# DRAM bytes (read + write) per two-site update of the ensemble kernel on this
# workload, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum,
# one pass, -k ensemble_kernel -c 1) of a 304-sample batch of the same ring of
# 64 at chi = 128: 3.728e11 + 4.921e11 bytes over 15716 updates. The launch
# runs the same 304 CTAs as the full batch, so the bytes per update carry over;
# the line's traffic is this times the updates of one launch.
# (profiles/ensemble_kernel_ring64_chi128_launches.md gives the command.)
DRAM_BYTES_PER_UPDATE = 5.503e7


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
    ap.add_argument("--tts-ring32", type=int, default=0, metavar="K",
                    help="also time K full ring32_heisenberg_T2 circuits (chi 64, mixed) and report the "
                         "time-to-<Z> of its 10^4 samples, extrapolated from the K timed ones")
    ap.add_argument("--three-site", action="store_true",
                    help="bond-2 gates as one three-site update (tepai_params.three_site) instead of "
                         "swap routing; compare events/s, not updates/s (each split counts as one update)")
    ap.add_argument("--three-site-steps", type=int, default=2,
                    help="also time this many steps of the same circuits with three-site updates "
                         "(0 = skip); reported as the line's three_site object")
    ap.add_argument("--launch-variant", type=int, default=0,
                    help="tepai_params.launch_variant (0 = library default; 2 = CUDA-core Jacobi, "
                         "7 = tensor-core Jacobi), for A/B runs")
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
    """One bench sample through the FP64 oracle, as it stands. The sample's
    set-up (interpreter start, imports, the shared start state's canonical
    form, the circuit draw) is outside the timed region: only the evolution of
    the sample's events is timed."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    window, offset = args
    import workloads as W
    from oracle import mps as omps
    from oracle import planner, sampler
    prob, par, init = W.bench_workload(1, window_steps=window, sample_offset=offset)
    plan = planner.make_plan(prob, par.T, par.n_steps, par.delta, par.variant)
    ev = sampler.sample_events(plan, par.seed, offset, par.steps_run())
    m = omps.canonicalize(init[0], prob.periodic)
    t = time.perf_counter()
    omps.run_events(m, plan, ev, [par.steps_run()], par.chi_max, par.cutoff, floor_rel=4e-6)
    dt = time.perf_counter() - t
    return m.stats["gate_updates"] + m.stats["swap_updates"], dt


def oracle_sample(window: int, offsets, procs: int):
    """The FP64 oracle on `procs` host processes (one BLAS thread each), one
    bench sample per process. Returns (updates, aggregate updates/s): the sum
    over processes of each one's updates per second of evolution."""
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(window, o) for o in offsets])
    return sum(u for u, _ in res), sum(u / t for u, t in res if t > 0)


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
    procs = cpu_cores()
    window = 1
    batch = procs
    for w in range(a.warmup):
        oracle_sample(window, [10_000_000 + w * batch + i for i in range(batch)], procs)
    rates, t0 = [], time.perf_counter()
    for s in range(a.steps):
        _, r = oracle_sample(window, [20_000_000 + s * batch + i for i in range(batch)], procs)
        rates.append(r)
    wall = time.perf_counter() - t0
    val = sum(rates) / len(rates)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * wall / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "ring64_xxz_chi128_window", "n": 64, "chi_max": 128,
                       "window_steps": window, "batch": batch, "init": "shared random MPS at chi=128",
                       "l2": "host CPU run"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": f"{batch} samples x {window} Trotter step(s) per step, one process "
                                       f"(1 BLAS thread) per sample on every core of the affinity mask "
                                       f"(nproc {procs}); evolution timed, set-up not"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- time to <Z>, ring of 8
def _sv_ring8_chunk(args):
    """State-vector oracle values of samples [lo, hi) of ring8_heisenberg_T1."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    lo, hi = args
    import workloads as W
    from oracle import run as orun
    prob, par, _ = W.workload(W.RING8)
    r = orun.run(prob, par, use_statevector=True, samples=range(lo, hi))
    return r["v"], r["sign"]


def ring8_oracle_mean():
    """Exact state-vector oracle estimate of ring8_heisenberg_T1 (all circuits,
    spawned processes with one BLAS thread each). Returns (mean [M][1], seconds)."""
    import numpy as np
    import workloads as W
    from oracle import estimator, planner
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    prob, par, _ = W.workload(W.RING8)
    chunks = [(lo, min(lo + 25, par.n_samples)) for lo in range(0, par.n_samples, 25)]
    t = time.perf_counter()
    with mp.get_context("spawn").Pool(cpu_cores()) as pool:
        res = pool.map(_sv_ring8_chunk, chunks)
    dt = time.perf_counter() - t
    v = np.concatenate([r[0] for r in res])
    sg = np.concatenate([r[1] for r in res])
    plan = planner.make_plan(prob, par.T, par.n_steps, par.delta, par.variant)
    g = np.array([planner.gnorm_at(plan, j) for j in planner.snapshot_steps(par.n_steps, par.n_snapshots)])
    mean, _, _ = estimator.estimate(v, sg, g)
    return mean, dt


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
    ref_mean, t_oracle = ring8_oracle_mean()
    return {"config": "ring8_heisenberg_T1 (N=2000, 1000 samples, chi_max=16, <Z_0> at 10 times)",
            "mixed_batched_s": t_mixed, "fp64_batched_s": t_fp64_batched,
            "fp64_one_sample_per_launch_s": t_one, "one_per_launch_subset": subset,
            "speedup_vs_fp64_one_per_launch": t_one / t_mixed,
            "max_abs_err_mixed_vs_fp64": err,
            "err_per_snapshot_mixed_vs_oracle": [float(x) for x in abs(rm["mean"] - ref_mean)[:, 0]],
            "err_per_snapshot_fp64_vs_oracle": [float(x) for x in abs(rf["mean"] - ref_mean)[:, 0]],
            "oracle": f"exact state vector on all {par.n_samples} circuits, {cpu_cores()} host processes, "
                      f"{t_oracle:.1f} s",
            "stderr_fp64": float(rf["stderr"].max()),
            "mixed_continuous_s": t_cont,
            "events_per_sample_finite_n": rm["stats"]["events"] / par.n_samples,
            "events_per_sample_continuous": rc["stats"]["events"] / par.n_samples,
            "sampler_phase_share_continuous": rc["stats"]["phase_cycles"]["sampler"]
            / max(1.0, float(sum(rc["stats"]["phase_cycles"].values()))),
            "sampler_phase_share_finite_n": rm["stats"]["phase_cycles"]["sampler"]
            / max(1.0, float(sum(rm["stats"]["phase_cycles"].values()))),
            "max_abs_diff_continuous_vs_finite_n": float(abs(rc["mean"] - rm["mean"]).max())}


# ---------------------------------------------------------------- time to <Z>, ring of 32
def tts_ring32(T, W, local, k):
    """ring32_heisenberg_T2 (n = 32, fields U[-2, 2], T = 2, N = 8000, chi 64,
    cutoff 1e-10, mixed precision, all <Z_i> at 20 times): K full circuits are
    evolved and timed (one launch, persistent CTAs); the time for the workload's
    10^4 samples is extrapolated as ceil(10^4 / K) such launches, which holds
    while K is a multiple of the CTAs of a launch. Labelled as an extrapolation."""
    prob, par, ex = W.workload(W.RING32)
    run_par = W.Params(**{**par.__dict__, "n_samples": k, "sample_offset": 7_000_000})
    ctx = T.tepai_create(local)
    try:
        t = time.perf_counter()
        r = T.tepai_run(ctx, prob, run_par)
        dt = time.perf_counter() - t
    finally:
        T.tepai_destroy(ctx)
    st = r["stats"]
    waves = math.ceil(par.n_samples / k)
    return {"config": "ring32_heisenberg_T2 (n=32, N=8000, chi_max=64, cutoff 1e-10, mixed, <Z_i> at 20 times)",
            "timed_samples": k, "timed_s": dt, "grid_ctas": st["grid_ctas"],
            "events_per_sample": st["mean_nu"], "updates": st["gate_updates"] + st["swap_updates"],
            "max_chi": st["max_chi"], "max_discarded_weight": st["max_discarded_weight"],
            "extrapolated_time_to_Z_s": dt * waves, "extrapolation": f"{waves} launches of {k} samples",
            "stderr_max_at_k": float(r["stderr"].max()),
            "stderr_max_extrapolated": float(r["stderr"].max()) * math.sqrt(k / par.n_samples)}


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
    if a.launch_variant:
        par = W.Params(**{**par.__dict__, "launch_variant": a.launch_variant})
    if a.three_site:
        par = W.Params(**{**par.__dict__, "three_site": 1})
    stream = torch.cuda.current_stream()
    run = T.DeviceRun(prob, par, init, stream=stream)
    base = 1_000_000 * (rank + 1)

    def step(i, r=None):
        r = r or run
        r.set_sample_offset(base + i * batch)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.execute()
        e1.record(stream)
        st = r.stats()              # synchronises the stream
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
    upd, flops, kms, events, sweeps, qrm, tcf, reorth = 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0
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
        tcf += st["tc_flops"]
        reorth += st["jacobi_reorth"]
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

    # the same circuits (the first timed steps' samples) with bond-2 gates as
    # three-site updates instead of swap routing: sampled events/s is the rate
    # to compare, since a three-site update counts two splits per event where
    # swap routing counts three updates
    three = None
    if world == 1 and not a.three_site and a.three_site_steps > 0:
        run3 = T.DeviceRun(prob, W.Params(**{**par.__dict__, "three_site": 1}), init, stream=stream)
        step(0, run3)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        ev3, up3, k3 = 0.0, 0.0, 0.0
        n3 = min(a.three_site_steps, a.steps)
        for i in range(n3):
            ms, st = step(a.warmup + i, run3)
            k3 += ms
            ev3 += st["events"]
            up3 += st["gate_updates"] + st["swap_updates"]
        torch.cuda.synchronize()
        el3 = time.perf_counter() - t3
        run3.release()
        del run3
        three = {"events_per_s": ev3 / el3, "updates_per_s": up3 / el3, "steps": n3,
                 "ms_per_step": 1e3 * el3 / n3, "kernel_ms": k3,
                 "events_per_s_swap_routing": events / elapsed,
                 "events_speedup": (ev3 / el3) / max(events / elapsed, 1e-30),
                 "note": "tepai_params.three_site = 1 on the samples of the first timed steps"}

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
    # roofline denominators measured on this device by the library's own
    # microbenchmarks (FP32 FMA, tcgen05 TF32), taken after the timed region
    peaks = T.tepai_measure_peaks(local)
    peak = peaks["fp32_tflops"]
    achieved = flops / (kms / 1e3) / 1e12
    tc_rate = tcf / (kms / 1e3) / 1e12
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
                     "frac": achieved / peak, "traffic": DRAM_BYTES_PER_UPDATE * upd / a.steps,
                     "traffic_note": "DRAM bytes per launch: ncu bytes per update on a 304-sample batch of this "
                                     "workload x updates per launch; algorithmic site-tensor bytes are 64 chi^2 "
                                     "= 1.05 MB per update",
                     "peak_note": "FP32 FMA throughput of this GPU, measured (tepai_measure_peaks); "
                                  "achieved = algorithmic flops (736 chi^3 per square update) per second "
                                  "of ensemble-kernel time"},
        "tensor_pipe": {"tc_flops_per_s": tc_rate * 1e12, "tf32_peak_tflops": peaks["tf32_tflops"],
                        "frac_of_tf32_peak": tc_rate / peaks["tf32_tflops"] if peaks["tf32_tflops"] else None,
                        "note": "tcgen05 MMA flops issued (3xTF32: three MMAs per product) per second of "
                                "kernel time, against the measured TF32 MMA peak"},
        "measured_peaks": peaks,
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
                  "kernel_ms": kms, "not_converged": nconv, "fp64_reorth_svds": reorth,
                  "max_chi": maxchi, "grid_ctas": grid, "tensor_core_jacobi": bool(tcf > 0),
                  "three_site": bool(a.three_site)},
    }
    if three is not None:
        line["three_site"] = three
    if not a.no_tts and world == 1:
        line["tts_ring8"] = tts_ring8(T, W, torch, local)
    if a.tts_ring32 and world == 1:
        line["tts_ring32"] = tts_ring32(T, W, local, a.tts_ring32)
    if not a.no_cpu_baseline and world == 1:
        procs = cpu_cores()
        u, rate = oracle_sample(1, [base + 900_000 + i for i in range(procs)], procs)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": f"{procs} samples x 1 Trotter step of the same workload ({u:.0f} "
                                          f"updates), one process (1 BLAS thread) per sample on every core "
                                          f"of the affinity mask (nproc {procs}); evolution timed, set-up not"}
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
