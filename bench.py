#!/usr/bin/env python
"""Benchmark of the LJ Verlet-list MD hot path: particle-steps/s at 16.4M atoms, mixed vs FP64.

One "step" is one velocity-Verlet step of the whole path (kick/drift, displacement check,
list rebuild when due, force over the list, energy and virial reductions).  Timed with CUDA
events on the library's stream, inputs resident in HBM (and far larger than L2).  Prints one
JSON line.  ``--impl reference`` times the FP64 CPU oracle on a bounded sample instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
For N > 1 launch under torch.distributed.run: every rank advances an independent replica
(the method has no data-path exchange on one box), and the job value is the sum.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LJ particle-steps/s at 16.4M atoms, mixed vs FP64 form; roofline fraction"
UNIT = "particle-steps/s"

# FCC workloads: M^3 cells x 4 at density rho (L = M (4/rho)^(1/3)), Eq. 2 truncation.
WORKLOADS = {
    "fcc16m_rho0.5": dict(M=160, rho=0.5, T=1.0, seed=3, cutoff=2.5, margin=0.5, dt=0.005),
    "fcc16m_rho0.8": dict(M=160, rho=0.8, T=0.9, seed=4, cutoff=2.5, margin=0.5, dt=0.005),
    "fcc1m_rho0.5": dict(M=64, rho=0.5, T=1.0, seed=2, cutoff=2.5, margin=0.5, dt=0.005),
    "fcc4k_rho0.5": dict(M=10, rho=0.5, T=1.0, seed=1, cutoff=2.5, margin=0.5, dt=0.005),
}

# Measured peaks of the non-tensor pipes of this GPU type (GB300, 152 SMs, 2070 MHz max): a kernel of
# independent FMA chains (8 per thread, 256-thread blocks, 4 and 8 blocks per SM), best of 5 launches
# timed with CUDA events.  FP32 FFMA 75.8 TFLOP/s (94 % of 152 x 128 lanes x 2 x 2.07 GHz); FP64 DFMA
# 1.008 TFLOP/s.
FP32_PEAK_TFLOPS = 75.8
FP64_PEAK_TFLOPS = 1.008
ALU_PEAK_SOURCE = "measured: FMA-chain kernel on GB300 (FP32 75.8, FP64 1.008 TFLOP/s)"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x, dist=None, device="cuda"):
    """Largest x over the ranks of the process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def mups(n, steps, seconds):
    """Speed in millions of particle updates per second (Sec. 3.3, Sec. 4.5): N k / (10^6 t) for
    N particles advanced k steps in t seconds."""
    return n * steps / (1e6 * seconds)


def replica_seed(base, rank):
    """Each rank advances an independent replica (no data-path exchange between ranks)."""
    return base + 1000 * rank


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_force_pipe_fcc1m_rho0.5.md")
FORCE_SOURCE = os.path.join(ROOT, "paper_1012_2677_gb300", "csrc", "kernels_tile.cu")


def recorded_traffic(kernel_name, N):
    """DRAM bytes of one force launch at N particles, scaled by N from the per-particle traffic in
    the committed ncu summary of a smaller case of the same kernel, if the kernel source is
    unchanged since the counters were taken (else None).  The summary's lines 'key: value'
    give kernel, source_sha and dram_bytes_per_particle."""
    rec = {}
    try:
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if line.startswith("- ") and ": " in line:
                    k, v = line[2:].split(": ", 1)
                    rec[k.strip().strip("`")] = v.strip().strip("`")
    except OSError:
        return None
    if rec.get("source_sha") != source_sha(FORCE_SOURCE) or rec.get("kernel") != kernel_name:
        return None
    try:
        return round(float(rec["dram_bytes_per_particle"]) * N)
    except (KeyError, ValueError):
        return None


def force_kernel_work(N, entries, form, energy=True):
    """Algorithmic bytes and flops of one force launch.

    bytes (the scope table's count): each list entry once as a 4-byte index and each particle's own
    position and force once, 32 B in the mixed form (16 B each) and 64 B in the FP64 form; partner
    positions come from on-chip memory (cell-sorted tiles) and count zero.
    stored_bytes (this library's layout): 2-byte entries (indices into the key's staged tile), an
    8-byte row, the own position record (mixed: 16 B fixed point; FP64: 32 B) and the force (mixed:
    16 B; FP64: 32 B).
    flops: 22 per list entry (Alg. 6 with the r^2 < r_c^2 select: 3 difference, 5 r^2, 1
    reciprocal, 4 r^6 and r^14, 3 coefficient, 3 force, 3 accumulation), 3 more for the partner's
    update with the half list (FP64 form), 8 more with the energy and virial."""
    half = form == "fp64"
    own = 32 if form == "mixed" else 64
    bytes_ = 4 * entries + own * N
    stored = 2 * entries + N * (8 + own)
    flops = entries * (22 + (3 if half else 0) + (8 if energy else 0))
    return bytes_, stored, flops


def roofline(kernel, ms, bytes_, flops, peaks, alu_peak, alu_name, peak_kind, traffic=None, extra=None):
    """Roofline block of one kernel: achieved algorithmic bytes and flops per launch over its mean
    launch time, each against its measured peak; `bound` names the larger fraction."""
    gbs = bytes_ / (ms * 1e-3) / 1e9
    tfs = flops / (ms * 1e-3) / 1e12
    hbm = {"achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(gbs / peaks["hbm_gbs"], 4),
           "peak_source": peak_kind + " (copy bandwidth)"}
    alu = {"achieved": round(tfs, 3), "peak": alu_peak, "unit": "TFLOP/s", "frac": round(tfs / alu_peak, 4),
           "peak_source": ALU_PEAK_SOURCE, "pipe": alu_name}
    main, other = (hbm, alu) if hbm["frac"] >= alu["frac"] else (alu, hbm)
    out = {"bound": "hbm" if main is hbm else "alu", "achieved": main["achieved"], "peak": main["peak"],
           "unit": main["unit"], "frac": main["frac"], "traffic": traffic, "peak_source": main["peak_source"],
           ("alu" if main is hbm else "hbm"): other, "kernel": kernel, "kernel_ms": round(ms, 4),
           "algorithmic_bytes_per_launch": int(bytes_), "algorithmic_flops_per_launch": int(flops)}
    if extra:
        out.update(extra)
    return out


def run_ours(args, wl, world, rank, local):
    import torch
    from paper_1012_2677_gb300 import ljmd

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    seed = replica_seed(wl["seed"], rank)  # independent replica per rank
    peaks, peak_kind = measured_peaks()

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed_run(precision, list_form, with_clocks):
        """Warm-up, then the timed steps between CUDA events on the library's stream (per-phase
        events on while timing).  Returns the system (still open) and the measurements."""
        sy = ljmd.System(cutoff=wl["cutoff"], margin=wl["margin"], precision=precision, list_form=list_form,
                         energy_every=1, stream=stream)
        sy.init_lattice(wl["M"], wl["rho"], wl["T"], seed)
        sy.step(wl["dt"], args.warmup)
        torch.cuda.synchronize()
        st0 = sy.stats()
        sy.set_profiling(True)
        clocks = ClockSampler(local) if with_clocks else None
        if clocks:
            clocks.start()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sy.step(wl["dt"], args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop() if clocks else None
        ms_ = reduce_max(e0.elapsed_time(e1), dist)
        prof = sy.profile()
        st1 = sy.stats()
        sy.set_profiling(False)
        return sy, dict(ms=ms_, prof=prof, st0=st0, st1=st1, clocks=clk)

    # ---- the headline: mixed form, automatic list form
    s, m = timed_run(ljmd.LJ_MIXED, ljmd.LJ_LIST_AUTO, True)
    N = s.n
    ms, prof, st0, st1 = m["ms"], m["prof"], m["st0"], m["st1"]
    value = job_value(N * args.steps, world, ms * 1e-3)
    pe, ke, vir = s.energies()
    entries = st1["list_entries"]
    half = st1["list_form"] == ljmd.LJ_LIST_HALF  # the automatic list form of this density
    # the mixed form on tiles: the pipelined kernel with the full list, the single-buffer one with the half
    kernel_name = "k_force_tile" if half else "k_force_pipe"
    f_ms = prof["force_ms"] / max(prof["force_launches"], 1)
    b, stored, fl = force_kernel_work(N, entries, "mixed")
    roof = roofline(kernel_name, f_ms, b, fl, peaks, FP32_PEAK_TFLOPS, "fp32", peak_kind,
                    traffic=recorded_traffic(kernel_name, N),
                    extra={"stored_list": {"bytes_per_launch": int(stored),
                                           "hbm_frac": round(stored / (f_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                                           "note": "2-byte tile-local entries, 8-byte rows, 16-byte records"}})
    breakdown = {k: round(prof[k], 3) for k in ("force_ms", "integrate_ms", "rebuild_ms", "energy_ms")}
    breakdown.update({k: prof[k] for k in ("force_launches", "integrate_launches", "rebuilds", "energy_launches")})
    x_mixed, f_mixed, box = None, None, s.box
    if rank == 0 and not args.no_cpu_baseline and not args.skip_cpu:
        x_mixed, _, f_mixed, _ = s.get_state()
    s.close()

    # ---- the FP64 form on the same workload and window (half list: its pair arithmetic is FP64)
    fp64 = None
    x64 = f64 = None
    if not args.no_fp64:
        s64, m64 = timed_run(ljmd.LJ_FP64, ljmd.LJ_LIST_HALF, False)
        p64 = m64["prof"]
        e64 = m64["st1"]["list_entries"]
        f64_ms = p64["force_ms"] / max(p64["force_launches"], 1)
        b64, stored64, fl64 = force_kernel_work(N, e64, "fp64")
        fp64 = {"value": job_value(N * args.steps, world, m64["ms"] * 1e-3), "unit": UNIT,
                "ms_per_step": m64["ms"] / args.steps, "steps": args.steps, "warmup": args.warmup, "list": "half",
                "rebuilds": m64["st1"]["rebuilds"] - m64["st0"]["rebuilds"],
                "speedup_mixed_over_fp64": (m64["ms"] / args.steps) / (ms / args.steps),
                "roofline": roofline("k_force_pipe (FP64, half list)", f64_ms, b64, fl64, peaks, FP64_PEAK_TFLOPS,
                                     "fp64", peak_kind),
                "phases": {k: round(p64[k], 3) for k in ("force_ms", "integrate_ms", "rebuild_ms")}}
        if rank == 0 and not args.no_cpu_baseline and not args.skip_cpu:
            x64, _, f64, _ = s64.get_state()
        s64.close()

    # ---- end to end through the public API with host buffers: H2D of the initial state from pinned
    # memory, K steps, D2H of the final state and energies, all inside the timed region
    e2e = None
    if not args.no_e2e:
        s2 = ljmd.System(cutoff=wl["cutoff"], margin=wl["margin"], precision=ljmd.LJ_MIXED,
                         list_form=ljmd.LJ_LIST_AUTO, energy_every=1, stream=stream)
        s2.init_lattice(wl["M"], wl["rho"], wl["T"], seed)
        x0 = torch.empty((N, 3), dtype=torch.float64).pin_memory()
        v0 = torch.empty((N, 3), dtype=torch.float64).pin_memory()
        ljmd.ljmd_get_state(s2.h, x0, v0, None, None, 0)
        xo = torch.empty((N, 3), dtype=torch.float64).pin_memory()
        vo = torch.empty((N, 3), dtype=torch.float64).pin_memory()

        def job():
            ljmd.ljmd_set_state(s2.h, N, s2.box, x0, v0)
            s2.step(wl["dt"], args.steps)
            ljmd.ljmd_get_state(s2.h, xo, vo, None, None, 0)
            s2.energies()

        job()  # untimed: the system's one-time allocations (list, tiles) happen in the first job
        torch.cuda.synchronize()
        # three timed jobs from the same start (identical work); the median is reported, since the
        # host copies' speed varies from job to job on a shared host
        jobs = []
        for _ in range(3):
            barrier()
            t0 = time.perf_counter()
            job()
            torch.cuda.synchronize()
            t_job = time.perf_counter() - t0
            barrier()
            jobs.append(reduce_max(t_job, dist))
        t_e2e = sorted(jobs)[1]
        e2e = {"value": job_value(N * args.steps, world, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": 2 * 24 * N / args.steps, "d2h_bytes_per_step": (2 * 24 * N + 24) / args.steps,
               "jobs_s": [round(t, 5) for t in jobs],
               "note": "set_state from pinned host + K steps + get_state/energies to host, per K-step job; "
                       "median of three timed jobs from the same start, after one untimed job that makes "
                       "the system's allocations"}
        s2.close()

    batched = None if args.no_batch else run_batched(args, stream, world, rank, barrier, peaks, peak_kind)
    replica = None if args.no_replica else run_paper_replica(stream)
    adjoint = None if args.no_adjoint else run_adjoint(stream, peaks, peak_kind)
    truncation = None if args.no_truncation else run_truncation(stream)
    small = None if args.no_small else run_small(stream)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 pair arithmetic, f64 state and sums", "data": "synthetic FCC start, Gaussian velocities",
        "config": {"workload": args.workload, "N": N, "density": wl["rho"], "T": wl["T"], "cutoff": wl["cutoff"],
                   "margin": wl["margin"], "dt": wl["dt"], "list": "half" if half else "full",
                   "parallelism": "replicas x%d" % world,
                   "l2": "inputs larger than L2 (state and list ~%.1f GB)" % ((N * 250 + 4 * entries) / 1e9)},
        "roofline": roof,
        "fp64": fp64,
        "e2e": e2e,
        "gpu_launches": st1["kernel_launches"] - st0["kernel_launches"],
        "clocks": m["clocks"],
        "phases": breakdown,
        "list": {"entries_per_particle": entries / N, "rebuilds": st1["rebuilds"] - st0["rebuilds"],
                 "mean_lifetime_steps": args.steps / max(st1["rebuilds"] - st0["rebuilds"], 1)},
        "energies_final": {"pe_per_particle": pe / N, "ke_per_particle": ke / N, "virial": vir},
        "batched": batched,
        "paper_replica": replica,
        "adjoint": adjoint,
        "truncation": truncation,
        "small_system": small,
        "pair_interactions_per_s": entries * args.steps * world / (ms * 1e-3),
    }
    if rank == 0 and not args.no_cpu_baseline and not args.skip_cpu:
        base, acc = cpu_baseline(wl, args.cpu_seconds, x_mixed, f_mixed, box, x64, f64)
        out["cpu_baseline"] = base
        out["accuracy_vs_oracle"] = acc
        if not args.no_cpu_verlet:
            out["cpu_verlet_list"] = cpu_verlet_list(wl)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return out if rank == 0 else None


def run_paper_replica(stream):
    """The paper's benchmark configuration on one GPU (Sec. 4.5): 500,000 particles (FCC 50^3 x 4) in
    a 100^3 box (rho = 0.5), r_c = 2.5, r_s = 2.8, dt = 0.001, |v| = 0.9 in random directions,
    150 warm-up steps and 1000 timed steps; MUPS = N steps / (1e6 s).  The list rule is the margin/2
    displacement rule and, beside it, the large displacement check of Alg. 2."""
    import torch
    from paper_1012_2677_gb300 import ljmd, synth
    out = {}
    for name, mode in (("half_margin", ljmd.LJ_VALID_HALF_MARGIN), ("half_margin_ldc", ljmd.LJ_VALID_HALF_MARGIN_LDC)):
        with ljmd.System(cutoff=2.5, margin=0.3, precision=ljmd.LJ_MIXED, energy_every=0, stream=stream) as s:
            s.init_lattice(50, 0.5, 1.0, 6)
            x, _, _, _ = s.get_state()
            v = 0.9 * synth.unit_vectors(len(x), 6)
            s.set_validity(mode, 16384)
            s.set_state(x, v, 100.0)
            s.step(0.001, 150)
            torch.cuda.synchronize()
            st0 = s.stats()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(0.001, 1000)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            st1 = s.stats()
        nr = st1["rebuilds"] - st0["rebuilds"]
        out[name] = {"mups": mups(len(x), 1000, ms * 1e-3), "ms_per_step": ms / 1000, "rebuilds": nr,
                     "mean_lifetime_steps": 1000 / max(nr, 1)}
    out["paper_context"] = {"mups_per_xeon_x5570_core": 2.73, "mups_per_power6_process": 1.65,
                            "lifetime_steps_power6": 51.2, "note": "FP64 CPU figures of Tables 2-3 and Sec. 5.2"}
    return out


def run_batched(args, stream, world, rank, barrier, peaks, peak_kind):
    """Batched-replica workload: 256 replicas, N ~ U[500, 50000], rho ~ U[0.3, 0.9], T ~ U[0.7, 1.5]
    (FCC filled then thinned), r_c 2.5, margin 0.3, dt 0.004, mixed form; tiles autotuned, steps
    replayed as a captured 10-step CUDA graph.  Timed with the host clock around one batch call
    (graph replays, one synchronisation at the end); the force kernel's roofline from CUDA events
    around plain launches afterwards."""
    import torch
    from paper_1012_2677_gb300 import ljmd, synth
    n, box, x, v, _ = synth.batch_workload(256, 1000 + 100 * rank)
    K = 10
    steps = max(K, (args.batch_steps // K) * K)
    with ljmd.Batch(n, box, cutoff=2.5, margin=0.3, stream=stream) as b:
        b.set_state(x, v)
        tile, lanes, tune_ms = b.autotune(trials=3)
        b.step(0.004, 2 * K, graph_steps=K)  # warm-up: capture and first replays
        torch.cuda.synchronize()
        st0 = b.stats()
        barrier()
        t0 = time.perf_counter()
        b.step(0.004, steps, graph_steps=K)  # returns after the stream is synchronised
        dt_s = time.perf_counter() - t0
        st1 = b.stats()
        f_ms = b.time_force(trials=5)
    N = int(n.sum())
    bb, stored, fl = force_kernel_work(N, st1["list_entries"], "mixed", energy=False)
    return {"workload": "256 replicas, N in [500, 50000] (%d particles), rho in [0.3, 0.9], T in [0.7, 1.5], "
                        "margin 0.3, dt 0.004" % N,
            "value": N * steps * world / dt_s, "unit": UNIT, "steps": steps, "ms_per_step": dt_s / steps * 1e3,
            "graph_steps": K, "autotuned": {"tile_cells": tile, "lanes": lanes, "cost_ms": round(tune_ms, 4)},
            "rebuilds": st1["rebuilds"] - st0["rebuilds"],
            "gpu_launches": st1["kernel_launches"] - st0["kernel_launches"],
            "roofline": roofline("k_force_batch", f_ms, bb, fl, peaks, FP32_PEAK_TFLOPS, "fp32", peak_kind),
            "timing": "host clock around one ljmd_batch_step call (graph replays, one synchronisation at the end)"}


def run_adjoint(stream, peaks, peak_kind):
    """Differentiable-trajectory workload: 32,000 particles (FCC 20^3 x 4 thinned), rho 0.6, T 1.2,
    50 steps, loss over the last 10, checkpoints every 10; forward + checkpointed reverse pass.  The
    adjoint kernel's roofline from its CUDA-event phase timer."""
    import numpy as np
    import torch
    from paper_1012_2677_gb300 import ljmd, synth
    x, L = synth.fcc_thinned(32000, 0.6, 5)
    v = synth.thermal_velocities(len(x), 1.2, 5)
    res = {}
    for name, prec in (("mixed", ljmd.LJ_MIXED), ("fp64", ljmd.LJ_FP64)):
        with ljmd.System(cutoff=2.5, margin=0.5, precision=prec, energy_every=0, stream=stream) as s:
            s.traj_loss_grad(x, v, L, 0.005, 50, 10, 10)  # warm-up (allocations, first constructions)
            times = []
            for _ in range(3):  # timed without the phase timers (their events perturb small launches)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                loss, gx, gv, gth = s.traj_loss_grad(x, v, L, 0.005, 50, 10, 10)
                times.append(time.perf_counter() - t0)
            t = sorted(times)[1]
            s.set_profiling(True)  # one more call for the adjoint kernel's time
            s.traj_loss_grad(x, v, L, 0.005, 50, 10, 10)
            prof = s.profile()
            st = s.stats()
        a_ms = prof["adjoint_ms"] / max(prof["adjoint_launches"], 1)
        E, n = st["list_entries"], len(x)
        # per list entry 12 flops (difference, r^2, cutoff test); per pair inside r_c (the continuum
        # fraction (r_c / r_s)^3 of the entries) 83 more: u, u', u'', the sigma derivatives, the
        # Hessian-vector row, force and parameter sums.  Bytes: 4 per entry, and per particle the
        # position (16 B mixed, 32 B FP64), w, H w and F (32 B each).
        inner = (2.5 / 3.0) ** 3
        flops = E * (12 + 83 * inner)
        bytes_ = 4 * E + n * ((16 if name == "mixed" else 32) + 96)
        res[name] = {"seconds": t, "particle_steps_per_s": n * 50 / t, "loss": loss,
                     "grad_norm_x0": float(np.linalg.norm(gx)), "dloss_deps": gth[0], "dloss_dsigma": gth[1],
                     "roofline": roofline("k_adjoint_tile", a_ms, bytes_, flops, peaks,
                                          FP32_PEAK_TFLOPS if name == "mixed" else FP64_PEAK_TFLOPS,
                                          "fp32" if name == "mixed" else "fp64", peak_kind,
                                          extra={"launches": prof["adjoint_launches"]})}
    res["note"] = ("forward 50 steps + reverse pass (one Hessian-vector product per state, segments recomputed); "
                   "seconds: median of 3 calls after a warm-up call, host clock with the stream synchronised")
    return res


def run_small(stream):
    """The small FP64 configuration (FCC 10^3 x 4, rho 0.5, T 1, seed 1, dt 0.005, 100 steps, energies
    every step) in both forms, timed with CUDA events after 20 warm-up steps: a size where launch and
    synchronisation costs, not the kernels, set the rate."""
    import torch
    from paper_1012_2677_gb300 import ljmd
    out = {}
    for name, prec in (("fp64", ljmd.LJ_FP64), ("mixed", ljmd.LJ_MIXED)):
        with ljmd.System(cutoff=2.5, margin=0.5, precision=prec, list_form=ljmd.LJ_LIST_AUTO, energy_every=1,
                         stream=stream) as s:
            s.init_lattice(10, 0.5, 1.0, 1)
            s.step(0.005, 20)
            torch.cuda.synchronize()
            st0 = s.stats()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(0.005, 100)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            st1 = s.stats()
            n = s.n
        out[name] = {"value": n * 100 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / 100,
                     "rebuilds": st1["rebuilds"] - st0["rebuilds"],
                     "gpu_launches": st1["kernel_launches"] - st0["kernel_launches"]}
    out["workload"] = "FCC 10^3 x 4 (4,000 particles), rho 0.5, T 1, seed 1, dt 0.005, 100 steps"
    return out


def drift_stats(E, n, dt):
    """(max |E(t) - E(0)| / |E(0)|, rms of (E(t) - E(0)) / |E(0)|, least-squares slope of E / N)."""
    import numpy as np
    e0 = abs(E[0])
    t = np.arange(len(E)) * dt
    return (float(np.abs(E - E[0]).max() / e0), float(np.sqrt(((E - E[0]) ** 2).mean()) / e0),
            float(np.polyfit(t, E / n, 1)[0]))


def run_truncation(stream):
    """Energy conservation of each truncation of the potential (Sec. 2.1: Eq. 2, the constant shift,
    the plain cut) at r_c = 2.5 and 3.0 on the small FP64 configuration (FCC 10^3 x 4, rho 0.5, T 1,
    seed 1, dt 0.005, 1000 steps, FP64 form): drift and slope of the total energy per particle."""
    import torch
    from paper_1012_2677_gb300 import ljmd
    steps, dt = 1000, 0.005
    out = {}
    for rc in (2.5, 3.0):
        for name, mode in (("quadratic", ljmd.LJ_TRUNC_QUADRATIC), ("shift", ljmd.LJ_TRUNC_SHIFT),
                           ("cut", ljmd.LJ_TRUNC_CUT)):
            log = torch.zeros((steps + 8, 4), dtype=torch.float64, device="cuda")
            with ljmd.System(cutoff=rc, margin=0.5, truncation=mode, precision=ljmd.LJ_FP64,
                             list_form=ljmd.LJ_LIST_AUTO, energy_every=1, stream=stream) as s:
                s.init_lattice(10, 0.5, 1.0, 1)
                s.set_energy_log(log)
                s.step(dt, steps)
                n = s.n
            rec = log.cpu().numpy()[:steps + 1]
            mx, rms, slope = drift_stats(rec[:, 1] + rec[:, 2], n, dt)
            out["rc%.1f_%s" % (rc, name)] = {"max_rel_drift": mx, "rms_rel_drift": rms, "slope_per_particle": slope}
    out["workload"] = "FCC 10^3 x 4, rho 0.5, T 1, seed 1, dt 0.005, 1000 steps, FP64 form"
    return out


def _oracle_sample_rate(wl, target_s, x=None, L=None, sample_seed=7):
    """Oracle (all-pairs FP64) on a sample of the workload: forces on S particles against all N, on
    the given state (else the FCC start, displaced).  Returns (rate, cores, description, seconds, idx, F)."""
    import oracle as O
    from paper_1012_2677_gb300 import synth
    if x is None:
        x, L = O.fcc_lattice(wl["M"], wl["rho"])
        x = O.wrap(x + synth.displacements(len(x), 0.05, sample_seed), L)
    N = len(x)
    p = O.LJParams(rc_over_sigma=wl["cutoff"])
    idx = synth.subset(N, 64, sample_seed)
    t0 = time.perf_counter()
    O.forces_sample(x, L, idx, p)
    t_small = time.perf_counter() - t0
    S = int(max(64, min(N, 64 * target_s / max(t_small, 1e-6))))
    idx = synth.subset(N, S, sample_seed + 1)
    t0 = time.perf_counter()
    F = O.forces_sample(x, L, idx, p)
    t = time.perf_counter() - t0
    return S / t, O.num_threads(), "all-pairs FP64 forces on %d of %d particles (%.1f s)" % (S, N, t), t, idx, F


def _force_error(f, idx, F):
    import numpy as np
    rms = float(np.sqrt((F ** 2).sum(1).mean()))
    err = float(np.sqrt(((f[idx] - F) ** 2).sum(1)).max() / rms)
    return {"max_dF_over_rms_F": err, "rms_F": rms, "sample": int(len(idx))}


def cpu_baseline(wl, seconds, x_mixed=None, f_mixed=None, L=None, x64=None, f64=None):
    """The oracle timed on the host cores on a bounded sample; the same sample (forces of the
    mixed form's final state) gives the measured error of the GPU forces against the oracle, and a
    small second sample that of the FP64 form's final state."""
    rate, cores, desc, _, idx, F = _oracle_sample_rate(wl, seconds, x_mixed, L)
    base = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    acc = {}
    if f_mixed is not None:
        acc["mixed"] = _force_error(f_mixed, idx, F)
        acc["mixed"]["tolerance"] = 1e-5
    if x64 is not None:
        import oracle as O
        from paper_1012_2677_gb300 import synth
        idx64 = synth.subset(len(x64), 512, 17)
        acc["fp64"] = _force_error(f64, idx64, O.forces_sample(x64, L, idx64, O.LJParams(rc_over_sigma=wl["cutoff"])))
        acc["fp64"]["tolerance"] = 1e-11
    acc["state"] = "after the timed steps (liquid), forces as the GPU last computed them"
    return base, acc


def cpu_verlet_list(wl, target_steps=None):
    """The paper's Verlet-list method on the host cores in FP64 (oracle/cellverlet.c: cell sort, half
    list, branch-free force with Newton's third law, velocity-Verlet, margin/2 rebuilds) on the full
    workload, a few steps after its first construction."""
    import oracle as O
    from oracle import cellverlet as CV
    x, L = O.fcc_lattice(wl["M"], wl["rho"])
    v = O.init_velocities(len(x), wl["T"], wl["seed"])
    N = len(x)
    steps = target_steps or int(min(100, max(3, 6e7 // N)))
    t0 = time.perf_counter()
    r = CV.run(x, v, L, wl["dt"], steps, wl["margin"], O.LJParams(rc_over_sigma=wl["cutoff"]))
    wall = time.perf_counter() - t0
    return {"value": N * steps / r["seconds"], "unit": UNIT, "cores": O.num_threads(),
            "kind": "cell-list + sorted Verlet list (Alg. 1, 4-6), FP64, OpenMP",
            "sample": "%d particles, %d steps after the first construction (%d constructions in all, %.1f s of "
                      "%.1f s wall)" % (N, steps, r["rebuilds"], r["seconds"], wall),
            "pairs_per_particle": r["pairs"] / N}


def run_reference(args, wl, world, rank):
    """The oracle on the host cores, each step a bounded sample of the workload."""
    if rank != 0:
        return None
    import numpy as np
    import oracle as O
    from paper_1012_2677_gb300 import synth
    x, L = O.fcc_lattice(wl["M"], wl["rho"])
    N = len(x)
    x = O.wrap(x + synth.displacements(N, 0.05, 7), L)
    p = O.LJParams(rc_over_sigma=wl["cutoff"])
    budget = max(30.0, min(150.0, 1.0 * (args.steps + args.warmup)))
    t0 = time.perf_counter()
    O.forces_sample(x, L, synth.subset(N, 16, 1), p)
    per_particle = (time.perf_counter() - t0) / 16
    S = int(max(4, min(N, budget / (args.steps + args.warmup) / max(per_particle, 1e-9))))
    for w in range(args.warmup):
        O.forces_sample(x, L, synth.subset(N, S, 100 + w), p)
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.forces_sample(x, L, synth.subset(N, S, 1000 + k), p)
    t = time.perf_counter() - t0
    value = S * args.steps / t
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic FCC start",
        "config": {"workload": args.workload, "N": N, "density": wl["rho"], "cutoff": wl["cutoff"],
                   "margin": wl["margin"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": "each step: all-pairs FP64 forces on %d of %d particles" % (S, N)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="fcc16m_rho0.5", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-replica", action="store_true")
    ap.add_argument("--no-truncation", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-cpu-verlet", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=100)
    ap.add_argument("--skip-cpu", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_env()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        out = run_reference(args, wl, world, rank)
    else:
        out = run_ours(args, wl, world, rank, local)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
