"""Benchmark of the staggered RHMC hot path on GB300.

One step = one RHMC trajectory (heatbath, minimum-norm MD with the fermion
force from the multi-shift CG, Metropolis) on the 16^4, N_f = 2, m = 0.02,
beta = 5.6 workload: 12-pole MD rational in fp32 with fp64 reliable updates,
fp64 heatbath and Metropolis inversions (24 poles), 10 outer steps with 5
gauge substeps per fermion half step (acceptance 0.85), tau = 1.  Synthetic data: a Haar-random start thermalised
by the recipe of paper_1010_5433_gb300/workload.py (quenched, then 100
dynamical trajectories) and the warm-up trajectories.

Prints one JSON line: trajectories/hour of the mixed path (value), the
fp64 path from the same configuration with the same random numbers (paired
trajectories), the end-to-end figure through host buffers (the timed
trajectories replayed), the roofline of the dominant kernel measured live
with CUDA events, the 48^4 Dslash roofline point (inputs larger than L2),
the oracle's CPU baseline and the SM clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")    # the CPU baseline runs on one core

import argparse
import json
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash HBM GB/s (% peak); RHMC trajectories/hour mixed+batched vs FP64 at equal ΔH"
from paper_1010_5433_gb300.workload import MD_LINKS, WORKLOAD, make_hmc  # noqa: E402
ROOFLINE_POINT_DIMS = (48, 48, 48, 48)
L2_FLUSH_BYTES = 512 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling clocks and throttle reasons every 200 ms.  The
    tool's start-up (NVML initialisation) can hold the driver for a few
    hundred ms, so the caller waits for the first sample before it starts the
    timed region and then keeps only the samples taken inside it."""

    def __init__(self, index):
        self.index = index
        self.lines = []                  # (host time, csv line)
        self.proc = None
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout=5.0):
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.02)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if self.window:
            inside = [x for x in lines if self.window[0] <= x[0] <= self.window[1]]
            lines = inside or lines
        for _, ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- replicas (N > 1)
# One independent chain per rank, no data-path collective: the job's rate is
# every rank's trajectories over the slowest rank's time.
def replica_seed(seed, rank):
    return seed + 1000 * rank


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, seconds):
    """Trajectories per hour of the whole job."""
    return world * steps / seconds * 3600.0


def workload_config(world):
    """The workload both arms report (the GPU arm adds how it ran)."""
    return {"workload": WORKLOAD["workload"], "lattice": "x".join(str(d) for d in WORKLOAD["dims"]),
            "global_batch": world, "parallelism": f"replicas{world}" if world > 1 else "single"}


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_1010_5433_gb300 import stag, workload

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOAD
    dims = tuple(w["dims"])
    V = int(np.prod(dims))
    rats = workload.rationals()
    seed = replica_seed(w["seed"], rank)
    ctx = stag.stag_create(dims, True, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    md_prec = MD_LINKS[args.md_links][0]

    # start: Haar-random links, quenched then dynamical thermalisation, then the warm-up trajectories
    t_therm = time.time()
    therm_plaq = workload.thermalise(stag, ctx, rats, seed, md_prec)
    t_therm = time.time() - t_therm
    counter = 0
    warm = []
    for k in range(args.warmup):
        warm.append(stag.stag_md_trajectory(ctx, make_hmc(stag, rats, md_prec, seed, counter)))
        counter += 1
    start_field = np.empty(4 * V * 18)
    stag.stag_store_gauge(ctx, start_field)
    c0 = counter            # both arms and the end-to-end run draw from here on

    def timed(prec, steps, profile):
        if profile:
            stag.stag_profile_begin(ctx, 1)
        launches0 = stag.stag_launch_count(ctx)
        trajs = []
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            clk.wait_first()                  # the sampler's start-up stays outside the timed region
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push(f"timed_{'fp64' if prec == 0 else 'mixed'}")
            t_in = time.perf_counter()
            e0.record(stream)
            for k in range(steps):
                flush.zero_()                 # inputs fit in L2: flush between trajectories
                trajs.append(stag.stag_md_trajectory(ctx, make_hmc(stag, rats, prec, seed, c0 + k)))
            e1.record(stream)
            torch.cuda.synchronize()
            clk.window = (t_in, time.perf_counter())
            torch.cuda.nvtx.range_pop()
        if world > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1)
        launches = stag.stag_launch_count(ctx) - launches0
        prof = None
        if profile:
            prof = [stag.stag_profile_read(ctx, kk) for kk in PROFILE_KINDS]
            stag.stag_profile_begin(ctx, 0)
        return ms, trajs, clk.summary(), launches, prof

    # ---- the mixed path (headline)
    ms, trajs, clocks, launches, prof = timed(md_prec, args.steps, True)
    ms = max_over_ranks(ms, world, dev)
    value = job_rate(world, args.steps, ms / 1e3)
    # ---- the plain fp64 path from the same configuration with the same random numbers
    stag.stag_load_gauge(ctx, start_field)
    steps64 = max(2, args.steps // 2)
    ms64, trajs64, _, _, _ = timed(stag.STAG_FP64, steps64, False)
    ms64 = max_over_ranks(ms64, world, dev)
    value64 = job_rate(world, steps64, ms64 / 1e3)
    # ---- end to end through the C ABI with host buffers (pinned), copies timed:
    # the timed mixed trajectories replayed from the same start with the same counters
    host = torch.empty(4 * V * 18, dtype=torch.float64, pin_memory=True)
    host.copy_(torch.from_numpy(start_field))
    hnp = host.numpy()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    e2e_trajs = []
    for k in range(args.steps):
        stag.stag_load_gauge(ctx, hnp)                                   # H2D of the configuration
        e2e_trajs.append(stag.stag_md_trajectory(ctx, make_hmc(stag, rats, md_prec, seed, c0 + k)))
        stag.stag_store_gauge(ctx, hnp)                                  # D2H of the updated configuration
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = job_rate(world, args.steps, e2e_s)

    # ---- roofline of the dominant kernel, from the live sampled events
    hbm, peak_kind = peaks()
    names = PROFILE_NAMES
    kern = []
    for nm, pr in zip(names, prof):
        avg_ms = pr.sampled_ms / max(pr.sampled, 1)
        kern.append({"kernel": nm, "launches": pr.launches, "sampled": pr.sampled, "avg_us": avg_ms * 1e3,
                     "bytes_per_launch": pr.bytes_per_launch, "est_total_ms": avg_ms * pr.launches,
                     "achieved_gbs": pr.bytes_per_launch / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0})
    kern = [k for k in kern if k["launches"] > 0]
    dom = max(kern, key=lambda k: k["est_total_ms"])
    traffic = NCU_TRAFFIC.get(dom["kernel"])
    roofline = {"bound": "hbm", "kernel": dom["kernel"], "achieved": round(dom["achieved_gbs"], 1), "peak": hbm,
                "unit": "GB/s", "frac": round(dom["achieved_gbs"] / hbm, 4),
                "traffic": traffic["bytes_per_unit"] if traffic else None,
                "traffic_source": traffic["source"] if traffic else None,
                "peak_source": peak_kind,
                "note": "unit = one solver iteration; 16^4 fields are L2-resident inside a trajectory; achieved = "
                        "the multi-shift CG iteration's algorithmic bytes (2 link passes + (8 + 4 n_live) spinor "
                        "passes) / CUDA-event time of every persistent launch on the context's stream divided by "
                        "its iterations; the fp32 iterations (MD solves) and the float-float ones (heatbath, "
                        "Metropolis) are timed apart",
                "kernels": kern}

    point = dslash_roofline_point(hbm) if rank == 0 else None
    force_point = force_dslash_point(hbm, clocks.get("sm_max_mhz")) if rank == 0 else None
    asq_point = asqtad_dslash_point(hbm) if rank == 0 else None
    stag.stag_destroy(ctx)
    chains = batched_chains() if world == 1 else None

    dh = [t.dH for t in trajs]
    dh64 = [t.dH for t in trajs64]
    paired = {"trajectories": steps64,
              "mean_abs_dH": [float(np.mean(np.abs(dh[:steps64]))), float(np.mean(np.abs(dh64)))],
              "acceptance": [float(np.mean([t.accepted for t in trajs[:steps64]])),
                             float(np.mean([t.accepted for t in trajs64]))],
              "max_abs_dH_difference": float(np.max(np.abs(np.array(dh[:steps64]) - np.array(dh64))))}
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "trajectories/hour",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(workload_config(world), l2="flushed between steps", md_links=MD_LINKS[args.md_links][1]),
        "roofline": roofline,
        "e2e": {"value": round(e2e, 2), "unit": "trajectories/hour", "h2d_bytes_per_step": V * 4 * 18 * 8,
                "d2h_bytes_per_step": V * 4 * 18 * 8},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "trajectories": {"mixed": {"dH": [round(x, 5) for x in dh], "accepted": [t.accepted for t in trajs],
                                   "mean_abs_dH": float(np.mean(np.abs(dh))),
                                   "cg_iterations_per_traj": float(np.mean([t.cg_iterations for t in trajs])),
                                   "reliable_updates_per_traj": float(np.mean([t.reliable_updates for t in trajs])),
                                   "seconds_breakdown": {k: round(float(np.mean([getattr(t, "t_" + k) for t in trajs])), 4)
                                                         for k in ("heatbath", "fermion", "gauge", "metropolis")},
                                   "plaquette": trajs[-1].plaq},
                         "fp64": {"value": round(value64, 2), "unit": "trajectories/hour", "steps": steps64,
                                  "arithmetic": "FP64 path: float-float (hi + lo floats, ~48-bit) solver iterations "
                                                "with IEEE fp64 sums and scalars, fp64 gauge force and link update",
                                  "dH": [round(x, 5) for x in dh64], "accepted": [t.accepted for t in trajs64],
                                  "mean_abs_dH": float(np.mean(np.abs(dh64))),
                                  "cg_iterations_per_traj": float(np.mean([t.cg_iterations for t in trajs64])),
                                  "seconds_breakdown": {k: round(float(np.mean([getattr(t, "t_" + k) for t in trajs64])), 4)
                                                        for k in ("heatbath", "fermion", "gauge", "metropolis")}},
                         "paired_mixed_vs_fp64": paired,
                         "speedup_mixed_vs_fp64": round(value / value64, 3),
                         "warmup_dH": [round(t.dH, 4) for t in warm],
                         "thermalisation": {"plaquette_by_decade": [round(float(np.mean(therm_plaq[i:i + 10])), 5)
                                                                    for i in range(0, len(therm_plaq), 10)],
                                            "seconds": round(t_therm, 1)},
                         "e2e_replays_timed": all(a.dH == b.dH for a, b in zip(trajs, e2e_trajs)),
                         "e2e_max_abs_dH_difference": max(abs(a.dH - b.dH) for a, b in zip(trajs, e2e_trajs))},
        "dslash_roofline_point": point,
        "force_dslash_point": force_point,
        "asqtad_dslash_point": asq_point,
        "batched_chains": chains,
    }
    return out


# kernels whose live timing the library records (STAG_PK_*): the three-kernel
# iteration's kernels, and the persistent solver in fp32 arithmetic (the MD
# solves) and in float-float (the heatbath and Metropolis solves)
PROFILE_KINDS = (0, 1, 2, 3, 5)
PROFILE_NAMES = ("dslash_oe", "dslash_eo_A", "update", "persistent_iteration_fp32", "persistent_iteration_ff")

# DRAM traffic of the dominant kernel per unit (one solver iteration) from an
# ncu capture of the same kernel on the same 16^4 lattice; empty once the
# kernel has changed since the capture.  The capture is cold-cache (ncu
# flushes caches between passes): one read of the working set, then L2 hits.
NCU_TRAFFIC = {
    "persistent_iteration_fp32": {
        "bytes_per_unit": 840685,
        "source": "ncu --set full of k_ms_persistent<float, FMT_F32_12, 1, 1, 256> on 16^4: one whole "
                  "40-iteration solve of the 12-pole MD rational (solve_bench --prec 2 --tol 0.11), "
                  "dram__bytes_read.sum 33.18 MB + dram__bytes_write.sum 0.44 MB per launch / 40 iterations",
    },
}


def batched_chains():
    """The 8-chain workload (2x8^4, 2x12^4, 2x16^4, 2x16^3x8, Nf=2, m=0.05,
    beta=5.5): one batched trajectory call per step against the same chains
    one after another, from identical fields with identical random numbers."""
    from paper_1010_5433_gb300 import batch_bench
    r = batch_bench.run(steps=2, warmup=1)
    b, q = r["batched"], r["sequential"]
    return {"workload": r["workload"], "batched_traj_per_hour": round(b["traj_per_hour"], 1),
            "sequential_traj_per_hour": round(q["traj_per_hour"], 1), "speedup": round(r["speedup"], 3),
            "acceptance": [b["acceptance"], q["acceptance"]], "mean_abs_dH": [b["mean_abs_dH"], q["mean_abs_dH"]],
            "batched_kernel": b.get("batched_kernel"), "launch_shape": b.get("launch_shape")}


def dslash_roofline_point(hbm):
    """Standalone D_oe at 48^4 (fp32 links 382 MB: larger than L2) in every
    precision, CUDA-event timed over 20 launches after 3 warm-ups."""
    from paper_1010_5433_gb300 import dslash_bench
    return dslash_bench.run(ROOFLINE_POINT_DIMS, (1, 2, 3, 0), 1, 20, hbm)


def asqtad_dslash_point(hbm):
    """The improved (asqtad) operator's D_oe at 48^4, fp32 fat and Naik
    links: 8 + 8 links of 72 B and the two spinors, 1200 B per site."""
    from paper_1010_5433_gb300 import asqtad_bench
    return asqtad_bench.dslash_point(ROOFLINE_POINT_DIMS, 20, hbm, precs=(1,), rebuild=False)


# the many-source force Dslash of the 2+1-flavour workload: Y_i = D_oe X_i for
# 2 flavours x 2 pseudo-fermions x 15 shifts = 60 sources on 32^3 x 8, bf16
# 12-real links, fp32 spinors
FORCE_POINT_DIMS = (32, 32, 32, 8)
FORCE_POINT_SOURCES = 60
# algorithmic flops per output site: per source 8 hops of an SU(3) matrix
# times a colour vector (66 flops each) and their signed sum (7 vector adds,
# 42 flops); per link the rebuild of row 3 from rows 1-2 (42 flops), once
FLOPS_PER_SITE_SOURCE = 8 * 66 + 42
FLOPS_PER_SITE_LINKS = 8 * 42
# FP32 peak without tensor cores: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock
FP32_LANES = 152 * 128


def force_dslash_point(hbm, sm_mhz):
    """The 60-source bf16-12 Dslash against min(HBM, FP32 ALU): the bound is
    the longer of the algorithmic bytes at the measured copy bandwidth and
    the algorithmic flops at the FP32 peak."""
    from paper_1010_5433_gb300 import dslash_bench
    r = dslash_bench.run(FORCE_POINT_DIMS, (3,), FORCE_POINT_SOURCES, 10, hbm)
    b = r["bf16_12"]
    sites = int(np.prod(FORCE_POINT_DIMS)) // 2
    flops = sites * (FORCE_POINT_SOURCES * FLOPS_PER_SITE_SOURCE + FLOPS_PER_SITE_LINKS)
    mhz = sm_mhz or 2070.0
    fp32_peak = FP32_LANES * 2 * mhz * 1e6
    t_hbm = sites * b["bytes_per_site"] / (hbm * 1e9)
    t_alu = flops / fp32_peak
    t = b["us"] * 1e-6
    return {"lattice": r["lattice"], "sources": FORCE_POINT_SOURCES, "links": "bf16, 12 reals", "us": b["us"],
            "achieved_gbs": b["achieved_gbs"], "achieved_tflops": round(flops / t / 1e12, 2),
            "bound_us": {"hbm": round(t_hbm * 1e6, 2), "fp32_alu": round(t_alu * 1e6, 2)},
            "fp32_peak_tflops": round(fp32_peak / 1e12, 1), "peak_clock_mhz": mhz,
            "frac_of_min_bound": round(max(t_hbm, t_alu) / t, 4)}


# ---------------------------------------------------------------- CPU baseline (the oracle)
def oracle_sample(seed=1, n_it=4):
    """Seconds the oracle (numpy, fp64, as it stands) takes on a bounded
    sample of the 16^4 workload: one multi-shift CG iteration with 12 shifts
    (the mean of n_it), one fermion force, one Wilson force, one link update;
    plus the cores the sample kept busy (process CPU time over wall time)."""
    import synthetic as syn
    from oracle import actions, dirac, integrator, lattice as lat, solvers
    w = WORKLOAD
    dims = tuple(w["dims"])
    u = syn.haar_gauge(dims, seed)
    eta, par = lat.eta(dims), lat.parity(dims)
    b = syn.gaussian_fermion(dims, seed + 1, on_parity=0)
    shifts = list(np.geomspace(1e-5, 3.0, 12))
    try:                                 # BLAS on one thread where the control is installed
        from threadpoolctl import threadpool_limits
        limit = threadpool_limits(1)
    except ImportError:
        limit = None
    wall0, cpu0 = time.perf_counter(), time.process_time()
    t0 = time.perf_counter()
    xs, _, _ = solvers.multishift_cg(lambda v: dirac.a_op(u, v, w["mass"], eta, par, shifts[0]), b, shifts, 0.0,
                                     max_iter=n_it)
    t_iter = (time.perf_counter() - t0) / n_it
    t0 = time.perf_counter()
    actions.fermion_force(u, xs, [1.0] * len(xs), eta, par)
    t_ff = time.perf_counter() - t0
    t0 = time.perf_counter()
    f = actions.wilson_force(u, w["beta"])
    t_gf = time.perf_counter() - t0
    t0 = time.perf_counter()
    integrator.update_links(u, f, 0.01)
    t_up = time.perf_counter() - t0
    cores = (time.process_time() - cpu0) / (time.perf_counter() - wall0)
    if limit is not None:
        limit.restore_original_limits()
    return {"cg_iteration": t_iter, "fermion_force": t_ff, "gauge_force": t_gf, "link_update": t_up,
            "sample_s": n_it * t_iter + t_ff + t_gf + t_up, "cores": cores}


def _oracle_sample_job(seed):
    return oracle_sample(seed)


# lattices of the oracle's Dslash rate: the 4^4, 16^4 and 32^3 x 8 workloads
ORACLE_DSLASH_DIMS = ((4, 4, 4, 4), (16, 16, 16, 16), (32, 32, 32, 8))


def oracle_dslash_rate(reps=3):
    """The oracle's D_oe (numpy, fp64, whole-lattice arrays, as it stands) on
    one core: milliseconds per application and the equivalent GB/s of the
    FP64 Dslash's algorithmic bytes (8 links x 144 B + 2 spinors x 48 B =
    1248 B per output site), best of reps."""
    import synthetic as syn
    from oracle import dirac, lattice as lat
    try:
        from threadpoolctl import threadpool_limits
        limit = threadpool_limits(1)
    except ImportError:
        limit = None
    out = []
    for dims in ORACLE_DSLASH_DIMS:
        u = syn.near_identity_gauge(dims, 3)
        eta, par = lat.eta(dims), lat.parity(dims)
        psi = syn.gaussian_fermion(dims, 4, on_parity=0)
        best = None
        for _ in range(reps):
            t0 = time.perf_counter()
            dirac.d_block(u, psi, eta, par, 1)
            t = time.perf_counter() - t0
            best = t if best is None else min(best, t)
        vh = int(np.prod(dims)) // 2
        out.append({"lattice": "x".join(str(d) for d in dims), "ms": round(best * 1e3, 3),
                    "equivalent_gbs": round(vh * 1248 / best / 1e9, 4)})
    if limit is not None:
        limit.restore_original_limits()
    return out


def traj_seconds(t, per_traj):
    return (per_traj["cg_iterations"] * t["cg_iteration"] + per_traj["fermion_forces"] * t["fermion_force"]
            + per_traj["gauge_forces"] * t["gauge_force"] + per_traj["link_updates"] * t["link_update"])


def cpu_baseline(per_traj, all_cores=True):
    """The oracle's trajectories/hour on the host: the bounded sample timed on
    one core and scaled by the work of one trajectory (per_traj: CG
    iterations, force evaluations, link updates); then, with all_cores, the
    same sample as one independent process per host core at once (spawned,
    so that no process inherits a CUDA context), whose summed rate is the
    host's throughput for independent chains.  `cores` is the processes that
    ran (each one thread, BLAS held to one)."""
    one = oracle_sample(1)
    t1 = traj_seconds(one, per_traj)
    work = (f"{per_traj['cg_iterations']} CG iterations, {per_traj['fermion_forces']} fermion forces, "
            f"{per_traj['gauge_forces']} gauge forces, {per_traj['link_updates']} link updates per trajectory")
    single = {"value": round(3600.0 / t1, 4), "cores": max(1.0, round(one["cores"], 1)), "seconds_per_traj": round(t1, 1),
              "sample": f"16^4: 4 multi-shift CG iterations (12 shifts), 1 fermion force, 1 Wilson force, 1 link "
                        f"update ({one['sample_s']:.1f} s), scaled by {work}"}
    out = {"value": single["value"], "unit": "trajectories/hour", "cores": single["cores"], "kind": "oracle",
           "sample": single["sample"], "seconds_per_traj": single["seconds_per_traj"], "single_core": single,
           "dslash_single_core": oracle_dslash_rate()}
    nproc = os.cpu_count() or 1
    if all_cores and nproc > 1:
        import multiprocessing as mp
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(nproc) as pool:
            res = pool.map(_oracle_sample_job, list(range(1, nproc + 1)))
        wall = time.perf_counter() - t0
        rate = sum(3600.0 / traj_seconds(r, per_traj) for r in res)
        out.update({"value": round(rate, 4), "cores": nproc,
                    "sample": f"{nproc} processes at once (one per host core, nproc = {nproc}), each the "
                              f"single-core sample with its own seed; summed rate ({wall:.1f} s wall)",
                    "seconds_per_traj": round(float(np.mean([traj_seconds(r, per_traj) for r in res])), 1)})
    return out


def work_per_traj(cg_iterations):
    w = WORKLOAD
    no, ng = w["n_outer"], w["n_gauge"]
    return {"cg_iterations": int(cg_iterations), "fermion_forces": 2 * no + 1,
            "gauge_forces": 2 * no * (2 * ng + 1), "link_updates": 2 * no * 2 * ng}


# CG iterations of one 16^4 trajectory of this workload (all solves: MD,
# heatbath, Metropolis), as the mixed path measured them on GB300 (20 816 per
# trajectory over 100 equilibrium trajectories at n_outer = 10); only used to
# scale the reference arm's sample, which runs without a GPU run before it.
REF_CG_ITERATIONS = 20816


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--md-links", default="12", choices=sorted(MD_LINKS),
                    help="link format of the fp32 MD inversions (the paper's: 12 reals)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        per = work_per_traj(REF_CG_ITERATIONS)
        for _ in range(args.warmup):
            pass                                  # the oracle has nothing to warm up
        vals = [cpu_baseline(per, all_cores=False) for _ in range(args.steps)]
        v = float(np.mean([x["value"] for x in vals]))
        cb = dict(vals[-1])
        cb["value"] = round(v, 4)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "trajectories/hour",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": round(3.6e6 / v, 1), "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": workload_config(args.gpus),
                          "cpu_baseline": cb,
                          "e2e": {"value": round(v, 4), "unit": "trajectories/hour", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        per = work_per_traj(out["trajectories"]["mixed"]["cg_iterations_per_traj"])
        out["cpu_baseline"] = cpu_baseline(per)
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
