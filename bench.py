"""Benchmark of the staggered RHMC hot path on GB300.

One step = one RHMC trajectory (heatbath, minimum-norm MD with the fermion
force from the multi-shift CG, Metropolis) on the 16^4, N_f = 2, m = 0.02,
beta = 5.6 workload: 12-pole MD rational in fp32 with fp64 reliable updates,
fp64 heatbath and Metropolis inversions (24 poles), 5 gauge substeps per
fermion half step, tau = 1.  Synthetic data: a Haar-random start thermalised
by quenched trajectories and by the warm-up trajectories themselves.

Prints one JSON line: trajectories/hour of the mixed path (value), the
fp64 path on the same configuration, the end-to-end figure through host
buffers, the roofline of the dominant kernel measured live with CUDA events,
the 48^4 Dslash roofline point (inputs larger than L2), the oracle's CPU
baseline and the SM clocks sampled during the timed region.

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
WORKLOAD = {
    "workload": "RHMC 16^4 Nf=2 unimproved staggered, m=0.02, beta=5.6, tau=1, 2MN n_outer=20 x n_gauge=5, "
                "12-pole MD rational (fp32 + fp64 reliable updates), 24-pole fp64 heatbath/Metropolis",
    "dims": [16, 16, 16, 16], "beta": 5.6, "mass": 0.02, "n_flavours": 2, "n_pf": 1, "tau": 1.0,
    "n_outer": 20, "n_gauge": 5, "tol_md": 1e-8, "tol_met": 1e-12,
    "rationals": {"md": "c2_md", "met": "c2_met", "hb": "c2_hb"},
    "seed": 0x5A0002, "quenched_thermalisation": 40,
}
# Work of one trajectory of this workload, used to scale the oracle's timed
# sample to trajectories/hour: fermion and gauge force evaluations and link
# updates follow from n_outer / n_gauge; CG iterations per solve are the
# workload's measured average (mixed MD solves, fp64 heatbath/Metropolis).
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
    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

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
            self.lines.append(line.strip())

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
        for ln in self.lines:
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


# ---------------------------------------------------------------- GPU path
def make_hmc(stag, rats, prec, seed, counter, n_flavours=1, **kw):
    w = WORKLOAD
    p = stag.stag_hmc()
    p.beta, p.tau, p.n_outer, p.n_gauge = w["beta"], w["tau"], w["n_outer"], w["n_gauge"]
    p.n_flavours = n_flavours
    if n_flavours:
        fl = p.flavour[0]
        fl.mass, fl.n_pf = w["mass"], w["n_pf"]
        fl.hb, fl.md, fl.met = rats["hb"].to_abi(), rats["md"].to_abi(), rats["met"].to_abi()
    p.tol_md, p.tol_met, p.max_iter = w["tol_md"], w["tol_met"], 20000
    p.md_prec = prec
    p.seed, p.counter = seed, counter
    for k, v in kw.items():
        setattr(p, k, v)
    return p


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


# link format of the fp32 MD inversions (the fp64 heatbath / Metropolis
# inversions always use the two-float store): stag_prec value, description.
# The paper stores two rows of every link and rebuilds the third (Sec. 5).
MD_LINKS = {"18": (1, "fp32, 18 reals per link"), "12": (2, "fp32, 12 reals per link (row 3 rebuilt)"),
            "bf16": (3, "bf16, 12 reals per link (row 3 rebuilt), fp32 arithmetic")}


def workload_config(world):
    """The workload both arms report (the GPU arm adds how it ran)."""
    return {"workload": WORKLOAD["workload"], "lattice": "x".join(str(d) for d in WORKLOAD["dims"]),
            "global_batch": world, "parallelism": f"replicas{world}" if world > 1 else "single"}


def run_gpu(args, rank, world, local_rank):
    import torch
    import synthetic as syn
    from paper_1010_5433_gb300 import rational, stag

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOAD
    dims = tuple(w["dims"])
    V = int(np.prod(dims))
    rats = {k: rational.load(v) for k, v in w["rationals"].items()}
    seed = replica_seed(w["seed"], rank)
    ctx = stag.stag_create(dims, True, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    md_prec = MD_LINKS[args.md_links][0]

    # start: Haar-random links, quenched thermalisation (no fermions), then warm-up trajectories
    u0 = syn.haar_gauge(dims, seed)     # [mu, t, z, y, x, 3, 3] = the host layout of the C ABI
    stag.stag_load_gauge(ctx, np.ascontiguousarray(u0).reshape(-1).view(np.float64))
    del u0
    for k in range(w["quenched_thermalisation"]):
        p = make_hmc(stag, rats, md_prec, seed, 10_000 + k, n_flavours=0)
        stag.stag_md_trajectory(ctx, p)
    counter = 0
    warm = []
    for k in range(args.warmup):
        warm.append(stag.stag_md_trajectory(ctx, make_hmc(stag, rats, md_prec, seed, counter)))
        counter += 1
    start_field = np.empty(4 * V * 18)
    stag.stag_store_gauge(ctx, start_field)

    def timed(prec, steps, counter0, profile):
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
            torch.cuda.nvtx.range_push(f"timed_{'fp64' if prec == 0 else 'mixed'}")
            e0.record(stream)
            for k in range(steps):
                flush.zero_()                 # inputs fit in L2: flush between trajectories
                trajs.append(stag.stag_md_trajectory(ctx, make_hmc(stag, rats, prec, seed, counter0 + k)))
            e1.record(stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        if world > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1)
        launches = stag.stag_launch_count(ctx) - launches0
        prof = None
        if profile:
            prof = [stag.stag_profile_read(ctx, kk) for kk in range(4)]
            stag.stag_profile_begin(ctx, 0)
        return ms, trajs, clk.summary(), launches, prof


    # ---- the mixed path (headline)
    ms, trajs, clocks, launches, prof = timed(md_prec, args.steps, counter, True)
    ms = max_over_ranks(ms, world, dev)
    counter += args.steps
    value = job_rate(world, args.steps, ms / 1e3)
    # ---- the plain fp64 path from the same configuration
    stag.stag_load_gauge(ctx, start_field)
    steps64 = max(2, args.steps // 2)
    ms64, trajs64, _, _, _ = timed(stag.STAG_FP64, steps64, 0, False)
    ms64 = max_over_ranks(ms64, world, dev)
    value64 = job_rate(world, steps64, ms64 / 1e3)
    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    host = torch.empty(4 * V * 18, dtype=torch.float64, pin_memory=True)
    host.copy_(torch.from_numpy(start_field))
    hnp = host.numpy()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        stag.stag_load_gauge(ctx, hnp)                                   # H2D of the configuration
        stag.stag_md_trajectory(ctx, make_hmc(stag, rats, md_prec, seed, 5000 + k))
        stag.stag_store_gauge(ctx, hnp)                                  # D2H of the updated configuration
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = job_rate(world, args.steps, e2e_s)

    # ---- roofline of the dominant kernel, from the live sampled events
    hbm, peak_kind = peaks()
    names = ["dslash_oe", "dslash_eo_A", "update", "persistent_iteration"]
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
                        "algorithmic bytes per iteration / CUDA-event time of every persistent launch on the "
                        "context's stream divided by its iterations",
                "kernels": kern}

    point = dslash_roofline_point(hbm) if rank == 0 else None
    stag.stag_destroy(ctx)
    chains = batched_chains() if world == 1 else None

    dh = [t.dH for t in trajs]
    dh64 = [t.dH for t in trajs64]
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
                                  "dH": [round(x, 5) for x in dh64], "accepted": [t.accepted for t in trajs64],
                                  "mean_abs_dH": float(np.mean(np.abs(dh64))),
                                  "cg_iterations_per_traj": float(np.mean([t.cg_iterations for t in trajs64])),
                                  "seconds_breakdown": {k: round(float(np.mean([getattr(t, "t_" + k) for t in trajs64])), 4)
                                                        for k in ("heatbath", "fermion", "gauge", "metropolis")}},
                         "speedup_mixed_vs_fp64": round(value / value64, 3),
                         "warmup_dH": [round(t.dH, 4) for t in warm]},
        "dslash_roofline_point": point,
        "batched_chains": chains,
    }
    return out


# DRAM traffic of the dominant kernel per unit (one solver iteration) from an
# ncu capture of the same kernel on the same 16^4 lattice; None once the
# kernel has changed since the capture.  The capture is cold-cache (ncu
# flushes caches between passes): one read of the working set, then L2 hits.
NCU_TRAFFIC = {
    "persistent_iteration": {
        "bytes_per_unit": round((33.118464e6 + 0.10752e6) / 39),
        "source": "profiles/persistent_fp32_12_16x4_ncu.md: dram__bytes_read+write over one 39-iteration launch "
                  "of k_ms_persistent<float, FMT_F32_12>",
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


# ---------------------------------------------------------------- CPU baseline (the oracle)
def cpu_baseline(per_traj):
    """Times the oracle (numpy, fp64) on a bounded sample of the
    16^4 workload -- multi-shift CG iterations with 12 shifts, one fermion
    force, one Wilson force, one link update -- and scales it by the work of
    one trajectory (per_traj: CG iterations, force evaluations, link updates).
    `cores` is measured: the sample's process CPU time over its wall time."""
    import synthetic as syn
    from oracle import actions, dirac, integrator, lattice as lat, solvers
    w = WORKLOAD
    dims = tuple(w["dims"])
    u = syn.haar_gauge(dims, 1)
    eta, par = lat.eta(dims), lat.parity(dims)
    b = syn.gaussian_fermion(dims, 2, on_parity=0)
    shifts = list(np.geomspace(1e-5, 3.0, 12))
    n_it = 4
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
    # cores actually busy: process CPU time over wall time of the sample
    cores = max(1.0, round((time.process_time() - cpu0) / (time.perf_counter() - wall0), 1))
    if limit is not None:
        limit.restore_original_limits()
    t_traj = (per_traj["cg_iterations"] * t_iter + per_traj["fermion_forces"] * t_ff
              + per_traj["gauge_forces"] * t_gf + per_traj["link_updates"] * t_up)
    sample_s = n_it * t_iter + t_ff + t_gf + t_up
    return {"value": round(3600.0 / t_traj, 4), "unit": "trajectories/hour", "cores": cores, "kind": "oracle",
            "sample": f"16^4: {n_it} multi-shift CG iterations (12 shifts), 1 fermion force, 1 Wilson force, "
                      f"1 link update ({sample_s:.1f} s), scaled by {per_traj['cg_iterations']} CG iterations, "
                      f"{per_traj['fermion_forces']} fermion forces, {per_traj['gauge_forces']} gauge forces, "
                      f"{per_traj['link_updates']} link updates per trajectory",
            "seconds_per_traj": round(t_traj, 1)}


def work_per_traj(cg_iterations):
    w = WORKLOAD
    no, ng = w["n_outer"], w["n_gauge"]
    return {"cg_iterations": int(cg_iterations), "fermion_forces": 2 * no + 1,
            "gauge_forces": 2 * no * (2 * ng + 1), "link_updates": 2 * no * 2 * ng}


# CG iterations of one 16^4 trajectory of this workload (all solves: MD,
# heatbath, Metropolis), as the mixed path measured them on GB300 (40 057 per
# trajectory over the bench's timed trajectories); only used to scale the
# reference arm's sample, which runs without a GPU run before it.
REF_CG_ITERATIONS = 40057


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
        vals = [cpu_baseline(per) for _ in range(args.steps)]
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
