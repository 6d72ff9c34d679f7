"""Independent chains of uneven volumes: one batched trajectory call per step
(every solve of all chains in one persistent launch) against the same chains
advanced one after another, from identical fields with identical random
numbers.  Default workload: 2 x 8^4, 2 x 12^4, 2 x 16^4, 2 x 16^3 x 8, Nf = 2,
m = 0.05, beta = 5.5, 12-pole MD rational, fp32 MD with fp64 reliable updates.

  python -m paper_1010_5433_gb300.batch_bench [--steps 3] [--warmup 1]
"""
import argparse
import json
import time

import numpy as np

CHAINS = [(8, 8, 8, 8)] * 2 + [(12, 12, 12, 12)] * 2 + [(16, 16, 16, 16)] * 2 + [(16, 16, 16, 8)] * 2


def run(chains=CHAINS, mass=0.05, beta=5.5, n_outer=10, n_gauge=5, steps=3, warmup=1, therm=2,
        rat_prefix="c4", seed=0x5A0004):
    import torch

    import synthetic as syn

    from . import rational, stag
    rats = {k: rational.load(f"{rat_prefix}_{k}") for k in ("md", "met", "hb")}
    stream = torch.cuda.current_stream()

    def hmc(k, counter, **kw):
        p = stag.stag_hmc()
        p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = beta, 1.0, n_outer, n_gauge, 1
        fl = p.flavour[0]
        fl.mass, fl.n_pf = mass, 1
        fl.hb, fl.md, fl.met = rats["hb"].to_abi(), rats["md"].to_abi(), rats["met"].to_abi()
        p.tol_md, p.tol_met, p.max_iter, p.md_prec = 1e-8, 1e-12, 20000, stag.STAG_FP32
        p.seed, p.counter = seed + k, counter
        for a, v in kw.items():
            setattr(p, a, v)
        return p

    n = len(chains)
    bat = [stag.stag_create(d, True, stream.cuda_stream) for d in chains]
    seq = [stag.stag_create(d, True, stream.cuda_stream) for d in chains]
    out = {"workload": " + ".join("x".join(map(str, d)) for d in chains), "mass": mass, "beta": beta,
           "n_outer": n_outer, "n_gauge": n_gauge, "chains": n,
           "sites": int(sum(np.prod(d) for d in chains))}
    try:
        # thermalise every chain once (warm-up without accept/reject), copy into both sets
        fields = []
        for k, d in enumerate(chains):
            u0 = syn.near_identity_gauge(d, seed + k)
            stag.stag_load_gauge(bat[k], np.ascontiguousarray(u0).reshape(-1).view(np.float64))
            for j in range(10):
                stag.stag_md_trajectory(bat[k], hmc(k, 10_000 + j, n_flavours=0, no_metropolis=1))
            for j in range(therm):
                stag.stag_md_trajectory(bat[k], hmc(k, 20_000 + j, no_metropolis=1))
            f = np.empty(4 * int(np.prod(d)) * 18)
            stag.stag_store_gauge(bat[k], f)
            stag.stag_load_gauge(seq[k], f)
            fields.append(f)
        res = {}
        for mode in ("batched", "sequential"):
            dh, acc, its = [], [], []
            phases = np.zeros(4)
            for step in range(warmup + steps):
                if step == warmup:
                    torch.cuda.synchronize()
                    if mode == "batched":
                        stag.stag_profile_begin(bat[0], 1 << 20)
                    t0 = time.perf_counter()
                ps = [hmc(k, step) for k in range(n)]
                if mode == "batched":
                    outs = stag.stag_md_trajectory_batch(bat, ps)
                else:
                    outs = [stag.stag_md_trajectory(seq[k], ps[k]) for k in range(n)]
                if step >= warmup:
                    dh += [o.dH for o in outs]
                    acc += [o.accepted for o in outs]
                    its += [o.cg_iterations for o in outs]
                    # phase times: the batch's own (the same in every record), or summed over chains
                    for o in (outs[:1] if mode == "batched" else outs):
                        phases += [o.t_heatbath, o.t_fermion, o.t_gauge, o.t_metropolis]
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            res[mode] = {"seconds": dt, "traj_per_hour": n * steps * 3600.0 / dt,
                         "mean_abs_dH": float(np.mean(np.abs(dh))), "acceptance": float(np.mean(acc)),
                         "cg_iterations_per_traj": float(np.mean(its)),
                         "phase_seconds": dict(zip(("heatbath", "fermion", "gauge", "metropolis"),
                                                   [round(float(x), 4) for x in phases]))}
            if mode == "batched":
                pr = stag.stag_profile_read(bat[0], stag.STAG_PK_BATCH)
                if pr.sampled:
                    us = pr.sampled_ms * 1e3 / pr.sampled
                    res[mode]["batched_kernel"] = {"iterations": pr.sampled, "us_per_iteration": us,
                                                   "bytes_per_iteration": pr.bytes_per_launch,
                                                   "GBps": pr.bytes_per_launch / (us * 1e-6) / 1e9}
                names = ("phase1", "barrier1", "phase2", "barrier2", "alpha", "phase3", "barrier3", "beta")
                res[mode]["batched_kernel_phases_us"] = {
                    "fp32": dict(zip(names, [round(x, 1) for x in stag.stag_profile_batch_phases(bat[0], 1)])),
                    "float_float": dict(zip(names, [round(x, 1) for x in stag.stag_profile_batch_phases(bat[0], 0)]))}
                stag.stag_profile_begin(bat[0], 0)
                res[mode]["launch_shape"] = {
                    name: dict(zip(("index", "threads_per_block", "blocks_per_sm"), stag.stag_batch_shape(bat[0], p)))
                    for name, p in (("fp32", stag.STAG_FP32), ("fp64", stag.STAG_FP64))}
        out.update(res)
        out["speedup"] = res["batched"]["traj_per_hour"] / res["sequential"]["traj_per_hour"]
        out["steps"], out["warmup"] = steps, warmup
    finally:
        for c in bat + seq:
            stag.stag_destroy(c)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--n-outer", type=int, default=10)
    a = ap.parse_args()
    print(json.dumps(run(steps=a.steps, warmup=a.warmup, n_outer=a.n_outer)))
