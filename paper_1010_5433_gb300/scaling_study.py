"""Volume scaling on GB300 at the paper's lattice shapes (Sec. 5 Table 2 for
the Dslash; Sec. 6 Fig. 3 and Tables 3-4 for the RHMC update).

Dslash: D_oe on 4 x 16^3, 32 x 32^3 and 4 x 48^3 (time extent first, as
the paper writes them) in every link format, with warm L2 (back-to-back
launches) and cold L2 (a 512 MB write before every launch), reported as
algorithmic GB/s and as a fraction of the measured copy bandwidth.

RHMC: trajectories per hour of the mixed path (fp32 MD on 12-real links,
fp64 heatbath and Metropolis) and of the fp64 path on L_s^3 x 4 lattices at
the paper's two masses: am = 1.0 with L_s = 32, 48, 64 and am = 0.01335 with
L_s = 16, 32, 48.  The paper states neither N_f, beta nor the integrator of
those runs; here N_f = 2 (one pseudo-fermion), beta = 5.6, tau = 1,
n_outer = 10 x n_gauge = 5, MD rationals of 6 (high mass) and 12 (low mass)
poles, 10- and 24-pole heatbath/Metropolis rationals.  Each lattice starts
hot, takes 10 quenched and 3 dynamical trajectories, then the timed ones.

  python -m paper_1010_5433_gb300.scaling_study [--dslash] [--rhmc] [--trajectories 3]
"""
import argparse
import json
import os
import time

import numpy as np

TABLE2 = [(16, 16, 16, 4), (32, 32, 32, 32), (48, 48, 48, 4)]      # (x, y, z, t)
TABLE3 = [("high", 1.0, 32), ("high", 1.0, 48), ("high", 1.0, 64),
          ("low", 0.01335, 16), ("low", 0.01335, 32), ("low", 0.01335, 48)]


def hbm():
    p = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    return json.load(open(p))["hbm_gbs"] if os.path.exists(p) else 6800.0


def dslash_table(reps=20):
    from . import dslash_bench
    out = []
    for dims in TABLE2:
        for flush in (False, True):
            r = dslash_bench.run(dims, (1, 2, 3, 0), 1, reps, hbm(), flush_l2=flush)
            r["paper_shape"] = f"{dims[3]}x{dims[0]}^3"
            out.append(r)
    return out


def rhmc_point(kind, mass, ls, trajectories, seed=0x5A0030):
    import torch

    import synthetic as syn
    from . import rational, stag
    dims = (ls, ls, ls, 4)
    V = int(np.prod(dims))
    rats = {k: rational.load(f"t3_{kind}_{k}") for k in ("md", "met", "hb")}
    stream = torch.cuda.current_stream()
    ctx = stag.stag_create(dims, True, stream.cuda_stream)

    def hmc(prec, counter, n_flavours=1):
        p = stag.stag_hmc()
        p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = 5.6, 1.0, 10, 5, n_flavours
        fl = p.flavour[0]
        fl.mass, fl.n_pf = mass, 1
        fl.hb, fl.md, fl.met = rats["hb"].to_abi(), rats["md"].to_abi(), rats["met"].to_abi()
        p.tol_md, p.tol_met, p.max_iter, p.md_prec = 1e-8, 1e-12, 40000, prec
        p.seed, p.counter = seed + ls, counter
        return p

    res = {"lattice": f"{ls}^3x4", "mass": mass}
    try:
        stag.stag_load_gauge(ctx, np.ascontiguousarray(syn.haar_gauge(dims, seed + ls)).reshape(-1).view(np.float64))
        for k in range(10):
            stag.stag_md_trajectory(ctx, hmc(stag.STAG_FP32_12, 1000 + k, n_flavours=0))
        for k in range(3):
            stag.stag_md_trajectory(ctx, hmc(stag.STAG_FP32_12, 2000 + k))
        start = np.empty(4 * V * 18)
        stag.stag_store_gauge(ctx, start)
        for name, prec in (("mixed", stag.STAG_FP32_12), ("fp64", stag.STAG_FP64)):
            stag.stag_load_gauge(ctx, start)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            trajs = [stag.stag_md_trajectory(ctx, hmc(prec, 3000 + k)) for k in range(trajectories)]
            dt = (time.perf_counter() - t0) / trajectories
            res[name] = {"seconds_per_traj": round(dt, 3), "traj_per_hour": round(3600 / dt, 1),
                         "cg_iterations_per_traj": int(np.mean([t.cg_iterations for t in trajs])),
                         "mean_abs_dH": round(float(np.mean([abs(t.dH) for t in trajs])), 4),
                         "accepted": [t.accepted for t in trajs],
                         "site_updates_per_second": round(V / dt, 1)}
        res["speedup_mixed_vs_fp64"] = round(res["fp64"]["seconds_per_traj"] / res["mixed"]["seconds_per_traj"], 3)
    finally:
        stag.stag_destroy(ctx)
    return res


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--dslash", action="store_true")
    ap.add_argument("--rhmc", action="store_true")
    ap.add_argument("--trajectories", type=int, default=3)
    a = ap.parse_args()
    if a.dslash or not a.rhmc:
        for r in dslash_table():
            print(json.dumps({"dslash": r}), flush=True)
    if a.rhmc or not a.dslash:
        for kind, mass, ls in TABLE3:
            print(json.dumps({"rhmc": rhmc_point(kind, mass, ls, a.trajectories)}), flush=True)
