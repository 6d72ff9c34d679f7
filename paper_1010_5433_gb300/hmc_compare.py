"""The metric's comparison (paper Sec. 4: Metropolis on dH): RHMC
trajectories per hour of the mixed path against the plain fp64 GPU path at
equal acceptance and <|dH|>, on the thermalised 16^4 N_f = 2 workload.

Both arms start from the same thermalised configuration and draw the same
random numbers trajectory by trajectory (the same Philox counters for the
momenta, the heatbath sources and the Metropolis uniform), so the chains
stay paired until an accept/reject decision differs.  Reported per arm:
acceptance, <|dH|>, <dH>, <exp(-dH)> with naive standard errors (the
trajectories are treated as independent), the mean event-timed seconds per
trajectory and trajectories per hour.

  python -m paper_1010_5433_gb300.hmc_compare [--trajectories 100]
         [--n-outer 10 ...] [--md-links 12] [--fp64-n-outer 10] [--n-pf 1 2 ...] [--no-fp64]
"""
import argparse
import json
import time

import numpy as np


def stats(trajs):
    dh = np.array([t.dH for t in trajs])
    acc = np.array([t.accepted for t in trajs], dtype=float)
    sec = np.array([t.seconds for t in trajs])
    n = len(dh)
    e = np.exp(-dh)
    return {"n": n, "acceptance": round(float(acc.mean()), 4),
            "acceptance_err": round(float(np.sqrt(acc.mean() * (1 - acc.mean()) / n)), 4),
            "mean_abs_dH": round(float(np.abs(dh).mean()), 5), "mean_abs_dH_err": round(float(np.abs(dh).std(ddof=1) / np.sqrt(n)), 5),
            "mean_dH": round(float(dh.mean()), 5), "mean_dH_err": round(float(dh.std(ddof=1) / np.sqrt(n)), 5),
            "mean_exp_minus_dH": round(float(e.mean()), 4), "mean_exp_minus_dH_err": round(float(e.std(ddof=1) / np.sqrt(n)), 4),
            "seconds_per_traj": round(float(sec.mean()), 4), "traj_per_hour": round(3600.0 / float(sec.mean()), 1),
            "cg_iterations_per_traj": round(float(np.mean([t.cg_iterations for t in trajs])), 1),
            "plaquette_mean": round(float(np.mean([t.plaq for t in trajs])), 5)}


def run(trajectories=100, n_outers=(20,), fp64_n_outer=None, md_links="12", warmup=5, log=print, n_pfs=(1,),
        fp64=True, splits=()):
    """Arms: the mixed path at every n_outer x n_pf (n_pf pseudo-fermions,
    s = 1 / (2 n_pf) each: the paper's multiple pseudo-fermions, Sec. 2), and
    the fp64 path at fp64_n_outer (default: the first n_outer) with one;
    splits: (n_outer, n_mid, n_gauge) of mixed-path arms with the Hasenbusch
    mass split of workload.py (ratio term outside, heavy term on the middle
    level)."""
    import torch

    from . import stag, workload as W
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    w = W.WORKLOAD
    dims = tuple(w["dims"])
    V = int(np.prod(dims))
    rats = W.rationals()
    seed = w["seed"]
    md_prec = W.MD_LINKS[md_links][0]
    ctx = stag.stag_create(dims, True, stream.cuda_stream)
    out = {"workload": w["workload"], "thermalisation": {}, "arms": {}}
    try:
        t0 = time.time()
        plaq = W.thermalise(stag, ctx, rats, seed, md_prec)
        for k in range(warmup):
            stag.stag_md_trajectory(ctx, W.make_hmc(stag, rats, md_prec, seed, 25_000 + k))
        out["thermalisation"] = {"quenched": w["quenched_thermalisation"], "dynamical": w["dynamical_thermalisation"],
                                 "n_outer": w["thermalisation_n_outer"], "warmup": warmup,
                                 "plaquette_by_decade": [round(float(np.mean(plaq[i:i + 10])), 5)
                                                         for i in range(0, len(plaq), 10)],
                                 "seconds": round(time.time() - t0, 1)}
        start = np.empty(4 * V * 18)
        stag.stag_store_gauge(ctx, start)
        arms = [("mixed", md_prec, no, npf) for npf in n_pfs for no in n_outers]
        if fp64:
            arms.append(("fp64", stag.STAG_FP64, fp64_n_outer or n_outers[0], 1))
        if splits:
            ratio, heavy = W.split_rationals()
        for no, nm, ng in splits:
            stag.stag_load_gauge(ctx, start)
            trajs = [stag.stag_md_trajectory(ctx, W.make_hmc_split(stag, ratio, heavy, md_prec, seed, 30_000 + k, no, nm,
                                                                   ng)) for k in range(trajectories)]
            key = f"split_n_outer_{no}_n_mid_{nm}_n_gauge_{ng}"
            out["arms"][key] = dict(stats(trajs), prec=int(md_prec), n_outer=no, n_mid=nm, n_gauge=ng,
                                    dH=[round(t.dH, 5) for t in trajs])
            log(f"{key}: " + json.dumps({k: v for k, v in out["arms"][key].items() if k != "dH"}))
        for name, prec, no, npf in arms:
            stag.stag_load_gauge(ctx, start)
            r_arm = rats if npf == 1 else W.rationals(npf)
            trajs = []
            for k in range(trajectories):
                trajs.append(stag.stag_md_trajectory(ctx, W.make_hmc(stag, r_arm, prec, seed, 30_000 + k, n_outer=no,
                                                                     n_pf=npf)))
            key = f"{name}_n_outer_{no}" + (f"_n_pf_{npf}" if npf > 1 else "")
            out["arms"][key] = dict(stats(trajs), prec=int(prec), n_outer=no, n_pf=npf,
                                    dH=[round(t.dH, 5) for t in trajs])
            log(f"{key}: " + json.dumps({k: v for k, v in out["arms"][key].items() if k != "dH"}))
    finally:
        stag.stag_destroy(ctx)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--trajectories", type=int, default=100)
    ap.add_argument("--n-outer", type=int, nargs="+", default=[20])
    ap.add_argument("--fp64-n-outer", type=int, default=None)
    ap.add_argument("--md-links", default="12")
    ap.add_argument("--n-pf", type=int, nargs="+", default=[1])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--split", nargs="*", default=[], help="n_outer:n_mid:n_gauge of Hasenbusch-split arms")
    ap.add_argument("--no-plain", action="store_true", help="only the split arms (and fp64 unless --no-fp64)")
    a = ap.parse_args()
    splits = tuple(tuple(int(v) for v in x.split(":")) for x in a.split)
    print(json.dumps(run(a.trajectories, () if a.no_plain else tuple(a.n_outer), a.fp64_n_outer or a.n_outer[0],
                         a.md_links, n_pfs=tuple(a.n_pf), fp64=not a.no_fp64, splits=splits)))
