"""Measurements of the improved (asqtad) staggered operator on one GPU: the
Dslash against its algorithmic bytes, the fat-link rebuild, multi-shift
solves and the force, and RHMC trajectories of a 16^4 N_f = 2 workload
(tree-level asqtad, m = 0.02, beta = 5.6, Wilson gauge action) from a start
thermalised with the unimproved operator and then with the improved one.

Algorithmic bytes of one improved Dslash per output site: 8 fat + 8 Naik
links (72 B each in fp32, 144 B as fp64 hi + lo) read once, the input and
output spinor once: 16 x 72 + 2 x 24 = 1200 B (fp32), 16 x 144 + 2 x 48 =
2400 B (fp64).  Times are CUDA events on the launching stream.

  python -m paper_1010_5433_gb300.asqtad_bench [--dslash-dims 48 48 48 48] [--solve-dims 16 16 16 16 32 32 32 32]
         [--trajectories 10] [--warmup 5] [--skip-hmc] [--skip-solve] [--skip-dslash]
"""
import argparse
import json
import time

import numpy as np

LINK_BYTES = {0: 2 * 1152, 1: 2 * 576}
NAMES = {0: "fp64", 1: "fp32"}
WORKLOAD = {
    "workload": "RHMC 16^4 Nf=2 asqtad (tree level, u0=1) staggered, m=0.02, beta=5.6 Wilson gauge, tau=1, "
                "2MN n_outer=10 x n_gauge=5, 14-pole MD rational on [m^2, m^2+64] (fp32 + fp64 reliable updates), "
                "24-pole fp64 heatbath/Metropolis",
    "dims": [16, 16, 16, 16], "beta": 5.6, "mass": 0.02, "u0": 1.0, "n_outer": 10, "n_gauge": 5, "tol_md": 1e-8,
    "tol_met": 1e-12, "rationals": {"md": "asqtad_md", "met": "asqtad_met", "hb": "asqtad_hb"},
    "seed": 0x5A0005, "quenched_thermalisation": 40, "unimproved_thermalisation": 60, "asqtad_thermalisation": 20,
}


def _near_identity_device(torch, dev, V, scale=0.05):
    g = torch.randn(4 * V * 18, dtype=torch.float64, device=dev).mul_(scale)
    gv = g.view(4 * V, 9, 2)
    for k in (0, 4, 8):
        gv[:, k, 0] += 1.0
    return g


def dslash_point(dims, reps=20, hbm_gbs=None, precs=(1, 0), rebuild=True):
    """D_oe with the improved operator in the given precisions (1 fp32, 0
    fp64), back-to-back launches; with rebuild, also the fat-link rebuild."""
    import torch

    from . import stag
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    V = int(np.prod(dims))
    vh = V // 2
    ctx = stag.stag_create(dims, True, stream.cuda_stream)
    res = {"lattice": "x".join(str(d) for d in dims), "reps": reps}
    try:
        g = _near_identity_device(torch, dev, V)
        stag.stag_load_gauge_device(ctx, g)
        stag.stag_set_action(ctx, stag.STAG_ACTION_ASQTAD, 1.0)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for prec in precs:
            dt = torch.float64 if prec == 0 else torch.float32
            s = 48 if prec == 0 else 24
            inp = torch.randn(3 * 2 * vh, dtype=dt, device=dev)
            out = torch.empty_like(inp)
            for _ in range(3):
                stag.stag_dslash(ctx, 1, prec, 1, inp, out)
            e[0].record(stream)
            for _ in range(reps):
                stag.stag_dslash(ctx, 1, prec, 1, inp, out)
            e[1].record(stream)
            torch.cuda.synchronize()
            t = e[0].elapsed_time(e[1]) / reps * 1e-3
            bps = LINK_BYTES[prec] + 2 * s
            gbs = vh * bps / t / 1e9
            r = {"us": round(t * 1e6, 2), "achieved_gbs": round(gbs, 1), "bytes_per_site": bps}
            if hbm_gbs:
                r["frac"] = round(gbs / hbm_gbs, 4)
            res[NAMES[prec]] = r
            del inp, out
        if not rebuild:
            return res
        # the fat-link rebuild: a reload marks the links stale, the next Dslash rebuilds them
        inp = torch.randn(3 * 2 * vh, dtype=torch.float32, device=dev)
        out = torch.empty_like(inp)
        ts = []
        for _ in range(3):
            e[0].record(stream)
            stag.stag_load_gauge_device(ctx, g)
            e[1].record(stream)
            stag.stag_dslash(ctx, 1, 1, 1, inp, out)
            e[2].record(stream)
            stag.stag_dslash(ctx, 1, 1, 1, inp, out)
            e[3].record(stream)
            torch.cuda.synchronize()
            ts.append(e[1].elapsed_time(e[2]) - e[2].elapsed_time(e[3]))
        res["fat_link_rebuild_us"] = round(min(ts) * 1e3, 1)
        res["fat_link_rebuild_links_per_s"] = round(4 * V / (min(ts) * 1e-3), 0)
    finally:
        stag.stag_destroy(ctx)
    return res


def solve_point(dims, mass=0.02, reps=3):
    """fp32 multi-shift solves (fp64 reliable updates) at the MD rational's
    shifts, and the fp32 fermion force of that rational (its own solve, the
    fp32 fat-link rebuild, Y = D_oe X and the reverse pass through the
    staples; the API solve also refines every shift and computes its true
    residual, so the two times are not to be subtracted)."""
    import torch

    from . import rational, stag
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    V = int(np.prod(dims))
    vh = V // 2
    md = rational.load("asqtad_md")
    shifts = list(md.beta)
    ctx = stag.stag_create(dims, True, stream.cuda_stream)
    res = {"lattice": "x".join(str(d) for d in dims), "shifts": len(shifts), "mass": mass}
    try:
        g = _near_identity_device(torch, dev, V, 0.3)
        stag.stag_load_gauge_device(ctx, g)
        stag.stag_set_action(ctx, stag.STAG_ACTION_ASQTAD, 1.0)
        b = torch.randn(3 * 2 * vh, dtype=torch.float64, device=dev)
        x = torch.empty(len(shifts) * 3 * 2 * vh, dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stag.stag_multishift_solve(ctx, mass, shifts, stag.STAG_FP32, 1, b, x, 1e-8, 20000)
        best = None
        for _ in range(reps):
            e0.record(stream)
            info = stag.stag_multishift_solve(ctx, mass, shifts, stag.STAG_FP32, 1, b, x, 1e-8, 20000)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        res["iterations"] = info.iterations
        res["reliable_updates"] = info.reliable_updates
        res["solve_ms"] = round(best, 2)
        res["us_per_iteration"] = round(best * 1e3 / info.iterations, 2)
        # algorithmic bytes of one iteration (two Dslash, 8 vector passes, 4 per shift)
        per_site = 2 * LINK_BYTES[1] + (8 + 4 * len(shifts)) * 24
        res["algorithmic_gbs"] = round(vh * per_site * info.iterations / (best * 1e-3) / 1e9, 1)
        r = md.to_abi()
        f = torch.empty(4 * 2 * 8 * vh, dtype=torch.float64, device=dev)
        stag.stag_fermion_force(ctx, mass, r, stag.STAG_FP32, 1, b, f, 1e-8, 20000)
        e0.record(stream)
        stag.stag_fermion_force(ctx, mass, r, stag.STAG_FP32, 1, b, f, 1e-8, 20000)
        e1.record(stream)
        torch.cuda.synchronize()
        res["force_ms"] = round(e0.elapsed_time(e1), 2)
    finally:
        stag.stag_destroy(ctx)
    return res


def hmc_run(trajectories=10, warmup=5, log=print):
    """Thermalised start (quenched, then unimproved, then improved dynamical
    trajectories), then `trajectories` timed improved trajectories of the
    workload; reports trajectories/hour, acceptance and <|dH|>."""
    import torch

    import synthetic as syn

    from . import rational, stag
    from . import workload as wl
    w = WORKLOAD
    dims = tuple(w["dims"])
    stream = torch.cuda.current_stream()
    ctx = stag.stag_create(dims, True, stream.cuda_stream)
    rats = {k: rational.load(v) for k, v in w["rationals"].items()}
    unimproved = wl.rationals()

    def hmc(counter, rr, n_flavours=1, **kw):
        p = wl.make_hmc(stag, rr, stag.STAG_FP32, w["seed"], counter, n_flavours=n_flavours, **kw)
        p.beta, p.n_outer, p.n_gauge, p.tol_md, p.tol_met = w["beta"], w["n_outer"], w["n_gauge"], w["tol_md"], \
            w["tol_met"]
        if n_flavours:
            p.flavour[0].mass = w["mass"]
        return p

    out = {"config": w}
    try:
        u0 = syn.haar_gauge(dims, w["seed"])
        stag.stag_load_gauge(ctx, np.ascontiguousarray(u0).reshape(-1).view(np.float64))
        t0 = time.time()
        for k in range(w["quenched_thermalisation"]):
            stag.stag_md_trajectory(ctx, hmc(10_000 + k, unimproved, n_flavours=0))
        for k in range(w["unimproved_thermalisation"]):
            stag.stag_md_trajectory(ctx, hmc(20_000 + k, unimproved))
        stag.stag_set_action(ctx, stag.STAG_ACTION_ASQTAD, w["u0"])
        plaq = []
        for k in range(w["asqtad_thermalisation"] + warmup):
            t = stag.stag_md_trajectory(ctx, hmc(30_000 + k, rats))
            plaq.append(t.plaq)
        out["thermalisation_s"] = round(time.time() - t0, 1)
        out["plaquette_after_thermalisation"] = plaq[-1]
        rs = []
        torch.cuda.synchronize()
        t0 = time.time()
        for k in range(trajectories):
            rs.append(stag.stag_md_trajectory(ctx, hmc(40_000 + k, rats)))
        torch.cuda.synchronize()
        dt = time.time() - t0
        dh = np.array([r.dH for r in rs])
        out.update({
            "trajectories": trajectories, "seconds_per_trajectory": round(dt / trajectories, 4),
            "trajectories_per_hour": round(3600.0 * trajectories / dt, 1),
            "acceptance": float(np.mean([r.accepted for r in rs])), "mean_abs_dH": float(np.mean(np.abs(dh))),
            "exp_minus_dH": float(np.mean(np.exp(-dh))),
            "cg_iterations_per_trajectory": float(np.mean([r.cg_iterations for r in rs])),
            "phase_s": {k: float(np.mean([getattr(r, k) for r in rs]))
                        for k in ("t_heatbath", "t_fermion", "t_gauge", "t_metropolis")},
            "plaquette": float(np.mean([r.plaq for r in rs])),
        })
        if log:
            log(json.dumps(out))
    finally:
        stag.stag_destroy(ctx)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--dslash-dims", type=int, nargs=4, default=[48, 48, 48, 48])
    ap.add_argument("--solve-dims", type=int, nargs="+", default=[16, 16, 16, 16, 32, 32, 32, 32])
    ap.add_argument("--trajectories", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--skip-hmc", action="store_true")
    ap.add_argument("--skip-solve", action="store_true")
    ap.add_argument("--skip-dslash", action="store_true")
    a = ap.parse_args()
    peak = None
    try:
        peak = json.load(open("MEASURED_PEAKS.json")).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    if not a.skip_dslash:
        print(json.dumps({"asqtad_dslash": dslash_point(tuple(a.dslash_dims), hbm_gbs=peak)}), flush=True)
    for k in range(0, 0 if a.skip_solve else len(a.solve_dims), 4):
        print(json.dumps({"asqtad_solve": solve_point(tuple(a.solve_dims[k:k + 4]))}), flush=True)
    if not a.skip_hmc:
        hmc_run(a.trajectories, a.warmup, log=lambda s: print(json.dumps({"asqtad_hmc": json.loads(s)}), flush=True))
