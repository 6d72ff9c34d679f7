"""Micro-benchmark of the library's multi-shift CG (paper Sec. 6): one solve
of (A + sigma_i) x_i = b with the 12-pole MD rational of the 16^4, m = 0.02
workload on a device-built near-identity SU(3) gauge field, in the requested
iteration precision; prints iterations, wall time and the per-kernel
event-timed profile.

  python -m paper_1010_5433_gb300.solve_bench [--dims 16 16 16 16] [--prec 1]
         [--nrhs 1] [--max-iter 400] [--width 0.3] [--tol 1e-30]
"""
import argparse
import json
import time


def run(dims, prec=1, nrhs=1, max_iter=400, width=0.3, mass=0.02, profile=True, tol=1e-30):
    import numpy as np
    import torch

    from . import rational, stag
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    V = int(np.prod(dims))
    vh = V // 2
    shifts = rational.load("c2_md").beta
    ctx = stag.stag_create(dims, True, stream.cuda_stream)
    try:
        g = torch.randn(4 * V * 18, dtype=torch.float64, device=dev).mul_(width)
        gv = g.view(4 * V, 9, 2)
        for k in (0, 4, 8):
            gv[:, k, 0] += 1.0
        # projected to SU(3) (rows 0, 1 orthonormalised, row 2 = (row 0 x row 1)*)
        # so that the 12-real formats, which rebuild row 2, see the same links
        u = torch.view_as_complex(g.view(4 * V, 3, 3, 2))
        r0 = u[:, 0] / torch.linalg.vector_norm(u[:, 0], dim=-1, keepdim=True)
        r1 = u[:, 1] - (r0.conj() * u[:, 1]).sum(-1, keepdim=True) * r0
        r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
        r2 = torch.linalg.cross(r0, r1, dim=-1).conj()
        g = torch.view_as_real(torch.stack([r0, r1, r2], dim=1)).reshape(-1).contiguous()
        stag.stag_load_gauge_device(ctx, g)
        del g, gv, u, r0, r1, r2
        b = torch.randn(nrhs * 3 * 2 * vh, dtype=torch.float64, device=dev)
        x = torch.empty(nrhs * len(shifts) * 3 * 2 * vh, dtype=torch.float64, device=dev)
        # identical warm-up solve: tunes, builds graphs and loads every kernel the timed one needs
        stag.stag_multishift_solve(ctx, mass, shifts, prec, nrhs, b, x, tol, max_iter, info=False, check=False)
        if profile:
            stag.stag_profile_begin(ctx, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = stag.stag_multishift_solve(ctx, mass, shifts, prec, nrhs, b, x, tol, max_iter, check=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out = {"lattice": "x".join(str(d) for d in dims), "prec": prec, "nrhs": nrhs, "status": st,
               "iterations": info.iterations, "seconds": round(dt, 4), "us_per_iteration": round(dt / max(info.iterations, 1) * 1e6, 2)}
        if profile:
            kinds = {"dslash_oe": stag.STAG_PK_DSLASH_OE, "dslash_eo_A": stag.STAG_PK_DSLASH_EO_A,
                     "update": stag.STAG_PK_UPDATE,
                     "persistent_iteration": stag.STAG_PK_PERSISTENT if prec else stag.STAG_PK_PERSISTENT_FF}
            for n, k in kinds.items():
                pr = stag.stag_profile_read(ctx, k)
                avg = pr.sampled_ms / max(pr.sampled, 1)
                out[n] = {"launches": pr.launches, "sampled": pr.sampled, "avg_us": round(avg * 1e3, 2),
                          "bytes_per_launch": round(pr.bytes_per_launch),
                          "achieved_gbs": round(pr.bytes_per_launch / (avg * 1e-3) / 1e9, 1) if avg > 0 else 0}
            ph = stag.stag_profile_phases(ctx)
            it = max(info.iterations, 1)
            out["persistent_phases_us_per_iteration"] = dict(zip(
                ["phase1_doe", "barrier1", "phase2_deo_A", "barrier2", "alpha_step", "phase3_update", "barrier3",
                 "beta_step", "reliable_updates", "alpha_sums", "alpha_arith", "alpha_sync", "beta_sums",
                 "beta_arith", "beta_rest"],
                [round(v / it, 2) for v in ph]))
    finally:
        stag.stag_destroy(ctx)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 16])
    ap.add_argument("--prec", type=int, default=1)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--max-iter", type=int, default=400)
    ap.add_argument("--width", type=float, default=0.3)
    # the default runs max_iter iterations; a loose tol (e.g. 0.11, above the first
    # reliable update at 0.1) gives one persistent launch of known length
    ap.add_argument("--tol", type=float, default=1e-30)
    a = ap.parse_args()
    print(json.dumps(run(tuple(a.dims), a.prec, a.nrhs, a.max_iter, a.width, tol=a.tol)))
