"""Micro-benchmark of the library's Dslash (paper Sec. 5, Table 2 measures
the same kernel): D_oe on one lattice in the requested precisions, CUDA-event
timed on the launching stream after warm-up, reported against the algorithmic
bytes per site (links once, input and output spinor once).

  python -m paper_1010_5433_gb300.dslash_bench [--dims 48 48 48 48] [--prec 1 2 3 0]
         [--nrhs 1] [--reps 20]
"""
import argparse
import json

LINK_BYTES = {0: 1152, 1: 576, 2: 384, 3: 192}
NAMES = {0: "fp64", 1: "fp32_18", 2: "fp32_12", 3: "bf16_12"}


def run(dims, precs=(1, 2, 3, 0), nrhs=1, reps=20, hbm_gbs=None, flush_l2=False):
    """flush_l2: write a 512 MB buffer before every timed launch and time the
    launches one by one (cold L2: lattices whose fields fit in the 129 MB L2
    are then read from HBM, as the paper's cache-less C1060 read them)."""
    import numpy as np
    import torch

    from . import stag
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    V = int(np.prod(dims))
    vh = V // 2
    ctx = stag.stag_create(dims, True, stream.cuda_stream)
    res = {"lattice": "x".join(str(d) for d in dims), "nrhs": nrhs, "reps": reps,
           "l2": "flushed before every launch" if flush_l2 else "warm (back-to-back launches)"}
    try:
        # a random field near the identity, built on the device (the values do
        # not change the timing; the 12-real formats rebuild row 2 from rows 0-1)
        g = torch.randn(4 * V * 18, dtype=torch.float64, device=dev).mul_(0.05)
        gv = g.view(4 * V, 9, 2)
        for k in (0, 4, 8):
            gv[:, k, 0] += 1.0
        stag.stag_load_gauge_device(ctx, g)
        torch.cuda.synchronize()
        del g, gv
        for prec in precs:
            dt = torch.float64 if prec == 0 else torch.float32
            s = 48 if prec == 0 else 24
            inp = torch.randn(nrhs * 3 * 2 * vh, dtype=dt, device=dev)
            out = torch.empty_like(inp)
            for _ in range(3):
                stag.stag_dslash(ctx, 1, prec, nrhs, inp, out)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if flush_l2:
                flush = torch.empty(128 << 20, dtype=torch.float32, device=dev)
                t = 0.0
                for _ in range(reps):
                    flush.zero_()
                    e0.record(stream)
                    stag.stag_dslash(ctx, 1, prec, nrhs, inp, out)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    t += e0.elapsed_time(e1)
                t = t / reps * 1e-3
                del flush
            else:
                e0.record(stream)
                for _ in range(reps):
                    stag.stag_dslash(ctx, 1, prec, nrhs, inp, out)
                e1.record(stream)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / reps * 1e-3
            bps = LINK_BYTES[prec] + 2 * s * nrhs
            gbs = vh * bps / t / 1e9
            r = {"us": round(t * 1e6, 2), "achieved_gbs": round(gbs, 1), "bytes_per_site": bps}
            if hbm_gbs:
                r["frac"] = round(gbs / hbm_gbs, 4)
            res[NAMES[prec]] = r
            del inp, out
    finally:
        stag.stag_destroy(ctx)
    return res


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[48, 48, 48, 48])
    ap.add_argument("--prec", type=int, nargs="+", default=[1, 2, 3, 0])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--flush-l2", action="store_true")
    a = ap.parse_args()
    print(json.dumps(run(tuple(a.dims), tuple(a.prec), a.nrhs, a.reps, flush_l2=a.flush_l2)))
