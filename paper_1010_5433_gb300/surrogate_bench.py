"""What the learned force surrogate gains: on one lattice, build a chain,
collect exact fermion forces as training samples, train the surrogate on the
GPU, then run paired trajectories (identical links, momenta and sources) with

  exact      the two-level integrator with n_outer fermion steps
  exact/2    the same with n_outer / 2 steps
  surrogate  n_outer / 2 exact-remainder steps, the surrogate on n_mid steps
             per half step in between (the Metropolis step stays exact)

and report mean |dH| and device seconds per trajectory for each.  Before the
trajectories it splits the exact force on C configurations into its mean over
K heatbath draws and the pseudo-fermion noise, F(U, phi) = Fbar(U) + n(phi):
the surrogate sees only U, so Fbar is all it can learn, and the report gives
the share of |F|^2 that Fbar carries and the share of |Fbar|^2 that the
trained network reproduces.

  python -m paper_1010_5433_gb300.surrogate_bench [--dims 8 8 8 8] [--mass 0.05]
"""
import argparse
import json
import time

import numpy as np


def force_decomposition(ctx, stag, rats, mass, n_pf, draws, counter0, seed, torch, Vh, surrogate=True):
    """Exact MD force of the loaded field for `draws` heatbath draws: second
    moment, noise variance and mean part (unbiased), and with the loaded
    surrogate F^ the residuals |F - F^|^2 and |Fbar - F^|^2 (sums over links)."""
    hb, md = rats["hb"], rats["md"]
    ns, hc = len(hb.beta), 3 * Vh
    xi = torch.empty(n_pf * hc * 2, dtype=torch.float64, device="cuda")
    xs = torch.empty(n_pf * ns * hc * 2, dtype=torch.float64, device="cuda")
    F = torch.empty(64 * Vh, dtype=torch.float64, device="cuda")
    Fs = []
    for k in range(draws):
        stag.stag_draw_sources(ctx, seed, counter0 + k, 0, n_pf, xi)
        stag.stag_multishift_solve(ctx, mass, hb.beta, stag.STAG_FP64, n_pf, xi, xs, 1e-12, 20000)
        phi = hb.a0 * xi                                   # heatbath phi = r_hb(A) xi
        xv, pv = xs.view(n_pf, ns, -1), phi.view(n_pf, -1)
        for i, a in enumerate(hb.alpha):
            pv += a * xv[:, i]
        stag.stag_fermion_force(ctx, mass, md.to_abi(), stag.STAG_FP32, n_pf, phi, F, 1e-8, 20000)
        Fs.append(F.clone())
    Fs = torch.stack(Fs)
    Fb = Fs.mean(0)
    noise = float(((Fs - Fb) ** 2).sum(1).mean()) * draws / (draws - 1)
    r = {"second_moment": float((Fs ** 2).sum(1).mean()), "noise": noise,
         "mean_part": float((Fb ** 2).sum()) - noise / draws}
    if surrogate:
        Fh = torch.empty_like(F)
        stag.stag_surrogate_force(ctx, Fh)
        r["residual"] = float(((Fs - Fh) ** 2).sum(1).mean())
        r["residual_of_mean"] = float(((Fb - Fh) ** 2).sum()) - noise / draws
    return r


def run(dims=(8, 8, 8, 8), rat_prefix="c4", mass=0.05, beta=5.6, n_outer=8, n_mid=3, n_gauge=4, therm=6,
        samples=8, train_steps=200, lr=3e-3, pairs=6, decomp_configs=3, draws=6, seed=0x5A0005, every=1):
    """every: chain trajectories between two training samples; the store is
    reserved for exactly `samples` configurations up front."""
    import torch

    import synthetic as syn

    from . import rational, stag
    rats = {k: rational.load(f"{rat_prefix}_{k}") for k in ("md", "met", "hb")}
    V = int(np.prod(dims))
    stream = torch.cuda.current_stream()
    ctx = stag.stag_create(dims, True, stream.cuda_stream)

    def hmc(counter, no, **kw):
        p = stag.stag_hmc()
        p.beta, p.tau, p.n_outer, p.n_gauge, p.n_flavours = beta, 1.0, no, n_gauge, 1
        fl = p.flavour[0]
        fl.mass, fl.n_pf = mass, 1
        fl.hb, fl.md, fl.met = rats["hb"].to_abi(), rats["md"].to_abi(), rats["met"].to_abi()
        p.tol_md, p.tol_met, p.max_iter, p.md_prec = 1e-8, 1e-12, 20000, stag.STAG_FP32
        p.seed, p.counter = seed, counter
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    out = {"lattice": "x".join(map(str, dims)), "mass": mass, "beta": beta, "n_outer": n_outer, "n_mid": n_mid}
    try:
        # start: SU(3) links near the identity; warm-up without accept/reject
        # (quenched, then dynamical) to leave the ordered start, then a
        # Metropolis chain from which every sample and test field is taken
        u0 = syn.near_identity_gauge(dims, seed)           # [mu, t, z, y, x, 3, 3], the host layout of the C ABI
        stag.stag_load_gauge(ctx, np.ascontiguousarray(u0).reshape(-1).view(np.float64))
        for k in range(20):
            stag.stag_md_trajectory(ctx, hmc(10_000 + k, 10, n_flavours=0, no_metropolis=1))
        for k in range(3):
            stag.stag_md_trajectory(ctx, hmc(20_000 + k, n_outer, no_metropolis=1))
        acc = []
        for k in range(therm):
            acc.append(stag.stag_md_trajectory(ctx, hmc(1 + k, n_outer)).accepted)
        out["thermalisation_acceptance"] = float(np.mean(acc))
        # training set: one exact-force sample per trajectory of the chain
        rng = np.random.default_rng(seed)
        p0 = np.concatenate([rng.standard_normal(n) * s for n, s in
                             [(768, 0.06), (32, 0.1), (1024, 0.05), (32, 0.1), (768, 0.05), (24, 0.0)]])
        stag.stag_surrogate_load(ctx, p0.astype(np.float32))
        stag.stag_surrogate_reserve(ctx, samples)
        t0 = time.perf_counter()
        for k in range(samples):
            for j in range(every):
                stag.stag_md_trajectory(ctx, hmc(100_000 + every * k + j, n_outer))
            stag.stag_surrogate_add_sample(ctx, hmc(0, n_outer), 5000 + k)
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        first, last = stag.stag_surrogate_train(ctx, train_steps, lr)
        torch.cuda.synchronize()
        out["training"] = {"samples": samples, "every": every, "links": samples * 4 * V, "steps": train_steps,
                           "loss_first": first, "loss_last": last, "seconds": round(time.perf_counter() - t0, 3),
                           "data_seconds": round(t_data, 3)}
        # what a function of U alone can learn, and what the trained network does learn
        dec = []
        for c in range(decomp_configs):
            stag.stag_md_trajectory(ctx, hmc(150 + c, n_outer))
            dec.append(force_decomposition(ctx, stag, rats, mass, 1, draws, 7000 + 100 * c, seed, torch, V // 2))
        if dec:
            d = {k: float(np.mean([x[k] for x in dec])) for k in dec[0]}
            out["force"] = {"configs": decomp_configs, "draws": draws,
                            "mean_share": d["mean_part"] / d["second_moment"],
                            "captured_share_of_mean": 1.0 - d["residual_of_mean"] / d["mean_part"],
                            "captured_share_of_force": 1.0 - d["residual"] / d["second_moment"]}
        # paired evaluation from the chain's configurations
        field = np.empty(4 * V * 18)
        res = {"exact": [], "exact_half": [], "surrogate": []}
        plaq = []
        for k in range(pairs):
            r = stag.stag_md_trajectory(ctx, hmc(200 + k, n_outer))     # advance the chain
            plaq.append(r.plaq)
            stag.stag_store_gauge(ctx, field)
            for name, kw in [("exact", dict(n_outer=n_outer)), ("exact_half", dict(n_outer=n_outer // 2)),
                             ("surrogate", dict(n_outer=n_outer // 2, use_surrogate=1, n_mid=n_mid))]:
                stag.stag_load_gauge(ctx, field)
                no = kw.pop("n_outer")
                r = stag.stag_md_trajectory(ctx, hmc(300 + k, no, no_metropolis=1, **kw))
                res[name].append((r.dH, r.seconds, r.cg_iterations))
            stag.stag_load_gauge(ctx, field)
        out["plaquette"] = float(np.mean(plaq))
        for name, v in res.items():
            a = np.array(v)
            out[name] = {"mean_abs_dH": float(np.mean(np.abs(a[:, 0]))), "seconds_per_traj": float(np.mean(a[:, 1])),
                         "cg_iterations": float(np.mean(a[:, 2])), "dH": [round(x, 5) for x in a[:, 0]]}
    finally:
        stag.stag_destroy(ctx)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[8, 8, 8, 8])
    ap.add_argument("--rationals", default="c4")
    ap.add_argument("--mass", type=float, default=0.05)
    ap.add_argument("--n-outer", type=int, default=8)
    ap.add_argument("--n-mid", type=int, default=3)
    ap.add_argument("--samples", type=int, default=8)
    ap.add_argument("--train-steps", type=int, default=200)
    ap.add_argument("--pairs", type=int, default=6)
    ap.add_argument("--decomp-configs", type=int, default=3)
    ap.add_argument("--draws", type=int, default=6)
    ap.add_argument("--n-gauge", type=int, default=4)
    ap.add_argument("--therm", type=int, default=6)
    ap.add_argument("--every", type=int, default=1, help="chain trajectories per training sample")
    a = ap.parse_args()
    print(json.dumps(run(tuple(a.dims), a.rationals, a.mass, n_outer=a.n_outer, n_mid=a.n_mid, n_gauge=a.n_gauge,
                         therm=a.therm, samples=a.samples, train_steps=a.train_steps, pairs=a.pairs,
                         decomp_configs=a.decomp_configs, draws=a.draws, every=a.every)))
