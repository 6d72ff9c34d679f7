"""Writes tests/golden/traj_8x4_asqtad.json: one RHMC trajectory of the
oracle (oracle/integrator.py with the improved operator of oracle/asqtad.py,
FP64) at the settings of the improved-staggered 16^4 N_f = 2 workload --
tree-level asqtad (u0 = 1), 14-pole MD rational of x^(-1/2) and 24-pole
heatbath and Metropolis rationals at m = 0.02 on [m^2, m^2 + 64]
(tests/golden/rationals.json), beta = 5.6 (Wilson gauge action), tau = 1,
n_outer = 10 outer minimum-norm steps with n_gauge = 5 gauge substeps -- on
an 8^4 lattice, so that the GPU trajectory at those settings can be
compared with the oracle without running the oracle on the GPU machine (tens of
minutes of numpy).  Inputs are the seeded synthetic fields named below;
nothing but oracle/ computes the stored values.

Stored: H0, H1, dH, S_f before and after, the final links' sum of squares
and their values at 64 fixed (mu, site) positions (paper Sec. 2, Sec. 4).

Run:  python tests/golden/make_traj_8x4_asqtad.py"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import synthetic as syn  # noqa: E402
from oracle import integrator  # noqa: E402
from oracle.rational import Rational  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SETUP = {"dims": [8, 8, 8, 8], "gauge": "near_identity", "gauge_seed": 0x5A0009, "gauge_width": 0.5,
         "mom_seed": 891, "xi_seed": 892, "mass": 0.02, "beta": 5.6, "tau": 1.0, "n_outer": 10, "n_gauge": 5,
         "rationals": "asqtad", "action": "asqtad", "u0": 1.0, "tol_md": 1e-12, "tol_met": 1e-13,
         "sample_seed": 893, "n_sample": 64}


def rationals(prefix):
    g = json.load(open(os.path.join(HERE, "rationals.json")))
    keys = ("s", "lo", "hi", "a0", "alpha", "beta", "err")
    return {k: Rational(*[g[prefix + "_" + k][kk] for kk in keys]) for k in ("md", "met", "hb")}


def inputs(s=SETUP):
    dims = tuple(s["dims"])
    u0 = syn.near_identity_gauge(dims, s["gauge_seed"], width=s["gauge_width"])
    mom0 = syn.gaussian_momenta(dims, s["mom_seed"])
    xi = syn.gaussian_fermion(dims, s["xi_seed"], on_parity=0)
    return dims, u0, mom0, xi


def sample_positions(s=SETUP):
    """(mu, t, z, y, x) of the sampled links."""
    dims = s["dims"]
    g = np.random.default_rng(s["sample_seed"])
    return [[int(g.integers(4))] + [int(g.integers(dims[3 - k])) for k in range(4)] for _ in range(s["n_sample"])]


def params(s=SETUP):
    r = rationals(s["rationals"])
    fl = integrator.Flavour(mass=s["mass"], hb=r["hb"], md=r["md"], met=r["met"])
    return integrator.HMCParams(dims=tuple(s["dims"]), beta=s["beta"], tau=s["tau"], n_outer=s["n_outer"],
                                n_gauge=s["n_gauge"], flavours=[fl], tol_md=s["tol_md"], tol_met=s["tol_met"],
                                action=s["action"], u0=s["u0"])


def main():
    t = time.time()
    dims, u0, mom0, xi = inputs()
    out = integrator.trajectory(integrator.Context(params()), u0, mom0, [[xi]])
    u1 = out["u"]
    pos = sample_positions()
    rec = {"setup": SETUP, "H0": out["H0"], "H1": out["H1"], "dH": out["dH"], "Sf0": out["Sf0"],
           "Sf1": out["Sf1"], "u_sumsq": float(np.sum(np.abs(u1) ** 2)),
           "u_sample": [[[float(v.real), float(v.imag)] for v in u1[tuple(p)].reshape(-1)] for p in pos],
           "u_sample_pos": pos, "oracle_seconds": round(time.time() - t, 1)}
    json.dump(rec, open(os.path.join(HERE, "traj_8x4_asqtad.json"), "w"), indent=1)
    print(f"dH {out['dH']:.10f} H0 {out['H0']:.6f} ({time.time() - t:.0f} s)")


if __name__ == "__main__":
    main()
