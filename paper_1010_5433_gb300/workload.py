"""The 16^4 N_f = 2 RHMC workload the benchmarks run (paper Sec. 2 and Sec. 4):
its parameters, the trajectory parameters of the C ABI for either arm, and
the seeded recipe of its thermalised start.  Host-side set-up only: every
trajectory runs in the library.

Start recipe (synthetic; the paper uses no public ensemble):
  Haar-random links (hot start) from the workload seed;
  40 quenched trajectories at beta = 5.6 (no fermions);
  100 dynamical trajectories with Metropolis at n_outer = 10 (half the
  outer steps: same equilibrium, half the cost), mixed path.
Measured on GB300: the plaquette climbs from 0.53 to 0.564 and levels off
after about 80 dynamical trajectories; <|dH|> at n_outer = 20 falls from
0.2 to 0.06 over the same span.

Outer step count.  The paper gives none; it is tuned to an acceptance near
0.8 at equilibrium (100 trajectories each from the thermalised start,
mixed path): n_outer = 20 gives acceptance 0.97, <|dH|> 0.064; 12 gives
0.94, 0.160; 10 gives 0.85, 0.225.  The workload runs n_outer = 10.
"""
import numpy as np

WORKLOAD = {
    "workload": "RHMC 16^4 Nf=2 unimproved staggered, m=0.02, beta=5.6, tau=1, 2MN n_outer=10 x n_gauge=5 "
                "(acceptance 0.85 at equilibrium), 12-pole MD rational (fp32 + fp64 reliable updates), 24-pole fp64 "
                "heatbath/Metropolis, thermalised start",
    "dims": [16, 16, 16, 16], "beta": 5.6, "mass": 0.02, "n_flavours": 2, "n_pf": 1, "tau": 1.0,
    "n_outer": 10, "n_gauge": 5, "tol_md": 1e-8, "tol_met": 1e-12,
    "rationals": {"md": "c2_md", "met": "c2_met", "hb": "c2_hb"},
    "seed": 0x5A0002, "quenched_thermalisation": 40, "dynamical_thermalisation": 100, "thermalisation_n_outer": 10,
}

# link format of the fp32 MD inversions (the fp64 heatbath / Metropolis
# inversions always use the two-float store): stag_prec value, description.
# The paper stores two rows of every link and rebuilds the third (Sec. 5).
MD_LINKS = {"18": (1, "fp32, 18 reals per link"), "12": (2, "fp32, 12 reals per link (row 3 rebuilt)"),
            "bf16": (3, "bf16, 12 reals per link (row 3 rebuilt), fp32 arithmetic")}


def rationals(n_pf=1):
    """MD, Metropolis and heatbath rationals of the workload's flavour split
    over n_pf pseudo-fermions (exponent s = 1 / (2 n_pf) per pseudo-fermion)."""
    from . import rational
    if n_pf == 1:
        return {k: rational.load(v) for k, v in WORKLOAD["rationals"].items()}
    return {k: rational.load(f"c2_pf{n_pf}_{k}") for k in ("md", "met", "hb")}


def make_hmc(stag, rats, prec, seed, counter, n_flavours=1, **kw):
    """stag_hmc of one trajectory of the workload (prec: the MD inversions'
    stag_prec; STAG_FP64 is the plain fp64 arm)."""
    w = WORKLOAD
    p = stag.stag_hmc()
    p.beta, p.tau, p.n_outer, p.n_gauge = w["beta"], w["tau"], w["n_outer"], w["n_gauge"]
    p.n_flavours = n_flavours
    if n_flavours:
        fl = p.flavour[0]
        fl.mass, fl.n_pf = w["mass"], kw.pop("n_pf", w["n_pf"])
        fl.hb, fl.md, fl.met = rats["hb"].to_abi(), rats["md"].to_abi(), rats["met"].to_abi()
    p.tol_md, p.tol_met, p.max_iter = w["tol_md"], w["tol_met"], 20000
    p.md_prec = prec
    p.seed, p.counter = seed, counter
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def thermalise(stag, ctx, rats, seed, md_prec, log=None):
    """Loads the hot start into ctx and runs the quenched and dynamical
    thermalisation of the recipe above; returns the plaquette history of the
    dynamical trajectories."""
    import synthetic as syn
    w = WORKLOAD
    dims = tuple(w["dims"])
    u0 = syn.haar_gauge(dims, seed)     # [mu, t, z, y, x, 3, 3] = the host layout of the C ABI
    stag.stag_load_gauge(ctx, np.ascontiguousarray(u0).reshape(-1).view(np.float64))
    del u0
    for k in range(w["quenched_thermalisation"]):
        stag.stag_md_trajectory(ctx, make_hmc(stag, rats, md_prec, seed, 10_000 + k, n_flavours=0))
    plaq = []
    for k in range(w["dynamical_thermalisation"]):
        t = stag.stag_md_trajectory(ctx, make_hmc(stag, rats, md_prec, seed, 20_000 + k,
                                                  n_outer=w["thermalisation_n_outer"]))
        plaq.append(t.plaq)
        if log:
            log(f"thermalisation {k}: dH {t.dH:+.4f} accepted {t.accepted} plaquette {t.plaq:.5f}")
    return plaq


# Hasenbusch mass split of the flavour (paper Sec. 2's multiple pseudo-fermions,
# extended by a heavier mass): det(A)^(1/2) = det(A_h)^(1/2) det(A / A_h)^(1/2)
# with m_h = 0.2; the ratio term at m on the outer level, the heavy term on the
# middle level.
HEAVY_MASS = 0.2


def split_rationals():
    from . import rational
    return ({k: rational.load(f"c2_ratio_{k}") for k in ("md", "met", "hb")},
            {k: rational.load(f"c2_heavy_{k}") for k in ("md", "met", "hb")})


def make_hmc_split(stag, ratio, heavy, prec, seed, counter, n_outer, n_mid, n_gauge=None):
    """stag_hmc of one trajectory with the mass split: flavour 0 the ratio
    term (mass m, outer level), flavour 1 the heavy term (mass m_h, middle
    level, n_mid steps per outer half step)."""
    w = WORKLOAD
    p = stag.stag_hmc()
    p.beta, p.tau, p.n_outer, p.n_gauge = w["beta"], w["tau"], n_outer, n_gauge or w["n_gauge"]
    p.n_flavours, p.n_mid = 2, n_mid
    for f, (mass, level, r) in enumerate(((w["mass"], 0, ratio), (HEAVY_MASS, 1, heavy))):
        fl = p.flavour[f]
        fl.mass, fl.n_pf, fl.level = mass, 1, level
        fl.hb, fl.md, fl.met = r["hb"].to_abi(), r["md"].to_abi(), r["met"].to_abi()
    p.tol_md, p.tol_met, p.max_iter = w["tol_md"], w["tol_met"], 20000
    p.md_prec = prec
    p.seed, p.counter = seed, counter
    return p
