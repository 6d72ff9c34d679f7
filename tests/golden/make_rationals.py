"""Writes tests/golden/rationals.json: the RHMC rational approximations of the
workloads, computed by the oracle's Remez (oracle/rational.py) and nothing
else.  Run:  python tests/golden/make_rationals.py

Each entry: r(x) = a0 + sum_i alpha_i / (x + beta_i) ~ x^(-s) on [lo, hi] with
its relative minimax error (entries with a "delta": ((x + delta) / x)^s, the
ratio term of a Hasenbusch mass split).  Exponents per pseudo-fermion s = N_f / (4 n_pf)
(MD and Metropolis) and -s/2 (heatbath, r_hb ~ x^(+s/2)); ranges
[m^2, 16 + m^2], the spectrum bound of A = m^2 - D_eo D_oe (entries with a
fifth field: [m^2, upper + m^2], the improved operator's wider bound).
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.rational import remez  # noqa: E402

# name: (s, m, n)
TABLE = {
    # 4^4, m = 0.1, N_f = 1, one pseudo-fermion: 8-pole MD rational of x^(-1/4)
    "c1_md": (0.25, 0.1, 8),
    "c1_met": (0.25, 0.1, 16),
    "c1_hb": (-0.125, 0.1, 16),
    # 16^4 and 24^4, m = 0.02, N_f = 2: 12-pole MD rational of x^(-1/2)
    "c2_md": (0.5, 0.02, 12),
    "c2_met": (0.5, 0.02, 24),
    "c2_hb": (-0.25, 0.02, 24),
    # 32^3x8, N_f = 2+1, two pseudo-fermions per flavour, 15 MD poles
    "c3_light_md": (0.25, 0.01, 15),
    "c3_light_met": (0.25, 0.01, 24),
    "c3_light_hb": (-0.125, 0.01, 24),
    "c3_strange_md": (0.125, 0.1, 15),
    "c3_strange_met": (0.125, 0.1, 18),
    "c3_strange_hb": (-0.0625, 0.1, 18),
    # chains, m = 0.05, N_f = 2, 12 poles
    "c4_md": (0.5, 0.05, 12),
    "c4_met": (0.5, 0.05, 20),
    "c4_hb": (-0.25, 0.05, 20),
    # volume-scaling study at the paper's masses am = 1.0 and 0.01335 (Sec. 6), N_f = 2
    "t3_high_md": (0.5, 1.0, 6),
    "t3_high_met": (0.5, 1.0, 10),
    "t3_high_hb": (-0.25, 1.0, 10),
    "t3_low_md": (0.5, 0.01335, 12),
    "t3_low_met": (0.5, 0.01335, 24),
    "t3_low_hb": (-0.25, 0.01335, 24),
    # 16^4, m = 0.02, N_f = 2 split over n_pf = 2, 3, 4 pseudo-fermions (s = 1 / (2 n_pf))
    "c2_pf2_md": (0.25, 0.02, 12),
    "c2_pf2_met": (0.25, 0.02, 20),
    "c2_pf2_hb": (-0.125, 0.02, 20),
    "c2_pf3_md": (1.0 / 6.0, 0.02, 12),
    "c2_pf3_met": (1.0 / 6.0, 0.02, 20),
    "c2_pf3_hb": (-1.0 / 12.0, 0.02, 20),
    "c2_pf4_md": (0.125, 0.02, 12),
    "c2_pf4_met": (0.125, 0.02, 20),
    "c2_pf4_hb": (-0.0625, 0.02, 20),
    # Hasenbusch mass split of the 16^4 workload: heavy term at m_h = 0.2, ratio term
    # ((x + delta) / x)^(1/2) at m = 0.02 with delta = m_h^2 - m^2 = 0.0396
    "c2_heavy_md": (0.5, 0.2, 8),
    "c2_heavy_met": (0.5, 0.2, 14),
    "c2_heavy_hb": (-0.25, 0.2, 14),
    "c2_ratio_md": (0.5, 0.02, 8, 0.0396),
    "c2_ratio_met": (0.5, 0.02, 12, 0.0396),
    "c2_ratio_hb": (-0.25, 0.02, 12, 0.0396),
    # the improved (asqtad, tree level) 16^4 N_f = 2 workload at m = 0.02: A's spectrum lies
    # in [m^2, m^2 + 58.8], so these approximate on [m^2, m^2 + 64]
    "asqtad_md": (0.5, 0.02, 14, 0.0, 64.0),
    "asqtad_met": (0.5, 0.02, 24, 0.0, 64.0),
    "asqtad_hb": (-0.25, 0.02, 24, 0.0, 64.0),
}


def main(names=None):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rationals.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name, spec in TABLE.items():
        s, m, n = spec[:3]
        delta = spec[3] if len(spec) > 3 else 0.0
        upper = spec[4] if len(spec) > 4 else 16.0
        if names and name not in names:
            continue
        if name in out and out[name]["n"] == n:
            continue
        t = time.time()
        r = remez(s, m * m, upper + m * m, n, dps=60 if n <= 16 else 100, delta=delta)
        d = r.as_dict()
        d["mass"] = m
        out[name] = d
        print(f"{name}: n={n} err={r.err:.3e} ({time.time() - t:.0f}s)", flush=True)
        json.dump(out, open(path, "w"), indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or None)
