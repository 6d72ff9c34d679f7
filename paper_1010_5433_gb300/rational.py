"""Rational approximations for RHMC (paper Sec. 2: separate rational
approximations and stopping residuals for the MD force and for the
Metropolis step; ref. [rhmc] Horvath, Kennedy, Sint).

Host-side set-up, not a step of the GPU path: it produces the coefficients
that the C ABI takes as input (stag_rational),

    r(x) = a0 + sum_i alpha_i / (x + beta_i)  ~  x^(-s)  on [lo, hi],

with the smallest maximum relative error (type (n, n), Remez exchange).
Per reference set the levelled equations

    P(t_j) - f(t_j) (1 + (-1)^j E) Q(t_j) = 0,   j = 0 .. 2n+1,   t = x / hi,

are solved by Newton's method in (P, Q, E) jointly, seeded by a few
linearised solves in which E multiplies the previous Q (Q = 1 at first);
the new reference set is the alternating set of local extrema of the
relative error, located on a logarithmic grid and polished by successive
parabolic interpolation.  Multiprecision (mpmath) keeps the monomial basis
usable for the degrees and condition numbers of RHMC (n <= 32, hi/lo <= 1e6).
"""
import mpmath as mp


class RationalApprox:
    def __init__(self, s, lo, hi, a0, alpha, beta, err):
        self.s, self.lo, self.hi = float(s), float(lo), float(hi)
        self.a0 = float(a0)
        self.alpha = [float(a) for a in alpha]
        self.beta = [float(b) for b in beta]
        self.err = float(err)
        self.delta = 0.0        # > 0: approximates ((x + delta) / x)^s

    @property
    def n(self):
        return len(self.alpha)

    def __call__(self, x):
        return self.a0 + sum(a / (x + b) for a, b in zip(self.alpha, self.beta))

    def to_abi(self):
        from . import stag
        return stag.make_rational(self.a0, self.alpha, self.beta)


def _horner(c, t):
    v = mp.mpf(0)
    for ck in reversed(c):
        v = v * t + ck
    return v


def _levelled_newton(ts, fs, n, z0):
    """Newton on F_j(p, q, E) = P(t_j) - f_j (1 + (-1)^j E) Q(t_j), Q monic."""
    m = 2 * n + 2
    z = list(z0)
    for _ in range(60):
        p, q, e = z[:n + 1], z[n + 1:2 * n + 1] + [mp.mpf(1)], z[-1]
        F = mp.matrix(m, 1)
        J = mp.matrix(m, m)
        for j, (t, f) in enumerate(zip(ts, fs)):
            sg = 1 if j % 2 == 0 else -1
            qv = _horner(q, t)
            F[j] = _horner(p, t) - f * (1 + sg * e) * qv
            tk = mp.mpf(1)
            for k in range(n + 1):
                J[j, k] = tk
                if k < n:
                    J[j, n + 1 + k] = -f * (1 + sg * e) * tk
                tk *= t
            J[j, m - 1] = -f * sg * qv
        dz = mp.lu_solve(J, F)
        z = [z[k] - dz[k] for k in range(m)]
        if mp.norm(dz) <= mp.mpf(10) ** (-(mp.mp.dps - 10)) * (1 + mp.norm(mp.matrix(z))):
            break
    return z


def _linearised(ts, fs, n, q_prev, sweeps=4):
    """Seed for Newton: E enters only through the previous Q, which makes the
    levelled equations linear in (P, Q, E); a few sweeps pick the branch
    whose Q has no root in the interval."""
    m = 2 * n + 2
    q = q_prev
    z = None
    for _ in range(sweeps):
        A = mp.matrix(m, m)
        rhs = mp.matrix(m, 1)
        for j, (t, f) in enumerate(zip(ts, fs)):
            sg = 1 if j % 2 == 0 else -1
            tk = mp.mpf(1)
            for k in range(n + 1):
                A[j, k] = tk
                if k < n:
                    A[j, n + 1 + k] = -f * tk
                tk *= t
            A[j, m - 1] = -sg * f * (_horner(q, t) if q is not None else 1)
            rhs[j] = f * t ** n
        sol = mp.lu_solve(A, rhs)
        z = [sol[k] for k in range(m)]
        q = z[n + 1:2 * n + 1] + [mp.mpf(1)]
    return z


def _extrema(err, tlo, m):
    """Alternating set of m local extrema of err on [tlo, 1] (log grid +
    parabolic polishing in log t)."""
    G = 40 * m
    us = [mp.log(tlo) * (1 - mp.mpf(k) / (G - 1)) for k in range(G)]
    es = [err(mp.e ** u) for u in us]
    cand = []
    for k in range(G):
        if 0 < k < G - 1:
            if abs(es[k]) < abs(es[k - 1]) or abs(es[k]) < abs(es[k + 1]):
                continue
            a, b, c = us[k - 1], us[k], us[k + 1]
            fa, fb, fc = abs(es[k - 1]), abs(es[k]), abs(es[k + 1])
            for _ in range(30):
                den = (b - a) * (fb - fc) - (b - c) * (fb - fa)
                if den == 0:
                    break
                x = b - ((b - a) ** 2 * (fb - fc) - (b - c) ** 2 * (fb - fa)) / (2 * den)
                if not (a < x < c) or abs(x - b) < mp.mpf(10) ** (-(mp.mp.dps // 2)):
                    break
                fx = abs(err(mp.e ** x))
                if x < b:
                    if fx >= fb:
                        c, fc, b, fb = b, fb, x, fx
                    else:
                        a, fa = x, fx
                else:
                    if fx >= fb:
                        a, fa, b, fb = b, fb, x, fx
                    else:
                        c, fc = x, fx
            cand.append((b, err(mp.e ** b)))
        else:
            cand.append((us[k], es[k]))
    alt = []
    for u, e in cand:
        if alt and (alt[-1][1] > 0) == (e > 0):
            if abs(e) > abs(alt[-1][1]):
                alt[-1] = (u, e)
        else:
            alt.append((u, e))
    while len(alt) > m:
        if abs(alt[0][1]) <= abs(alt[-1][1]):
            alt.pop(0)
        else:
            alt.pop()
    return alt


def remez(s, lo, hi, n, dps=None, max_iter=80, delta=0.0):
    """Relative-minimax r(x) ~ x^(-s) on [lo, hi] with n partial fractions;
    with delta > 0, r(x) ~ ((x + delta) / x)^s, the ratio term of a Hasenbusch
    mass split (x + delta is the spectrum of A at m_h^2 = m^2 + delta)."""
    if not (0 < lo < hi) or n < 1 or delta < 0:
        raise ValueError("need 0 < lo < hi, n >= 1 and delta >= 0")
    if delta > 0:
        return _ratio_by_moebius(s, lo, hi, n, delta, dps, max_iter)
    dps = dps or (30 + 3 * n)
    with mp.workdps(dps):
        s_m, hi_m, d_m = mp.mpf(s), mp.mpf(hi), mp.mpf(delta)
        tlo = mp.mpf(lo) / hi_m

        def f(t):
            x = t * hi_m
            return x ** (-s_m) * (x + d_m) ** s_m if d_m > 0 else x ** (-s_m)

        m = 2 * n + 2
        ts = [tlo ** ((1 + mp.cos(mp.pi * j / (m - 1))) / 2) for j in range(m)]
        fs = [f(t) for t in ts]
        z = _levelled_newton(ts, fs, n, _linearised(ts, fs, n, None))
        emax = None
        for _ in range(max_iter):
            p, q, e_lvl = z[:n + 1], z[n + 1:2 * n + 1] + [mp.mpf(1)], z[-1]

            def err(t):
                return _horner(p, t) / (_horner(q, t) * f(t)) - 1

            alt = _extrema(err, tlo, m)
            if len(alt) < m:
                raise RuntimeError("Remez: lost alternation")
            emax = max(abs(e) for _, e in alt)
            emin = min(abs(e) for _, e in alt)
            if emax - emin <= mp.mpf("1e-7") * emax:
                break
            ts = [mp.e ** u for u, _ in alt]
            fs = [f(t) for t in ts]
            z = _levelled_newton(ts, fs, n, _linearised(ts, fs, n, q))
        else:
            raise RuntimeError("Remez did not converge")
        # partial fractions: roots of Q are -beta_i / hi, residues P(t_i) / Q'(t_i)
        roots = mp.polyroots(list(reversed(q)), maxsteps=500, extraprec=3 * dps)
        dq = [k * q[k] for k in range(1, n + 1)]
        alpha, beta = [], []
        for t_i in roots:
            if abs(mp.im(t_i)) > mp.mpf(10) ** (-(dps // 3)):
                raise RuntimeError("Remez: complex pole")
            t_i = mp.re(t_i)
            alpha.append(_horner(p, t_i) / _horner(dq, t_i) * hi_m)
            beta.append(-t_i * hi_m)
        order = sorted(range(n), key=lambda i: beta[i])
        r = RationalApprox(s, lo, hi, p[n], [alpha[i] for i in order], [beta[i] for i in order], emax)
        r.delta = float(delta)
        return r


def _ratio_by_moebius(s, lo, hi, n, delta, dps, max_iter):
    """((x + delta) / x)^s on [lo, hi] through the change of variable
    y = x / (x + delta), under which the function is y^(-s) on
    [lo / (lo + delta), hi / (hi + delta)].  y is a Moebius function of x, so a
    type (n, n) rational in y is one in x and the relative minimax error is
    the same; each partial fraction maps as
        alpha / (y + beta) = alpha / (1 + beta) (1 + (delta - b) / (x + b)),
        b = beta delta / (1 + beta)."""
    with mp.workdps(dps or (30 + 3 * n)):
        d = mp.mpf(delta)
        ry = remez(s, float(mp.mpf(lo) / (lo + d)), float(mp.mpf(hi) / (hi + d)), n, dps, max_iter)
        a0 = mp.mpf(ry.a0)
        alpha, beta = [], []
        for a, bt in zip(ry.alpha, ry.beta):
            a, bt = mp.mpf(a), mp.mpf(bt)
            b = bt * d / (1 + bt)
            a0 += a / (1 + bt)
            alpha.append(a * (d - b) / (1 + bt))
            beta.append(b)
        order = sorted(range(n), key=lambda i: beta[i])
        r = RationalApprox(s, lo, hi, a0, [alpha[i] for i in order], [beta[i] for i in order], ry.err)
        r.delta = float(delta)
        return r


def rhmc_rationals(n_flavours, n_pf, mass, n_md, n_met, upper=16.0):
    """The three rationals of one flavour: MD and Metropolis ~ x^(-s), heatbath
    ~ x^(+s/2), s = N_f / (4 n_pf), on [m^2, upper + m^2] (the spectrum of A)."""
    s = n_flavours / (4.0 * n_pf)
    lo, hi = mass * mass, upper + mass * mass
    return {"md": remez(s, lo, hi, n_md), "met": remez(s, lo, hi, n_met), "hb": remez(-s / 2, lo, hi, n_met)}


# Rationals of the standard workloads: name -> (s, m, n).  MD poles as the
# workloads state them; heatbath and Metropolis degrees chosen for a relative
# error near 1e-14 or below.
WORKLOADS = {
    "c1_md": (0.25, 0.1, 8), "c1_met": (0.25, 0.1, 16), "c1_hb": (-0.125, 0.1, 16),
    "c2_md": (0.5, 0.02, 12), "c2_met": (0.5, 0.02, 24), "c2_hb": (-0.25, 0.02, 24),
    "c3_light_md": (0.25, 0.01, 15), "c3_light_met": (0.25, 0.01, 24), "c3_light_hb": (-0.125, 0.01, 24),
    "c3_strange_md": (0.125, 0.1, 15), "c3_strange_met": (0.125, 0.1, 18), "c3_strange_hb": (-0.0625, 0.1, 18),
    "c4_md": (0.5, 0.05, 12), "c4_met": (0.5, 0.05, 20), "c4_hb": (-0.25, 0.05, 20),
    # the volume-scaling study at the paper's two masses (Sec. 6, Tables 3-4: am = 1.0 and 0.01335), N_f = 2
    "t3_high_md": (0.5, 1.0, 6), "t3_high_met": (0.5, 1.0, 10), "t3_high_hb": (-0.25, 1.0, 10),
    "t3_low_md": (0.5, 0.01335, 12), "t3_low_met": (0.5, 0.01335, 24), "t3_low_hb": (-0.25, 0.01335, 24),
    # the 16^4 N_f = 2, m = 0.02 workload with n_pf = 2, 3, 4 pseudo-fermions (s = 1 / (2 n_pf)), Sec. 2
    "c2_pf2_md": (0.25, 0.02, 12), "c2_pf2_met": (0.25, 0.02, 20), "c2_pf2_hb": (-0.125, 0.02, 20),
    "c2_pf3_md": (1.0 / 6.0, 0.02, 12), "c2_pf3_met": (1.0 / 6.0, 0.02, 20), "c2_pf3_hb": (-1.0 / 12.0, 0.02, 20),
    "c2_pf4_md": (0.125, 0.02, 12), "c2_pf4_met": (0.125, 0.02, 20), "c2_pf4_hb": (-0.0625, 0.02, 20),
    # the 16^4 workload with a Hasenbusch mass split at m_h = 0.2: the heavy term x^(-1/2) at m_h and the
    # ratio term ((x + delta) / x)^(1/2) at m = 0.02, delta = m_h^2 - m^2 = 0.0396
    "c2_heavy_md": (0.5, 0.2, 8), "c2_heavy_met": (0.5, 0.2, 14), "c2_heavy_hb": (-0.25, 0.2, 14),
    "c2_ratio_md": (0.5, 0.02, 8, 0.0396), "c2_ratio_met": (0.5, 0.02, 12, 0.0396),
    "c2_ratio_hb": (-0.25, 0.02, 12, 0.0396),
    # the improved (asqtad, tree level) 16^4 N_f = 2 workload at m = 0.02: its A has a wider spectrum,
    # bounded by m^2 + (4 sum |c|)^2 = m^2 + 58.8, so these approximate on [m^2, m^2 + 64]
    "asqtad_md": (0.5, 0.02, 14, 0.0, 64.0), "asqtad_met": (0.5, 0.02, 24, 0.0, 64.0),
    "asqtad_hb": (-0.25, 0.02, 24, 0.0, 64.0),
}
TABLE_PATH = __import__("os").path.join(__import__("os").path.dirname(__file__), "rational_table.json")


def _spec(name):
    """(s, m, n, delta, upper) of a workload rational (delta 0 unless it is a
    mass ratio; the interval is [m^2, m^2 + upper], upper 16 unless given)."""
    w = WORKLOADS[name]
    return (w[0], w[1], w[2], w[3] if len(w) > 3 else 0.0, w[4] if len(w) > 4 else 16.0)


def load(name):
    """A workload rational from the shipped table (computed by remez above),
    or computed now if the table lacks it."""
    import json
    import os
    s, m, n, delta, upper = _spec(name)
    if os.path.exists(TABLE_PATH):
        tab = json.load(open(TABLE_PATH))
        if name in tab and tab[name]["n"] == n:
            d = tab[name]
            r = RationalApprox(d["s"], d["lo"], d["hi"], d["a0"], d["alpha"], d["beta"], d["err"])
            r.delta = d.get("delta", 0.0)
            return r
    return remez(s, m * m, upper + m * m, n, delta=delta)


def write_table(names=None):
    import json
    import os
    tab = json.load(open(TABLE_PATH)) if os.path.exists(TABLE_PATH) else {}
    for name in WORKLOADS:
        s, m, n, delta, upper = _spec(name)
        if (names and name not in names) or (name in tab and tab[name]["n"] == n):
            continue
        r = remez(s, m * m, upper + m * m, n, delta=delta)
        tab[name] = {"s": r.s, "lo": r.lo, "hi": r.hi, "n": r.n, "a0": r.a0, "alpha": r.alpha, "beta": r.beta,
                     "err": r.err, "mass": m}
        if delta:
            tab[name]["delta"] = delta
        json.dump(tab, open(TABLE_PATH, "w"), indent=1)
        print(name, r.n, r.err, flush=True)


if __name__ == "__main__":
    import sys
    write_table(sys.argv[1:] or None)
