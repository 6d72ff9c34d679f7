"""Minimax rational approximation for RHMC (paper Sec. 2: "different rational
approximations and stopping residuals for Metropolis step and Molecular
Dynamic"; ref. [rhmc] Horvath, Kennedy, Sint).

r(x) = alpha_0 + sum_i alpha_i / (x + beta_i)  approximates  x^(-s)  on
[lo, hi] with the smallest maximum RELATIVE error (the error metric is not
stated in the paper; relative minimax is the standard RHMC choice).

Method: classical Remez exchange for a type (n, n) rational P/Q with monic Q,
in multiprecision (mpmath).  Reference set of 2n+2 points x_j; the levelled
equations
        P(x_j) - f(x_j) Q(x_j) = (-1)^j E f(x_j) Q(x_j)
are solved by iterating the linear system in which the right-hand Q is the
previous iterate; the new reference set is the set of extrema of the
relative error e(x) = P(x) / (Q(x) f(x)) - 1 between its zeros.  Converged
when max|e| equals |E| to a relative 1e-6.  The partial fractions follow from
the roots of Q and the residues P(t_i) / Q'(t_i).
"""
import mpmath as mp


def _solve_levelled(ts, fs, n, q_old):
    """One linear solve of the levelled equations in the scaled variable t."""
    m = 2 * n + 2
    a = mp.matrix(m, m)
    rhs = mp.matrix(m, 1)
    for j, (t, f) in enumerate(zip(ts, fs)):
        tk = mp.mpf(1)
        for k in range(n + 1):                # P coefficients p_0..p_n
            a[j, k] = tk
            if k < n:                          # Q coefficients q_0..q_{n-1}
                a[j, n + 1 + k] = -f * tk
            tk *= t
        a[j, 2 * n + 1] = -((-1) ** j) * f * q_old(t)
        rhs[j] = f * t ** n
    z = mp.lu_solve(a, rhs)
    p = [z[k] for k in range(n + 1)]
    q = [z[n + 1 + k] for k in range(n)] + [mp.mpf(1)]
    return p, q, z[2 * n + 1]


def _polyval(c, t):
    acc = mp.mpf(0)
    for ck in reversed(c):
        acc = acc * t + ck
    return acc


def _golden_max(g, a, b, iters=80):
    """Maximiser of |g| on [a, b] (unimodal in each extremum interval)."""
    invphi = (mp.sqrt(5) - 1) / 2
    c = b - invphi * (b - a)
    d = a + invphi * (b - a)
    gc, gd = abs(g(c)), abs(g(d))
    for _ in range(iters):
        if gc > gd:
            b, d, gd = d, c, gc
            c = b - invphi * (b - a)
            gc = abs(g(c))
        else:
            a, c, gc = c, d, gd
            d = a + invphi * (b - a)
            gd = abs(g(d))
    cand = [(abs(g(a)), a), (abs(g(b)), b), (gc, c), (gd, d)]
    return max(cand)[1]


class Rational:
    """alpha_0 + sum_i alpha_i / (x + beta_i), with its minimax error."""

    def __init__(self, s, lo, hi, a0, alpha, beta, err, delta=0.0):
        self.s, self.lo, self.hi = s, lo, hi
        self.a0, self.alpha, self.beta, self.err = a0, alpha, beta, err
        self.delta = delta      # 0: x^(-s); > 0: x^(-s) (x + delta)^s

    def __call__(self, x):
        return self.a0 + sum(a / (x + b) for a, b in zip(self.alpha, self.beta))

    def as_dict(self):
        d = {"s": self.s, "lo": self.lo, "hi": self.hi, "n": len(self.alpha),
             "a0": self.a0, "alpha": list(self.alpha), "beta": list(self.beta),
             "err": self.err}
        if self.delta:
            d["delta"] = self.delta
        return d


def remez(s, lo, hi, n, dps=80, max_iter=60, verbose=False, delta=0.0):
    """Relative-minimax type (n, n) approximation of x^(-s) on [lo, hi], or,
    with delta > 0, of the mass-ratio function x^(-s) (x + delta)^s: for
    A = m^2 - D_eo D_oe with spectrum x, (x + delta) is the spectrum of the
    same operator at the heavier mass m_h^2 = m^2 + delta, so
    r(A) ~ (A_h / A)^s is the ratio term of a Hasenbusch mass split
    det(A)^s = det(A_h)^s det(A / A_h)^s."""
    with mp.workdps(dps):
        lo_m, hi_m, s_m, d_m = mp.mpf(lo), mp.mpf(hi), mp.mpf(s), mp.mpf(delta)
        scale = hi_m

        def f_t(t):                        # f as a function of t = x / hi
            x = t * scale
            return x ** (-s_m) * (x + d_m) ** s_m if d_m > 0 else x ** (-s_m)

        tlo = lo_m / scale
        m = 2 * n + 2
        # initial reference: Chebyshev points in log x
        ts = [tlo * (1 / tlo) ** ((1 - mp.cos(mp.pi * j / (m - 1))) / 2) for j in range(m)]
        q_prev = None
        err = None
        for it in range(max_iter):
            fs = [f_t(t) for t in ts]
            q_old = (lambda t: mp.mpf(1)) if q_prev is None else (lambda t, c=q_prev: _polyval(c, t))
            for _ in range(30):
                p, q, e_lvl = _solve_levelled(ts, fs, n, q_old)
                q_new = q
                q_old = (lambda t, c=q_new: _polyval(c, t))
                # stop the inner linearisation once Q is stationary at the points
                if _ > 0 and abs(e_lvl - e_prev) <= abs(e_lvl) * mp.mpf(10) ** (-(dps // 3)):
                    break
                e_prev = e_lvl
            q_prev = q

            def e(t):
                return _polyval(p, t) / (_polyval(q, t) * f_t(t)) - 1

            # zeros of e between consecutive reference points
            zs = []
            for j in range(m - 1):
                a_, b_ = ts[j], ts[j + 1]
                ea = e(a_)
                for _ in range(100):
                    c_ = (a_ + b_) / 2
                    ec = e(c_)
                    if (ec > 0) == (ea > 0):
                        a_, ea = c_, ec
                    else:
                        b_ = c_
                zs.append((a_ + b_) / 2)
            edges = [tlo] + zs + [mp.mpf(1)]
            new_ts = []
            for j in range(m):
                a_, b_ = edges[j], edges[j + 1]
                # search in log t, where the extrema are spread evenly
                g = lambda u: e(mp.e ** u)
                new_ts.append(mp.e ** _golden_max(g, mp.log(a_), mp.log(b_)))
            new_ts[0], new_ts[-1] = tlo, mp.mpf(1)
            emax = max(abs(e(t)) for t in new_ts)
            if verbose:
                print(it, mp.nstr(e_lvl, 8), mp.nstr(emax, 8))
            ts = new_ts
            if abs(emax - abs(e_lvl)) <= mp.mpf("1e-6") * abs(e_lvl):
                err = emax
                break
        if err is None:
            raise RuntimeError("Remez did not converge")
        roots = mp.polyroots(list(reversed(q)), maxsteps=400, extraprec=4 * dps)
        dq = [k * q[k] for k in range(1, n + 1)]
        alpha, beta = [], []
        for t_i in roots:
            t_i = mp.re(t_i) if abs(mp.im(t_i)) < mp.mpf(10) ** (-dps // 2) else t_i
            if isinstance(t_i, mp.mpc):
                raise RuntimeError("complex pole")
            c_i = _polyval(p, t_i) / _polyval(dq, t_i)
            alpha.append(float(c_i * scale))
            beta.append(float(-t_i * scale))
        order = sorted(range(n), key=lambda i: beta[i])
        alpha = [alpha[i] for i in order]
        beta = [beta[i] for i in order]
        r = Rational(float(s), float(lo), float(hi), float(p[n]), alpha, beta, float(err))
        r.delta = float(delta)
        return r


def apply_rational(r, solve_shifted, phi):
    """r(A) phi = alpha_0 phi + sum_i alpha_i (A + beta_i)^(-1) phi, given the
    multi-shift solutions X_i = (A + beta_i)^(-1) phi from solve_shifted."""
    xs = solve_shifted(phi, r.beta)
    out = r.a0 * phi
    for a, x in zip(r.alpha, xs):
        out = out + a * x
    return out
