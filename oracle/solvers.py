"""Krylov solvers (paper Sec. 6: CG is "the optimal choice" for staggered
fermions; shifted systems for RHMC use a multi-shift solver, ref. [shift] =
B. Jegerlehner, hep-lat/9612014).

`apply(v)` is any Hermitian positive-definite operator on numpy arrays.
Norms are ||v||^2 = sum over all entries of Re^2 + Im^2.
"""
import numpy as np


def _dot(a, b):
    return np.vdot(a, b)


def _norm2(a):
    return float(np.real(np.vdot(a, a)))


def cg(apply, b, tol, max_iter=100000, x0=None):
    """Textbook conjugate gradient for apply(x) = b.

    Stops when the recursive residual satisfies ||r|| <= tol ||b||; returns
    (x, iterations, true relative residual ||b - A x|| / ||b||).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = _norm2(r)
    bb = _norm2(b)
    k = 0
    while rr > tol * tol * bb and k < max_iter:
        q = apply(p)
        alpha = rr / float(np.real(_dot(p, q)))
        x = x + alpha * p
        r = r - alpha * q
        rr_new = _norm2(r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        k += 1
    true_res = np.sqrt(_norm2(b - apply(x)) / bb)
    return x, k, true_res


def multishift_cg(apply0, b, shifts, tol, max_iter=100000):
    """Solve (A + sigma_i) x_i = b for every shift with one Krylov space.

    apply0(v) = (A + sigma_0) v for the base shift sigma_0 = min(shifts).
    Start: x_i = 0, r = p = p_i = b, zeta_{-1} = zeta_0 = 1, alpha_{-1} = 1,
    beta_{-1} = 0.  Iteration k (standard CG signs):
        alpha_k   = (r, r) / (p, A0 p)
        zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
                    [alpha_k beta_{k-1} (zeta_{k-1} - zeta_k)
                     + zeta_{k-1} alpha_{k-1} (1 + (sigma_i - sigma_0) alpha_k)]
        alpha_k^i = alpha_k zeta_{k+1} / zeta_k ;   x_i += alpha_k^i p_i
        r        -= alpha_k A0 p ;  beta_k = (r', r') / (r, r)
        beta_k^i  = beta_k (zeta_{k+1} / zeta_k)^2
        p_i       = zeta_{k+1} r' + beta_k^i p_i ;  p = r' + beta_k p
    Shift i is frozen once |zeta^i| ||r|| <= tol ||b|| (its residual is
    zeta^i r); the loop ends when the base system converges.
    Returns (list of x_i, iterations, list of per-shift iteration counts).
    """
    shifts = np.asarray(shifts, dtype=float)
    n = len(shifts)
    s0 = float(np.min(shifts))
    ds = shifts - s0
    x = [np.zeros_like(b) for _ in range(n)]
    ps = [b.copy() for _ in range(n)]
    r = b.copy()
    p = b.copy()
    zeta_prev = np.ones(n)
    zeta = np.ones(n)
    alpha_prev = 1.0
    beta_prev = 0.0
    bb = _norm2(b)
    rr = bb
    live = np.ones(n, dtype=bool)
    iters_at = np.zeros(n, dtype=int)
    k = 0
    while k < max_iter and np.any(live):
        q = apply0(p)
        alpha = rr / float(np.real(_dot(p, q)))
        zeta_next = np.empty(n)
        for i in range(n):
            if not live[i]:
                zeta_next[i] = zeta[i]
                continue
            den = (alpha * beta_prev * (zeta_prev[i] - zeta[i])
                   + zeta_prev[i] * alpha_prev * (1.0 + ds[i] * alpha))
            zeta_next[i] = zeta[i] * zeta_prev[i] * alpha_prev / den
            x[i] = x[i] + (alpha * zeta_next[i] / zeta[i]) * ps[i]
        r = r - alpha * q
        rr_new = _norm2(r)
        beta = rr_new / rr
        for i in range(n):
            if not live[i]:
                continue
            beta_i = beta * (zeta_next[i] / zeta[i]) ** 2
            ps[i] = zeta_next[i] * r + beta_i * ps[i]
        p = r + beta * p
        zeta_prev, zeta = zeta, zeta_next
        alpha_prev, beta_prev = alpha, beta
        rr = rr_new
        k += 1
        for i in range(n):
            if live[i] and abs(zeta[i]) * np.sqrt(rr) <= tol * np.sqrt(bb):
                live[i] = False
                iters_at[i] = k
    iters_at[live] = k
    return x, k, iters_at
