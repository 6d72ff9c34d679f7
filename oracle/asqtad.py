"""Improved staggered (asqtad) operator and its fermion force.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper runs standard, unimproved staggered fermions (Sec. 2).  The
improved operator here is the a^2-improved ("asqtad") staggered action of
Lepage, PRD 59 (1999) 074502, and Orginos, Toussaint, Sugar, PRD 60 (1999)
054503, written out from its construction:

  D psi(x) = 1/2 sum_mu eta_mu(x) [ V_mu(x) psi(x+mu) - V_mu(x-mu)^dag psi(x-mu)
                                  + W_mu(x) psi(x+3mu) - W_mu(x-3mu)^dag psi(x-3mu) ]

* W_mu(x) = c_N U_mu(x) U_mu(x+mu) U_mu(x+2mu), the Naik term: with
  c_N = -1/24 and a one-hop coefficient of 9/8 at U = 1 the free derivative
  is 9/8 sin p - 1/24 sin 3p = p + O(p^5).
* V_mu(x), the fat link: a sum over paths from x to x+mu.  The product
  over the three orthogonal directions rho of (1 + delta_rho^2 / 4), with
  delta_rho^2 the covariant second difference, cancels the coupling to
  gluons of momentum pi in any orthogonal direction; expanded it is the
  1-link term (1/8), 6 three-link staples (1/16 each), 24 five-link
  staples (1/64) and 48 seven-link staples (1/384).  The Lepage term,
  -(1/16) per double-width staple in each of the 6 orthogonal directions
  with +3/8 moved to the 1-link term, removes the O(a^2) low-momentum
  distortion this smearing introduces; the Naik normalisation adds 1/8
  more to the 1-link term.  Resulting coefficients:
      1-link 5/8, 3-staple 1/16, 5-staple 1/64, 7-staple 1/384,
      Lepage -1/16, Naik -1/24,
  each path of n links divided by u0^(n-1) (tadpole factor u0; u0 = 1 gives
  the tree-level action).  At U = 1: V = 9/8, W = -1/24.

Boundary conditions: the antiperiodic time boundary of the fermions is put
into the thin links (every t-link leaving the last time slice times -1)
before the paths are multiplied, so that each path carries the sign of the
boundary crossings it makes; eta carries no boundary sign here.

Fields are whole-lattice arrays as in the rest of the oracle:
gauge U[mu, t, z, y, x, 3, 3], field psi[t, z, y, x, 3].  A signed step
s = +(nu+1) or -(nu+1) moves by +nu_hat or -nu_hat.
"""
import itertools

import numpy as np

from . import lattice as lat
from .su3 import T, dag


def coefficients(u0=1.0):
    """Path coefficients of the asqtad action, tadpole-improved by u0."""
    return {
        "one": 5.0 / 8.0,
        "staple3": 1.0 / 16.0 / u0 ** 2,
        "staple5": 1.0 / 64.0 / u0 ** 4,
        "staple7": 1.0 / 384.0 / u0 ** 6,
        "lepage": -1.0 / 16.0 / u0 ** 4,
        "naik": -1.0 / 24.0 / u0 ** 2,
    }


def fat_paths(mu):
    """Every path of the fat link V_mu as (coefficient name, steps)."""
    m = mu + 1
    perp = [d for d in range(4) if d != mu]
    paths = [("one", [m])]
    for nu in perp:
        for sn in (1, -1):
            a = sn * (nu + 1)
            paths.append(("staple3", [a, m, -a]))
            paths.append(("lepage", [a, a, m, -a, -a]))
    for nu, rho in itertools.permutations(perp, 2):
        for sn, sr in itertools.product((1, -1), repeat=2):
            a, b = sn * (nu + 1), sr * (rho + 1)
            paths.append(("staple5", [a, b, m, -b, -a]))
    for nu, rho, sig in itertools.permutations(perp, 3):
        for sn, sr, ss in itertools.product((1, -1), repeat=3):
            a, b, c = sn * (nu + 1), sr * (rho + 1), ss * (sig + 1)
            paths.append(("staple7", [a, b, c, m, -c, -b, -a]))
    return paths


def naik_path(mu):
    return [mu + 1] * 3


def boundary_signed_links(u, antiperiodic_t=True):
    """Thin links with the fermions' time boundary sign folded in."""
    up = u.copy()
    if antiperiodic_t:
        up[3, -1] = -up[3, -1]
    return up


def _at(f, d):
    """g(x) = f(x + d) for an integer offset d = (dx, dy, dz, dt), periodic."""
    return np.roll(f, shift=(-d[3], -d[2], -d[1], -d[0]), axis=(0, 1, 2, 3))


def _walk(u, steps):
    """The links met along a path started at every site x: a list of
    (link field A_k over x, offset of the link's site, direction, forward),
    where A_k = U_nu(x + d) for a forward step and U_nu(x + d - nu)^dag for
    a backward one, d the position reached before the step."""
    d = np.zeros(4, dtype=int)
    out = []
    for s in steps:
        nu = abs(s) - 1
        e = np.eye(4, dtype=int)[nu]
        if s > 0:
            out.append((_at(u[nu], d), d.copy(), nu, True))
            d = d + e
        else:
            d = d - e
            out.append((dag(_at(u[nu], d)), d.copy(), nu, False))
    return out, d


def path_product(u, steps):
    """Product of the links along the path, for every start site."""
    links, _ = _walk(u, steps)
    p = links[0][0]
    for a, _, _, _ in links[1:]:
        p = p @ a
    return p


def fat_long_links(u, u0=1.0, antiperiodic_t=True):
    """(V, W): fat and Naik links [4, t, z, y, x, 3, 3] of the thin links u."""
    c = coefficients(u0)
    up = boundary_signed_links(u, antiperiodic_t)
    v = np.zeros_like(u)
    w = np.zeros_like(u)
    for mu in range(4):
        for name, steps in fat_paths(mu):
            v[mu] += c[name] * path_product(up, steps)
        w[mu] = c["naik"] * path_product(up, naik_path(mu))
    return v, w


def _hop(link, psi, mu, n):
    """sum of the forward and backward n-hops along mu through the given links
    (without eta):  link(x) psi(x + n mu) - link(x - n mu)^dag psi(x - n mu)."""
    d = np.zeros(4, dtype=int)
    d[mu] = n
    fwd = np.einsum("...ij,...j->...i", link, _at(psi, d))
    bwd = _at(np.einsum("...ij,...j->...i", dag(link), psi), -d)
    return fwd - bwd


def dslash(v, w, psi, eta0):
    """D psi for fat links v, Naik links w and phases eta0 (no boundary sign)."""
    out = np.zeros_like(psi)
    for mu in range(4):
        out += 0.5 * eta0[mu][..., None] * (_hop(v[mu], psi, mu, 1) + _hop(w[mu], psi, mu, 3))
    return out


def restrict(psi, par, p):
    return np.where((par == p)[..., None], psi, 0.0)


def d_block(v, w, psi, eta0, par, out_parity):
    """D_{out, in}: a field on parity 1-out_parity to one on out_parity."""
    return restrict(dslash(v, w, restrict(psi, par, 1 - out_parity), eta0), par, out_parity)


def a_op(v, w, psi_e, mass, eta0, par, shift=0.0):
    """(A + shift) psi_e,  A = m^2 - D_eo D_oe on even sites."""
    tmp = d_block(v, w, psi_e, eta0, par, 1)
    return (mass * mass + shift) * restrict(psi_e, par, 0) - d_block(v, w, tmp, eta0, par, 0)


def dense_dslash(v, w, eta0):
    """D as a dense matrix by applying it to unit vectors (tiny lattices)."""
    shape = v.shape[1:5]
    n = 3 * int(np.prod(shape))
    mat = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1.0
        mat[:, k] = dslash(v, w, e.reshape(shape + (3,)), eta0).reshape(n)
    return mat


def norm_bound(u0=1.0):
    """Upper bound of ||D||: every hop term of direction mu is at most the
    sum of |coefficients| of its paths (products of unitary links), and
    1/2 (T - T^-1) has norm <= 1 per term, so ||D|| <= sum_mu (||V|| + ||W||)."""
    c = coefficients(u0)
    fat = abs(c["one"]) + 6 * abs(c["staple3"]) + 24 * abs(c["staple5"]) + 48 * abs(c["staple7"]) \
        + 6 * abs(c["lepage"])
    return 4.0 * (fat + abs(c["naik"]))


def _coeff_of_i_t(m):
    """Re tr(i T_a M) for every a: shape [..., 8]."""
    return np.real(1j * np.einsum("aij,...ji->...a", T, m))


def fermion_force(u, xs, alphas, par, u0=1.0, antiperiodic_t=True):
    """Force F_a(y, nu) = d S / d omega_a under U_nu(y) -> exp(i omega_a T_a) U_nu(y)
    of S = sum_i alpha_i phi^dag X_i, X_i = (A + beta_i)^(-1) phi (even fields).

    As for the unimproved operator, d(phi^dag (A+beta)^(-1) phi) =
    sum_x eps(x) Z(x)^dag (dD Z)(x) with Z = X (even) + D_oe X (odd), which
    collects into  dS = sum_{x,mu} Re tr[dV_mu(x) Xv_mu(x) + dW_mu(x) Xw_mu(x)],
      Xv_mu(x) = sum_i alpha_i eps(x) eta_mu(x) Z_i(x+mu) Z_i(x)^dag,
      Xw_mu(x) = sum_i alpha_i eps(x) eta_mu(x) Z_i(x+3mu) Z_i(x)^dag.
    Every path product c A_1 ... A_n of V or W then contributes, for each of
    its links, with R_k = A_{k+1} ... A_n X A_1 ... A_{k-1}:
      F_a += c Re tr[i T_a U R_k]                 (link met forward, A_k = U)
      F_a += c Re tr[i T_a U (-U^dag R_k U^dag)]  (met backward, A_k = U^dag)
    Everything is evaluated with the boundary-signed links, which have the
    same derivative.  The sign is pinned by finite differences of S.
    """
    dims = (u.shape[4], u.shape[3], u.shape[2], u.shape[1])
    eta0 = lat.eta(dims, antiperiodic_t=False)
    epsx = np.where(par == 0, 1.0, -1.0)
    c = coefficients(u0)
    up = boundary_signed_links(u, antiperiodic_t)
    v, w = fat_long_links(u, u0, antiperiodic_t)
    xv = np.zeros_like(u)
    xw = np.zeros_like(u)
    for a_i, x in zip(alphas, xs):
        z = restrict(x, par, 0) + d_block(v, w, x, eta0, par, 1)
        for mu in range(4):
            d1 = np.zeros(4, dtype=int)
            d1[mu] = 1
            s = (a_i * epsx * eta0[mu])[..., None, None]
            xv[mu] += s * (_at(z, d1)[..., :, None] * np.conj(z)[..., None, :])
            xw[mu] += s * (_at(z, 3 * d1)[..., :, None] * np.conj(z)[..., None, :])
    g = np.zeros_like(u)
    eye = np.broadcast_to(np.eye(3, dtype=complex), u.shape[1:])
    for mu in range(4):
        terms = [(c[name], steps, xv[mu]) for name, steps in fat_paths(mu)]
        terms.append((c["naik"], naik_path(mu), xw[mu]))
        for coef, steps, xm in terms:
            links, _ = _walk(up, steps)
            n = len(links)
            pre = [eye]
            for a, _, _, _ in links:
                pre.append(pre[-1] @ a)
            suf = [eye] * (n + 1)
            for k in range(n - 1, -1, -1):
                suf[k] = links[k][0] @ suf[k + 1]
            for k, (_, d, nu, fwd) in enumerate(links):
                r = suf[k + 1] @ xm @ pre[k]
                if fwd:
                    g[nu] += coef * _at(r, -d)
                else:
                    r_at = _at(r, -d)
                    g[nu] -= coef * (dag(up[nu]) @ r_at @ dag(up[nu]))
    return np.stack([_coeff_of_i_t(up[nu] @ g[nu]) for nu in range(4)])
