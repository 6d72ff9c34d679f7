"""HISQ staggered operator (highly improved staggered quarks) and its force.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper runs unimproved staggered fermions (Sec. 2).  HISQ (Follana et al.,
PRD 75 (2007) 054502) smears twice with a unitary projection in between:

  V = F7[U]          fat7 smearing of the thin links: 1-link 1/8, 3-staple 1/16,
                     5-staple 1/64, 7-staple 1/384 (the product of (1 + delta^2/4)
                     over the orthogonal directions, oracle/asqtad.py)
  W = V (V^dag V)^(-1/2)          the U(3) projection (polar factor) of V
  X = F7L[W]         fat7 again with a doubled Lepage term: -2/16 per
                     double-width staple and +6/8 moved to the 1-link, which
                     cancels the O(a^2) low-momentum distortion of both
                     smearings; +1/8 more on the 1-link for the Naik
                     normalisation: 1-link 1, 3-staple 1/16, 5-staple 1/64,
                     7-staple 1/384, Lepage -1/8
  N = -1/24 W(x) W(x+mu) W(x+2mu) the Naik link, from the projected links
                     (light quarks: no mass-dependent correction)

and D is the operator of oracle/asqtad.py with fat links X and Naik links N.
At U = 1: X = 9/8, N = -1/24, the asqtad free field.  The time boundary sign
sits in the thin links before the first smearing (the projection commutes
with a sign).

The force runs the chain rule backwards through the three maps with matrix
cotangents C (Re tr[C dA] for an arbitrary variation dA of a matrix A):
through a path product a link met forward gets the rest of the loop R, a
link met backward R^dag; through the projection, with Q = V^dag V = E L E^dag,
  C_V = Q^(-1/2) C_W + (M + M^dag) V^dag,  M = E (F o (E^dag C_W V E)) E^dag,
F_ij the divided differences of x^(-1/2) at the eigenvalues of Q; and
F_a = Re tr[i T_a U C_U] for U -> exp(i omega_a T_a) U.
"""
import numpy as np

from . import asqtad, lattice as lat
from .su3 import T, dag

FAT7 = {"one": 1.0 / 8.0, "staple3": 1.0 / 16.0, "staple5": 1.0 / 64.0, "staple7": 1.0 / 384.0, "lepage": 0.0}
LEVEL2 = {"one": 1.0, "staple3": 1.0 / 16.0, "staple5": 1.0 / 64.0, "staple7": 1.0 / 384.0, "lepage": -1.0 / 8.0}
NAIK = -1.0 / 24.0


def smear(links, coef):
    """sum over the fat paths of every direction of coef[class] x path product."""
    out = np.zeros_like(links)
    for mu in range(4):
        for name, steps in asqtad.fat_paths(mu):
            if coef[name] != 0.0:
                out[mu] += coef[name] * asqtad.path_product(links, steps)
    return out


def project_u3(v):
    """W = V (V^dag V)^(-1/2), by the eigen-decomposition of V^dag V."""
    q = dag(v) @ v
    lam, e = np.linalg.eigh(q)
    return v @ (e * lam[..., None, :] ** -0.5) @ dag(e)


def hisq_links(u, antiperiodic_t=True):
    """(X, N, W, V): level-2 fat links, Naik links, the projected and the
    level-1 links [4, t, z, y, x, 3, 3] of the thin links u."""
    up = asqtad.boundary_signed_links(u, antiperiodic_t)
    v = smear(up, FAT7)
    w = project_u3(v)
    x = smear(w, LEVEL2)
    n = np.stack([NAIK * asqtad.path_product(w, asqtad.naik_path(mu)) for mu in range(4)])
    return x, n, w, v


def path_cotangents(links, outer, coef, naik_outer=None):
    """Matrix cotangent of every link of `links` for the functional
    sum_{x,mu} Re tr[S_mu(x) outer_mu(x)] with S = sum_paths coef x path
    product (plus, with naik_outer, Re tr[Naik_mu(x) naik_outer_mu(x)] for the
    Naik path of coefficient NAIK)."""
    c = np.zeros_like(links)
    for mu in range(4):
        terms = [(coef[name], steps, outer[mu]) for name, steps in asqtad.fat_paths(mu) if coef[name] != 0.0]
        if naik_outer is not None:
            terms.append((NAIK, asqtad.naik_path(mu), naik_outer[mu]))
        for cf, steps, xm in terms:
            walk, _ = asqtad._walk(links, steps)
            n = len(walk)
            eye = np.broadcast_to(np.eye(3, dtype=complex), links.shape[1:])
            pre = [eye]
            for a, _, _, _ in walk:
                pre.append(pre[-1] @ a)
            suf = [eye] * (n + 1)
            for k in range(n - 1, -1, -1):
                suf[k] = walk[k][0] @ suf[k + 1]
            for k, (_, d, nu, fwd) in enumerate(walk):
                r = asqtad._at(suf[k + 1] @ xm @ pre[k], -d)
                c[nu] += cf * (r if fwd else dag(r))
    return c


def project_cotangent(v, c_w):
    """C_V from C_W through W = V (V^dag V)^(-1/2)."""
    q = dag(v) @ v
    lam, e = np.linalg.eigh(q)
    s = lam ** -0.5
    li, lj = lam[..., :, None], lam[..., None, :]
    si, sj = s[..., :, None], s[..., None, :]
    same = np.abs(li - lj) <= 1e-12 * np.maximum(np.abs(li), np.abs(lj))
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(same, -0.5 * si ** 3, (si - sj) / (li - lj))
    q_inv_sqrt = (e * s[..., None, :]) @ dag(e)
    k = dag(e) @ (c_w @ v) @ e
    m = e @ (f * k) @ dag(e)
    return q_inv_sqrt @ c_w + (m + dag(m)) @ dag(v)


def _coeff_of_i_t(m):
    return np.real(1j * np.einsum("aij,...ji->...a", T, m))


def fermion_force(u, xs, alphas, par, antiperiodic_t=True):
    """F_a = d S / d omega_a of S = sum_i alpha_i phi^dag X_i through the HISQ
    links, X_i = (A + beta_i)^(-1) phi on even sites (as oracle/asqtad.py,
    whose outer-product fields Xv, Xw are the cotangents of X and N)."""
    dims = (u.shape[4], u.shape[3], u.shape[2], u.shape[1])
    eta0 = lat.eta(dims, antiperiodic_t=False)
    epsx = np.where(par == 0, 1.0, -1.0)
    up = asqtad.boundary_signed_links(u, antiperiodic_t)
    x, n, w, v = hisq_links(u, antiperiodic_t)
    xv = np.zeros_like(u)
    xw = np.zeros_like(u)
    for a_i, xsol in zip(alphas, xs):
        z = asqtad.restrict(xsol, par, 0) + asqtad.d_block(x, n, xsol, eta0, par, 1)
        for mu in range(4):
            d1 = np.zeros(4, dtype=int)
            d1[mu] = 1
            s = (a_i * epsx * eta0[mu])[..., None, None]
            xv[mu] += s * (asqtad._at(z, d1)[..., :, None] * np.conj(z)[..., None, :])
            xw[mu] += s * (asqtad._at(z, 3 * d1)[..., :, None] * np.conj(z)[..., None, :])
    c_w = path_cotangents(w, xv, LEVEL2, naik_outer=xw)
    c_v = project_cotangent(v, c_w)
    c_u = path_cotangents(up, c_v, FAT7)
    return np.stack([_coeff_of_i_t(up[nu] @ c_u[nu]) for nu in range(4)])
