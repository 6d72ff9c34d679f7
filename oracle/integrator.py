"""RHMC trajectory (paper Sec. 2 and Sec. 4; ref. [rhmc] Horvath, Kennedy,
Sint; ref. [hmc] Duane, Kennedy, Pendleton, Roweth).

  * pseudo-fermion heatbath  phi = r_hb(A) xi,  xi ~ exp(-xi^dag xi)
  * multi-step integrator: the fermion force on the outer level, the gauge
    force on an inner level with n_gauge substeps per outer half step
  * both levels use the second-order minimum-norm scheme
        p += -lam h F;  U-update h/2;  p += -(1-2 lam) h F;  U-update h/2;  p += -lam h F
    with lam = 0.1931833275037836 (Omelyan, Mryglod, Folk 2002; the paper
    names the scheme but not the constant)
  * optionally (not in the paper: the learned-surrogate workload) three levels:
    the remainder F_f - F^ on the outer level, the surrogate force F^
    (oracle/surrogate.py) on n_mid minimum-norm steps per outer half step,
    the gauge level inside those; the levels add up to the exact force, so
    the integrator stays reversible and area-preserving for any F^
  * a flavour term may sit on that middle level instead of the outer one
    (Flavour.level = 1): a Hasenbusch mass split puts the heavy term, whose
    force is large and whose solves are cheap, on the middle level and the
    light-over-heavy ratio term, small force and expensive solves, outside
    (the paper's multiple pseudo-fermions, Sec. 2, extended by a mass split)
  * Metropolis on dH = H_f - H_i with H = 1/2 sum p_a^2 + S_g + S_f, where the
    final S_f uses the Metropolis rational (tighter than the MD one, Sec. 2)
    and the initial S_f = xi^dag xi.
  * the fermion operator is the paper's unimproved one, or (action =
    "asqtad" or "hisq", not in the paper) the improved operators of
    oracle/asqtad.py and oracle/hisq.py with their fermion forces; the gauge
    action stays Wilson's either way.
Everything here is float64 (the oracle reference for all precision modes).
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import asqtad, dirac, hisq, lattice as lat, solvers, su3
from . import surrogate as sur
from .actions import fermion_action, fermion_force, wilson_action, wilson_force

LAMBDA_2MN = 0.1931833275037836


@dataclass
class Flavour:
    mass: float
    hb: object          # rational for the heatbath, ~ x^(+s/2)
    md: object          # rational for the MD force, ~ x^(-s)
    met: object         # rational for the Metropolis action, ~ x^(-s)
    n_pf: int = 1
    level: int = 0      # 0: outer integration level; 1: the middle level


@dataclass
class HMCParams:
    dims: tuple
    beta: float
    tau: float
    n_outer: int
    n_gauge: int
    flavours: List[Flavour] = field(default_factory=list)
    tol_md: float = 1e-10
    tol_met: float = 1e-14
    antiperiodic_t: bool = True
    action: str = "unimproved"     # or "asqtad", "hisq"
    u0: float = 1.0                # tadpole factor of the asqtad paths


class Context:
    def __init__(self, p: HMCParams):
        self.p = p
        self.eta = lat.eta(p.dims, p.antiperiodic_t)
        self.par = lat.parity(p.dims)

    def shifted_solves(self, u, mass, phi, betas, tol):
        if self.p.action in ("asqtad", "hisq"):
            if self.p.action == "asqtad":
                fat, naik = asqtad.fat_long_links(u, self.p.u0, self.p.antiperiodic_t)
            else:
                fat, naik, _, _ = hisq.hisq_links(u, self.p.antiperiodic_t)
            eta0 = lat.eta(self.p.dims, antiperiodic_t=False)

            def apply0(v, s0=min(betas)):
                return asqtad.a_op(fat, naik, v, mass, eta0, self.par, s0)
        else:
            def apply0(v, s0=min(betas)):
                return dirac.a_op(u, v, mass, self.eta, self.par, s0)
        xs, _, _ = solvers.multishift_cg(apply0, phi, betas, tol)
        return xs

    def rational_apply(self, u, mass, rat, phi, tol):
        xs = self.shifted_solves(u, mass, phi, rat.beta, tol)
        out = rat.a0 * phi
        for a, x in zip(rat.alpha, xs):
            out = out + a * x
        return out, xs

    def fermion_force_total(self, u, phis, level=None):
        """Summed force of the flavour terms on one integration level (all with level None)."""
        f = np.zeros(u.shape[:5] + (8,))
        for fl, phi_list in zip(self.p.flavours, phis):
            if level is not None and fl.level != level:
                continue
            for phi in phi_list:
                xs = self.shifted_solves(u, fl.mass, phi, fl.md.beta, self.p.tol_md)
                if self.p.action == "asqtad":
                    f += asqtad.fermion_force(u, xs, fl.md.alpha, self.par, self.p.u0, self.p.antiperiodic_t)
                elif self.p.action == "hisq":
                    f += hisq.fermion_force(u, xs, fl.md.alpha, self.par, self.p.antiperiodic_t)
                else:
                    f += fermion_force(u, xs, fl.md.alpha, self.eta, self.par)
        return f

    def fermion_action_total(self, u, phis, tol):
        s = 0.0
        for fl, phi_list in zip(self.p.flavours, phis):
            for phi in phi_list:
                xs = self.shifted_solves(u, fl.mass, phi, fl.met.beta, tol)
                s += fermion_action(phi, xs, fl.met)
        return s


def update_links(u, mom, h):
    """U_mu(x) <- exp(i h P_mu(x)) U_mu(x)."""
    return np.einsum("...ij,...jk->...ik", su3.expi_coeffs(mom, h), u)


def gauge_level(u, mom, h, n, beta):
    """n minimum-norm steps of size h/n with the gauge force only."""
    d = h / n
    for _ in range(n):
        mom = mom - LAMBDA_2MN * d * wilson_force(u, beta)
        u = update_links(u, mom, d / 2)
        mom = mom - (1 - 2 * LAMBDA_2MN) * d * wilson_force(u, beta)
        u = update_links(u, mom, d / 2)
        mom = mom - LAMBDA_2MN * d * wilson_force(u, beta)
    return u, mom


def surrogate_force(u, params):
    """F^ of the links u for the network params (oracle/surrogate.py); a true
    "quant" entry evaluates the network as tensor cores do (bf16 inputs of
    every product)."""
    f, G = sur.features_and_generators(u)
    return sur.surrogate_force(params, f, G, quant=bool(params.get("quant", False)))


def middle_level(u, mom, h, n_mid, n_gauge, beta, force):
    """n_mid minimum-norm steps of size h/n_mid with force(u), the gauge
    level for the link updates."""
    d = h / n_mid
    for _ in range(n_mid):
        mom = mom - LAMBDA_2MN * d * force(u)
        u, mom = gauge_level(u, mom, d / 2, n_gauge, beta)
        mom = mom - (1 - 2 * LAMBDA_2MN) * d * force(u)
        u, mom = gauge_level(u, mom, d / 2, n_gauge, beta)
        mom = mom - LAMBDA_2MN * d * force(u)
    return u, mom


def surrogate_level(u, mom, h, n_mid, n_gauge, beta, params):
    """n_mid minimum-norm steps of size h/n_mid with the surrogate force F^,
    the gauge level for the link updates."""
    return middle_level(u, mom, h, n_mid, n_gauge, beta, lambda v: surrogate_force(v, params))


def md_evolve(ctx, u, mom, phis, tau, n_outer, n_gauge, surrogate=None, n_mid=1):
    """Two-level minimum-norm integration of length tau; three levels when
    surrogate params are given (outer force F_f - F^, middle F^) or a flavour
    has level 1 (outer: the level-0 terms, middle: the level-1 terms), the
    gauge level innermost."""
    p = ctx.p
    e = tau / n_outer
    mid_terms = any(fl.level == 1 for fl in p.flavours)

    def outer_force(u):
        f = ctx.fermion_force_total(u, phis, level=0 if mid_terms else None)
        return f if surrogate is None else f - surrogate_force(u, surrogate)

    def middle_force(u):
        f = ctx.fermion_force_total(u, phis, level=1) if mid_terms else 0.0
        return f if surrogate is None else f + surrogate_force(u, surrogate)

    def inner(u, mom):
        if surrogate is None and not mid_terms:
            return gauge_level(u, mom, e / 2, n_gauge, p.beta)
        return middle_level(u, mom, e / 2, n_mid, n_gauge, p.beta, middle_force)

    for _ in range(n_outer):
        mom = mom - LAMBDA_2MN * e * outer_force(u)
        u, mom = inner(u, mom)
        mom = mom - (1 - 2 * LAMBDA_2MN) * e * outer_force(u)
        u, mom = inner(u, mom)
        mom = mom - LAMBDA_2MN * e * outer_force(u)
    return u, mom


def heatbath(ctx, u, xis):
    """phi = r_hb(A) xi for every pseudo-fermion (the first FP64 inversion)."""
    phis = []
    for fl, xi_list in zip(ctx.p.flavours, xis):
        phis.append([ctx.rational_apply(u, fl.mass, fl.hb, xi, ctx.p.tol_met)[0] for xi in xi_list])
    return phis


def hamiltonian_kinetic(mom):
    return 0.5 * float(np.sum(mom * mom))


def trajectory(ctx, u0, mom0, xis, uniform=None, surrogate=None, n_mid=1, phis=None):
    """One RHMC trajectory with supplied momenta mom0 [4,t,z,y,x,8] and
    Gaussian sources xis (per flavour, per pseudo-fermion, even fields);
    surrogate params select the three-level integrator.  With phis given
    (per flavour, per pseudo-fermion) the heatbath is skipped and the initial
    S_f is phi^dag r_met(A) phi.

    Returns dict with the final links and momenta (before accept/reject),
    dH, the pieces of H and, if `uniform` is given, the Metropolis decision
    accept = uniform < exp(-dH)."""
    p = ctx.p
    if phis is None:
        phis = heatbath(ctx, u0, xis)
        s_f0 = sum(float(np.real(np.vdot(x, x))) for xl in xis for x in xl)
    else:
        s_f0 = ctx.fermion_action_total(u0, phis, p.tol_met)
    h0 = hamiltonian_kinetic(mom0) + wilson_action(u0, p.beta) + s_f0
    u1, mom1 = md_evolve(ctx, u0, mom0, phis, p.tau, p.n_outer, p.n_gauge, surrogate, n_mid)
    u1 = su3.reunitarize(u1)
    s_f1 = ctx.fermion_action_total(u1, phis, p.tol_met)
    h1 = hamiltonian_kinetic(mom1) + wilson_action(u1, p.beta) + s_f1
    dh = h1 - h0
    out = {"u": u1, "mom": mom1, "dH": dh, "H0": h0, "H1": h1, "Sf0": s_f0, "Sf1": s_f1,
           "phis": phis}
    if uniform is not None:
        out["accept"] = bool(uniform < np.exp(-dh)) if np.isfinite(dh) else False
    return out
