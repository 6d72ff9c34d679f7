"""Pins for the oracle's forces and MD (paper Sec. 2 and Sec. 4): finite
differences of the actions, reversibility, dH scaling, <exp(-dH)> = 1."""
import numpy as np
import pytest

import synthetic as syn
from oracle import actions, dirac, integrator, lattice as lat, rational, solvers, su3


def _fd(action, u, mu, site, a, d):
    """Fourth-order central difference of action along exp(i w T_a) on one link."""
    s = lambda k: action(_perturb(u, mu, site, a, k * d))
    return (8 * (s(1) - s(-1)) - (s(2) - s(-2))) / (12 * d)


def _perturb(u, mu, site, a, delta):
    up = u.copy()
    gen = np.zeros(8)
    gen[a] = 1.0
    up[(mu,) + site] = su3.expi_coeffs(gen, delta) @ u[(mu,) + site]
    return up


def test_wilson_force_finite_difference():
    dims = (4, 2, 2, 4)
    u = syn.haar_gauge(dims, 61)
    beta = 5.5
    f = actions.wilson_force(u, beta)
    rg = np.random.default_rng(0)
    for _ in range(6):
        mu = int(rg.integers(4))
        site = tuple(int(rg.integers(n)) for n in u.shape[1:5])
        a = int(rg.integers(8))
        fd = _fd(lambda uu: actions.wilson_action(uu, beta), u, mu, site, a, 1e-3)
        assert abs(fd - f[(mu,) + site + (a,)]) < 1e-8 * max(1.0, abs(fd))


def test_fermion_force_finite_difference():
    dims = (2, 2, 2, 4)
    u = syn.near_identity_gauge(dims, 71, width=0.5)
    eta, par = lat.eta(dims), lat.parity(dims)
    mass = 0.2
    r = rational.remez(0.5, mass ** 2, 16 + mass ** 2, 4, dps=40)
    phi = syn.gaussian_fermion(dims, 72, on_parity=0)

    def s_f(uu):
        s0 = min(r.beta)
        xs = solvers.multishift_cg(lambda v: dirac.a_op(uu, v, mass, eta, par, s0),
                                   phi, r.beta, 1e-15)[0]
        return actions.fermion_action(phi, xs, r), xs

    _, xs = s_f(u)
    f = actions.fermion_force(u, xs, r.alpha, eta, par)
    rg = np.random.default_rng(1)
    for _ in range(8):
        mu = int(rg.integers(4))
        site = tuple(int(rg.integers(n)) for n in u.shape[1:5])
        a = int(rg.integers(8))
        fd = _fd(lambda uu: s_f(uu)[0], u, mu, site, a, 1e-3)
        assert abs(fd - f[(mu,) + site + (a,)]) < 1e-7 * max(1.0, abs(fd)), (fd, f[(mu,) + site + (a,)])


def _small_params(dims, n_outer, n_gauge=2, mass=0.2, tau=0.5):
    lo, hi = mass ** 2, 16 + mass ** 2
    fl = integrator.Flavour(mass=mass,
                            hb=rational.remez(-0.25, lo, hi, 8, dps=40),
                            md=rational.remez(0.5, lo, hi, 6, dps=40),
                            met=rational.remez(0.5, lo, hi, 10, dps=40))
    return integrator.HMCParams(dims=dims, beta=5.5, tau=tau, n_outer=n_outer, n_gauge=n_gauge,
                                flavours=[fl], tol_md=1e-13, tol_met=1e-14)


@pytest.fixture(scope="module")
def params_2x4():
    return _small_params((2, 2, 2, 2), 4)


def test_reversibility_fp64(params_2x4):
    ctx = integrator.Context(params_2x4)
    dims = params_2x4.dims
    u0 = syn.near_identity_gauge(dims, 81)
    mom0 = syn.gaussian_momenta(dims, 82)
    phis = [[syn.gaussian_fermion(dims, 83, on_parity=0)]]
    u1, m1 = integrator.md_evolve(ctx, u0, mom0, phis, 0.5, 4, 2)
    u2, m2 = integrator.md_evolve(ctx, u1, -m1, phis, 0.5, 4, 2)
    assert np.abs(u2 - u0).max() < 1e-12
    assert np.abs(m2 + mom0).max() < 1e-11


def test_dh_scales_as_step_squared():
    """For a second-order integrator dH = O(eps^2) on one trajectory."""
    dims = (2, 2, 2, 2)
    dhs = []
    for n in (4, 8):
        p = _small_params(dims, n, n_gauge=4, tau=0.5)
        ctx = integrator.Context(p)
        out = integrator.trajectory(ctx, syn.near_identity_gauge(dims, 91),
                                    syn.gaussian_momenta(dims, 92),
                                    [[syn.gaussian_fermion(dims, 93, on_parity=0)]])
        dhs.append(abs(out["dH"]))
    ratio = dhs[0] / dhs[1]
    assert 2.5 < ratio < 6.5, dhs


@pytest.mark.slow
def test_exp_minus_dh_averages_to_one():
    """Creutz's identity <exp(-dH)> = 1 over an equilibrium Markov chain."""
    dims = (2, 2, 2, 2)
    p = _small_params(dims, 3, n_gauge=2, tau=1.0)
    ctx = integrator.Context(p)
    rg = syn.rng(2024)
    u = syn.near_identity_gauge(dims, 101)
    vals = []
    for k in range(70):
        mom = rg.standard_normal((4,) + u.shape[1:5] + (8,))
        xi = syn.gaussian_fermion(dims, 5000 + k, on_parity=0)
        out = integrator.trajectory(ctx, u, mom, [[xi]], uniform=rg.random())
        if k >= 10:
            vals.append(np.exp(-out["dH"]))
        if out["accept"]:
            u = out["u"]
    vals = np.array(vals)
    err = vals.std() / np.sqrt(len(vals))
    assert abs(vals.mean() - 1.0) < 4 * err + 0.02, (vals.mean(), err)


def _two_flavour_params(dims, n_outer, n_gauge=2, tau=0.5):
    """N_f = 2 + 1 with two pseudo-fermions each: s = N_f / (4 n_pf)."""
    fls = []
    for mass, nf in ((0.2, 2), (0.5, 1)):
        s = nf / 8.0
        lo, hi = mass ** 2, 16 + mass ** 2
        fls.append(integrator.Flavour(mass=mass, n_pf=2,
                                      hb=rational.remez(-s / 2, lo, hi, 8, dps=40),
                                      md=rational.remez(s, lo, hi, 6, dps=40),
                                      met=rational.remez(s, lo, hi, 10, dps=40)))
    return integrator.HMCParams(dims=dims, beta=5.5, tau=tau, n_outer=n_outer, n_gauge=n_gauge,
                                flavours=fls, tol_md=1e-13, tol_met=1e-14)


def _sources(dims, seed):
    return [[syn.gaussian_fermion(dims, seed + 10 * f + k, on_parity=0) for k in range(2)] for f in range(2)]


def test_heatbath_and_metropolis_rationals_agree_for_every_pseudo_fermion():
    """phi = r_hb(A) xi with r_hb ~ A^(s/2) and r_met ~ A^(-s) give
    phi^dag r_met(A) phi = xi^dag xi up to the two approximations' errors,
    for each flavour and pseudo-fermion (a wrong exponent or sign in either
    rational, or a flavour's mass crossed, breaks it by orders of magnitude)."""
    dims = (2, 2, 2, 4)
    p = _two_flavour_params(dims, 2)
    ctx = integrator.Context(p)
    u = syn.near_identity_gauge(dims, 111)
    xis = _sources(dims, 112)
    phis = integrator.heatbath(ctx, u, xis)
    for fl, xl, pl in zip(p.flavours, xis, phis):
        bound = 2 * fl.hb.err + fl.met.err + 1e-10
        for xi, phi in zip(xl, pl):
            want = float(np.real(np.vdot(xi, xi)))
            got = integrator.Context(integrator.HMCParams(dims=dims, beta=p.beta, tau=p.tau, n_outer=1, n_gauge=1,
                                                           flavours=[fl], tol_md=p.tol_md, tol_met=p.tol_met)
                                     ).fermion_action_total(u, [[phi]], p.tol_met)
            assert abs(got - want) < 3 * bound * want, (got, want, bound)


def test_dh_scales_as_step_squared_two_flavours_two_pseudo_fermions():
    """The summed force of 2 flavours x 2 pseudo-fermions is the gradient of
    the summed action: dH = O(eps^2).  Dropping or double-counting one term
    leaves dH at a constant instead."""
    dims = (2, 2, 2, 2)
    dhs = []
    for n in (4, 8):
        p = _two_flavour_params(dims, n, n_gauge=4, tau=0.5)
        out = integrator.trajectory(integrator.Context(p), syn.near_identity_gauge(dims, 121),
                                    syn.gaussian_momenta(dims, 122), _sources(dims, 123))
        dhs.append(abs(out["dH"]))
    ratio = dhs[0] / dhs[1]
    assert 2.5 < ratio < 6.5, dhs
