"""Pins for the oracle's force surrogate: the plaquette generators reproduce
the Wilson force exactly, finite differences of the summed plaquette and
rectangle loops fix every generator, gauge invariance of the features and
covariance of the surrogate force, finite differences of the loss for the
hand-written backward pass."""
import numpy as np
import pytest

import synthetic as syn
from oracle import actions, lattice as lat, su3, surrogate as sur

DIMS = (4, 4, 2, 4)
PLAQ = [8 * i + j for i in range(3) for j in (0, 1)]
RECT = [8 * i + j for i in range(3) for j in range(2, 8)]


@pytest.fixture(scope="module")
def u():
    return syn.near_identity_gauge(DIMS, 401, width=0.6)


@pytest.fixture(scope="module")
def fg(u):
    return sur.features_and_generators(u)


def test_plaquette_generators_give_the_wilson_force(u, fg):
    f, G = fg
    beta = 5.6
    w = np.zeros(f.shape)
    w[..., PLAQ] = -beta / 3.0
    F = np.einsum("...k,...ka->...a", w, G)
    np.testing.assert_allclose(F, actions.wilson_force(u, beta), atol=1e-12)


def _loop_sum(u, kind):
    """sum over loops of Re tr / 3: kind 'plaq' or 'rect' (every 1x2 and 2x1 loop once)."""
    s = 0.0
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            if kind == "plaq" and nu > mu:
                s += np.sum(np.real(np.trace(actions.plaquette_field(u, mu, nu), axis1=-2, axis2=-1))) / 3
            if kind == "rect":       # 2 in mu, 1 in nu, starting at x
                um = lambda sh: sur._at(u, mu, sh)   # noqa: E731
                un = lambda sh: sur._at(u, nu, sh)   # noqa: E731
                loop = sur._mm(um([]), um([(mu, 1)]), un([(mu, 1), (mu, 1)]), su3.dag(um([(mu, 1), (nu, 1)])),
                               su3.dag(um([(nu, 1)])), su3.dag(un([])))
                s += np.sum(np.real(np.trace(loop, axis1=-2, axis2=-1))) / 3
    return s


@pytest.mark.parametrize("kind,idx", [("plaq", PLAQ), ("rect", RECT)])
def test_generators_are_derivatives_of_loop_sums(u, fg, kind, idx):
    """d/d omega_a of the summed loops through a link = sum of G over its staples / 3."""
    f, G = fg
    rg = np.random.default_rng(7)
    for _ in range(4):
        mu = int(rg.integers(4))
        site = tuple(int(rg.integers(n)) for n in u.shape[1:5])
        a = int(rg.integers(8))

        def s_of(d):
            up = u.copy()
            gen = np.zeros(8)
            gen[a] = 1.0
            up[(mu,) + site] = su3.expi_coeffs(gen, d) @ u[(mu,) + site]
            return _loop_sum(up, kind)
        h = 1e-3
        fd = (8 * (s_of(h) - s_of(-h)) - (s_of(2 * h) - s_of(-2 * h))) / (12 * h)
        an = np.sum(G[(mu,) + site][idx, a]) / 3.0
        assert abs(fd - an) < 1e-8, (kind, fd, an)


def test_features_invariant_and_force_covariant(u, fg):
    f, G = fg
    g = syn.random_gauge_transform(DIMS, 402)
    ug = np.stack([np.einsum("...ij,...jk,...lk->...il", g, u[mu], np.conj(lat.shift_fwd(g, mu)))
                   for mu in range(4)])
    f2, G2 = sur.features_and_generators(ug)
    np.testing.assert_allclose(f2, f, atol=1e-12)
    p = sur.init_params(1)
    F1 = su3.coeffs_to_matrix(sur.surrogate_force(p, f, G))
    F2 = su3.coeffs_to_matrix(sur.surrogate_force(p, f2, G2))
    np.testing.assert_allclose(F2, np.einsum("...ij,...jk,...lk->...il", g, F1, np.conj(g)), atol=1e-12)


def test_backward_matches_finite_differences(fg):
    f, G = fg
    rg = np.random.default_rng(3)
    F = rg.standard_normal(G.shape[:-2] + (8,))
    p = sur.init_params(2, scale=1.0)
    _, grad = sur.loss_and_grad(p, f, G, F)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        for _ in range(3):
            idx = tuple(int(rg.integers(n)) for n in p[name].shape)
            h = 1e-5
            pp = {k: v.copy() for k, v in p.items()}
            pm = {k: v.copy() for k, v in p.items()}
            pp[name][idx] += h
            pm[name][idx] -= h
            fd = (sur.loss_and_grad(pp, f, G, F)[0] - sur.loss_and_grad(pm, f, G, F)[0]) / (2 * h)
            assert abs(fd - grad[name][idx]) < 1e-7 * max(1.0, abs(fd)), (name, idx, fd, grad[name][idx])


def test_bf16_round_known_values():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159265])
    np.testing.assert_array_equal(sur.bf16_round(x), [1.0, 1.0, 1.0 + 2 ** -7, -3.140625])


def _three_level_params(n_outer, n_gauge, tau=0.5, mass=0.2):
    from oracle import integrator, rational
    lo, hi = mass ** 2, 16 + mass ** 2
    fl = integrator.Flavour(mass=mass, hb=rational.remez(-0.25, lo, hi, 8, dps=40),
                            md=rational.remez(0.5, lo, hi, 6, dps=40), met=rational.remez(0.5, lo, hi, 10, dps=40))
    return integrator.HMCParams(dims=(2, 2, 2, 2), beta=5.5, tau=tau, n_outer=n_outer, n_gauge=n_gauge,
                                flavours=[fl], tol_md=1e-13, tol_met=1e-14)


def _strong_network(seed):
    """A network whose force is of the size of the fermion force (not fitted
    to it): a plain test of the splitting, not of the learning."""
    p = sur.init_params(seed, scale=1.0)
    p["W3"] *= 4.0
    p["b3"] += 0.5
    return p


def test_three_level_with_zero_network_is_the_two_level_integrator():
    """F^ = 0 makes each surrogate level n_mid pairs of gauge levels of the
    same step: the trajectory equals the two-level one with 2 n_mid n_gauge
    gauge steps per half step (step sizes are powers of two: exactly)."""
    from oracle import integrator
    dims = (2, 2, 2, 2)
    zero = {k: np.zeros_like(v) for k, v in sur.init_params(0).items()}
    zero["W1"] = sur.init_params(1)["W1"]          # hidden layers alive, output weights zero
    args = (syn.near_identity_gauge(dims, 611), syn.gaussian_momenta(dims, 612),
            [[syn.gaussian_fermion(dims, 613, on_parity=0)]])
    three = integrator.trajectory(integrator.Context(_three_level_params(2, 1)), *args, surrogate=zero, n_mid=2)
    two = integrator.trajectory(integrator.Context(_three_level_params(2, 4)), *args)
    assert np.array_equal(three["u"], two["u"]) and np.array_equal(three["mom"], two["mom"])
    assert three["dH"] == two["dH"]


def test_three_level_dh_vanishes_as_step_squared():
    """Outer F_f - F^ plus middle F^ integrate the exact force for any F^:
    with a large, unfitted F^ dH still falls as eps^2.  A sign slip in the
    remainder would integrate F_f + 2 F^ (or leave F^ twice) and dH would
    tend to a nonzero limit instead."""
    from oracle import integrator
    dims = (2, 2, 2, 2)
    net = _strong_network(7)
    u0 = syn.near_identity_gauge(dims, 621)
    f, G = sur.features_and_generators(u0)
    fs = sur.surrogate_force(net, f, G)
    pr = _three_level_params(2, 1)
    ctx = integrator.Context(pr)
    phi = [[syn.gaussian_fermion(dims, 623, on_parity=0)]]
    ff = ctx.fermion_force_total(u0, integrator.heatbath(ctx, u0, phi))
    assert np.linalg.norm(fs) > 0.5 * np.linalg.norm(ff)       # F^ is not small
    dhs = []
    for n in (4, 8):
        out = integrator.trajectory(integrator.Context(_three_level_params(n, 1)), u0,
                                    syn.gaussian_momenta(dims, 622), phi, surrogate=net, n_mid=1)
        dhs.append(abs(out["dH"]))
    assert 2.5 < dhs[0] / dhs[1] < 6.5, dhs


def test_three_level_is_reversible():
    from oracle import integrator
    dims = (2, 2, 2, 2)
    net = _strong_network(8)
    ctx = integrator.Context(_three_level_params(2, 1))
    u0, mom0 = syn.near_identity_gauge(dims, 631), syn.gaussian_momenta(dims, 632)
    phis = [[syn.gaussian_fermion(dims, 633, on_parity=0)]]
    u1, m1 = integrator.md_evolve(ctx, u0, mom0, phis, 0.5, 2, 1, surrogate=net, n_mid=2)
    u2, m2 = integrator.md_evolve(ctx, u1, -m1, phis, 0.5, 2, 1, surrogate=net, n_mid=2)
    assert np.abs(u2 - u0).max() < 1e-11 and np.abs(m2 + mom0).max() < 1e-10


def test_quantised_network_stays_within_the_bf16_bound(fg):
    """Pins the oracle's tensor-core mode (quant=True: bf16 inputs of every
    product, straight-through gradients) against the exact network, which
    finite differences pin: the loss, all 2648 gradient components and the
    force lie within lambda = 3 probabilistic bf16 bounds of the exact ones
    (tests/bf16_bounds.py: first-order running-error bound per link, summed
    over the links in quadrature) and within the rigorous worst-case bound,
    and differ from them visibly (the mode does round).  The same bounds
    reject the network with a transposed W2 or a dropped output bias."""
    from tests.bf16_bounds import LAMBDA, network_bounds, ratio
    f, G = fg
    p = sur.init_params(6, scale=1.0)
    pd = {k: (sur.bf16_round(v) if k.startswith("W") else v) for k, v in p.items()}
    F = np.random.default_rng(4).standard_normal(G.shape[:-2] + (8,))
    exact, worst, prob = network_bounds(pd, f, G, F)
    loss_x, grad_x = sur.loss_and_grad(pd, f, G, F, quant=False)
    assert abs(loss_x - exact["loss"]) < 1e-12 * exact["loss"]           # the bounds' own exact network
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        np.testing.assert_allclose(grad_x[k], exact[k], rtol=1e-10, atol=1e-14)

    def ratios(q, bound):
        loss_q, grad_q = sur.loss_and_grad(q, f, G, F, quant=True)
        r = [ratio(loss_q, exact["loss"], bound["loss"])]
        r += [ratio(grad_q[k], exact[k], bound[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
        return r + [ratio(sur.surrogate_force(q, f, G, quant=True), exact["force"], bound["force"])]

    r_prob = ratios(pd, {k: LAMBDA * v for k, v in prob.items()})
    assert max(r_prob) <= 1.0, r_prob
    assert max(ratios(pd, worst)) <= 1.0
    assert max(r_prob) > 1e-3, r_prob                                    # the quantised mode does round
    assert max(ratios(dict(pd, W2=pd["W2"].T.copy()), {k: LAMBDA * v for k, v in prob.items()})) > 1.0
    assert max(ratios(dict(pd, b3=0 * pd["b3"]), {k: LAMBDA * v for k, v in prob.items()})) > 1.0
