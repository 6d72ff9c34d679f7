"""Pins for the oracle's Hasenbusch mass split (the paper's multiple
pseudo-fermions, Sec. 2, extended by a heavier mass): the ratio rational
((x + delta) / x)^s, its action and force, and the three-level integrator
with the heavy term on the middle level.

With A = m^2 - D_eo D_oe and A_h = A + delta (delta = m_h^2 - m^2),
det(A)^s = det(A_h)^s det(A / A_h)^s: the heavy term is an ordinary flavour
at mass m_h, the ratio term phi^dag (A_h / A)^s phi at mass m, whose rational
r(x) ~ ((x + delta) / x)^s needs the same multi-shift solves as x^(-s)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import actions, dirac, integrator, lattice as lat, rational, solvers, su3

M, MH = 0.2, 0.6
DELTA = MH ** 2 - M ** 2
LO, HI = M ** 2, 16 + M ** 2


@pytest.fixture(scope="module")
def rats():
    return {"ratio_md": rational.remez(0.5, LO, HI, 6, dps=40, delta=DELTA),
            "ratio_met": rational.remez(0.5, LO, HI, 10, dps=40, delta=DELTA),
            "ratio_hb": rational.remez(-0.25, LO, HI, 10, dps=40, delta=DELTA),
            "heavy_md": rational.remez(0.5, MH ** 2, 16 + MH ** 2, 6, dps=40),
            "heavy_met": rational.remez(0.5, MH ** 2, 16 + MH ** 2, 10, dps=40),
            "heavy_hb": rational.remez(-0.25, MH ** 2, 16 + MH ** 2, 10, dps=40),
            "light": rational.remez(0.5, LO, HI, 10, dps=40)}


def test_ratio_rational_equioscillates_and_is_positive(rats):
    """Chebyshev alternation of the relative error of a 3-pole ratio rational
    (large enough an error to resolve in doubles): 2n+1 sign changes and
    2n+2 extrema of equal magnitude; positive partial fractions for the
    6-pole one."""
    r = rational.remez(0.5, LO, HI, 3, dps=40, delta=DELTA)
    x = np.exp(np.linspace(np.log(LO), np.log(HI), 200001))
    e = r(x) * (x / (x + DELTA)) ** 0.5 - 1.0
    cuts = [0] + [k for k in range(1, len(e)) if (e[k] > 0) != (e[k - 1] > 0)] + [len(e)]
    ext = np.array([e[a:b][np.argmax(np.abs(e[a:b]))] for a, b in zip(cuts[:-1], cuts[1:])])
    assert len(ext) == 2 * len(r.alpha) + 2
    assert np.all(np.sign(ext[1:]) == -np.sign(ext[:-1]))
    np.testing.assert_allclose(np.abs(ext), r.err, rtol=2e-3)
    r6 = rats["ratio_md"]
    assert r6.a0 > 0 and min(r6.alpha) > 0 and min(r6.beta) > 0


def test_mass_split_reproduces_the_light_rational(rats):
    """((x + delta) / x)^s (x + delta)^(-s) = x^(-s): the ratio rational at x
    times the heavy rational at x + delta (its own spectral variable)
    equals the light rational within the three approximation errors."""
    x = np.geomspace(LO, HI, 4001)
    lhs = rats["ratio_met"](x) * rats["heavy_met"](x + DELTA)
    rhs = rats["light"](x)
    bound = rats["ratio_met"].err + rats["heavy_met"].err + rats["light"].err + 1e-14
    assert np.abs(lhs / rhs - 1).max() <= 1.01 * bound


def test_ratio_rational_of_the_operator_matches_eigendecomposition(rats):
    dims = (2, 2, 2, 2)
    u = syn.near_identity_gauge(dims, 81, width=0.8)
    eta, par = lat.eta(dims), lat.parity(dims)
    phi = syn.gaussian_fermion(dims, 82, on_parity=0)
    a = dirac.dense_a(u, M, eta, par)
    w, v = np.linalg.eigh(a)
    ev = dirac.even_indices(par)
    exact = v @ (((w + DELTA) / w) ** 0.5 * (v.conj().T @ phi.reshape(-1)[ev]))
    r = rats["ratio_met"]
    s0 = min(r.beta)
    got = rational.apply_rational(
        r, lambda b, betas: solvers.multishift_cg(lambda y: dirac.a_op(u, y, M, eta, par, s0), b, betas, 1e-14)[0],
        phi).reshape(-1)[ev]
    assert np.linalg.norm(got - exact) <= 1.01 * r.err * np.linalg.norm(exact) + 1e-12


def _fd(action, u, mu, site, a, d):
    def s(k):
        up = u.copy()
        gen = np.zeros(8)
        gen[a] = 1.0
        up[(mu,) + site] = su3.expi_coeffs(gen, k * d) @ u[(mu,) + site]
        return action(up)
    return (8 * (s(1) - s(-1)) - (s(2) - s(-2))) / (12 * d)


def test_ratio_force_finite_difference(rats):
    """The ratio term's force is the standard formula with the ratio
    rational's (alpha_i, beta_i): checked against 4th-order finite differences
    of phi^dag r(A) phi."""
    dims = (2, 2, 2, 4)
    u = syn.near_identity_gauge(dims, 83, width=0.5)
    eta, par = lat.eta(dims), lat.parity(dims)
    r = rats["ratio_md"]
    phi = syn.gaussian_fermion(dims, 84, on_parity=0)

    def s_f(uu):
        xs = solvers.multishift_cg(lambda v: dirac.a_op(uu, v, M, eta, par, min(r.beta)), phi, r.beta, 1e-15)[0]
        return actions.fermion_action(phi, xs, r), xs

    _, xs = s_f(u)
    f = actions.fermion_force(u, xs, r.alpha, eta, par)
    rg = np.random.default_rng(2)
    for _ in range(6):
        mu = int(rg.integers(4))
        site = tuple(int(rg.integers(n)) for n in u.shape[1:5])
        a = int(rg.integers(8))
        fd = _fd(lambda uu: s_f(uu)[0], u, mu, site, a, 1e-3)
        assert abs(fd - f[(mu,) + site + (a,)]) < 1e-7 * max(1.0, abs(fd)), (fd, f[(mu,) + site + (a,)])


def test_ratio_heatbath_and_metropolis_are_consistent(rats):
    """phi = r_hb(A) xi makes phi^dag r_met(A) phi = xi^dag xi within the
    two rationals' errors (r_hb^2 r_met = 1)."""
    dims = (2, 2, 2, 4)
    u = syn.haar_gauge(dims, 85)
    eta, par = lat.eta(dims), lat.parity(dims)
    xi = syn.gaussian_fermion(dims, 86, on_parity=0)
    ctx = integrator.Context(integrator.HMCParams(dims=dims, beta=5.5, tau=1.0, n_outer=1, n_gauge=1))
    phi, _ = ctx.rational_apply(u, M, rats["ratio_hb"], xi, 1e-15)
    s, _ = ctx.rational_apply(u, M, rats["ratio_met"], phi, 1e-15)
    xx = float(np.real(np.vdot(xi, xi)))
    assert abs(float(np.real(np.vdot(phi, s))) - xx) <= (2 * rats["ratio_hb"].err + rats["ratio_met"].err) * xx * 1.01 \
        + 1e-12 * xx


def _split_params(dims, n_outer, n_mid, levels=(0, 1)):
    fls = [integrator.Flavour(mass=M, hb=None, md=None, met=None, level=levels[0]),
           integrator.Flavour(mass=MH, hb=None, md=None, met=None, level=levels[1])]
    return integrator.HMCParams(dims=dims, beta=5.5, tau=0.5, n_outer=n_outer, n_gauge=4, flavours=fls,
                                tol_md=1e-13, tol_met=1e-14), n_mid


def _with_rats(prm, rats):
    prm.flavours[0].hb, prm.flavours[0].md, prm.flavours[0].met = rats["ratio_hb"], rats["ratio_md"], rats["ratio_met"]
    prm.flavours[1].hb, prm.flavours[1].md, prm.flavours[1].met = rats["heavy_hb"], rats["heavy_md"], rats["heavy_met"]
    return prm


def test_split_integrator_dh_scales_as_step_squared_and_is_reversible(rats):
    """The heavy term's force on the middle level and the ratio term's on the
    outer one add up to the gradient of the split action: dH = O(eps^2)
    (a term on the wrong level twice, or on none, leaves dH at a constant)."""
    dims = (2, 2, 2, 2)
    u0 = syn.near_identity_gauge(dims, 87)
    mom0 = syn.gaussian_momenta(dims, 88)
    xis = [[syn.gaussian_fermion(dims, 89, on_parity=0)], [syn.gaussian_fermion(dims, 90, on_parity=0)]]
    dhs = []
    for n in (4, 8):
        prm, n_mid = _split_params(dims, n, 2)
        out = integrator.trajectory(integrator.Context(_with_rats(prm, rats)), u0, mom0, xis, n_mid=n_mid)
        dhs.append(out["dH"])
    ratio = abs(dhs[0] / dhs[1])
    assert 3.0 < ratio < 5.0, dhs            # second order: 4 for small steps
    # reversibility: forward, flip the momenta, back with the same pseudo-fermions
    prm, n_mid = _split_params(dims, 2, 2)
    ctx = integrator.Context(_with_rats(prm, rats))
    fwd = integrator.trajectory(ctx, u0, mom0, xis, n_mid=n_mid)
    back = integrator.trajectory(ctx, fwd["u"], -fwd["mom"], None, n_mid=n_mid, phis=fwd["phis"])
    assert np.abs(back["u"] - u0).max() < 1e-12
    assert abs(fwd["dH"] + back["dH"]) < 1e-9


def test_split_integrator_on_one_level_is_the_two_level_scheme(rats):
    """Both terms on the outer level: the same trajectory as the plain
    two-level integrator with the two flavours summed."""
    dims = (2, 2, 2, 2)
    u0 = syn.near_identity_gauge(dims, 91, width=0.6)
    mom0 = syn.gaussian_momenta(dims, 92)
    xis = [[syn.gaussian_fermion(dims, 93, on_parity=0)], [syn.gaussian_fermion(dims, 94, on_parity=0)]]
    prm, _ = _split_params(dims, 3, 2, levels=(0, 0))
    a = integrator.trajectory(integrator.Context(_with_rats(prm, rats)), u0, mom0, xis, n_mid=5)
    prm1, _ = _split_params(dims, 3, 2, levels=(0, 0))
    b = integrator.trajectory(integrator.Context(_with_rats(prm1, rats)), u0, mom0, xis, n_mid=1)
    assert np.abs(a["u"] - b["u"]).max() == 0.0 and a["dH"] == b["dH"]
