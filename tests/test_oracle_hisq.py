"""Pins for the oracle's HISQ operator and force (oracle/hisq.py; Follana et
al. 2007): the free-field spectrum, the U(3) projection (unitary, the
identity on unitary links, its cotangent by finite differences), gauge
covariance, the level-1 coefficients by path counting, and the force by
finite differences of the action."""
import numpy as np
import pytest

import synthetic as syn
from oracle import asqtad, hisq, lattice as lat, rational, solvers, su3
from oracle import integrator as itg


def _free_spectrum(dims, antiperiodic_t):
    ps = []
    for mu, L in enumerate(dims):
        ps.append(np.pi * (2 * np.arange(L) + 1) / L if (mu == 3 and antiperiodic_t) else 2 * np.pi * np.arange(L) / L)
    grids = np.meshgrid(*ps, indexing="ij")
    vals = sum((9 / 8 * np.sin(g) - 1 / 24 * np.sin(3 * g)) ** 2 for g in grids).reshape(-1)
    return np.sort(np.repeat(vals, 3))


@pytest.mark.parametrize("dims,apt", [((4, 4, 4, 4), True), ((2, 4, 2, 6), True), ((4, 2, 4, 2), False)])
def test_free_field_spectrum(dims, apt):
    """At U = 1 the two smearings give X = 9/8 and N = -1/24: the asqtad free field."""
    x, n, w, v = hisq.hisq_links(syn.unit_gauge(dims), apt)
    d = asqtad.dense_dslash(x, n, lat.eta(dims, antiperiodic_t=False))
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(-(d @ d))), _free_spectrum(dims, apt), atol=1e-12)


def test_projection_is_unitary_and_fixes_unitary_links():
    dims = (4, 4, 2, 4)
    u = syn.haar_gauge(dims, 3)
    np.testing.assert_allclose(hisq.project_u3(u), u, atol=1e-13)
    _, _, w, v = hisq.hisq_links(u)
    eye = np.broadcast_to(np.eye(3), w.shape)
    np.testing.assert_allclose(su3.dag(w) @ w, eye, atol=1e-12)
    assert np.abs(v - w).max() > 0.1          # the fat7 links are not unitary


def test_projection_cotangent_by_finite_differences():
    """d/dt Re tr[C_W W(V + t E)] at t = 0 equals Re tr[C_V E] for random V, E, C_W."""
    g = np.random.default_rng(5)
    shape = (7, 3, 3)
    v = np.eye(3) + 0.4 * (g.normal(size=shape) + 1j * g.normal(size=shape))
    e = g.normal(size=shape) + 1j * g.normal(size=shape)
    c = g.normal(size=shape) + 1j * g.normal(size=shape)
    cv = hisq.project_cotangent(v, c)
    h = 1e-4

    def f(t):
        return np.real(np.einsum("kij,kji->k", c, hisq.project_u3(v + t * e)))
    fd = (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
    np.testing.assert_allclose(fd, np.real(np.einsum("kij,kji->k", cv, e)), rtol=1e-8, atol=1e-9)


def test_level1_coefficients_by_counting():
    """dV_mu(x)/d eps for an abelian phase on one link: the fat7 1-link term
    (1/8) on (x, mu), one 3-staple (1/16) on (x + nu, mu), six 7-staples
    (6/384) on (x + nu + rho + sig, mu), and on the first leg (x, nu) of the
    paths opening with +nu: 1/16 + 4/64 + 8/384."""
    dims = (6, 6, 6, 6)
    x0 = np.array([2, 2, 2, 2])
    e = np.eye(4, dtype=int)
    mu, nu, rho, sig = 1, 0, 2, 3
    cases = [(x0, mu, 1 / 8), (x0 + e[nu], mu, 1 / 16), (x0 - e[nu] + e[rho] + e[sig], mu, 6 / 384),
             (x0, nu, 1 / 16 + 4 / 64 + 8 / 384), (x0 + 2 * e[nu], mu, 0.0)]
    h = 1e-5
    t, z, y, x = x0[3], x0[2], x0[1], x0[0]
    for site, d, expect in cases:
        vals = []
        for s in (h, -h):
            u = syn.unit_gauge(dims).copy()
            u[d, site[3], site[2], site[1], site[0]] = np.exp(1j * s) * np.eye(3)
            vals.append(hisq.smear(asqtad.boundary_signed_links(u, False), hisq.FAT7)[mu, t, z, y, x])
        np.testing.assert_allclose((vals[0] - vals[1]) / (2 * h), 1j * expect * np.eye(3), atol=1e-9)


def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    u = syn.haar_gauge(dims, 5)
    g = syn.random_gauge_transform(dims, 6)
    up = np.stack([np.einsum("...ij,...jk,...lk->...il", g, u[mu], np.conj(lat.shift_fwd(g, mu))) for mu in range(4)])
    x, n, _, _ = hisq.hisq_links(u)
    xg, ng, _, _ = hisq.hisq_links(up)
    for mu in range(4):
        g3 = g
        for _ in range(3):
            g3 = lat.shift_fwd(g3, mu)
        np.testing.assert_allclose(xg[mu], g @ x[mu] @ su3.dag(lat.shift_fwd(g, mu)), atol=1e-12)
        np.testing.assert_allclose(ng[mu], g @ n[mu] @ su3.dag(g3), atol=1e-13)


def _rat(a0, alpha, beta):
    return rational.Rational(0.0, 0.0, 0.0, a0, np.array(alpha), np.array(beta), 0.0)


def _action(u, phi, rat, mass, par, apt):
    dims = (u.shape[4], u.shape[3], u.shape[2], u.shape[1])
    x, n, _, _ = hisq.hisq_links(u, apt)
    eta0 = lat.eta(dims, antiperiodic_t=False)
    xs, _, _ = solvers.multishift_cg(lambda y: asqtad.a_op(x, n, y, mass, eta0, par, min(rat.beta)), phi, rat.beta,
                                     1e-14)
    s = rat.a0 * np.vdot(phi, phi) + sum(a * np.vdot(phi, xx) for a, xx in zip(rat.alpha, xs))
    return float(np.real(s)), xs


@pytest.mark.parametrize("apt", [True, False])
def test_force_by_finite_differences(apt):
    dims = (4, 4, 4, 4)
    u = syn.near_identity_gauge(dims, 81, width=0.5)
    par = lat.parity(dims)
    mass = 0.4
    rat = _rat(0.1, [0.3, 0.7], [0.05, 1.5])
    phi = syn.gaussian_fermion(dims, 82, on_parity=0)
    _, xs = _action(u, phi, rat, mass, par, apt)
    f = hisq.fermion_force(u, xs, rat.alpha, par, apt)
    for (nu, t, z, y, x, a) in [(3, 3, 1, 2, 0, 2), (0, 1, 3, 0, 2, 5), (2, 0, 2, 1, 3, 7)]:
        def s_at(dl):
            up = u.copy()
            up[nu, t, z, y, x] = su3.expi_hermitian(dl * su3.T[a]) @ u[nu, t, z, y, x]
            return _action(up, phi, rat, mass, par, apt)[0]
        dl = 1e-3
        fd = (-s_at(2 * dl) + 8 * s_at(dl) - 8 * s_at(-dl) + s_at(-2 * dl)) / (12 * dl)
        assert abs(f[nu, t, z, y, x, a] - fd) < 1e-8 * max(1.0, abs(fd)), (nu, a, f[nu, t, z, y, x, a], fd)


def test_trajectory_reversible():
    rat = _rat(0.2, [0.4, 0.9], [0.1, 2.0])
    hb = _rat(1.2, [-0.3, -0.5], [0.2, 3.0])
    fl = itg.Flavour(mass=0.5, hb=hb, md=rat, met=rat)
    p = itg.HMCParams(dims=(4, 4, 4, 4), beta=5.5, tau=0.5, n_outer=2, n_gauge=2, flavours=[fl], tol_md=1e-13,
                      tol_met=1e-13, action="hisq")
    ctx = itg.Context(p)
    u0 = syn.near_identity_gauge(p.dims, 91)
    mom = syn.gaussian_momenta(p.dims, 92)
    phis = [[syn.gaussian_fermion(p.dims, 93, on_parity=0)]]
    u1, m1 = itg.md_evolve(ctx, u0, mom, phis, p.tau, p.n_outer, p.n_gauge)
    u2, m2 = itg.md_evolve(ctx, u1, -m1, phis, p.tau, p.n_outer, p.n_gauge)
    assert np.max(np.abs(u2 - u0)) < 1e-12
    assert np.max(np.abs(m2 + mom)) < 1e-11


def test_projection_equals_newton_polar_iteration():
    """The polar factor by the eigen-decomposition of V^dag V (the oracle's)
    equals Newton's iteration W <- (W + W^(-dag)) / 2 from W = V, an
    independent method, on the level-1 links of a hot field."""
    dims = (4, 2, 4, 2)
    _, _, w, v = hisq.hisq_links(syn.haar_gauge(dims, 13))
    x = v.copy()
    for _ in range(30):
        x = 0.5 * (x + su3.dag(np.linalg.inv(x)))
    np.testing.assert_allclose(x, w, atol=1e-12)
