"""Pins for the oracle's improved (asqtad) staggered operator and force
(oracle/asqtad.py; Lepage 1999, Orginos-Toussaint-Sugar 1999): the free-field
spectrum in closed form, the fat-link coefficients by path counting,
gauge covariance, anti-Hermiticity, dense solves, the force by finite
differences of the action, and the trajectory's reversibility and dH scaling."""
import numpy as np
import pytest

import synthetic as syn
from oracle import asqtad, lattice as lat, rational, solvers, su3
from oracle import integrator as itg


def _free_spectrum(dims, antiperiodic_t, u0=1.0):
    """Closed form: -D^2 = sum_mu s(p_mu)^2 on plane waves, one per colour,
    with s(p) = c1 sin p + c_N sin 3p, c1 the fat link at U = 1 (9/8 at
    u0 = 1) and c_N = -1/24 / u0^2 (p_t = pi (2n+1) / L_t with antiperiodic time)."""
    c1 = 5 / 8 + 6 / 16 / u0 ** 2 + 24 / 64 / u0 ** 4 + 48 / 384 / u0 ** 6 - 6 / 16 / u0 ** 4
    cn = -1 / 24 / u0 ** 2
    ps = []
    for mu, L in enumerate(dims):
        if mu == 3 and antiperiodic_t:
            ps.append(np.pi * (2 * np.arange(L) + 1) / L)
        else:
            ps.append(2 * np.pi * np.arange(L) / L)
    grids = np.meshgrid(*ps, indexing="ij")
    vals = sum((c1 * np.sin(g) + cn * np.sin(3 * g)) ** 2 for g in grids).reshape(-1)
    return np.sort(np.repeat(vals, 3))


@pytest.mark.parametrize("dims,apt,u0", [((4, 4, 4, 4), True, 1.0), ((2, 4, 2, 6), True, 1.0),
                                         ((4, 2, 4, 2), False, 0.87), ((2, 2, 2, 8), True, 0.9)])
def test_free_field_spectrum(dims, apt, u0):
    u = syn.unit_gauge(dims)
    v, w = asqtad.fat_long_links(u, u0, apt)
    d = asqtad.dense_dslash(v, w, lat.eta(dims, antiperiodic_t=False))
    ev = np.sort(np.linalg.eigvalsh(-(d @ d)))
    np.testing.assert_allclose(ev, _free_spectrum(dims, apt, u0), atol=1e-12)


def test_path_counts():
    """85 fat paths per direction, each from x to x + mu, of the stated lengths."""
    for mu in range(4):
        paths = asqtad.fat_paths(mu)
        assert len(paths) == 85
        lengths = {"one": 1, "staple3": 3, "staple5": 5, "staple7": 7, "lepage": 5}
        counts = {}
        for name, steps in paths:
            assert len(steps) == lengths[name]
            net = np.zeros(4, dtype=int)
            for s in steps:
                net[abs(s) - 1] += np.sign(s)
            assert list(net) == [1 if d == mu else 0 for d in range(4)]
            counts[name] = counts.get(name, 0) + 1
        assert counts == {"one": 1, "staple3": 6, "staple5": 24, "staple7": 48, "lepage": 6}
        assert len({tuple(s) for _, s in paths}) == 85


def _phase_on_link(dims, site, nu, eps):
    """U = 1 except an abelian phase exp(i eps) on link (site, nu)."""
    u = syn.unit_gauge(dims).copy()
    x, y, z, t = site
    u[nu, t, z, y, x] = np.exp(1j * eps) * np.eye(3)
    return u


@pytest.mark.parametrize("u0", [1.0, 0.8])
def test_fat_link_coefficients_by_counting(u0):
    """dV_mu(x)/d eps for an abelian phase exp(i eps) on a single link equals
    i (or -i, for a link met backward) times the sum of the coefficients of
    the paths through that link, counted by hand:
      link (x, mu): the 1-link term only;
      (x +- nu, mu): one 3-staple;  (x + nu + rho, mu): two 5-staples (both orders);
      (x + nu + rho + sig, mu): six 7-staples;  (x + 2 nu, mu): one Lepage path;
      (x, nu) first leg of every path opening with +nu: one 3-staple, four
      5-staples, eight 7-staples, one Lepage path; (x + mu, nu) the same, met backward;
      (x + nu, nu): the Lepage path's second step.
    The Naik link W_mu(x) has each of its three links once."""
    dims = (6, 6, 6, 6)     # paths reach 2 sites across, so nothing wraps onto x
    c = asqtad.coefficients(u0)
    x0 = np.array([2, 2, 2, 2])
    mu, nu, rho, sig = 1, 0, 2, 3
    e = np.eye(4, dtype=int)
    leg = c["staple3"] + 4 * c["staple5"] + 8 * c["staple7"] + c["lepage"]
    cases = [
        (x0, mu, c["one"]),
        (x0 + e[nu], mu, c["staple3"]),
        (x0 - e[rho], mu, c["staple3"]),
        (x0 + e[nu] - e[rho], mu, 2 * c["staple5"]),
        (x0 - e[nu] + e[rho] + e[sig], mu, 6 * c["staple7"]),
        (x0 + 2 * e[sig], mu, c["lepage"]),
        (x0, nu, leg),
        (x0 + e[mu], nu, -leg),
        (x0 - e[rho], rho, -leg),
        (x0 + e[nu], nu, c["lepage"]),
        (x0 + e[mu] + e[nu], nu, -c["lepage"]),
        (x0 + 3 * e[nu], mu, 0.0),
    ]
    h = 1e-5
    t, z, y, x = x0[3], x0[2], x0[1], x0[0]
    for site, dnu, expect in cases:
        vp, _ = asqtad.fat_long_links(_phase_on_link(dims, tuple(site), dnu, h), u0, False)
        vm, _ = asqtad.fat_long_links(_phase_on_link(dims, tuple(site), dnu, -h), u0, False)
        deriv = (vp[mu, t, z, y, x] - vm[mu, t, z, y, x]) / (2 * h)
        np.testing.assert_allclose(deriv, 1j * expect * np.eye(3), atol=1e-9)
    for k in range(3):
        _, wp = asqtad.fat_long_links(_phase_on_link(dims, tuple(x0 + k * e[mu]), mu, h), u0, False)
        _, wm = asqtad.fat_long_links(_phase_on_link(dims, tuple(x0 + k * e[mu]), mu, -h), u0, False)
        deriv = (wp[mu, t, z, y, x] - wm[mu, t, z, y, x]) / (2 * h)
        np.testing.assert_allclose(deriv, 1j * c["naik"] * np.eye(3), atol=1e-9)


def test_time_boundary_signs():
    """With antiperiodic time the fat t-link leaving the last slice and the
    Naik t-links that cross it change sign, spatial fat links do not."""
    dims = (4, 4, 4, 4)
    u = syn.near_identity_gauge(dims, 31)
    v1, w1 = asqtad.fat_long_links(u, 1.0, True)
    v0, w0 = asqtad.fat_long_links(u, 1.0, False)
    np.testing.assert_allclose(v1[:3], v0[:3], atol=1e-15)
    np.testing.assert_allclose(v1[3, :3], v0[3, :3], atol=1e-15)
    np.testing.assert_allclose(v1[3, 3], -v0[3, 3], atol=1e-15)
    np.testing.assert_allclose(w1[:3], w0[:3], atol=1e-15)
    np.testing.assert_allclose(w1[3, 0], w0[3, 0], atol=1e-15)
    np.testing.assert_allclose(w1[3, 1:], -w0[3, 1:], atol=1e-15)


def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    u = syn.haar_gauge(dims, 5)
    g = syn.random_gauge_transform(dims, 6)
    up = np.stack([np.einsum("...ij,...jk,...lk->...il", g, u[mu], np.conj(lat.shift_fwd(g, mu)))
                   for mu in range(4)])
    v, w = asqtad.fat_long_links(u)
    vg, wg = asqtad.fat_long_links(up)
    for mu in range(4):
        g3 = g
        for _ in range(3):
            g3 = lat.shift_fwd(g3, mu)
        np.testing.assert_allclose(vg[mu], g @ v[mu] @ su3.dag(lat.shift_fwd(g, mu)), atol=1e-13)
        np.testing.assert_allclose(wg[mu], g @ w[mu] @ su3.dag(g3), atol=1e-13)
    eta0 = lat.eta(dims, antiperiodic_t=False)
    psi = syn.gaussian_fermion(dims, 7, on_parity=None)
    lhs = asqtad.dslash(vg, wg, np.einsum("...ij,...j->...i", g, psi), eta0)
    rhs = np.einsum("...ij,...j->...i", g, asqtad.dslash(v, w, psi, eta0))
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_antihermitian_blocks_and_dense_a():
    dims = (4, 4, 4, 4)
    u = syn.near_identity_gauge(dims, 11)
    v, w = asqtad.fat_long_links(u)
    eta0, par = lat.eta(dims, antiperiodic_t=False), lat.parity(dims)
    a = syn.gaussian_fermion(dims, 1, on_parity=1)
    b = syn.gaussian_fermion(dims, 2, on_parity=0)
    lhs = np.vdot(a, asqtad.d_block(v, w, b, eta0, par, 1))
    rhs = -np.vdot(asqtad.d_block(v, w, a, eta0, par, 0), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    d2 = (2, 2, 2, 4)
    u2 = syn.haar_gauge(d2, 3)
    v2, w2 = asqtad.fat_long_links(u2, 0.9)
    e2, p2 = lat.eta(d2, antiperiodic_t=False), lat.parity(d2)
    d = asqtad.dense_dslash(v2, w2, e2)
    np.testing.assert_allclose(d, -d.conj().T, atol=1e-14)
    # A = m^2 - D_eo D_oe against the dense blocks, Hermitian, in [m^2, m^2 + ||D||^2]
    mass = 0.3
    ev_idx = np.flatnonzero(np.repeat(p2.reshape(-1) == 0, 3))
    od_idx = np.flatnonzero(np.repeat(p2.reshape(-1) == 1, 3))
    dense_a = mass ** 2 * np.eye(len(ev_idx)) - d[np.ix_(ev_idx, od_idx)] @ d[np.ix_(od_idx, ev_idx)]
    psi = syn.gaussian_fermion(d2, 9, on_parity=0)
    got = asqtad.a_op(v2, w2, psi, mass, e2, p2).reshape(-1)[ev_idx]
    np.testing.assert_allclose(got, dense_a @ psi.reshape(-1)[ev_idx], atol=1e-12)
    lam = np.linalg.eigvalsh(dense_a)
    assert lam.min() >= mass ** 2 - 1e-12
    assert lam.max() <= mass ** 2 + asqtad.norm_bound(0.9) ** 2


def test_multishift_matches_dense():
    dims = (2, 2, 4, 4)
    u = syn.haar_gauge(dims, 13)
    v, w = asqtad.fat_long_links(u)
    eta0, par = lat.eta(dims, antiperiodic_t=False), lat.parity(dims)
    mass = 0.2
    b = syn.gaussian_fermion(dims, 14, on_parity=0)
    shifts = [0.0, 0.05, 0.7, 3.0]
    xs, _, _ = solvers.multishift_cg(lambda x: asqtad.a_op(v, w, x, mass, eta0, par), b, shifts, 1e-13)
    ev_idx = np.flatnonzero(np.repeat(par.reshape(-1) == 0, 3))
    d = asqtad.dense_dslash(v, w, eta0)
    od_idx = np.flatnonzero(np.repeat(par.reshape(-1) == 1, 3))
    dense_a = mass ** 2 * np.eye(len(ev_idx)) - d[np.ix_(ev_idx, od_idx)] @ d[np.ix_(od_idx, ev_idx)]
    for s, x in zip(shifts, xs):
        ref = np.linalg.solve(dense_a + s * np.eye(len(ev_idx)), b.reshape(-1)[ev_idx])
        np.testing.assert_allclose(x.reshape(-1)[ev_idx], ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def _rat(a0, alpha, beta):
    """A partial-fraction sum with given coefficients (no fit: any positive
    alpha, beta give a valid action for the force test)."""
    return rational.Rational(0.0, 0.0, 0.0, a0, np.array(alpha), np.array(beta), 0.0)


def _action(u, phi, rat, mass, par, u0, apt):
    dims = (u.shape[4], u.shape[3], u.shape[2], u.shape[1])
    v, w = asqtad.fat_long_links(u, u0, apt)
    eta0 = lat.eta(dims, antiperiodic_t=False)
    xs, _, _ = solvers.multishift_cg(lambda x: asqtad.a_op(v, w, x, mass, eta0, par, min(rat.beta)),
                                     phi, rat.beta, 1e-14)
    s = rat.a0 * np.vdot(phi, phi) + sum(a * np.vdot(phi, x) for a, x in zip(rat.alpha, xs))
    return float(np.real(s)), xs


@pytest.mark.parametrize("apt,u0", [(True, 1.0), (False, 0.85)])
def test_force_by_finite_differences(apt, u0):
    """F_a(y, nu) against the 4th-order central difference of S_f under
    U_nu(y) -> exp(i delta T_a) U_nu(y), on t-links of the boundary slice
    and on spatial links."""
    dims = (4, 4, 4, 4)
    u = syn.near_identity_gauge(dims, 41, width=0.5)
    par = lat.parity(dims)
    mass = 0.4
    rat = _rat(0.1, [0.3, 0.7], [0.05, 1.5])
    phi = syn.gaussian_fermion(dims, 42, on_parity=0)
    _, xs = _action(u, phi, rat, mass, par, u0, apt)
    f = asqtad.fermion_force(u, xs, rat.alpha, par, u0, apt)
    for (nu, t, z, y, x, a) in [(3, 3, 1, 2, 0, 2), (3, 0, 2, 2, 1, 7), (0, 1, 3, 0, 2, 0), (2, 2, 0, 1, 3, 4)]:
        def s_at(dl):
            up = u.copy()
            up[nu, t, z, y, x] = su3.expi_hermitian(dl * su3.T[a]) @ u[nu, t, z, y, x]
            return _action(up, phi, rat, mass, par, u0, apt)[0]
        dl = 1e-3
        fd = (-s_at(2 * dl) + 8 * s_at(dl) - 8 * s_at(-dl) + s_at(-2 * dl)) / (12 * dl)
        assert abs(f[nu, t, z, y, x, a] - fd) < 1e-8 * max(1.0, abs(fd)), (nu, t, z, y, x, a, f[nu, t, z, y, x, a], fd)


def _small_params(n_outer, apt=True):
    rat = _rat(0.2, [0.4, 0.9], [0.1, 2.0])
    hb = _rat(1.2, [-0.3, -0.5], [0.2, 3.0])
    fl = itg.Flavour(mass=0.5, hb=hb, md=rat, met=rat)
    return itg.HMCParams(dims=(4, 4, 4, 4), beta=5.5, tau=0.5, n_outer=n_outer, n_gauge=2, flavours=[fl],
                         tol_md=1e-13, tol_met=1e-13, antiperiodic_t=apt, action="asqtad", u0=0.9)


def test_trajectory_reversible():
    """Forward trajectory, momenta flipped, back again: the links return to
    1e-12 per component (fp64 MD with the asqtad force)."""
    p = _small_params(2)
    ctx = itg.Context(p)
    u0 = syn.near_identity_gauge(p.dims, 51)
    mom = syn.gaussian_momenta(p.dims, 52)
    phis = [[syn.gaussian_fermion(p.dims, 53, on_parity=0)]]
    u1, m1 = itg.md_evolve(ctx, u0, mom, phis, p.tau, p.n_outer, p.n_gauge)
    u2, m2 = itg.md_evolve(ctx, u1, -m1, phis, p.tau, p.n_outer, p.n_gauge)
    assert np.max(np.abs(u2 - u0)) < 1e-12
    assert np.max(np.abs(m2 + mom)) < 1e-11


def test_dh_scales_as_step_squared():
    """Energy violation of the second-order scheme: dH(eps) / dH(eps/2) ~ 4."""
    dims = (4, 4, 4, 4)
    u0 = syn.near_identity_gauge(dims, 61)
    mom = syn.gaussian_momenta(dims, 62)
    phis = [[syn.gaussian_fermion(dims, 63, on_parity=0)]]
    dh = []
    for n in (2, 4):
        p = _small_params(n)
        ctx = itg.Context(p)
        r = itg.trajectory(ctx, u0, mom, None, phis=phis)
        dh.append(abs(r["dH"]))
    ratio = dh[0] / dh[1]
    assert 3.0 < ratio < 5.5, (dh, ratio)


def test_one_hop_skeleton_is_the_unimproved_operator():
    """With the boundary-signed thin links as fat links and no Naik term the
    improved operator's hop structure is the paper's unimproved D (pinned
    separately by its own free-field spectrum and dense solves)."""
    from oracle import dirac
    dims = (4, 2, 4, 6)
    u = syn.haar_gauge(dims, 71)
    psi = syn.gaussian_fermion(dims, 72, on_parity=None)
    v = asqtad.boundary_signed_links(u, True)
    got = asqtad.dslash(v, np.zeros_like(u), psi, lat.eta(dims, antiperiodic_t=False))
    np.testing.assert_allclose(got, dirac.dslash(u, psi, lat.eta(dims, True)), atol=1e-14)
