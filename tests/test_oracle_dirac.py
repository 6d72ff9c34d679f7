"""Pins for the oracle's staggered operator (paper Sec. 2): closed-form
free-field spectrum, anti-Hermiticity, gauge covariance and dense solves."""
import numpy as np
import pytest

import synthetic as syn
from oracle import dirac, lattice as lat, solvers


def _free_spectrum(dims, antiperiodic_t):
    """Closed form: -D^2 = sum_mu sin^2 p_mu on plane waves, p_mu = 2 pi n / L
    (p_t = pi (2n+1) / L_t with antiperiodic time), one per colour."""
    ps = []
    for mu, L in enumerate(dims):
        if mu == 3 and antiperiodic_t:
            ps.append(np.pi * (2 * np.arange(L) + 1) / L)
        else:
            ps.append(2 * np.pi * np.arange(L) / L)
    grids = np.meshgrid(*ps, indexing="ij")
    vals = sum(np.sin(g) ** 2 for g in grids).reshape(-1)
    return np.sort(np.repeat(vals, 3))


@pytest.mark.parametrize("dims,apt", [((2, 2, 2, 2), False), ((4, 4, 4, 4), True), ((2, 4, 2, 4), True)])
def test_free_field_spectrum(dims, apt):
    u = syn.unit_gauge(dims)
    d = dirac.dense_dslash(u, lat.eta(dims, apt))
    ev = np.sort(np.linalg.eigvalsh(-(d @ d)))
    np.testing.assert_allclose(ev, _free_spectrum(dims, apt), atol=1e-12)


def test_antihermitian_blocks():
    dims = (4, 4, 4, 4)
    u = syn.near_identity_gauge(dims, 11)
    eta, par = lat.eta(dims), lat.parity(dims)
    a = syn.gaussian_fermion(dims, 1, on_parity=1)   # odd
    b = syn.gaussian_fermion(dims, 2, on_parity=0)   # even
    lhs = np.vdot(a, dirac.d_block(u, b, eta, par, 1))          # <a, D_oe b>
    rhs = -np.vdot(dirac.d_block(u, a, eta, par, 0), b)         # -<D_eo a, b>
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    d = dirac.dense_dslash(syn.near_identity_gauge((2, 2, 2, 2), 3), lat.eta((2, 2, 2, 2)))
    np.testing.assert_allclose(d, -d.conj().T, atol=1e-14)


def test_gauge_covariance():
    dims = (4, 2, 4, 2)
    u = syn.haar_gauge(dims, 5)
    g = syn.random_gauge_transform(dims, 6)
    eta = lat.eta(dims)
    up = np.stack([np.einsum("...ij,...jk,...lk->...il", g, u[mu], np.conj(lat.shift_fwd(g, mu)))
                   for mu in range(4)])
    psi = syn.gaussian_fermion(dims, 7, on_parity=None)
    lhs = dirac.dslash(up, np.einsum("...ij,...j->...i", g, psi), eta)
    rhs = np.einsum("...ij,...j->...i", g, dirac.dslash(u, psi, eta))
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_a_operator_matches_dense_and_is_hpd():
    dims = (2, 2, 2, 2)
    u = syn.near_identity_gauge(dims, 21)
    eta, par = lat.eta(dims), lat.parity(dims)
    mass = 0.1
    a = dirac.dense_a(u, mass, eta, par)
    np.testing.assert_allclose(a, a.conj().T, atol=1e-14)
    w = np.linalg.eigvalsh(a)
    assert w.min() >= mass ** 2 - 1e-12 and w.max() <= mass ** 2 + 16 + 1e-12
    psi = syn.gaussian_fermion(dims, 4, on_parity=0)
    ev = dirac.even_indices(par)
    got = dirac.a_op(u, psi, mass, eta, par).reshape(-1)[ev]
    np.testing.assert_allclose(got, a @ psi.reshape(-1)[ev], atol=1e-13)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_cg_matches_dense_inverse(dims):
    u = syn.near_identity_gauge(dims, 31)
    eta, par = lat.eta(dims), lat.parity(dims)
    mass = 0.1
    b = syn.gaussian_fermion(dims, 8, on_parity=0)
    x, its, res = solvers.cg(lambda v: dirac.a_op(u, v, mass, eta, par), b, 1e-13)
    ev = dirac.even_indices(par)
    xd = np.linalg.solve(dirac.dense_a(u, mass, eta, par), b.reshape(-1)[ev])
    got = x.reshape(-1)[ev]
    assert np.linalg.norm(got - xd) <= 1e-12 * np.linalg.norm(xd)
    assert res <= 1e-12


def test_multishift_matches_dense_and_first_zeta():
    dims = (2, 2, 2, 2)
    u = syn.near_identity_gauge(dims, 41)
    eta, par = lat.eta(dims), lat.parity(dims)
    mass = 0.1
    shifts = [0.003, 0.02, 0.1, 0.7, 3.0]
    b = syn.gaussian_fermion(dims, 9, on_parity=0)
    s0 = min(shifts)
    apply0 = lambda v: dirac.a_op(u, v, mass, eta, par, s0)
    xs, its, per = solvers.multishift_cg(apply0, b, shifts, 1e-13)
    ev = dirac.even_indices(par)
    a = dirac.dense_a(u, mass, eta, par)
    for s, x in zip(shifts, xs):
        xd = np.linalg.solve(a + s * np.eye(len(ev)), b.reshape(-1)[ev])
        assert np.linalg.norm(x.reshape(-1)[ev] - xd) <= 1e-11 * np.linalg.norm(xd)
    # after one iteration: zeta_1 = 1 / (1 + (sigma - sigma_0) alpha_0) and
    # x_sigma = alpha_0 zeta_1 b exactly (first CG step of the shifted system)
    x1, _, _ = solvers.multishift_cg(apply0, b, shifts, 0.0, max_iter=1)
    bb = np.vdot(b, b).real
    alpha0 = bb / np.vdot(b, apply0(b)).real
    for s, x in zip(shifts, x1):
        zeta1 = 1.0 / (1.0 + (s - s0) * alpha0)
        np.testing.assert_allclose(x, alpha0 * zeta1 * b, rtol=1e-13, atol=1e-15)
    # iteration counts: larger shifts converge no later than smaller ones
    assert all(per[i] >= per[i + 1] for i in range(len(per) - 1))
