"""Pins for the oracle's Remez rational approximation (paper Sec. 2)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import dirac, lattice as lat, rational, solvers


@pytest.fixture(scope="module")
def r_quarter():
    return rational.remez(0.25, 0.01, 16.01, 6, dps=50)


def test_equioscillation(r_quarter):
    """Chebyshev alternation: the relative error has 2n+2 extrema of equal
    magnitude and alternating sign, including both end points."""
    r = r_quarter
    x = np.exp(np.linspace(np.log(r.lo), np.log(r.hi), 200001))
    e = r(x) * x ** r.s - 1.0
    assert np.isclose(np.abs(e).max(), r.err, rtol=1e-4)
    # local extrema of the sampled error
    idx = [0] + [i for i in range(1, len(e) - 1)
                 if (e[i] - e[i - 1]) * (e[i + 1] - e[i]) <= 0] + [len(e) - 1]
    ext = e[idx]
    ext = ext[np.abs(ext) > 0.5 * r.err]
    n = len(r.alpha)
    assert len(ext) == 2 * n + 2
    assert np.all(np.sign(ext[1:]) == -np.sign(ext[:-1]))
    np.testing.assert_allclose(np.abs(ext), r.err, rtol=1e-3)


def test_positive_partial_fractions(r_quarter):
    assert r_quarter.a0 > 0
    assert all(a > 0 for a in r_quarter.alpha) and all(b > 0 for b in r_quarter.beta)
    rh = rational.remez(-0.125, 0.01, 16.01, 5, dps=50)     # heatbath-type x^(+1/8)
    assert all(b > 0 for b in rh.beta)


def test_rational_of_matrix_matches_eigendecomposition(r_quarter):
    """r(A) phi vs V diag(lambda^(-s)) V^dag phi from the dense A on 2^4,
    within the approximation's relative error bound."""
    dims = (2, 2, 2, 2)
    mass = 0.1
    u = syn.near_identity_gauge(dims, 51)
    eta, par = lat.eta(dims), lat.parity(dims)
    phi = syn.gaussian_fermion(dims, 52, on_parity=0)
    a = dirac.dense_a(u, mass, eta, par)
    w, v = np.linalg.eigh(a)
    ev = dirac.even_indices(par)
    exact = v @ (w ** -r_quarter.s * (v.conj().T @ phi.reshape(-1)[ev]))
    s0 = min(r_quarter.beta)
    got = rational.apply_rational(
        r_quarter,
        lambda b, betas: solvers.multishift_cg(
            lambda y: dirac.a_op(u, y, mass, eta, par, s0), b, betas, 1e-14)[0],
        phi).reshape(-1)[ev]
    assert np.linalg.norm(got - exact) <= 1.01 * r_quarter.err * np.linalg.norm(exact) + 1e-12
