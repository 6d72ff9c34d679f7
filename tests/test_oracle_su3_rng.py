"""Pins for the oracle's SU(3) algebra and its counter-based generator."""
import numpy as np
import scipy.linalg

import synthetic as syn
from oracle import philox, su3


def test_generators_normalised():
    g = np.einsum("aij,bji->ab", su3.T, su3.T)
    np.testing.assert_allclose(g, 0.5 * np.eye(8), atol=1e-15)
    for a in range(8):
        np.testing.assert_allclose(su3.T[a], su3.T[a].conj().T)
        assert abs(np.trace(su3.T[a])) < 1e-15


def test_coeff_roundtrip_and_exp_matches_scipy():
    r = np.random.default_rng(0).standard_normal((5, 8))
    h = su3.coeffs_to_matrix(r)
    np.testing.assert_allclose(su3.matrix_to_coeffs(h), r, atol=1e-14)
    e = su3.expi_coeffs(r, 0.7)
    for k in range(5):
        np.testing.assert_allclose(e[k], scipy.linalg.expm(0.7j * h[k]), atol=1e-13)
        np.testing.assert_allclose(np.linalg.det(e[k]), 1.0, atol=1e-13)


def test_reunitarize_and_third_row():
    u = syn.haar_gauge((2, 2, 2, 2), 3).reshape(-1, 3, 3)
    np.testing.assert_allclose(su3.third_row(u), u[:, 2, :], atol=1e-13)
    noisy = u + 1e-3 * np.random.default_rng(1).standard_normal(u.shape)
    w = su3.reunitarize(noisy)
    eye = np.einsum("nij,nkj->nik", w, np.conj(w))
    np.testing.assert_allclose(eye, np.broadcast_to(np.eye(3), eye.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(w), 1.0, atol=1e-14)
    np.testing.assert_allclose(su3.reunitarize(u), u, atol=1e-14)   # idempotent on SU(3)


def test_philox_matches_numpy_and_known_answer():
    # numpy's Philox bit generator is Philox4x64-10; it increments the
    # counter before each block, so a state counter c yields block c + 1
    for key, ctr in [((7, 9), 5), ((0, 0), 0), ((2**64 - 1, 123), 2**40)]:
        raw = np.random.Philox(counter=np.array([ctr, 0, 0, 0], dtype=np.uint64),
                               key=np.array(key, dtype=np.uint64)).random_raw(4)
        assert [int(v) for v in raw] == philox.philox4x64((ctr + 1, 0, 0, 0), key)
    # Random123 known-answer vector for philox4x64-10 at zero counter and key
    assert philox.philox4x64((0, 0, 0, 0), (0, 0)) == [
        0x16554d9eca36314c, 0xdb20fe9d672d0fdc, 0xd7e772cee186176b, 0x7e68b68aec7ba23b]


def test_gaussian_draws_moments():
    g = np.array([philox.gaussians4(1234, 5, i, 0) for i in range(20000)]).reshape(-1)
    assert abs(g.mean()) < 0.02 and abs(g.var() - 1) < 0.02
