"""The seeded input generators that feed both the oracle and the CUDA path:
SU(3) by construction, Haar moments fixed by character orthogonality
(E tr U = 0, E |tr U|^2 = 1, and E (tr U)^3 = 1, which separates SU(3) from
U(3)), the near-identity recipe's generator coefficients, the fermion and
momentum draws' variances and support, and determinism per seed."""
import numpy as np
import pytest

import synthetic as syn

DIMS = (4, 4, 4, 8)


def _su3_violation(u):
    m = u.reshape(-1, 3, 3)
    eye = np.eye(3)
    unit = np.abs(np.einsum("nij,nkj->nik", m, m.conj()) - eye).max()
    det = np.abs(np.linalg.det(m) - 1.0).max()
    return unit, det


@pytest.mark.parametrize("make", [syn.haar_gauge, syn.near_identity_gauge])
def test_links_are_su3(make):
    unit, det = _su3_violation(make(DIMS, 11))
    assert unit < 1e-13 and det < 1e-13


def test_haar_moments():
    t = np.trace(syn.haar_gauge(DIMS, 12).reshape(-1, 3, 3), axis1=1, axis2=2)
    n = t.size                                  # 4 * 512 links
    assert abs(t.mean()) < 5 / np.sqrt(n)       # E tr U = 0, Var = 1
    assert abs(np.mean(np.abs(t) ** 2) - 1.0) < 5 / np.sqrt(n)
    assert abs(np.mean(t ** 3) - 1.0) < 0.3     # SU(3): one invariant in V x V x V


def test_near_identity_generator_coefficients():
    width = 0.3
    u = syn.near_identity_gauge(DIMS, 13, width=width).reshape(-1, 3, 3)
    w, v = np.linalg.eig(u)
    h = np.einsum("nij,nj,nkj->nik", v, np.angle(w), np.linalg.inv(v).transpose(0, 2, 1))
    t = syn._gell_mann_half()
    c = 2.0 * np.einsum("nij,aji->na", h, t).real / width   # tr(T_a T_b) = delta_ab / 2
    assert abs(c.mean()) < 0.05
    assert abs(c.var() - 1.0) < 0.05
    assert np.abs(c.mean(axis=0)).max() < 0.15


def test_fermion_and_momentum_draws():
    f = syn.gaussian_fermion(DIMS, 14, on_parity=1)
    par = syn.parity(DIMS)
    assert np.all(f[par == 0] == 0)
    on = f[par == 1]
    assert abs(on.real.var() - 0.5) < 0.05 and abs(on.imag.var() - 0.5) < 0.05
    full = syn.gaussian_fermion(DIMS, 14, on_parity=None)
    assert np.count_nonzero(full) == full.size
    p = syn.gaussian_momenta(DIMS, 15)
    assert p.shape == (4,) + syn.shape_of(DIMS) + (8,)
    assert abs(p.mean()) < 0.03 and abs(p.var() - 1.0) < 0.03


def test_seeded_and_shaped():
    for make in (syn.haar_gauge, syn.near_identity_gauge, syn.gaussian_momenta, syn.gaussian_fermion):
        a, b, c = make(DIMS, 21), make(DIMS, 21), make(DIMS, 22)
        assert np.array_equal(a, b) and not np.array_equal(a, c)
    g = syn.random_gauge_transform(DIMS, 23)
    assert g.shape == syn.shape_of(DIMS) + (3, 3)
    unit, det = _su3_violation(g)
    assert unit < 1e-13 and det < 1e-13
    assert syn.haar_gauge(DIMS, 1).shape == (4,) + syn.shape_of(DIMS) + (3, 3)
