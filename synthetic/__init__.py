"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds none of the method's arithmetic: it only draws random
numbers with numpy's PCG64 and shapes them into gauge links, momenta and
fermion sources.  Both the CUDA path and the CPU oracle receive what it
produces; neither is imported here.

Array conventions (whole lattice, float64 / complex128):
  gauge    U[mu, t, z, y, x, 3, 3]   mu = 0..3 for x, y, z, t
  momenta  p[mu, t, z, y, x, 8]      coefficients of sum_a p_a lambda_a / 2
  fermion  psi[t, z, y, x, 3]
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _gell_mann_half():
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l / 2


def shape_of(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx)


def near_identity_gauge(dims, seed, width=0.3):
    """U = exp(i * width * sum_a r_a T_a), r_a ~ N(0, 1) per link: the 4^4
    test configuration's recipe.  The exponential is taken with numpy's
    Hermitian eigensolver (a library routine)."""
    g = rng(seed)
    r = g.standard_normal((4,) + shape_of(dims) + (8,))
    h = width * np.einsum("...a,aij->...ij", r, _gell_mann_half())
    w, v = np.linalg.eigh(h)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def haar_gauge(dims, seed):
    """Haar-random SU(3) links (hot start): QR of a complex Gaussian matrix
    with the phases of R's diagonal moved into Q, then det fixed to 1."""
    g = rng(seed)
    z = (g.standard_normal((4,) + shape_of(dims) + (3, 3))
         + 1j * g.standard_normal((4,) + shape_of(dims) + (3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    q[..., :, 2] = q[..., :, 2] / det[..., None]   # unit-modulus det -> 1
    return q


def unit_gauge(dims):
    return np.broadcast_to(np.eye(3, dtype=complex), (4,) + shape_of(dims) + (3, 3)).copy()


def gaussian_momenta(dims, seed):
    return rng(seed).standard_normal((4,) + shape_of(dims) + (8,))


def parity(dims):
    Lt, Lz, Ly, Lx = shape_of(dims)
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    return (x + y + z + t) % 2


def gaussian_fermion(dims, seed, on_parity=0):
    """Complex Gaussian field with Re, Im ~ N(0, 1/2) (density exp(-psi^dag psi))
    on the sites of one parity, zero elsewhere (on_parity=None: everywhere)."""
    g = rng(seed)
    f = (g.standard_normal(shape_of(dims) + (3,)) + 1j * g.standard_normal(shape_of(dims) + (3,))) / np.sqrt(2)
    if on_parity is None:
        return f
    return np.where((parity(dims) == on_parity)[..., None], f, 0.0)


def random_gauge_transform(dims, seed):
    """One Haar-random SU(3) matrix per site, shape [t, z, y, x, 3, 3]."""
    return haar_gauge(dims, seed)[0]
