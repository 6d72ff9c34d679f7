"""Unimproved staggered Dirac operator and its even/odd blocks (paper Sec. 2).

  D psi(x) = 1/2 sum_mu eta_mu(x) [ U_mu(x) psi(x+mu) - U_mu(x-mu)^dag psi(x-mu) ]
  M = m + D,   D^dag = -D,   M^dag M = m^2 - D^2.

D only connects sites of opposite parity, so with even/odd ordering
D = [[0, D_eo], [D_oe, 0]] and det M is carried by the even block
  A = m^2 - D_eo D_oe = m^2 + D_eo D_eo^dag       (Hermitian, spectrum in [m^2, m^2+16]).
The 1/2 normalisation is the reading taken where the paper is silent: it makes
the free-field spectrum of -D^2 equal to sum_mu sin^2(p_mu).

Fields here are whole-lattice arrays [t, z, y, x, 3]; a field "on parity p"
is one that vanishes on the other parity.
"""
import numpy as np

from . import lattice as lat
from .su3 import dag


def dslash(u, psi, eta):
    """D psi on the whole lattice; u [4, t, z, y, x, 3, 3], psi [t, z, y, x, 3]."""
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = np.einsum("...ij,...j->...i", u[mu], lat.shift_fwd(psi, mu))
        bwd_at_src = np.einsum("...ij,...j->...i", dag(u[mu]), psi)  # U_mu(y)^dag psi(y)
        bwd = lat.shift_bwd(bwd_at_src, mu)                          # taken at y = x - mu
        sgn_bwd = lat.shift_bwd(eta[mu], mu)                         # eta of link (x - mu, mu)
        out += 0.5 * (eta[mu][..., None] * fwd - sgn_bwd[..., None] * bwd)
    return out


def restrict(psi, par, p):
    """Zero the sites whose parity is not p."""
    return np.where((par == p)[..., None], psi, 0.0)


def d_block(u, psi, eta, par, out_parity):
    """D_{out, in}: takes a field on parity 1-out_parity, returns it on out_parity."""
    return restrict(dslash(u, restrict(psi, par, 1 - out_parity), eta), par, out_parity)


def a_op(u, psi_e, mass, eta, par, shift=0.0):
    """(A + shift) psi_e with A = m^2 - D_eo D_oe, psi_e an even field."""
    tmp = d_block(u, psi_e, eta, par, 1)     # D_oe psi_e
    return (mass * mass + shift) * restrict(psi_e, par, 0) - d_block(u, tmp, eta, par, 0)


def dense_dslash(u, eta):
    """D as a dense (3V x 3V) matrix by applying it to unit vectors (tiny lattices)."""
    shape = u.shape[1:5]
    n = 3 * int(np.prod(shape))
    mat = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1.0
        mat[:, k] = dslash(u, e.reshape(shape + (3,)), eta).reshape(n)
    return mat


def even_indices(par):
    """Flat indices (site*3 + colour) of the even-site components."""
    sites = np.flatnonzero(par.reshape(-1) == 0)
    return (sites[:, None] * 3 + np.arange(3)).reshape(-1)


def dense_a(u, mass, eta, par):
    """A = m^2 - D_eo D_oe as a dense matrix on the even components."""
    d = dense_dslash(u, eta)
    n = d.shape[0]
    ev = even_indices(par)
    od = np.setdiff1d(np.arange(n), ev)
    d_eo = d[np.ix_(ev, od)]
    d_oe = d[np.ix_(od, ev)]
    return mass * mass * np.eye(len(ev)) - d_eo @ d_oe
