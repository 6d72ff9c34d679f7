"""SU(3) algebra used by the MD update (paper Sec. 4: gauge update
U <- exp(i eps P) U in single precision, reunitarisation in double).

Conventions
  T_a = lambda_a / 2 (Gell-Mann matrices), tr(T_a T_b) = delta_ab / 2.
  A momentum / force on a link is the Hermitian traceless matrix
  P = sum_a p_a T_a, stored as its 8 real coefficients p_a = 2 tr(T_a P).
  U(eps) = exp(i eps P) U solves dU/dt = i P U.
"""
import numpy as np


def gell_mann():
    """The eight Gell-Mann matrices lambda_a, shape [8, 3, 3] complex."""
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j
    l[1][1, 0] = 1j
    l[2][0, 0] = 1
    l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j
    l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j
    l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


T = gell_mann() / 2.0


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def coeffs_to_matrix(p):
    """P = sum_a p_a T_a for p of shape [..., 8]."""
    return np.einsum("...a,aij->...ij", p, T)


def matrix_to_coeffs(h):
    """p_a = 2 Re tr(T_a H) for Hermitian H of shape [..., 3, 3]."""
    return 2.0 * np.real(np.einsum("aij,...ji->...a", T, h))


def traceless_hermitian_part(m):
    """TH(M) = (M + M^dag)/2 - tr(M + M^dag)/6 * 1."""
    h = 0.5 * (m + dag(m))
    tr = np.trace(h, axis1=-2, axis2=-1)
    return h - (tr / 3.0)[..., None, None] * np.eye(3)


def expi_hermitian(h):
    """exp(i H) for Hermitian H by its eigen-decomposition (float64)."""
    w, v = np.linalg.eigh(h)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def expi_coeffs(p, eps):
    """exp(i eps sum_a p_a T_a)."""
    return expi_hermitian(eps * coeffs_to_matrix(p))


def reunitarize(u):
    """Project onto SU(3): Gram-Schmidt on rows 1 and 2, then row 3 is the
    complex conjugate of their cross product (paper Sec. 4 and Sec. 5: the
    third row of an SU(3) link is fixed by the first two)."""
    r0 = u[..., 0, :]
    r0 = r0 / np.sqrt(np.sum(np.abs(r0) ** 2, axis=-1))[..., None]
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1)[..., None] * r0
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1))[..., None]
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def third_row(u):
    """conj(row0 x row1): the row that 12-real storage rebuilds (Sec. 5)."""
    return np.conj(np.cross(u[..., 0, :], u[..., 1, :]))
