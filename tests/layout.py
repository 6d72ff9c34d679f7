"""Test-side layout helpers: move whole-lattice numpy fields ([t, z, y, x, ...])
to and from the half-lattice structure-of-arrays layout of the C ABI.  Pure
index bookkeeping, written independently of both the oracle and the
library."""
import numpy as np


def parity_flat(dims):
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((x + y + z + t) % 2).reshape(-1)


def to_half(psi, dims, parity):
    """psi [t, z, y, x, 3] complex -> [3, Vh] complex (sites of `parity`, h = s >> 1)."""
    flat = psi.reshape(-1, 3)
    return np.ascontiguousarray(flat[parity_flat(dims) == parity].T)


def from_half(half, dims, parity):
    """[3, Vh] -> whole-lattice field, zero on the other parity."""
    Lx, Ly, Lz, Lt = dims
    out = np.zeros((Lx * Ly * Lz * Lt, 3), dtype=complex)
    out[parity_flat(dims) == parity] = half.T
    return out.reshape(Lt, Lz, Ly, Lx, 3)


def gauge_host(u):
    """[4, t, z, y, x, 3, 3] complex -> contiguous float64 host layout of the C ABI."""
    return np.ascontiguousarray(u.astype(np.complex128)).reshape(-1).view(np.float64)


def gauge_from_host(buf, dims):
    Lx, Ly, Lz, Lt = dims
    return buf.view(np.complex128).reshape(4, Lt, Lz, Ly, Lx, 3, 3)


def mom_to_abi(mom, dims):
    """[4, t, z, y, x, 8] -> [4][2][8][Vh] (the momentum/force layout)."""
    par = parity_flat(dims)
    out = np.empty((4, 2, 8, len(par) // 2))
    for mu in range(4):
        flat = mom[mu].reshape(-1, 8)
        for p in range(2):
            out[mu, p] = flat[par == p].T
    return out


def mom_from_abi(arr, dims):
    Lx, Ly, Lz, Lt = dims
    par = parity_flat(dims)
    out = np.empty((4, Lx * Ly * Lz * Lt, 8))
    for mu in range(4):
        for p in range(2):
            out[mu][par == p] = arr[mu, p].T
    return out.reshape(4, Lt, Lz, Ly, Lx, 8)


def half_to_complex64(h):
    return np.ascontiguousarray(h.astype(np.complex64))


def rel_err(a, b):
    return float(np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1)))


def bf16_round(x32):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32)
