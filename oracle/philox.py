"""Counter-based Philox4x64-10 generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11) and the Gaussian draws
built on it.  The paper does not say how its RNG works; a counter-based
generator lets the GPU draw momenta and pseudo-fermion sources in any order
and still be compared draw by draw with this plain restatement.

Philox4x64 round on counter (c0, c1, c2, c3) and key (k0, k1):
    (h0, l0) = M0 * c0,  (h1, l1) = M1 * c2     (128-bit products)
    c' = (h1 ^ c1 ^ k0,  l1,  h0 ^ c3 ^ k1,  l0)
    then k0 += W0, k1 += W1 (mod 2^64);  10 rounds.

Draw layout used by the method (both sides):
  block(key=(seed, stream), counter=(index, counter_lo, counter_hi, 0)) -> 4 x u64
  uniform   u = ((x >> 11) + 0.5) * 2^-53  in (0, 1)
  Gaussian  Box-Muller on the two uniforms of words (0, 1) and of (2, 3):
            g = sqrt(-2 ln u_a) * (cos 2 pi u_b, sin 2 pi u_b)
"""
import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
MASK = (1 << 64) - 1


def philox4x64(ctr, key, rounds=10):
    c = [int(v) & MASK for v in ctr]
    k0, k1 = int(key[0]) & MASK, int(key[1]) & MASK
    for r in range(rounds):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        h0, l0 = p0 >> 64, p0 & MASK
        h1, l1 = p1 >> 64, p1 & MASK
        c = [h1 ^ c[1] ^ k0, l1, h0 ^ c[3] ^ k1, l0]
    return c


def uniform_from_u64(x):
    return ((x >> 11) + 0.5) * (2.0 ** -53)


def gaussians4(seed, stream, index, counter):
    """Four N(0,1) numbers from one Philox block."""
    w = philox4x64((index, counter & MASK, (counter >> 64) & MASK, 0), (seed, stream))
    u = [uniform_from_u64(v) for v in w]
    r0 = np.sqrt(-2.0 * np.log(u[0]))
    r1 = np.sqrt(-2.0 * np.log(u[2]))
    return [r0 * np.cos(2 * np.pi * u[1]), r0 * np.sin(2 * np.pi * u[1]),
            r1 * np.cos(2 * np.pi * u[3]), r1 * np.sin(2 * np.pi * u[3])]


def draw_momenta(dims, seed, counter):
    """Momenta [4, t, z, y, x, 8]: link (mu, s) with s lexicographic takes the
    normals of blocks 2 (mu V + s) + j, j = 0, 1, as p_{4j..4j+3} (stream 1)."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    out = np.empty((4, V, 8))
    for mu in range(4):
        for s in range(V):
            for j in range(2):
                out[mu, s, 4 * j:4 * j + 4] = gaussians4(seed, 1, 2 * (mu * V + s) + j, counter)
    return out.reshape(4, Lt, Lz, Ly, Lx, 8)


def draw_source_half(vh, seed, counter, stream):
    """One source on the even sites in half-lattice order [3, Vh]: site h takes
    the first six normals of blocks 2h and 2h + 1, times sqrt(1/2), as
    (Re, Im) of colours 0..2 (stream 0x100 + stream)."""
    out = np.empty((3, vh), dtype=complex)
    for h in range(vh):
        g = gaussians4(seed, 0x100 + stream, 2 * h, counter) + gaussians4(seed, 0x100 + stream, 2 * h + 1, counter)
        for c in range(3):
            out[c, h] = np.sqrt(0.5) * (g[2 * c] + 1j * g[2 * c + 1])
    return out
