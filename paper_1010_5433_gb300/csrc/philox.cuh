// Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11),
// usable on host and device.  Round: (h0,l0) = M0*c0, (h1,l1) = M1*c2,
// c' = (h1^c1^k0, l1, h0^c3^k1, l0); key += (W0, W1) between rounds.
#pragma once
#include <stdint.h>

struct Philox4 { uint64_t v[4]; };

__host__ __device__ inline void mul128(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
#ifdef __CUDA_ARCH__
    lo = a * b;
    hi = __umul64hi(a, b);
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    lo = (uint64_t)p;
    hi = (uint64_t)(p >> 64);
#endif
}

__host__ __device__ inline Philox4 philox4x64_10(Philox4 c, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        uint64_t h0, l0, h1, l1;
        mul128(M0, c.v[0], h0, l0);
        mul128(M1, c.v[2], h1, l1);
        Philox4 n;
        n.v[0] = h1 ^ c.v[1] ^ k0;
        n.v[1] = l1;
        n.v[2] = h0 ^ c.v[3] ^ k1;
        n.v[3] = l0;
        c = n;
    }
    return c;
}

// uniform in (0, 1) from the top 53 bits
__host__ __device__ inline double philox_uniform(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1.0p-53; }

// Block `index` of stream `stream` at trajectory counter `counter`:
// key = (seed, stream), counter words = (index, counter, 0, 0).
__host__ __device__ inline Philox4 philox_block(uint64_t seed, uint64_t stream, uint64_t index, uint64_t counter) {
    Philox4 c;
    c.v[0] = index; c.v[1] = counter; c.v[2] = 0; c.v[3] = 0;
    return philox4x64_10(c, seed, stream);
}

enum : uint64_t { RNG_STREAM_MOMENTA = 1, RNG_STREAM_METROPOLIS = 3, RNG_STREAM_SOURCES = 0x100 };
