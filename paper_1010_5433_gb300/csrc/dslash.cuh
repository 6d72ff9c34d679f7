// The staggered Dslash kernel template (Sec. 2, Sec. 3, Sec. 5 / Table 2).
//
// One thread per output site and chunk of NR right-hand sides.  Each of the
// eight links of the site is loaded once (coalesced, structure of arrays) and
// applied to all NR sources before the next link is fetched, so the link
// traffic is shared by the right-hand sides.  What happens to the result
// (plain store, A-operator epilogue, reductions) is supplied by an Epi functor.
#pragma once
#include "common.cuh"

enum LinkFmt { FMT_F64 = 0, FMT_F32_18 = 1, FMT_F32_12 = 2, FMT_BF16_12 = 3 };

struct LinkPtrs {
    const float* hi;
    const float* lo;
    const uint16_t* b16;
};

template <typename R, int FMT> struct LinkFetch;
template <> struct LinkFetch<double, FMT_F64> {
    __device__ __forceinline__ static Su3<double> get(const LinkPtrs& L, int mu, int par, int h, int Vh) {
        return load_link_d(L.hi, L.lo, link_block_f(mu, par, Vh), h, Vh);
    }
};
template <> struct LinkFetch<DF, FMT_F64> {
    __device__ __forceinline__ static Su3<DF> get(const LinkPtrs& L, int mu, int par, int h, int Vh) {
        return load_link_df(L.hi, L.lo, link_block_f(mu, par, Vh), h, Vh);
    }
};
template <> struct LinkFetch<float, FMT_F32_18> {
    __device__ __forceinline__ static Su3<float> get(const LinkPtrs& L, int mu, int par, int h, int Vh) {
        return load_link_f<3>(L.hi + link_block_f(mu, par, Vh), h, Vh);
    }
};
template <> struct LinkFetch<float, FMT_F32_12> {
    __device__ __forceinline__ static Su3<float> get(const LinkPtrs& L, int mu, int par, int h, int Vh) {
        return load_link_f<2>(L.hi + link_block_f(mu, par, Vh), h, Vh);
    }
};
template <> struct LinkFetch<float, FMT_BF16_12> {
    __device__ __forceinline__ static Su3<float> get(const LinkPtrs& L, int mu, int par, int h, int Vh) {
        return load_link_bf(L.b16 + link_block_b(mu, par, Vh), h, Vh);
    }
};

// Source of the hops: the field itself ...
template <typename R> struct SrcPlain {
    const typename V2T<R>::T* __restrict__ in;
    template <int NR> __device__ __forceinline__ void prepare(int r0, int nrhs) {}
    // slot: the source's index inside the thread's chunk (compile-time after unrolling)
    __device__ __forceinline__ Vec3<R> load(int slot, int rhs, int h, int Vh) const {
        return load_vec<R>(in + (size_t)rhs * 3 * Vh, h, Vh);
    }
};

// ... or an fp64 field read as float-float: every double split into hi + lo
// floats with integer operations only (GB300's fp64 pipes are slow), so that
// the fp64 operator runs its arithmetic in float-float (Sec. 5's two-float
// representation) on the fp32 pipes.  hi keeps the top 23 mantissa bits (an
// exact float), lo is the remaining 29 bits rounded to float: hi + lo carries
// ~48 bits.  Magnitudes below 2^-126 (and lo parts below float range) flush
// to zero; magnitudes above float range become infinite.
__device__ __forceinline__ DF df_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;     // float exponent field of hi
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (e <= 0) return DF(0.f, 0.f);
    if (e >= 255) return DF(__uint_as_float(sign | 0x7F800000u), 0.f);
    const float hi = __uint_as_float(sign | ((unsigned int)e << 23) | (unsigned int)(m >> 29));
    // lo = low29 x 2^(e - 127 - 52): the integer part converts exactly up to 2^24 and rounds above
    const int el = e - 52;                                    // exponent field of 2^(e - 127 - 52)
    float lo = 0.f;
    if (el > 0) {
        lo = (float)(unsigned int)(m & 0x1FFFFFFFull) * __uint_as_float((unsigned int)el << 23);
        lo = __uint_as_float(__float_as_uint(lo) | sign);
    }
    return DF(hi, lo);
}
// hi + lo as a double: each float widened exactly by integer operations, one fp64 add
__device__ __forceinline__ double df_widen(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xFF;
    if (e == 0) return 0.0;                                   // zero (float denormals flushed)
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned long long ed = e == 0xFF ? 0x7FFull : (unsigned long long)(e - 127 + 1023);
    return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double df_join(DF v) { return df_widen(v.hi) + df_widen(v.lo); }

// CG = false: read-only path (__ldg), for fields no block of the launch
// writes; CG = true: L2 loads (__ldcg), for fields that other blocks of a
// persistent launch wrote before a grid barrier (the non-coherent cache may
// still hold an older copy of those lines).
template <bool CG>
struct SrcD2DFT {
    const double2* __restrict__ in;
    template <int NR> __device__ __forceinline__ void prepare(int r0, int nrhs) {}
    __device__ __forceinline__ Vec3<DF> load(int slot, int rhs, int h, int Vh) const {
        const double2* p = in + (size_t)rhs * 3 * Vh;
        Vec3<DF> v;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 d = CG ? __ldcg(p + (size_t)c * Vh + h) : __ldg(p + (size_t)c * Vh + h);
            v.c[c].re = df_split(d.x);
            v.c[c].im = df_split(d.y);
        }
        return v;
    }
};
typedef SrcD2DFT<false> SrcD2DF;
typedef SrcD2DFT<true> SrcD2DFcg;
template <typename R> struct SrcFor { typedef SrcPlain<R> type; typedef typename V2T<R>::T io; };
template <> struct SrcFor<DF> { typedef SrcD2DF type; typedef double2 io; };

// Accumulate the hops of one site for NR sources:
//   sum_mu [ sf U_mu(x) in(x+mu) - sb U_mu(x-mu)^dag in(x-mu) ]
// (the factor 1/2 is left to the epilogue).  With TPS threads per site, thread
// `sub` takes the hops of mu = sub, sub + TPS, ... (TPS <= 4), or, for TPS = 8,
// the forward (even sub) or backward (odd sub) hop of mu = sub / 2; the TPS
// partial sums are then added with warp shuffles.
// bf16 links, one thread per site and source: every load of the site (eight
// links' raw words, eight neighbour spinors) is issued before the first
// product, so a warp keeps ~12 KB in flight instead of one hop's worth
template <class Src>
__device__ __forceinline__ void dslash_site_bf16_prefetch(const Geom& g, int out_par, const LinkPtrs& L,
                                                          const Src& src, int r0, int h, Vec3<float>& acc) {
    Nbr n;
    site_neighbours(g, h, out_par, n);
    uint4 la[8];
    uint2 lb[8];
    Vec3<float> v[8];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const uint16_t* bf = L.b16 + link_block_b(mu, out_par, g.Vh);
        const uint16_t* bb = L.b16 + link_block_b(mu, 1 - out_par, g.Vh);
        la[2 * mu] = __ldg(reinterpret_cast<const uint4*>(bf) + h);
        lb[2 * mu] = __ldg(reinterpret_cast<const uint2*>(bf + 8 * (size_t)g.Vh) + h);
        la[2 * mu + 1] = __ldg(reinterpret_cast<const uint4*>(bb) + n.bwd[mu]);
        lb[2 * mu + 1] = __ldg(reinterpret_cast<const uint2*>(bb + 8 * (size_t)g.Vh) + n.bwd[mu]);
    }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        v[2 * mu] = src.load(0, r0, n.fwd[mu], g.Vh);
        v[2 * mu + 1] = src.load(0, r0, n.bwd[mu], g.Vh);
    }
    zero(acc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        mac_uv(acc, n.sf[mu], unpack_link_bf(la[2 * mu], lb[2 * mu]), v[2 * mu]);
        mac_udv(acc, -n.sb[mu], unpack_link_bf(la[2 * mu + 1], lb[2 * mu + 1]), v[2 * mu + 1]);
    }
}

template <typename R, int FMT, int NR, int TPS, class Src>
__device__ __forceinline__ void dslash_site(const Geom& g, int out_par, const LinkPtrs& L, const Src& src,
                                            int r0, int nrhs, int h, int sub, Vec3<R> (&acc)[NR]) {
    if constexpr (FMT == FMT_BF16_12 && TPS == 1 && NR == 1) {
        dslash_site_bf16_prefetch(g, out_par, L, src, r0, h, acc[0]);
        return;
    }
    Nbr n;
    site_neighbours(g, h, out_par, n);
#pragma unroll
    for (int r = 0; r < NR; ++r) zero(acc[r]);
#pragma unroll
    for (int m = 0; m < (TPS >= 4 ? 1 : 4 / TPS); ++m) {
        const int mu = TPS == 8 ? (sub >> 1) : (TPS == 4 ? sub : sub + m * TPS);
        const bool do_fwd = TPS < 8 || (sub & 1) == 0;
        const bool do_bwd = TPS < 8 || (sub & 1) == 1;
        if (do_fwd) {
            Su3<R> u = LinkFetch<R, FMT>::get(L, mu, out_par, h, g.Vh);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (r0 + r < nrhs) {
                    Vec3<R> v = src.load(r, r0 + r, n.fwd[mu], g.Vh);
                    mac_uv(acc[r], (R)n.sf[mu], u, v);
                }
            }
        }
        if (do_bwd) {
            Su3<R> w = LinkFetch<R, FMT>::get(L, mu, 1 - out_par, n.bwd[mu], g.Vh);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (r0 + r < nrhs) {
                    Vec3<R> v = src.load(r, r0 + r, n.bwd[mu], g.Vh);
                    mac_udv(acc[r], -(R)n.sb[mu], w, v);
                }
            }
        }
    }
}

template <int TPS, typename R>
__device__ __forceinline__ R group_sum(R v) {
#pragma unroll
    for (int o = TPS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid: blockIdx.x = site_block * nchunk + chunk, so that the chunks of one
// site block run back to back and re-read its links from L2.  A block of
// blockDim.x threads covers blockDim.x / TPS sites.
template <typename R, int FMT, int NR, int TPS, class Src, class Epi>
__global__ void __launch_bounds__(STAG_RED_BLOCK)
k_dslash(Geom g, int out_par, LinkPtrs L, Src src, int nrhs, int nchunk, Epi epi) {
    if (epi.halted()) return;
    const int chunk = blockIdx.x % nchunk;
    const int sblock = blockIdx.x / nchunk;
    const int sub = TPS > 1 ? (int)(threadIdx.x % TPS) : 0;
    const int h = sblock * (blockDim.x / TPS) + threadIdx.x / TPS;
    const int r0 = chunk * NR;
    Vec3<R> acc[NR];
    const bool inside = h < g.Vh;
    src.template prepare<NR>(r0, nrhs);
    if (inside) {
        dslash_site<R, FMT, NR, TPS>(g, out_par, L, src, r0, nrhs, h, sub, acc);
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) zero(acc[r]);
    }
    if (TPS > 1) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[r].c[c].re = group_sum<TPS>(acc[r].c[c].re);
                acc[r].c[c].im = group_sum<TPS>(acc[r].c[c].im);
            }
    }
    epi.template finish<NR>(g, h, inside && sub == 0, r0, nrhs, acc);
}

// Plain epilogue: out = scale * acc  (scale = 1/2 for D itself).
template <typename R> struct EpiStore {
    typename V2T<R>::T* out;
    R scale;
    __device__ __forceinline__ bool halted() const { return false; }
    template <int NR>
    __device__ __forceinline__ void finish(const Geom& g, int h, bool valid, int r0, int nrhs, Vec3<R> (&acc)[NR]) {
        if (!valid) return;
        const size_t rs = (size_t)3 * g.Vh;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (r0 + r >= nrhs) continue;
            Vec3<R> o;
#pragma unroll
            for (int c = 0; c < 3; ++c) o.c[c] = scale * acc[r].c[c];
            store_vec<R>(out + (size_t)(r0 + r) * rs, h, g.Vh, o);
        }
    }
};

// The same two epilogues for the float-float operator on fp64 fields
struct EpiStoreD2 {
    double2* out;
    DF scale;
    __device__ __forceinline__ bool halted() const { return false; }
    template <int NR>
    __device__ __forceinline__ void finish(const Geom& g, int h, bool valid, int r0, int nrhs, Vec3<DF> (&acc)[NR]) {
        if (!valid) return;
        const size_t rs = (size_t)3 * g.Vh;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (r0 + r >= nrhs) continue;
            double2* o = out + (size_t)(r0 + r) * rs;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                o[(size_t)c * g.Vh + h] = make_double2(df_join(scale * acc[r].c[c].re), df_join(scale * acc[r].c[c].im));
        }
    }
};
struct EpiAopD2 {
    double2* out;
    const double2* aux;
    DF c0;
    __device__ __forceinline__ bool halted() const { return false; }
    template <int NR>
    __device__ __forceinline__ void finish(const Geom& g, int h, bool valid, int r0, int nrhs, Vec3<DF> (&acc)[NR]) {
        if (!valid) return;
        const size_t rs = (size_t)3 * g.Vh;
        const DF half(0.5f);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (r0 + r >= nrhs) continue;
            const double2* a = aux + (size_t)(r0 + r) * rs;
            double2* o = out + (size_t)(r0 + r) * rs;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double2 ad = __ldg(a + (size_t)c * g.Vh + h);
                const DF re = c0 * df_split(ad.x) - half * acc[r].c[c].re;
                const DF im = c0 * df_split(ad.y) - half * acc[r].c[c].im;
                o[(size_t)c * g.Vh + h] = make_double2(df_join(re), df_join(im));
            }
        }
    }
};

// A-operator epilogue: out = c0 * aux - 1/2 acc (aux on the output parity).
template <typename R> struct EpiAop {
    typename V2T<R>::T* out;
    const typename V2T<R>::T* aux;
    R c0;
    __device__ __forceinline__ bool halted() const { return false; }
    template <int NR>
    __device__ __forceinline__ void finish(const Geom& g, int h, bool valid, int r0, int nrhs, Vec3<R> (&acc)[NR]) {
        if (!valid) return;
        const size_t rs = (size_t)3 * g.Vh;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (r0 + r >= nrhs) continue;
            Vec3<R> a = load_vec<R>(aux + (size_t)(r0 + r) * rs, h, g.Vh);
            Vec3<R> o;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o.c[c].re = c0 * a.c[c].re - (R)0.5 * acc[r].c[c].re;
                o.c[c].im = c0 * a.c[c].im - (R)0.5 * acc[r].c[c].im;
            }
            store_vec<R>(out + (size_t)(r0 + r) * rs, h, g.Vh, o);
        }
    }
};

// sources per thread: every link load serves NR of them.  Four is the
// measured optimum for the force's many-source Y_i = D_oe X_i as well (60
// sources on 32^3 x 8: 311 us at NR = 4, 473 us at NR = 8, whose extra
// registers halve the resident warps).
inline int dslash_nr_for(int nrhs) { return nrhs >= 2 ? 4 : 1; }

// Threads per site: enough threads to fill the GPU at small volumes (about
// 2^19 in flight), one per site once the lattice alone provides them.
inline int dslash_tps_for(long long vh) {
    long long t = (1LL << 19) / (vh > 0 ? vh : 1);
    return t >= 8 ? 8 : t >= 4 ? 4 : t >= 2 ? 2 : 1;
}

#define STAG_DSLASH_BLOCK 128
