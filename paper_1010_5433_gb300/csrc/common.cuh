// Device-side building blocks shared by the libstag kernels: complex and
// SU(3) arithmetic, even/odd geometry with staggered phases, the gauge-link
// store (Sec. 5, Fig. 2 of the paper) and the spinor layout.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "stag.h"

#define STAG_MAX_RHS 8          // independent Krylov spaces solved together
#define STAG_RED_BLOCK 256      // threads of every reducing kernel
#define STAG_MAX_RED_BLOCKS 65536

// ---------------------------------------------------------------- geometry
// Half index h of a site of parity p: h = s >> 1 with s = x + Lx(y + Ly(z + Lz t)).
// With Lxh = Lx/2:  xh = h % Lxh,  (y, z, t) from h / Lxh,  x = 2 xh + ((y+z+t+p) & 1).
struct Geom {
    int L[4];
    int Lxh;
    int Vh;
    int V;
    int apt;   // antiperiodic time boundary for the fermions
};

// Neighbour half indices and link signs of one site (Sec. 2, unimproved staggered):
// fwd[mu] = h(x+mu), bwd[mu] = h(x-mu) on the other parity; sf[mu] = eta_mu(x) with
// the boundary sign of link (x, mu); sb[mu] the same for link (x-mu, mu).
struct Nbr {
    int fwd[4], bwd[4];
    float sf[4], sb[4];
    int x[4];
};

__device__ __forceinline__ void site_neighbours(const Geom& g, int h, int par, Nbr& n) {
    int xh = h % g.Lxh;
    int yzt = h / g.Lxh;
    int y = yzt % g.L[1];
    int zt = yzt / g.L[1];
    int z = zt % g.L[2];
    int t = zt / g.L[2];
    int x = 2 * xh + ((y + z + t + par) & 1);
    n.x[0] = x; n.x[1] = y; n.x[2] = z; n.x[3] = t;
    int xp = (x + 1 == g.L[0]) ? 0 : x + 1;
    int xm = (x == 0) ? g.L[0] - 1 : x - 1;
    n.fwd[0] = (xp >> 1) + g.Lxh * yzt;
    n.bwd[0] = (xm >> 1) + g.Lxh * yzt;
    int sy = g.Lxh, sz = g.Lxh * g.L[1], st = sz * g.L[2];
    n.fwd[1] = (y + 1 == g.L[1]) ? h - (g.L[1] - 1) * sy : h + sy;
    n.bwd[1] = (y == 0) ? h + (g.L[1] - 1) * sy : h - sy;
    n.fwd[2] = (z + 1 == g.L[2]) ? h - (g.L[2] - 1) * sz : h + sz;
    n.bwd[2] = (z == 0) ? h + (g.L[2] - 1) * sz : h - sz;
    n.fwd[3] = (t + 1 == g.L[3]) ? h - (g.L[3] - 1) * st : h + st;
    n.bwd[3] = (t == 0) ? h + (g.L[3] - 1) * st : h - st;
    float e1 = (x & 1) ? -1.f : 1.f;
    float e2 = ((x + y) & 1) ? -1.f : 1.f;
    float e3 = ((x + y + z) & 1) ? -1.f : 1.f;
    n.sf[0] = n.sb[0] = 1.f;
    n.sf[1] = n.sb[1] = e1;
    n.sf[2] = n.sb[2] = e2;
    n.sf[3] = n.sb[3] = e3;
    if (g.apt) {
        if (t == g.L[3] - 1) n.sf[3] = -n.sf[3];
        if (t == 0) n.sb[3] = -n.sb[3];
    }
}

// ---------------------------------------------------------------- float-float reals
// DF = hi + lo with two floats: the representation of Sec. 5 / Fig. 2 of the
// paper, used "directly" (the option the paper names and leaves aside on
// hardware with fast doubles).  On GB300 fp32 issue is ~64x fp64 issue, so
// fp64-accurate (about 48-bit) Dslash and solver vectors run on the fp32
// pipes.  Arithmetic: Knuth's two-sum / Dekker's fast two-sum for addition,
// an FMA-based exact product for multiplication (error-free transformations).
struct DF {
    float hi, lo;
    __host__ __device__ __forceinline__ DF() {}
    __host__ __device__ __forceinline__ DF(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ __forceinline__ DF(float v) : hi(v), lo(0.f) {}
    __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ DF(double v) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    }
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    return DF(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
    float s = a + b;
    return DF(s, b - (s - a));
}
__device__ __forceinline__ DF operator+(DF a, DF b) {
    DF s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ DF __shfl_xor_sync(unsigned int mask, DF v, int lane_mask) {
    return DF(__shfl_xor_sync(mask, v.hi, lane_mask), __shfl_xor_sync(mask, v.lo, lane_mask));
}
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = a - b; }

// ---------------------------------------------------------------- complex / SU(3)
template <typename R> struct Cx { R re, im; };

template <typename R> __host__ __device__ __forceinline__ Cx<R> mk(R a, R b) { Cx<R> c; c.re = a; c.im = b; return c; }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R> __host__ __device__ __forceinline__ Cx<R> conj(Cx<R> a) { return mk(a.re, -a.im); }
// acc += a * b
template <typename R> __host__ __device__ __forceinline__ void cmac(Cx<R>& acc, Cx<R> a, Cx<R> b) {
    acc.re += a.re * b.re - a.im * b.im;
    acc.im += a.re * b.im + a.im * b.re;
}
// acc += conj(a) * b
template <typename R> __host__ __device__ __forceinline__ void cmacc(Cx<R>& acc, Cx<R> a, Cx<R> b) {
    acc.re += a.re * b.re + a.im * b.im;
    acc.im += a.re * b.im - a.im * b.re;
}

template <typename R> struct Vec3 { Cx<R> c[3]; };
template <typename R> struct Su3 { Cx<R> e[3][3]; };

template <typename R> __device__ __forceinline__ void zero(Vec3<R>& v) {
#pragma unroll
    for (int i = 0; i < 3; ++i) v.c[i] = mk<R>(0, 0);
}

// acc += s * U v
template <typename R> __device__ __forceinline__ void mac_uv(Vec3<R>& acc, R s, const Su3<R>& u, const Vec3<R>& v) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Cx<R> t = mk<R>(0, 0);
#pragma unroll
        for (int j = 0; j < 3; ++j) cmac(t, u.e[i][j], v.c[j]);
        acc.c[i].re += s * t.re;
        acc.c[i].im += s * t.im;
    }
}
// acc += s * U^dag v
template <typename R> __device__ __forceinline__ void mac_udv(Vec3<R>& acc, R s, const Su3<R>& u, const Vec3<R>& v) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Cx<R> t = mk<R>(0, 0);
#pragma unroll
        for (int j = 0; j < 3; ++j) cmacc(t, u.e[j][i], v.c[j]);
        acc.c[i].re += s * t.re;
        acc.c[i].im += s * t.im;
    }
}

// Float-float versions (the fp64 operator): each output component sums its
// six products with error-free products of the high parts (FMA) and a
// compensated running sum, the cross terms and rounding errors gathered in the
// low word, and is renormalised once per link (the compensated dot product of
// Ogita, Rump and Oishi, 2005) -- about half the fp32 operations of chained
// float-float multiplies and adds.  s is a staggered sign, exactly +1 or -1.
__device__ __forceinline__ void df_mac(DF& acc, const DF& a, const DF& b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float sum = acc.hi + p;             // two-sum of acc.hi and p
    const float bv = sum - acc.hi;
    const float err = (acc.hi - (sum - bv)) + (p - bv);
    acc.hi = sum;
    acc.lo += e + err;
}
__device__ __forceinline__ DF df_neg_if(const DF& a, bool neg) { return neg ? DF(-a.hi, -a.lo) : a; }
__device__ __forceinline__ void df_renorm(DF& v) { v = df_two_sum(v.hi, v.lo); }

template <> __device__ __forceinline__ void mac_uv<DF>(Vec3<DF>& acc, DF s, const Su3<DF>& u, const Vec3<DF>& v) {
    const bool neg = s.hi < 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        DF re = acc.c[i].re, im = acc.c[i].im;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const DF ur = df_neg_if(u.e[i][j].re, neg), ui = df_neg_if(u.e[i][j].im, neg);
            df_mac(re, ur, v.c[j].re);          // s (u v).re = s (ur vr - ui vi)
            df_mac(re, DF(-ui.hi, -ui.lo), v.c[j].im);
            df_mac(im, ur, v.c[j].im);          // s (u v).im = s (ur vi + ui vr)
            df_mac(im, ui, v.c[j].re);
        }
        df_renorm(re);
        df_renorm(im);
        acc.c[i].re = re;
        acc.c[i].im = im;
    }
}
template <> __device__ __forceinline__ void mac_udv<DF>(Vec3<DF>& acc, DF s, const Su3<DF>& u, const Vec3<DF>& v) {
    const bool neg = s.hi < 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        DF re = acc.c[i].re, im = acc.c[i].im;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const DF ur = df_neg_if(u.e[j][i].re, neg), ui = df_neg_if(u.e[j][i].im, neg);
            df_mac(re, ur, v.c[j].re);          // s (u^dag v).re = s (ur vr + ui vi)
            df_mac(re, ui, v.c[j].im);
            df_mac(im, ur, v.c[j].im);          // s (u^dag v).im = s (ur vi - ui vr)
            df_mac(im, DF(-ui.hi, -ui.lo), v.c[j].re);
        }
        df_renorm(re);
        df_renorm(im);
        acc.c[i].re = re;
        acc.c[i].im = im;
    }
}

template <typename R> __device__ __forceinline__ Su3<R> mul(const Su3<R>& a, const Su3<R>& b) {
    Su3<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Cx<R> t = mk<R>(0, 0);
#pragma unroll
            for (int k = 0; k < 3; ++k) cmac(t, a.e[i][k], b.e[k][j]);
            c.e[i][j] = t;
        }
    return c;
}
// a * b^dag
template <typename R> __device__ __forceinline__ Su3<R> mul_nd(const Su3<R>& a, const Su3<R>& b) {
    Su3<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Cx<R> t = mk<R>(0, 0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                // a_ik * conj(b_jk)
                t.re += a.e[i][k].re * b.e[j][k].re + a.e[i][k].im * b.e[j][k].im;
                t.im += a.e[i][k].im * b.e[j][k].re - a.e[i][k].re * b.e[j][k].im;
            }
            c.e[i][j] = t;
        }
    return c;
}
// a^dag * b
template <typename R> __device__ __forceinline__ Su3<R> mul_dn(const Su3<R>& a, const Su3<R>& b) {
    Su3<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Cx<R> t = mk<R>(0, 0);
#pragma unroll
            for (int k = 0; k < 3; ++k) cmacc(t, a.e[k][i], b.e[k][j]);
            c.e[i][j] = t;
        }
    return c;
}

// third row of an SU(3) matrix from the first two: conj(row0 x row1) (Sec. 5)
template <typename R> __device__ __forceinline__ void rebuild_row2(Su3<R>& u) {
    const Cx<R>* a = u.e[0];
    const Cx<R>* b = u.e[1];
    u.e[2][0] = conj(a[1] * b[2] - a[2] * b[1]);
    u.e[2][1] = conj(a[2] * b[0] - a[0] * b[2]);
    u.e[2][2] = conj(a[0] * b[1] - a[1] * b[0]);
}

// ---------------------------------------------------------------- gauge store
// Two-float store of Sec. 5 / Fig. 2: every real a is held as hi = (float)a and
// lo = (float)(a - hi).  Both arrays share one layout, structure of arrays per
// (mu, parity) block of Vh links:
//   float4 plane 0: u00 u01   plane 1: u02 u10   plane 2: u11 u12   plane 3: u20 u21
//   float2 plane 4: u22
// i.e. 18 floats x Vh per block, block (mu, par) at offset (2 mu + par) * 18 Vh.
// The 12-real format reads planes 0-2 (rows 0 and 1) and rebuilds row 2.
// bf16 copy: per block a uint4 plane (u00 u01 u02 u10) and a uint2 plane (u11 u12),
// 12 bf16 x Vh per block.
__host__ __device__ __forceinline__ size_t link_block_f(int mu, int par, int Vh) { return (size_t)(2 * mu + par) * 18 * Vh; }
__host__ __device__ __forceinline__ size_t link_block_b(int mu, int par, int Vh) { return (size_t)(2 * mu + par) * 12 * Vh; }

__device__ __forceinline__ float4 ldg_stream(const float4* p) { return __ldg(p); }

template <int ROWS>
__device__ __forceinline__ Su3<float> load_link_f(const float* __restrict__ blk, int h, int Vh) {
    const float4* p4 = reinterpret_cast<const float4*>(blk);
    Su3<float> u;
    float4 a = ldg_stream(p4 + h);
    float4 b = ldg_stream(p4 + Vh + h);
    float4 c = ldg_stream(p4 + 2 * Vh + h);
    u.e[0][0] = mk(a.x, a.y); u.e[0][1] = mk(a.z, a.w);
    u.e[0][2] = mk(b.x, b.y); u.e[1][0] = mk(b.z, b.w);
    u.e[1][1] = mk(c.x, c.y); u.e[1][2] = mk(c.z, c.w);
    if (ROWS == 3) {
        float4 d = ldg_stream(p4 + 3 * Vh + h);
        float2 e = __ldg(reinterpret_cast<const float2*>(blk + 16 * (size_t)Vh) + h);
        u.e[2][0] = mk(d.x, d.y); u.e[2][1] = mk(d.z, d.w);
        u.e[2][2] = mk(e.x, e.y);
    } else {
        rebuild_row2(u);
    }
    return u;
}

// Two-float split of a double x (Sec. 5): hi = x rounded to float, lo = the
// remainder rounded to float, then (hi, lo) made canonical, hi = RN(hi + lo).
// A remainder that rounds up to exactly half an ulp of hi makes hi + lo a
// tie that a later split of the same double resolves to the even neighbour;
// the canonical pair is the one that split gives, so a store (hi + lo as a
// double) followed by a load reproduces (hi, lo) bit for bit.
__device__ __forceinline__ void hl_canonical(float& hi, float& lo) {
    const float s = __fadd_rn(hi, lo);
    lo = __fsub_rn(lo, __fsub_rn(s, hi));
    hi = s;
}

__device__ __forceinline__ Su3<double> load_link_d(const float* __restrict__ hi, const float* __restrict__ lo,
                                                   size_t blk, int h, int Vh) {
    const float4* ph = reinterpret_cast<const float4*>(hi + blk);
    const float4* pl = reinterpret_cast<const float4*>(lo + blk);
    Su3<double> u;
    float vh[18], vl[18];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 a = __ldg(ph + (size_t)k * Vh + h);
        float4 b = __ldg(pl + (size_t)k * Vh + h);
        vh[4 * k] = a.x; vh[4 * k + 1] = a.y; vh[4 * k + 2] = a.z; vh[4 * k + 3] = a.w;
        vl[4 * k] = b.x; vl[4 * k + 1] = b.y; vl[4 * k + 2] = b.z; vl[4 * k + 3] = b.w;
    }
    float2 e = __ldg(reinterpret_cast<const float2*>(hi + blk + 16 * (size_t)Vh) + h);
    float2 f = __ldg(reinterpret_cast<const float2*>(lo + blk + 16 * (size_t)Vh) + h);
    vh[16] = e.x; vh[17] = e.y; vl[16] = f.x; vl[17] = f.y;
#pragma unroll
    for (int k = 0; k < 9; ++k)
        u.e[k / 3][k % 3] = mk((double)vh[2 * k] + (double)vl[2 * k], (double)vh[2 * k + 1] + (double)vl[2 * k + 1]);
    return u;
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// rows 0-1 of a bf16 link from its two words (uint4: u00 u01 u02 u10, uint2: u11 u12), row 2 rebuilt
__device__ __forceinline__ Su3<float> unpack_link_bf(const uint4 a, const uint2 b) {
    Su3<float> u;
    u.e[0][0] = mk(bf_lo(a.x), bf_hi(a.x)); u.e[0][1] = mk(bf_lo(a.y), bf_hi(a.y));
    u.e[0][2] = mk(bf_lo(a.z), bf_hi(a.z)); u.e[1][0] = mk(bf_lo(a.w), bf_hi(a.w));
    u.e[1][1] = mk(bf_lo(b.x), bf_hi(b.x)); u.e[1][2] = mk(bf_lo(b.y), bf_hi(b.y));
    rebuild_row2(u);
    return u;
}
__device__ __forceinline__ Su3<float> load_link_bf(const uint16_t* __restrict__ blk, int h, int Vh) {
    const uint4* p4 = reinterpret_cast<const uint4*>(blk);
    const uint2* p2 = reinterpret_cast<const uint2*>(blk + 8 * (size_t)Vh);
    return unpack_link_bf(__ldg(p4 + h), __ldg(p2 + h));
}

// ---------------------------------------------------------------- spinors
// Half-lattice field: [rhs][colour][Vh] complex, complex = float2 / double2.
template <typename R> struct V2T;
template <> struct V2T<float> { typedef float2 T; };
template <> struct V2T<double> { typedef double2 T; };
template <> struct V2T<DF> { typedef float4 T; };   // (re.hi, re.lo, im.hi, im.lo)

__device__ __forceinline__ Cx<DF> cx_of(float4 a) { return mk(DF(a.x, a.y), DF(a.z, a.w)); }
__device__ __forceinline__ float4 f4_of(Cx<DF> v) { return make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }

template <typename R>
__device__ __forceinline__ Vec3<R> load_vec(const typename V2T<R>::T* __restrict__ f, int h, int Vh) {
    Vec3<R> v;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        typename V2T<R>::T a = __ldg(f + (size_t)c * Vh + h);
        v.c[c] = mk(a.x, a.y);
    }
    return v;
}
template <typename R>
__device__ __forceinline__ Vec3<R> load_vec_cg(const typename V2T<R>::T* f, int h, int Vh) {
    Vec3<R> v;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        typename V2T<R>::T a = __ldcg(f + (size_t)c * Vh + h);
        v.c[c] = mk(a.x, a.y);
    }
    return v;
}
template <typename R>
__device__ __forceinline__ void store_vec(typename V2T<R>::T* f, int h, int Vh, const Vec3<R>& v) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        typename V2T<R>::T a;
        a.x = v.c[c].re;
        a.y = v.c[c].im;
        f[(size_t)c * Vh + h] = a;
    }
}

template <typename R> __device__ __forceinline__ double re_dot(const Vec3<R>& a, const Vec3<R>& b) {
    R s = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) s += a.c[c].re * b.c[c].re + a.c[c].im * b.c[c].im;
    return (double)s;
}

// float-float spinors: load / store the float4 planes
template <>
__device__ __forceinline__ Vec3<DF> load_vec<DF>(const float4* __restrict__ f, int h, int Vh) {
    Vec3<DF> v;
#pragma unroll
    for (int c = 0; c < 3; ++c) v.c[c] = cx_of(__ldg(f + (size_t)c * Vh + h));
    return v;
}
template <>
__device__ __forceinline__ Vec3<DF> load_vec_cg<DF>(const float4* f, int h, int Vh) {
    Vec3<DF> v;
#pragma unroll
    for (int c = 0; c < 3; ++c) v.c[c] = cx_of(__ldcg(f + (size_t)c * Vh + h));
    return v;
}
template <>
__device__ __forceinline__ void store_vec<DF>(float4* f, int h, int Vh, const Vec3<DF>& v) {
#pragma unroll
    for (int c = 0; c < 3; ++c) f[(size_t)c * Vh + h] = f4_of(v.c[c]);
}

// the two-float gauge store read as float-float links (no conversion at all)
__device__ __forceinline__ Su3<DF> load_link_df(const float* __restrict__ hi, const float* __restrict__ lo,
                                                size_t blk, int h, int Vh) {
    const float4* ph = reinterpret_cast<const float4*>(hi + blk);
    const float4* pl = reinterpret_cast<const float4*>(lo + blk);
    float vh[18], vl[18];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 a = __ldg(ph + (size_t)k * Vh + h);
        float4 b = __ldg(pl + (size_t)k * Vh + h);
        vh[4 * k] = a.x; vh[4 * k + 1] = a.y; vh[4 * k + 2] = a.z; vh[4 * k + 3] = a.w;
        vl[4 * k] = b.x; vl[4 * k + 1] = b.y; vl[4 * k + 2] = b.z; vl[4 * k + 3] = b.w;
    }
    float2 e = __ldg(reinterpret_cast<const float2*>(hi + blk + 16 * (size_t)Vh) + h);
    float2 f = __ldg(reinterpret_cast<const float2*>(lo + blk + 16 * (size_t)Vh) + h);
    vh[16] = e.x; vh[17] = e.y; vl[16] = f.x; vl[17] = f.y;
    Su3<DF> u;
#pragma unroll
    for (int k = 0; k < 9; ++k) u.e[k / 3][k % 3] = mk(DF(vh[2 * k], vl[2 * k]), DF(vh[2 * k + 1], vl[2 * k + 1]));
    return u;
}
template <typename R> __device__ __forceinline__ double norm2(const Vec3<R>& a) { return re_dot(a, a); }

// ---------------------------------------------------------------- reductions
// Block-wide sum of N doubles; result valid in thread 0.  Fixed tree order, so
// the same launch shape gives bit-identical sums.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N]) {
    __shared__ double sm[N][32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) sm[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double s = (lane < nw) ? sm[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[k] = s;
        }
    }
}

// Sum n partials in a fixed order by the whole block; result in thread 0.
// Lane `lane`'s share of a warp's sum of p[0..n): p[lane] + p[lane + 32] +
// ..., added in that order, with the loads of up to 8 terms issued before
// the first add (one L2 round trip instead of one per term).
__device__ __forceinline__ double lane_strided_sum(const double* p, int n, int lane) {
    double v = 0.0;
    for (int i0 = lane; i0 < n; i0 += 32 * 8) {
        double t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) t[k] = (i0 + 32 * k < n) ? __ldcg(p + i0 + 32 * k) : 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (i0 + 32 * k < n) v += t[k];
    }
    return v;
}

__device__ __forceinline__ double block_sum_array(const double* p, int n) {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[0] += __ldcg(p + i);
    block_sum<1>(v);
    return v[0];
}

// Last-block election: each block calls this after writing its partials
// (thread 0 only, after __threadfence).  Returns true in the last block.
__device__ __forceinline__ bool elect_last_block(unsigned int* counter, unsigned int total) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int prev = atomicAdd(counter, 1u);
        last = (prev == total - 1);
        if (last) *counter = 0u;   // reset for the next launch
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}
