// Improved (asqtad) staggered fermions: the fat and Naik links built from the
// thin links, and the fermion force through them (Lepage, PRD 59 (1999)
// 074502; Orginos, Toussaint, Sugar, PRD 60 (1999) 054503).  The paper runs
// unimproved staggered fermions (Sec. 2); this is the improved operator on the
// same even/odd multi-shift machinery (asqtad.cuh holds its Dslash).
//
// Fat link of direction mu at x, as nested staples
//   S_s[A](y) = L(y, s) A(y + s) L(y + mu, s)^dag,   L(y, +nu) = U_nu(y),
//                                                    L(y, -nu) = U_nu(y - nu)^dag,
//   V = c1 U_mu + sum_nu S_nu[ c3 U_mu + sum_rho S_rho[ c5 U_mu + c7 sum_sig S_sig[U_mu] ] ]
//       + cL sum_nu S_nu[S_nu[U_mu]]
// with nu, rho, sig signed, mutually orthogonal and orthogonal to mu:
// 1 + 6 + 24 + 48 + 6 paths.  Coefficients (tadpole factor u0): 5/8, 1/16 u0^-2,
// 1/64 u0^-4, 1/384 u0^-6, -1/16 u0^-4; Naik W = -1/24 u0^-2 U_mu(x) U_mu(x+mu) U_mu(x+2mu).
// V and W carry neither eta nor the time boundary sign: every path of V_t
// from the last time slice crosses the boundary an odd number of times and
// every other path of V an even number, so the Dslash applies the thin
// links' hop sign to V and the sign of the three t-links to W.
//
// Arithmetic of the rebuild: float-float (hi + lo floats, ~48 bits) on the
// fp32 pipes (GB300's fp64 rate is ~1/64 of fp32), read from the two-float
// thin-link store and written to two-float stores of the same layout, so the
// fp32 Dslash reads the rounded fat links (hi) and the fp64 one all of them;
// before an fp32 MD force the rebuild runs in fp32 from the hi words.
//
// Force: dS = sum Re tr[dV Xv + dW Xw] with the outer-product fields Xv, Xw
// of the solutions (k_asq_outer), differentiated through the nested staples
// by a reverse pass (k_asq_fwd_*, k_asq_bwd_*); k_asq_force, one gather per
// thin link over the path incidences of its direction, is the same sum in
// another order, kept as a cross-check (STAG_ASQ_FORCE=gather).
#include <cstring>
#include <vector>

#include "asqtad.cuh"
#include "internal.h"

namespace {
constexpr int AB = 128;

__device__ __forceinline__ int a_hidx(const Geom& g, const int c[4]) {
    return (c[0] >> 1) + g.Lxh * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}
__device__ __forceinline__ void a_coords(const Geom& g, int par, int h, int c[4]) {
    int xh = h % g.Lxh, r = h / g.Lxh;
    c[1] = r % g.L[1]; r /= g.L[1];
    c[2] = r % g.L[2]; c[3] = r / g.L[2];
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + par) & 1);
}
// move c by one step along signed direction s (+-(nu+1))
__device__ __forceinline__ void a_move(const Geom& g, int c[4], int s) {
    const int nu = (s > 0 ? s : -s) - 1;
    c[nu] += s > 0 ? 1 : -1;
    if (c[nu] < 0) c[nu] += g.L[nu];
    if (c[nu] >= g.L[nu]) c[nu] -= g.L[nu];
}

template <typename R> __device__ __forceinline__ Su3<R> dagger(const Su3<R>& a) {
    Su3<R> b;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) b.e[i][j] = conj(a.e[j][i]);
    return b;
}
template <typename R> __device__ __forceinline__ void axpy(Su3<R>& acc, R c, const Su3<R>& a) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            acc.e[i][j].re += c * a.e[i][j].re;
            acc.e[i][j].im += c * a.e[i][j].im;
        }
}
template <typename R> __device__ __forceinline__ Su3<R> scaled(R c, const Su3<R>& a) {
    Su3<R> b;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) b.e[i][j] = mk(c * a.e[i][j].re, c * a.e[i][j].im);
    return b;
}

// 3x3 products a b and a b^dag.  In float-float each entry's six real
// products are summed with error-free products and a compensated running sum
// (df_mac, Ogita-Rump-Oishi) and renormalised once, about half the work of
// chained float-float multiplies and adds.
__device__ __forceinline__ Su3<float> mm(const Su3<float>& a, const Su3<float>& b) { return mul(a, b); }
__device__ __forceinline__ Su3<float> mm_nd(const Su3<float>& a, const Su3<float>& b) { return mul_nd(a, b); }
__device__ __forceinline__ Su3<DF> mm(const Su3<DF>& a, const Su3<DF>& b) {
    Su3<DF> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            DF re(0.f), im(0.f);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                df_mac(re, a.e[i][k].re, b.e[k][j].re);
                df_mac(re, -a.e[i][k].im, b.e[k][j].im);
                df_mac(im, a.e[i][k].re, b.e[k][j].im);
                df_mac(im, a.e[i][k].im, b.e[k][j].re);
            }
            df_renorm(re);
            df_renorm(im);
            c.e[i][j] = mk(re, im);
        }
    return c;
}
__device__ __forceinline__ Su3<DF> mm_nd(const Su3<DF>& a, const Su3<DF>& b) {
    Su3<DF> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            DF re(0.f), im(0.f);
#pragma unroll
            for (int k = 0; k < 3; ++k) {   // a_ik conj(b_jk)
                df_mac(re, a.e[i][k].re, b.e[j][k].re);
                df_mac(re, a.e[i][k].im, b.e[j][k].im);
                df_mac(im, a.e[i][k].im, b.e[j][k].re);
                df_mac(im, -a.e[i][k].re, b.e[j][k].im);
            }
            df_renorm(re);
            df_renorm(im);
            c.e[i][j] = mk(re, im);
        }
    return c;
}

// thin link U_nu(c)
template <typename R, int FMT>
__device__ __forceinline__ Su3<R> thin(const Geom& g, const LinkPtrs& L, const int c[4], int nu) {
    return LinkFetch<R, FMT>::get(L, nu, (c[0] + c[1] + c[2] + c[3]) & 1, a_hidx(g, c), g.Vh);
}
// the link met on a step from c along s, c moved to the step's end
template <typename R, int FMT>
__device__ __forceinline__ Su3<R> walk(const Geom& g, const LinkPtrs& L, int c[4], int s) {
    if (s > 0) {
        const Su3<R> u = thin<R, FMT>(g, L, c, s - 1);
        a_move(g, c, s);
        return u;
    }
    a_move(g, c, s);
    return dagger(thin<R, FMT>(g, L, c, -s - 1));
}
// S_s[A](y) = L(y, s) A L(y + mu, s)^dag, A the value at y + s
template <typename R, int FMT>
__device__ __forceinline__ Su3<R> staple(const Geom& g, const LinkPtrs& L, const int y[4], int mu, int s,
                                         const Su3<R>& a) {
    int c[4] = {y[0], y[1], y[2], y[3]};
    const Su3<R> first = walk<R, FMT>(g, L, c, s);
    int d[4] = {y[0], y[1], y[2], y[3]};
    a_move(g, d, mu + 1);
    const Su3<R> last = walk<R, FMT>(g, L, d, s);   // L(y + mu, s)
    return mm_nd(mm(first, a), last);
}

struct AsqCoef {
    float c[6][2];   // one, staple3, staple5, staple7, lepage, naik as float-float (hi, lo)
};
__device__ __forceinline__ DF cf(const AsqCoef& k, int i) { return DF(k.c[i][0], k.c[i][1]); }

// float-float -> two-float store (hi, lo canonical, as the thin links)
__device__ __forceinline__ void store_df(float* hi, float* lo, size_t blk, int h, int Vh, const Su3<DF>& u) {
    float vh[18], vl[18];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        DF re = u.e[k / 3][k % 3].re, im = u.e[k / 3][k % 3].im;
        hl_canonical(re.hi, re.lo);
        hl_canonical(im.hi, im.lo);
        vh[2 * k] = re.hi; vl[2 * k] = re.lo;
        vh[2 * k + 1] = im.hi; vl[2 * k + 1] = im.lo;
    }
    float4* h4 = reinterpret_cast<float4*>(hi + blk);
    float4* l4 = reinterpret_cast<float4*>(lo + blk);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h4[(size_t)k * Vh + h] = make_float4(vh[4 * k], vh[4 * k + 1], vh[4 * k + 2], vh[4 * k + 3]);
        l4[(size_t)k * Vh + h] = make_float4(vl[4 * k], vl[4 * k + 1], vl[4 * k + 2], vl[4 * k + 3]);
    }
    reinterpret_cast<float2*>(hi + blk + 16 * (size_t)Vh)[h] = make_float2(vh[16], vh[17]);
    reinterpret_cast<float2*>(lo + blk + 16 * (size_t)Vh)[h] = make_float2(vl[16], vl[17]);
}

template <typename R> __device__ __forceinline__ R coef_as(const AsqCoef& k, int i);
template <> __device__ __forceinline__ float coef_as<float>(const AsqCoef& k, int i) { return k.c[i][0] + k.c[i][1]; }
template <> __device__ __forceinline__ DF coef_as<DF>(const AsqCoef& k, int i) { return cf(k, i); }

__device__ __forceinline__ Su3<DF> as_df(const Su3<DF>& u) { return u; }
__device__ __forceinline__ Su3<DF> as_df(const Su3<float>& u) {
    Su3<DF> d;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) d.e[i][j] = mk(DF(u.e[i][j].re), DF(u.e[i][j].im));
    return d;
}

// one thread per fat link (mu, x): V and W in float-float (R = DF, from the
// two-float thin links) or in fp32 (R = float, from their hi words; stored
// with zero lo words)
template <typename R, int FMT>
__global__ void __launch_bounds__(AB) k_fatten(Geom g, LinkPtrs L, AsqCoef k, float* fhi, float* flo, float* lhi,
                                               float* llo) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int blk = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    int x[4];
    a_coords(g, par, h, x);
    Su3<R> v = scaled(coef_as<R>(k, 0), thin<R, FMT>(g, L, x, mu));
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        for (int sn = -1; sn <= 1; sn += 2) {
            const int a = sn * (nu + 1);
            int y1[4] = {x[0], x[1], x[2], x[3]};
            a_move(g, y1, a);
            Su3<R> q = scaled(coef_as<R>(k, 1), thin<R, FMT>(g, L, y1, mu));
            for (int rho = 0; rho < 4; ++rho) {
                if (rho == mu || rho == nu) continue;
                for (int sr = -1; sr <= 1; sr += 2) {
                    const int b = sr * (rho + 1);
                    int y2[4] = {y1[0], y1[1], y1[2], y1[3]};
                    a_move(g, y2, b);
                    Su3<R> t = scaled(coef_as<R>(k, 2), thin<R, FMT>(g, L, y2, mu));
                    const int sig = 6 - mu - nu - rho;     // the remaining direction
                    for (int ss = -1; ss <= 1; ss += 2) {
                        const int c = ss * (sig + 1);
                        int y3[4] = {y2[0], y2[1], y2[2], y2[3]};
                        a_move(g, y3, c);
                        axpy(t, coef_as<R>(k, 3), staple<R, FMT>(g, L, y2, mu, c, thin<R, FMT>(g, L, y3, mu)));
                    }
                    axpy(q, R(1.f), staple<R, FMT>(g, L, y1, mu, b, t));
                }
            }
            axpy(v, R(1.f), staple<R, FMT>(g, L, x, mu, a, q));
            // Lepage: the double-width staple in the same direction
            int y2[4] = {y1[0], y1[1], y1[2], y1[3]};
            a_move(g, y2, a);
            const Su3<R> inner = staple<R, FMT>(g, L, y1, mu, a, thin<R, FMT>(g, L, y2, mu));
            axpy(v, coef_as<R>(k, 4), staple<R, FMT>(g, L, x, mu, a, inner));
        }
    }
    store_df(fhi, flo, link_block_f(mu, par, g.Vh), h, g.Vh, as_df(v));
    int c[4] = {x[0], x[1], x[2], x[3]};
    Su3<R> w = walk<R, FMT>(g, L, c, mu + 1);
    w = mm(w, walk<R, FMT>(g, L, c, mu + 1));
    w = mm(w, walk<R, FMT>(g, L, c, mu + 1));
    store_df(lhi, llo, link_block_f(mu, par, g.Vh), h, g.Vh, as_df(scaled(coef_as<R>(k, 5), w)));
}

// ---------------------------------------------------------------- force
// Path incidences of every thin-link direction: each (mu, path of V_mu or
// W_mu, position k on it) whose k-th step runs along +-nu, listed under nu.
struct AsqInc {
    signed char s[7];
    unsigned char len, k, mu, cls, pad;
};
constexpr int ASQ_MAX_INC = 512;
__constant__ AsqInc c_inc[4][ASQ_MAX_INC];
__constant__ int c_ninc[4];

template <typename R> __device__ __forceinline__ R from_f64(double d);
template <> __device__ __forceinline__ float from_f64<float>(double d) { return (float)d; }
template <> __device__ __forceinline__ DF from_f64<DF>(double d) { return df_split(d); }
template <typename R> struct FieldT { typedef typename V2T<R>::T T; };
template <> struct FieldT<DF> { typedef double2 T; };

template <typename R> __device__ __forceinline__ Vec3<R> load_z(const typename FieldT<R>::T* f, int h, int Vh);
template <> __device__ __forceinline__ Vec3<float> load_z<float>(const float2* f, int h, int Vh) {
    return load_vec<float>(f, h, Vh);
}
template <> __device__ __forceinline__ Vec3<DF> load_z<DF>(const double2* f, int h, int Vh) {
    Vec3<DF> v;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 d = __ldg(f + (size_t)c * Vh + h);
        v.c[c] = mk(df_split(d.x), df_split(d.y));
    }
    return v;
}

// Xv_mu(x) += sum alpha_s eps(x) (hop sign) Z(x+mu) Z(x)^dag, Xw_mu(x) the
// same with Z(x+3mu): Z = X on even sites, Y = D_oe X on odd ones.  The
// fields are [mu][par][18][Vh] reals of R (Xw after Xv).
template <typename R>
__global__ void __launch_bounds__(AB) k_asq_outer(Geom g, int nsrc, int nshift, const double* __restrict__ alpha,
                                                  double coef, const typename FieldT<R>::T* xs,
                                                  const typename FieldT<R>::T* ys, R* xv, R* xw) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int blk = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    Nbr n;
    site_neighbours(g, h, par, n);
    Nbr3 m3;
    site_neighbours3(g, n, m3);
    const typename FieldT<R>::T* here = par == 0 ? xs : ys;
    const typename FieldT<R>::T* there = par == 0 ? ys : xs;
    const double eps = par == 0 ? 1.0 : -1.0;
    Su3<R> mv, mw;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) { mv.e[i][j] = mk<R>(R(0), R(0)); mw.e[i][j] = mk<R>(R(0), R(0)); }
    const size_t rs = (size_t)3 * g.Vh;
    for (int q = 0; q < nsrc; ++q) {
        for (int s = 0; s < nshift; ++s) {
            const size_t off = ((size_t)q * nshift + s) * rs;
            const Vec3<R> zx = load_z<R>(here + off, h, g.Vh);
            const Vec3<R> z1 = load_z<R>(there + off, n.fwd[mu], g.Vh);
            const Vec3<R> z3 = load_z<R>(there + off, m3.fwd[mu], g.Vh);
            const R a1 = from_f64<R>(coef * alpha[s] * eps * (double)n.sf[mu]);
            const R a3 = from_f64<R>(coef * alpha[s] * eps * (double)m3.sf[mu]);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const Cx<R> p1 = mk(a1 * z1.c[i].re, a1 * z1.c[i].im);
                const Cx<R> p3 = mk(a3 * z3.c[i].re, a3 * z3.c[i].im);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    cmac(mv.e[i][j], p1, conj(zx.c[j]));
                    cmac(mw.e[i][j], p3, conj(zx.c[j]));
                }
            }
        }
    }
    R* ov = xv + (size_t)blk * 18 * g.Vh + h;
    R* ow = xw + (size_t)blk * 18 * g.Vh + h;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        ov[(size_t)(2 * k) * g.Vh] += mv.e[k / 3][k % 3].re;
        ov[(size_t)(2 * k + 1) * g.Vh] += mv.e[k / 3][k % 3].im;
        ow[(size_t)(2 * k) * g.Vh] += mw.e[k / 3][k % 3].re;
        ow[(size_t)(2 * k + 1) * g.Vh] += mw.e[k / 3][k % 3].im;
    }
}

template <typename R>
__device__ __forceinline__ Su3<R> load_x(const R* f, int mu, const Geom& g, const int c[4]) {
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const R* p = f + (size_t)(2 * mu + par) * 18 * g.Vh + a_hidx(g, c);
    Su3<R> m;
#pragma unroll
    for (int k = 0; k < 9; ++k) m.e[k / 3][k % 3] = mk(p[(size_t)(2 * k) * g.Vh], p[(size_t)(2 * k + 1) * g.Vh]);
    return m;
}

// F_a = Re tr[i T_a (U Gf - Gb U^dag)] of thin link (blk = 2 nu + par, h),
// written (mode 0) or added (mode 1) in the momentum layout
template <typename R>
__device__ __forceinline__ void put_asq_force(const Geom& g, const Su3<R>& u, const Su3<R>& gf, const Su3<R>& gb,
                                              double* out, int blk, int h, int mode) {
    Su3<R> w = mm(u, gf);
    const Su3<R> b = mm_nd(gb, u);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            w.e[i][j].re -= b.e[i][j].re;
            w.e[i][j].im -= b.e[i][j].im;
        }
    // Re tr(i T_a W), T_a = lambda_a / 2
    const R hf = R(0.5f);
    R f[8];
    f[0] = -hf * (w.e[1][0].im + w.e[0][1].im);
    f[1] = -hf * (w.e[0][1].re - w.e[1][0].re);
    f[2] = -hf * (w.e[0][0].im - w.e[1][1].im);
    f[3] = -hf * (w.e[2][0].im + w.e[0][2].im);
    f[4] = -hf * (w.e[0][2].re - w.e[2][0].re);
    f[5] = -hf * (w.e[2][1].im + w.e[1][2].im);
    f[6] = -hf * (w.e[1][2].re - w.e[2][1].re);
    f[7] = -(w.e[0][0].im + w.e[1][1].im - R(2.f) * w.e[2][2].im) * R(0.28867513459481287);   // 1/(2 sqrt 3)
    double* o = out + ((size_t)blk * 8) * g.Vh + h;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const double fa = (double)f[a];
        if (mode) o[(size_t)a * g.Vh] += fa;
        else o[(size_t)a * g.Vh] = fa;
    }
}

// One thread per thin link (nu, y): over every incidence of nu, the rest of
// the path's loop R = A_{k+1} .. A_n X_mu(x) A_1 .. A_{k-1} (x the path's
// start), summed with the path coefficient into Gf (link met forward) or Gb
// (met backward); then F_a = Re tr[i T_a (U Gf - Gb U^dag)], which is
// d S / d omega_a under U -> exp(i omega_a T_a) U.
template <typename R, int FMT>
__global__ void __launch_bounds__(AB) k_asq_force(Geom g, LinkPtrs L, AsqCoef k, const R* __restrict__ xv,
                                                  const R* __restrict__ xw, double* out, int mode) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int blk = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
    const int nu = blk >> 1, par = blk & 1;
    int y[4];
    a_coords(g, par, h, y);
    Su3<R> gf, gb;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) { gf.e[i][j] = mk<R>(R(0), R(0)); gb.e[i][j] = mk<R>(R(0), R(0)); }
    const int ninc = c_ninc[nu];
    for (int e = 0; e < ninc; ++e) {
        const AsqInc& in = c_inc[nu][e];
        const int len = in.len, kk = in.k, mu = in.mu;
        const bool fwd = in.s[kk] > 0;
        // start of the path: undo the steps before k from the link's near end
        int x[4] = {y[0], y[1], y[2], y[3]};
        if (!fwd) a_move(g, x, -in.s[kk]);
        for (int j = kk - 1; j >= 0; --j) a_move(g, x, -in.s[j]);
        // the far end of link k, where the rest of the path goes on
        int c[4] = {y[0], y[1], y[2], y[3]};
        if (fwd) a_move(g, c, in.s[kk]);
        Su3<R> m;
        bool have = false;
        for (int j = kk + 1; j < len; ++j) {
            const Su3<R> a = walk<R, FMT>(g, L, c, in.s[j]);
            m = have ? mm(m, a) : a;
            have = true;
        }
        const Su3<R> xm = load_x<R>(in.cls == 5 ? xw : xv, mu, g, x);
        m = have ? mm(m, xm) : xm;
        for (int j = 0; j < kk; ++j) m = mm(m, walk<R, FMT>(g, L, x, in.s[j]));
        axpy(fwd ? gf : gb, coef_as<R>(k, in.cls), m);
    }
    put_asq_force(g, thin<R, FMT>(g, L, y, nu), gf, gb, out, blk, h, mode);
}


// ---------------------------------------------------------------- force by reverse mode
// The force as the reverse pass of the nested staples of the fat link
// (the rebuild's structure), with every intermediate kept as a field:
//   T_{mu sig}(y) = c5 U_mu(y) + c7 sum_{s = +-sig} S_s[U_mu](y)            (sig unsigned, 12 fields)
//   Q_{mu nu}(y)  = c3 U_mu(y) + sum_rho S_rho[T_{mu, sig(nu, rho)}](y)      (nu signed, 24)
//   P_{mu nu}(y)  = S_nu[U_mu](y)                                           (the Lepage path's inner staple, 24)
//   V_mu(x) = c1 U_mu(x) + sum_nu S_nu[Q_{mu nu} + cL P_{mu nu}](x)
// with sig(nu, rho) the direction orthogonal to mu, nu and rho.  Cotangents
// (Re tr[C dA] for each intermediate A), from Xv = dS/dV:
//   CQ_{mu nu}(y) = L(x + mu, nu)^dag Xv_mu(x) L(x, nu),  x = y - nu    (that of P is cL CQ)
//   CT_{mu sig}(z) = sum over nu, rho with sig(nu, rho) = sig of L(y + mu, rho)^dag CQ_{mu nu}(y) L(y, rho), y = z - rho
// and the thin link U_al(z) collects: the direct terms of the 1-link,
// c3 U and c5 U pieces (al = mu), the inner U_mu of the seven-link and inner
// Lepage staples, the Naik products, and as a leg of every staple S_s with
// |s| = al: for a staple L1 A L2^dag with cotangent C, Re tr[(A L2^dag C) dL1]
// and Re tr[(C L1 A) d(L2^dag)], turned into Gf (link met forward) or Gb
// (met backward).  About 460 3x3 products per link against ~3000 for the
// per-link gather over the path incidences.
// Matrix fields: slot f, [f][par][18][Vh] reals of R.  Q and P enter the
// pass only as Q + cL P, which is stored instead of the two: 72 slots,
// T and CT at slot3(mu, sig), Q + cL P and CQ at slot6(mu, nu).
template <typename R>
__device__ __forceinline__ Su3<R> ld_f(const R* base, int slot, const Geom& g, const int c[4]) {
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const R* p = base + ((size_t)(2 * slot + par) * 18) * g.Vh + a_hidx(g, c);
    Su3<R> m;
#pragma unroll
    for (int k = 0; k < 9; ++k) m.e[k / 3][k % 3] = mk(p[(size_t)(2 * k) * g.Vh], p[(size_t)(2 * k + 1) * g.Vh]);
    return m;
}
template <typename R>
__device__ __forceinline__ void st_f(R* base, int slot, int par, int h, int Vh, const Su3<R>& m) {
    R* p = base + ((size_t)(2 * slot + par) * 18) * Vh + h;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        p[(size_t)(2 * k) * Vh] = m.e[k / 3][k % 3].re;
        p[(size_t)(2 * k + 1) * Vh] = m.e[k / 3][k % 3].im;
    }
}
// a link-layout field of R at (direction mu, parity, half index)
template <typename R>
__device__ __forceinline__ Su3<R> ld_half(const R* f, int mu, int par, int h, int Vh) {
    const R* p = f + (size_t)(2 * mu + par) * 18 * Vh + h;
    Su3<R> m;
#pragma unroll
    for (int e = 0; e < 9; ++e) m.e[e / 3][e % 3] = mk(p[(size_t)(2 * e) * Vh], p[(size_t)(2 * e + 1) * Vh]);
    return m;
}
// a staple leg's matrix cotangent: A L2^dag C for the first leg, C L1 A for
// the second (other = the staple's other leg)
template <typename R>
__device__ __forceinline__ Su3<R> leg_term(int leg, const Su3<R>& A, const Su3<R>& C, const Su3<R>& other) {
    return leg == 1 ? mm(mm_nd(A, other), C) : mm(mm(C, other), A);
}
// direction sig != mu (unsigned) and signed nu orthogonal to mu, numbered densely per mu
__device__ __forceinline__ int slot3(int mu, int sig) { return mu * 3 + sig - (sig > mu); }
__device__ __forceinline__ int slot6(int mu, int s) {
    const int d = (s > 0 ? s : -s) - 1;
    return mu * 6 + 2 * (d - (d > mu)) + (s < 0);
}
// L(y, s) without moving y
template <typename R, int FMT>
__device__ __forceinline__ Su3<R> lnk(const Geom& g, const LinkPtrs& L, const int y[4], int s) {
    int c[4] = {y[0], y[1], y[2], y[3]};
    return walk<R, FMT>(g, L, c, s);
}
template <typename R> __device__ __forceinline__ Su3<R> zero_m() {
    Su3<R> m;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) m.e[i][j] = mk<R>(R(0), R(0));
    return m;
}
template <typename R> __device__ __forceinline__ Su3<R> add_m(const Su3<R>& a, R c, const Su3<R>& b) {
    Su3<R> m = a;
    axpy(m, c, b);
    return m;
}

struct FwdArgs {
    Geom g;
    LinkPtrs L;
    AsqCoef k;
};

// T and then Q, P: one thread per (mu, site)
template <typename R, int FMT>
__global__ void __launch_bounds__(AB) k_asq_fwd_t(FwdArgs a, R* T) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * a.g.Vh) return;
    const Geom& g = a.g;
    const int blk = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    int x[4];
    a_coords(g, par, h, x);
    const Su3<R> umu = thin<R, FMT>(g, a.L, x, mu);
    for (int sig = 0; sig < 4; ++sig) {
        if (sig == mu) continue;
        Su3<R> t = scaled(coef_as<R>(a.k, 2), umu);
        for (int sg = -1; sg <= 1; sg += 2) {
            const int s = sg * (sig + 1);
            int y[4] = {x[0], x[1], x[2], x[3]};
            a_move(g, y, s);
            axpy(t, coef_as<R>(a.k, 3), staple<R, FMT>(g, a.L, x, mu, s, thin<R, FMT>(g, a.L, y, mu)));
        }
        st_f(T, slot3(mu, sig), par, h, g.Vh, t);
    }
}
template <typename R, int FMT>
__global__ void __launch_bounds__(AB) k_asq_fwd_qp(FwdArgs a, const R* __restrict__ T, R* QP) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * a.g.Vh) return;
    const Geom& g = a.g;
    const int blk = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    int x[4];
    a_coords(g, par, h, x);
    const Su3<R> umu = thin<R, FMT>(g, a.L, x, mu);
    for (int nd = 0; nd < 4; ++nd) {
        if (nd == mu) continue;
        for (int sn = -1; sn <= 1; sn += 2) {
            const int nu = sn * (nd + 1);
            Su3<R> q = scaled(coef_as<R>(a.k, 1), umu);
            for (int rd = 0; rd < 4; ++rd) {
                if (rd == mu || rd == nd) continue;
                const int sig = 6 - mu - nd - rd;
                for (int sr = -1; sr <= 1; sr += 2) {
                    const int rho = sr * (rd + 1);
                    int y[4] = {x[0], x[1], x[2], x[3]};
                    a_move(g, y, rho);
                    axpy(q, R(1.f), staple<R, FMT>(g, a.L, x, mu, rho, ld_f(T, slot3(mu, sig), g, y)));
                }
            }
            int y[4] = {x[0], x[1], x[2], x[3]};
            a_move(g, y, nu);
            axpy(q, coef_as<R>(a.k, 4), staple<R, FMT>(g, a.L, x, mu, nu, thin<R, FMT>(g, a.L, y, mu)));
            st_f(QP, slot6(mu, nu), par, h, g.Vh, q);
        }
    }
}
// CQ, then CT: one thread per (mu, site)
template <typename R, int FMT>
__global__ void __launch_bounds__(AB) k_asq_bwd_cq(FwdArgs a, const R* __restrict__ xv, R* CQ) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * a.g.Vh) return;
    const Geom& g = a.g;
    const int blk = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    int y[4];
    a_coords(g, par, h, y);
    for (int nd = 0; nd < 4; ++nd) {
        if (nd == mu) continue;
        for (int sn = -1; sn <= 1; sn += 2) {
            const int nu = sn * (nd + 1);
            int x[4] = {y[0], y[1], y[2], y[3]};
            a_move(g, x, -nu);
            int xm[4] = {x[0], x[1], x[2], x[3]};
            a_move(g, xm, mu + 1);
            const Su3<R> c = mm(mm(dagger(lnk<R, FMT>(g, a.L, xm, nu)), load_x<R>(xv, mu, g, x)), lnk<R, FMT>(g, a.L, x, nu));
            st_f(CQ, slot6(mu, nu), par, h, g.Vh, c);
        }
    }
}
template <typename R, int FMT>
__global__ void __launch_bounds__(AB) k_asq_bwd_ct(FwdArgs a, const R* __restrict__ CQ, R* CT) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * a.g.Vh) return;
    const Geom& g = a.g;
    const int blk = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    int z[4];
    a_coords(g, par, h, z);
    for (int sig = 0; sig < 4; ++sig) {
        if (sig == mu) continue;
        Su3<R> acc = zero_m<R>();
        for (int nd = 0; nd < 4; ++nd) {
            if (nd == mu || nd == sig) continue;
            const int rd = 6 - mu - sig - nd;
            for (int sn = -1; sn <= 1; sn += 2)
                for (int sr = -1; sr <= 1; sr += 2) {
                    const int nu = sn * (nd + 1), rho = sr * (rd + 1);
                    int y[4] = {z[0], z[1], z[2], z[3]};
                    a_move(g, y, -rho);
                    int ym[4] = {y[0], y[1], y[2], y[3]};
                    a_move(g, ym, mu + 1);
                    axpy(acc, R(1.f), mm(mm(dagger(lnk<R, FMT>(g, a.L, ym, rho)), ld_f(CQ, slot6(mu, nu), g, y)),
                                         lnk<R, FMT>(g, a.L, y, rho)));
                }
        }
        st_f(CT, slot3(mu, sig), par, h, g.Vh, acc);
    }
}
// the thin link U_al(z): direct terms, Naik, and every staple leg on it
template <typename R, int FMT>
__global__ void __launch_bounds__(AB) k_asq_bwd_links(FwdArgs a, const R* __restrict__ xv, const R* __restrict__ xw,
                                                      const R* __restrict__ T, const R* __restrict__ QP,
                                                      const R* __restrict__ CQ,
                                                      const R* __restrict__ CT, double* out, int mode) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * a.g.Vh) return;
    const Geom& g = a.g;
    const LinkPtrs& L = a.L;
    const int blk = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
    const int al = blk >> 1, par = blk & 1;
    int z[4];
    a_coords(g, par, h, z);
    const R c1 = coef_as<R>(a.k, 0), c3 = coef_as<R>(a.k, 1), c5 = coef_as<R>(a.k, 2), c7 = coef_as<R>(a.k, 3);
    const R cl = coef_as<R>(a.k, 4), cn = coef_as<R>(a.k, 5);
    Su3<R> gf = scaled(c1, load_x<R>(xv, al, g, z)), gb = zero_m<R>();
    // direct terms: U_al(z) as the c3 and c5 pieces, and as the inner link of
    // the seven-link and inner Lepage staples based at z - s
    for (int d = 0; d < 4; ++d) {
        if (d == al) continue;
        axpy(gf, c5, ld_f(CT, slot3(al, d), g, z));
        for (int sg = -1; sg <= 1; sg += 2) {
            const int s = sg * (d + 1);
            axpy(gf, c3, ld_f(CQ, slot6(al, s), g, z));
            int y[4] = {z[0], z[1], z[2], z[3]};
            a_move(g, y, -s);
            int ym[4] = {y[0], y[1], y[2], y[3]};
            a_move(g, ym, al + 1);
            const Su3<R> c = add_m(scaled(c7, ld_f(CT, slot3(al, d), g, y)), cl, ld_f(CQ, slot6(al, s), g, y));
            axpy(gf, R(1.f), mm(mm(dagger(lnk<R, FMT>(g, L, ym, s)), c), lnk<R, FMT>(g, L, y, s)));
        }
    }
    // Naik: W_al(x) = cN U(x) U(x+al) U(x+2al) with U_al(z) first, second, third;
    // the sites z + k al (k = 2, 1, -1, -2) as half-lattice indices computed
    // from scalars
    {
        const int La = g.L[al], za = z[al];
        int hk[4], pk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = q == 0 ? 2 : q == 1 ? 1 : q == 2 ? -1 : -2;
            const int ca = (za + k + 2 * La) % La;
            const int c0 = al == 0 ? ca : z[0], c1 = al == 1 ? ca : z[1];
            const int c2 = al == 2 ? ca : z[2], c3 = al == 3 ? ca : z[3];
            hk[q] = (c0 >> 1) + g.Lxh * (c1 + g.L[1] * (c2 + g.L[2] * c3));
            pk[q] = (c0 + c1 + c2 + c3) & 1;
        }
        const Su3<R> up2 = LinkFetch<R, FMT>::get(L, al, pk[0], hk[0], g.Vh);
        const Su3<R> up1 = LinkFetch<R, FMT>::get(L, al, pk[1], hk[1], g.Vh);
        const Su3<R> um1 = LinkFetch<R, FMT>::get(L, al, pk[2], hk[2], g.Vh);
        const Su3<R> um2 = LinkFetch<R, FMT>::get(L, al, pk[3], hk[3], g.Vh);
        axpy(gf, cn, mm(mm(up1, up2), load_x<R>(xw, al, g, z)));
        axpy(gf, cn, mm(mm(up1, ld_half<R>(xw, al, pk[2], hk[2], g.Vh)), um1));
        axpy(gf, cn, mm(mm(ld_half<R>(xw, al, pk[3], hk[3], g.Vh), um2), um1));
    }
    // legs: U_al(z) in the staples S_s, |s| = al, of every outer direction mu
    for (int mu = 0; mu < 4; ++mu) {
        if (mu == al) continue;
        for (int sg = -1; sg <= 1; sg += 2) {
            const int s = sg * (al + 1);
            for (int leg = 1; leg <= 2; ++leg) {
                // the staple's base y: leg 1 starts at y, leg 2 starts at y + mu
                int y[4] = {z[0], z[1], z[2], z[3]};
                if (leg == 2) a_move(g, y, -(mu + 1));
                if (s < 0) a_move(g, y, -s);
                int ys[4] = {y[0], y[1], y[2], y[3]};
                a_move(g, ys, s);
                int ym[4] = {y[0], y[1], y[2], y[3]};
                a_move(g, ym, mu + 1);
                // the other leg of the staple
                const Su3<R> other = leg == 1 ? lnk<R, FMT>(g, L, ym, s) : lnk<R, FMT>(g, L, y, s);
                // (inner value, cotangent) pairs of every staple of this geometry,
                // the leg's matrix cotangents summed in acc
                Su3<R> acc = leg_term(leg, ld_f(QP, slot6(mu, s), g, ys), load_x<R>(xv, mu, g, y), other);
                for (int nd = 0; nd < 4; ++nd) {
                    if (nd == mu || nd == al) continue;
                    const int sig = 6 - mu - nd - al;
                    for (int sn = -1; sn <= 1; sn += 2)
                        axpy(acc, R(1.f), leg_term(leg, ld_f(T, slot3(mu, sig), g, ys),
                                                   ld_f(CQ, slot6(mu, sn * (nd + 1)), g, y), other));
                }
                axpy(acc, R(1.f), leg_term(leg, thin<R, FMT>(g, L, ys, mu),
                                           add_m(scaled(cl, ld_f(CQ, slot6(mu, s), g, y)), c7,
                                                 ld_f(CT, slot3(mu, al), g, y)), other));
                // leg 1 with s > 0 and leg 2 with s < 0 meet U_al(z) forward
                if ((leg == 1) == (s > 0)) axpy(gf, R(1.f), acc);
                else axpy(gb, R(1.f), acc);
            }
        }
    }
    put_asq_force(g, thin<R, FMT>(g, L, z, al), gf, gb, out, blk, h, mode);
}

// host: the incidence table of every direction
struct IncTable {
    AsqInc inc[4][ASQ_MAX_INC];
    int n[4];
};
void build_incidences(IncTable* t) {
    std::memset(t, 0, sizeof(*t));
    for (int mu = 0; mu < 4; ++mu) {
        const int m = mu + 1;
        std::vector<std::pair<int, std::vector<int>>> paths;   // (class, steps)
        paths.push_back({0, {m}});
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            for (int sn = -1; sn <= 1; sn += 2) {
                const int a = sn * (nu + 1);
                paths.push_back({1, {a, m, -a}});
                paths.push_back({4, {a, a, m, -a, -a}});
                for (int rho = 0; rho < 4; ++rho) {
                    if (rho == mu || rho == nu) continue;
                    for (int sr = -1; sr <= 1; sr += 2) {
                        const int b = sr * (rho + 1);
                        paths.push_back({2, {a, b, m, -b, -a}});
                        const int sig = 6 - mu - nu - rho;
                        for (int ss = -1; ss <= 1; ss += 2) {
                            const int c = ss * (sig + 1);
                            paths.push_back({3, {a, b, c, m, -c, -b, -a}});
                        }
                    }
                }
            }
        }
        paths.push_back({5, {m, m, m}});
        for (auto& p : paths) {
            const int len = (int)p.second.size();
            for (int k = 0; k < len; ++k) {
                const int d = (p.second[k] > 0 ? p.second[k] : -p.second[k]) - 1;
                AsqInc& e = t->inc[d][t->n[d]++];
                for (int j = 0; j < len; ++j) e.s[j] = (signed char)p.second[j];
                e.len = (unsigned char)len;
                e.k = (unsigned char)k;
                e.mu = (unsigned char)mu;
                e.cls = (unsigned char)p.first;
            }
        }
    }
}

AsqCoef make_coef(const double (&c)[6]) {
    AsqCoef k;
    for (int i = 0; i < 6; ++i) {
        k.c[i][0] = (float)c[i];
        k.c[i][1] = (float)(c[i] - (double)k.c[i][0]);
    }
    return k;
}

size_t link_store_floats(const stag_ctx* ctx) { return (size_t)4 * 2 * 18 * ctx->g.Vh; }
}  // namespace

// ---------------------------------------------------------------- host side
AsqLinks asq_links(const stag_ctx* ctx) {
    const size_t n = link_store_floats(ctx);
    float* base = ctx->asq_store;
    return AsqLinks{LinkPtrs{base, base + n, nullptr}, LinkPtrs{base + 2 * n, base + 3 * n, nullptr}};
}

int asq_tps(const stag_ctx* ctx) {
    if (ctx->tps_force == 1 || ctx->tps_force == 2 || ctx->tps_force == 4 || ctx->tps_force == 8) return ctx->tps_force;
    return dslash_tps_for(ctx->g.Vh);
}

stag_status asq_ensure(stag_ctx* ctx) {
    if (!ctx->asqtad) return STAG_OK;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    const int want = ctx->asq_fp32_build ? 1 : 2;
    if (!ctx->asq_stale && ctx->asq_built == want) return STAG_OK;
    const AsqLinks A = asq_links(ctx);
    const long long n = 8LL * ctx->g.Vh;
    float *fh = const_cast<float*>(A.fat.hi), *fl = const_cast<float*>(A.fat.lo);
    float *lh = const_cast<float*>(A.lng.hi), *ll = const_cast<float*>(A.lng.lo);
    if (want == 2)
        k_fatten<DF, FMT_F64><<<nblocks(n, AB), AB, 0, ctx->stream>>>(ctx->g, link_ptrs(ctx), make_coef(ctx->asq_coef),
                                                                      fh, fl, lh, ll);
    else
        k_fatten<float, FMT_F32_18><<<nblocks(n, AB), AB, 0, ctx->stream>>>(ctx->g, link_ptrs(ctx),
                                                                            make_coef(ctx->asq_coef), fh, fl, lh, ll);
    CKL();
    ctx->asq_stale = false;
    ctx->asq_built = want;
    return STAG_OK;
}

stag_status asq_outer_begin(stag_ctx* ctx, stag_prec prec) {
    const size_t rs = prec == STAG_FP64 ? sizeof(DF) : sizeof(float);
    const size_t bytes = 2 * link_store_floats(ctx) * rs;
    void* p;
    CKS(ws_get(ctx, WS_ASQ_X, bytes, &p));
    CK(cudaMemsetAsync(p, 0, bytes, ctx->stream));
    return STAG_OK;
}

stag_status asq_outer_add(stag_ctx* ctx, stag_prec prec, int nsrc, int nshift, const double* alpha, const void* x,
                          const void* y, double coef) {
    if (nshift > 60) return STAG_ERR_ARG;
    CKS(stage_upload(ctx, ctx->scal, alpha, nshift * sizeof(double)));
    const long long n = 8LL * ctx->g.Vh;
    const size_t nl = link_store_floats(ctx);
    if (prec == STAG_FP64) {
        DF* xv = (DF*)ctx->ws[WS_ASQ_X];
        k_asq_outer<DF><<<nblocks(n, AB), AB, 0, ctx->stream>>>(ctx->g, nsrc, nshift, ctx->scal, coef,
                                                                (const double2*)x, (const double2*)y, xv, xv + nl);
    } else {
        float* xv = (float*)ctx->ws[WS_ASQ_X];
        k_asq_outer<float><<<nblocks(n, AB), AB, 0, ctx->stream>>>(ctx->g, nsrc, nshift, ctx->scal, coef,
                                                                   (const float2*)x, (const float2*)y, xv, xv + nl);
    }
    CKL();
    return STAG_OK;
}

template <typename R, int FMT>
static stag_status asq_force_reverse(stag_ctx* ctx, const R* xv, const R* xw, double* out, int mode) {
    const size_t slot = (size_t)2 * 18 * ctx->g.Vh;     // reals of one matrix field
    void* p;
    CKS(ws_get(ctx, WS_ASQ_F, 72 * slot * sizeof(R), &p));
    R* T = (R*)p;
    R* QP = T + 12 * slot;
    R* CQ = QP + 24 * slot;
    R* CT = CQ + 24 * slot;
    const FwdArgs a{ctx->g, link_ptrs(ctx), make_coef(ctx->asq_coef)};
    const int nb = nblocks(8LL * ctx->g.Vh, AB);
    k_asq_fwd_t<R, FMT><<<nb, AB, 0, ctx->stream>>>(a, T);
    k_asq_fwd_qp<R, FMT><<<nb, AB, 0, ctx->stream>>>(a, T, QP);
    k_asq_bwd_cq<R, FMT><<<nb, AB, 0, ctx->stream>>>(a, xv, CQ);
    k_asq_bwd_ct<R, FMT><<<nb, AB, 0, ctx->stream>>>(a, CQ, CT);
    k_asq_bwd_links<R, FMT><<<nb, AB, 0, ctx->stream>>>(a, xv, xw, T, QP, CQ, CT, out, mode);
    ctx->launches += 4;
    CKL();
    return STAG_OK;
}

stag_status asq_force_finish(stag_ctx* ctx, stag_prec prec, double* out, int mode) {
    CKS(asq_ensure(ctx));
    const long long n = 8LL * ctx->g.Vh;
    const size_t nl = link_store_floats(ctx);
    const AsqCoef k = make_coef(ctx->asq_coef);
    if (prec == STAG_FP64) {
        const DF* xv = (const DF*)ctx->ws[WS_ASQ_X];
        if (!ctx->asq_gather) return asq_force_reverse<DF, FMT_F64>(ctx, xv, xv + nl, out, mode);
        k_asq_force<DF, FMT_F64><<<nblocks(n, AB), AB, 0, ctx->stream>>>(ctx->g, link_ptrs(ctx), k, xv, xv + nl,
                                                                         out, mode);
    } else {
        const float* xv = (const float*)ctx->ws[WS_ASQ_X];
        if (!ctx->asq_gather) return asq_force_reverse<float, FMT_F32_18>(ctx, xv, xv + nl, out, mode);
        k_asq_force<float, FMT_F32_18><<<nblocks(n, AB), AB, 0, ctx->stream>>>(ctx->g, link_ptrs(ctx), k, xv,
                                                                               xv + nl, out, mode);
    }
    CKL();
    return STAG_OK;
}

extern "C" stag_status stag_set_action(stag_ctx* ctx, stag_action action, double u0) {
    if (!ctx) return STAG_ERR_ARG;
    if (action == STAG_ACTION_UNIMPROVED) {
        ctx->asqtad = false;
        return STAG_OK;
    }
    if (action != STAG_ACTION_ASQTAD || !(u0 > 0.0) || !(u0 <= 1.0)) return STAG_ERR_ARG;
    void* p;
    CKS(ws_get(ctx, WS_ASQ_LINKS, 4 * link_store_floats(ctx) * sizeof(float), &p));
    ctx->asq_store = (float*)p;
    const double u2 = u0 * u0, u4 = u2 * u2, u6 = u4 * u2;
    const double c[6] = {5.0 / 8.0, 1.0 / 16.0 / u2, 1.0 / 64.0 / u4, 1.0 / 384.0 / u6, -1.0 / 16.0 / u4,
                         -1.0 / 24.0 / u2};
    for (int i = 0; i < 6; ++i) ctx->asq_coef[i] = c[i];
    static IncTable table;      // the same for every context; built once
    static bool built = false;
    if (!built) {
        build_incidences(&table);
        built = true;
    }
    for (int d = 0; d < 4; ++d)
        if (table.n[d] > ASQ_MAX_INC) return STAG_ERR_ARG;
    CK(cudaMemcpyToSymbolAsync(c_inc, table.inc, sizeof(table.inc), 0, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyToSymbolAsync(c_ninc, table.n, sizeof(table.n), 0, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->asqtad = true;
    ctx->asq_stale = true;
    return STAG_OK;
}

extern "C" stag_status stag_asqtad_links(stag_ctx* ctx, double* host_fat, double* host_naik) {
    if (!ctx || !host_fat || !host_naik || !ctx->asqtad) return STAG_ERR_ARG;
    CKS(asq_ensure(ctx));
    const AsqLinks A = asq_links(ctx);
    const size_t bytes = (size_t)4 * ctx->g.V * 18 * sizeof(double);
    void* stage;
    CKS(ws_get(ctx, WS_STAGE, bytes, &stage));
    for (int which = 0; which < 2; ++which) {
        const LinkPtrs& l = which == 0 ? A.fat : A.lng;
        CKS(unpack_links(ctx, l.hi, l.lo, (double*)stage));
        CK(cudaMemcpyAsync(which == 0 ? host_fat : host_naik, stage, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return STAG_OK;
}
