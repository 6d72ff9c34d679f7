// Per-link kernels of the MD update (Sec. 2, Sec. 3 "one thread per link in
// the gauge update", Sec. 4 precisions): fermion force from the multi-shift
// solutions, Wilson gauge force, momentum kicks fused into both, the link
// update U <- exp(i eps P) U fused with the fp64 reunitarisation, the fp64
// action sums and the Philox draws of momenta and pseudo-fermion sources.
#include <cmath>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "philox.cuh"

namespace {
constexpr int FB = 128;

__device__ __forceinline__ int hidx(const Geom& g, const int c[4]) {
    return (c[0] >> 1) + g.Lxh * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}
__device__ __forceinline__ void link_coords(const Geom& g, int par, int h, int c[4]) {
    int xh = h % g.Lxh, r = h / g.Lxh;
    c[1] = r % g.L[1]; r /= g.L[1];
    c[2] = r % g.L[2]; c[3] = r / g.L[2];
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + par) & 1);
}
__device__ __forceinline__ void step(const Geom& g, int c[4], int mu, int d) {
    c[mu] += d;
    if (c[mu] < 0) c[mu] += g.L[mu];
    if (c[mu] >= g.L[mu]) c[mu] -= g.L[mu];
}

// coefficient a of Re tr(i T_a W), T_a = lambda_a / 2
template <typename R>
__device__ __forceinline__ void re_tr_i_t(const Su3<R>& w, R (&f)[8]) {
    const R h = (R)0.5;
    f[0] = -h * (w.e[1][0].im + w.e[0][1].im);
    f[1] = -h * (w.e[0][1].re - w.e[1][0].re);
    f[2] = -h * (w.e[0][0].im - w.e[1][1].im);
    f[3] = -h * (w.e[2][0].im + w.e[0][2].im);
    f[4] = -h * (w.e[0][2].re - w.e[2][0].re);
    f[5] = -h * (w.e[2][1].im + w.e[1][2].im);
    f[6] = -h * (w.e[1][2].re - w.e[2][1].re);
    f[7] = -(w.e[0][0].im + w.e[1][1].im - (R)2 * w.e[2][2].im) * (R)0.28867513459481287;  // 1/(2 sqrt 3)
}

// out[a] = coef F_a (mode 0) or out[a] += coef F_a (mode 1); momentum layout
__device__ __forceinline__ void put_force(double* out, int mu, int par, int h, int Vh, const double (&f)[8],
                                          double coef, int mode) {
    double* o = out + ((size_t)(2 * mu + par) * 8) * Vh + h;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        if (mode) o[(size_t)a * Vh] += coef * f[a];
        else o[(size_t)a * Vh] = coef * f[a];
    }
}

// Conversions between float and double by integer operations on the IEEE-754
// bit patterns, with the results of the conversion instructions (round to
// nearest even): those instructions issue on GB300's FP64 pipe, which is
// ~1/64 of the FP32 rate, and made up about half of the link update's FP64
// work.  Zeros, results outside the float normal range, Inf and NaN take the
// instruction.
__device__ __forceinline__ float f64_to_f32_rn(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;    // float exponent field
    if (e <= 0 || e >= 255) return __double2float_rn(d);
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    const unsigned int top = (unsigned int)((b >> 29) & 0x7FFFFFull);   // the 23 kept mantissa bits
    const unsigned int rest = (unsigned int)(b & 0x1FFFFFFFull);        // the 29 dropped ones
    const unsigned int up = (rest > 0x10000000u || (rest == 0x10000000u && (top & 1u))) ? 1u : 0u;
    // a carry out of the mantissa steps the exponent (to Inf past the largest float)
    return __uint_as_float(sign | ((((unsigned int)e << 23) | top) + up));
}
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)f;
    return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                            ((unsigned long long)(e - 127u + 1023u) << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// ---------------------------------------------------------------- fermion force
// F_a(x,mu) = sum_{k,i} alpha_i eps(x) eta_mu(x) Re tr[i T_a U_mu(x) Z(x+mu) Z(x)^dag],
// Z = X on even sites and Y = D_oe X on odd sites.  X, Y: [n_pf][nshift][3][Vh].
template <typename R, int FMT>
__global__ void __launch_bounds__(FB) k_fermion_force(Geom g, LinkPtrs L, int nsrc, int nshift,
                                                      const double* __restrict__ alpha,
                                                      const typename V2T<R>::T* __restrict__ X,
                                                      const typename V2T<R>::T* __restrict__ Y, double* out,
                                                      double coef, int mode) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int blk = (int)(idx / g.Vh);
    const int h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    Nbr n;
    site_neighbours(g, h, par, n);
    const int hf = n.fwd[mu];
    const typename V2T<R>::T* here = par == 0 ? X : Y;     // Z(x)
    const typename V2T<R>::T* there = par == 0 ? Y : X;    // Z(x+mu)
    Su3<R> m;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) m.e[i][j] = mk<R>(0, 0);
    const size_t rs = (size_t)3 * g.Vh;
    for (int k = 0; k < nsrc; ++k) {
        for (int s = 0; s < nshift; ++s) {
            const size_t off = ((size_t)k * nshift + s) * rs;
            Vec3<R> v = load_vec<R>(there + off, hf, g.Vh);
            Vec3<R> w = load_vec<R>(here + off, h, g.Vh);
            const R a = (R)alpha[s];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                Cx<R> av = a * v.c[i];
#pragma unroll
                for (int j = 0; j < 3; ++j) cmac(m.e[i][j], av, conj(w.c[j]));
            }
        }
    }
    Su3<R> u = LinkFetch<R, FMT>::get(L, mu, par, h, g.Vh);
    Su3<R> w = mul(u, m);
    R f[8];
    re_tr_i_t(w, f);
    const double sgn = (par == 0 ? 1.0 : -1.0) * (double)n.sf[mu];
    double fd[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) fd[a] = sgn * (double)f[a];
    put_force(out, mu, par, h, g.Vh, fd, coef, mode);
}

// ---------------------------------------------------------------- gauge force
// F_a = -(beta/3) Re tr(i T_a U_mu(x) Sigma_mu(x)), Sigma = sum of upper and lower staples.
// The fp32 instantiation is held to 128 registers (four blocks per SM: its
// 18 link gathers per thread are L2 latency), the fp64 one would spill there.
template <typename R, int FMT>
__global__ void __launch_bounds__(FB, std::is_same<R, float>::value ? 4 : 1) k_gauge_force(Geom g, LinkPtrs L, double beta, double* out, double coef,
                                                    int mode) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int blk = (int)(idx / g.Vh);
    const int h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    int x[4];
    link_coords(g, par, h, x);
    Su3<R> sig;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) sig.e[i][j] = mk<R>(0, 0);
    int xpm[4] = {x[0], x[1], x[2], x[3]};
    step(g, xpm, mu, +1);
    const int h_xpm = hidx(g, xpm);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        int xpn[4] = {x[0], x[1], x[2], x[3]};
        step(g, xpn, nu, +1);
        int xmn[4] = {x[0], x[1], x[2], x[3]};
        step(g, xmn, nu, -1);
        int xpmmn[4] = {xpm[0], xpm[1], xpm[2], xpm[3]};
        step(g, xpmmn, nu, -1);
        const int h_xpn = hidx(g, xpn), h_xmn = hidx(g, xmn), h_xpmmn = hidx(g, xpmmn);
        // upper: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        Su3<R> a = LinkFetch<R, FMT>::get(L, nu, 1 - par, h_xpm, g.Vh);
        Su3<R> b = LinkFetch<R, FMT>::get(L, mu, 1 - par, h_xpn, g.Vh);
        Su3<R> c = LinkFetch<R, FMT>::get(L, nu, par, h, g.Vh);
        Su3<R> up = mul_nd(mul_nd(a, b), c);
        // lower: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
        Su3<R> d = LinkFetch<R, FMT>::get(L, nu, par, h_xpmmn, g.Vh);
        Su3<R> e = LinkFetch<R, FMT>::get(L, mu, 1 - par, h_xmn, g.Vh);
        Su3<R> f = LinkFetch<R, FMT>::get(L, nu, 1 - par, h_xmn, g.Vh);
        // d^dag e^dag f = (e d)^dag f
        Su3<R> ed = mul(e, d);
        Su3<R> low = mul_dn(ed, f);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) sig.e[i][j] = sig.e[i][j] + up.e[i][j] + low.e[i][j];
    }
    Su3<R> u = LinkFetch<R, FMT>::get(L, mu, par, h, g.Vh);
    Su3<R> w = mul(u, sig);
    R fr[8];
    re_tr_i_t(w, fr);
    double fd[8];
    if constexpr (std::is_same<R, float>::value) {
        // the fp32 force scaled in fp32 and widened by integer operations
        // (no conversion or multiply on the FP64 pipe but put_force's FMA)
        const float sb = f64_to_f32_rn(-beta / 3.0);
#pragma unroll
        for (int a = 0; a < 8; ++a) fd[a] = f32_to_f64(sb * fr[a]);
    } else {
#pragma unroll
        for (int a = 0; a < 8; ++a) fd[a] = -(beta / 3.0) * (double)fr[a];
    }
    put_force(out, mu, par, h, g.Vh, fd, coef, mode);
}

// ---------------------------------------------------------------- link update + reunitarisation
// hi = the double rounded to float, lo = the (exact) remainder rounded to
// float, the pair made canonical (hl_canonical) as the load makes it
__device__ __forceinline__ void store_link_hl(float* hi, float* lo, size_t blk, int h, int Vh, const Su3<double>& u) {
    float vh[18], vl[18];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double re = u.e[k / 3][k % 3].re, im = u.e[k / 3][k % 3].im;
        float a = f64_to_f32_rn(re), b = f64_to_f32_rn(im);
        float la = f64_to_f32_rn(re - f32_to_f64(a)), lb = f64_to_f32_rn(im - f32_to_f64(b));
        hl_canonical(a, la);
        hl_canonical(b, lb);
        vh[2 * k] = a; vh[2 * k + 1] = b;
        vl[2 * k] = la; vl[2 * k + 1] = lb;
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

// Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1)  (Sec. 4: reunitarisation in double)
__device__ __forceinline__ void reunit(Su3<double>& u) {
    double n0 = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) n0 += u.e[0][j].re * u.e[0][j].re + u.e[0][j].im * u.e[0][j].im;
    n0 = rsqrt(n0);
#pragma unroll
    for (int j = 0; j < 3; ++j) u.e[0][j] = n0 * u.e[0][j];
    Cx<double> d = mk(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 3; ++j) cmacc(d, u.e[0][j], u.e[1][j]);
#pragma unroll
    for (int j = 0; j < 3; ++j) u.e[1][j] = u.e[1][j] - d * u.e[0][j];
    double n1 = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) n1 += u.e[1][j].re * u.e[1][j].re + u.e[1][j].im * u.e[1][j].im;
    n1 = rsqrt(n1);
#pragma unroll
    for (int j = 0; j < 3; ++j) u.e[1][j] = n1 * u.e[1][j];
    rebuild_row2(u);
}

// 1/sqrt(x) in float-float: the fp32 estimate refined by two Newton steps
// y <- y + y (1 - x y^2) / 2 (the error squares: about 2^-22, 2^-43, then the
// float-float rounding)
__device__ __forceinline__ DF df_rsqrt(const DF& x) {
    DF y(rsqrtf(x.hi));
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const DF r = DF(1.f) - x * (y * y);
        y = y + y * r * DF(0.5f);
    }
    return y;
}

// The same Gram-Schmidt in float-float for the fp32 link update (Sec. 4's
// reunitarisation in double precision, on the fp32 pipes: GB300 issues fp64
// at ~1/64 of the fp32 rate, and the fp64 version was nearly all of the
// update's time); the rows come out about 2^-46 from orthonormal.
__device__ __forceinline__ void reunit_df(Su3<DF>& u) {
    DF n0(0.f);
#pragma unroll
    for (int j = 0; j < 3; ++j) n0 = n0 + u.e[0][j].re * u.e[0][j].re + u.e[0][j].im * u.e[0][j].im;
    n0 = df_rsqrt(n0);
#pragma unroll
    for (int j = 0; j < 3; ++j) u.e[0][j] = n0 * u.e[0][j];
    Cx<DF> d = mk(DF(0.f), DF(0.f));
#pragma unroll
    for (int j = 0; j < 3; ++j) cmacc(d, u.e[0][j], u.e[1][j]);
#pragma unroll
    for (int j = 0; j < 3; ++j) u.e[1][j] = u.e[1][j] - d * u.e[0][j];
    DF n1(0.f);
#pragma unroll
    for (int j = 0; j < 3; ++j) n1 = n1 + u.e[1][j].re * u.e[1][j].re + u.e[1][j].im * u.e[1][j].im;
    n1 = df_rsqrt(n1);
#pragma unroll
    for (int j = 0; j < 3; ++j) u.e[1][j] = n1 * u.e[1][j];
    rebuild_row2(u);
}

// lo rounded to a multiple of 2^(E - 52), E the exponent of hi: hi + lo is
// then a double, so storing it (hi + lo as a double) and loading it again
// gives this pair back bit for bit.  A float-float lo can otherwise hold bits
// below the double's last place.  hi below 2^-74 (or zero) keeps its lo.
__device__ __forceinline__ float lo_on_double_grid(float hi, float lo) {
    const int e = (int)((__float_as_uint(hi) >> 23) & 0xFFu);   // biased exponent of hi
    if (e < 53 || e == 0xFF) return e == 0 ? 0.f : lo;
    const float q = __uint_as_float((unsigned int)(e - 52) << 23);        // 2^(E - 52)
    const float iq = __uint_as_float((unsigned int)(254 - (e - 52)) << 23);   // 1 / q, exact
    return rintf(lo * iq) * q;
}

// the float-float link into the two-float store: its value rounded to double
// precision, split canonically
__device__ __forceinline__ void store_link_df(float* hi, float* lo, size_t blk, int h, int Vh, const Su3<DF>& u) {
    float vh[18], vl[18];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        float a = u.e[k / 3][k % 3].re.hi, la = u.e[k / 3][k % 3].re.lo;
        float b = u.e[k / 3][k % 3].im.hi, lb = u.e[k / 3][k % 3].im.lo;
        la = lo_on_double_grid(a, la);
        lb = lo_on_double_grid(b, lb);
        hl_canonical(a, la);
        hl_canonical(b, lb);
        vh[2 * k] = a; vh[2 * k + 1] = b;
        vl[2 * k] = la; vl[2 * k + 1] = lb;
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

// P = sum_a p_a T_a as a Hermitian matrix
template <typename R>
__device__ __forceinline__ Su3<R> herm_from_coeffs(const double* p, size_t stride) {
    R c[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        if constexpr (std::is_same<R, float>::value) c[a] = f64_to_f32_rn(p[(size_t)a * stride]);
        else c[a] = p[(size_t)a * stride];
    }
    const R s3 = (R)0.57735026918962576;   // 1/sqrt(3)
    Su3<R> hm;
    hm.e[0][0] = mk<R>((R)0.5 * (c[2] + s3 * c[7]), 0);
    hm.e[1][1] = mk<R>((R)0.5 * (-c[2] + s3 * c[7]), 0);
    hm.e[2][2] = mk<R>(-s3 * c[7], 0);
    hm.e[0][1] = mk<R>((R)0.5 * c[0], -(R)0.5 * c[1]);
    hm.e[1][0] = conj(hm.e[0][1]);
    hm.e[0][2] = mk<R>((R)0.5 * c[3], -(R)0.5 * c[4]);
    hm.e[2][0] = conj(hm.e[0][2]);
    hm.e[1][2] = mk<R>((R)0.5 * c[5], -(R)0.5 * c[6]);
    hm.e[2][1] = conj(hm.e[1][2]);
    return hm;
}

// exp(i eps H) by a Taylor series in Horner form after scaling by 2^-k
// (||X|| <= 1/4), then k squarings (scaling and squaring, Moler & Van Loan).
template <typename R, int ORDER>
__device__ __forceinline__ Su3<R> expi(const Su3<R>& hm, R eps) {
    Su3<R> x;
    R nrm = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            x.e[i][j] = mk<R>(-eps * hm.e[i][j].im, eps * hm.e[i][j].re);   // i eps H
            nrm += x.e[i][j].re * x.e[i][j].re + x.e[i][j].im * x.e[i][j].im;
        }
    nrm = sqrt(nrm);
    int k = 0;
    while (nrm > (R)0.25 && k < 40) { nrm *= (R)0.5; ++k; }
    R sc = (R)1;
    for (int q = 0; q < k; ++q) sc *= (R)0.5;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) x.e[i][j] = sc * x.e[i][j];
    Su3<R> e;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) e.e[i][j] = mk<R>(i == j ? (R)1 : (R)0, 0);
    for (int n = ORDER; n >= 1; --n) {
        Su3<R> t = mul(x, e);
        const R inv = (R)1 / (R)n;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) e.e[i][j] = mk<R>((i == j ? (R)1 : (R)0) + inv * t.e[i][j].re, inv * t.e[i][j].im);
    }
    for (int q = 0; q < k; ++q) e = mul(e, e);
    return e;
}

__device__ __forceinline__ double to_f64(float f) { return f32_to_f64(f); }
__device__ __forceinline__ double to_f64(double d) { return d; }

// U <- reunitarise(exp(i eps P) U): the exponential and the product in R
// (fp32 in the mixed path, Sec. 4), the reunitarisation in double precision:
// float-float after the fp32 product, fp64 on the fp64 path.
template <typename R, int FMT, int ORDER>
__global__ void __launch_bounds__(FB) k_update_links(Geom g, float* hi, float* lo, const double* __restrict__ mom,
                                                     double eps) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int blk = (int)(idx / g.Vh);
    const int h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    LinkPtrs L{hi, lo, nullptr};
    Su3<R> u = LinkFetch<R, FMT>::get(L, mu, par, h, g.Vh);
    Su3<R> hm = herm_from_coeffs<R>(mom + ((size_t)blk * 8) * g.Vh + h, g.Vh);
    Su3<R> e = expi<R, ORDER>(hm, (R)eps);
    Su3<R> un = mul(e, u);
    if constexpr (std::is_same<R, float>::value) {
        Su3<DF> ud;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) ud.e[i][j] = mk(DF(un.e[i][j].re), DF(un.e[i][j].im));
        reunit_df(ud);
        store_link_df(hi, lo, link_block_f(mu, par, g.Vh), h, g.Vh, ud);
    } else {
        Su3<double> ud;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) ud.e[i][j] = mk(to_f64(un.e[i][j].re), to_f64(un.e[i][j].im));
        reunit(ud);
        store_link_hl(hi, lo, link_block_f(mu, par, g.Vh), h, g.Vh, ud);
    }
}

__global__ void __launch_bounds__(FB) k_reunitarize(Geom g, float* hi, float* lo) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int blk = (int)(idx / g.Vh);
    const int h = (int)(idx % g.Vh);
    const int mu = blk >> 1, par = blk & 1;
    Su3<double> u = load_link_d(hi, lo, link_block_f(mu, par, g.Vh), h, g.Vh);
    reunit(u);
    store_link_hl(hi, lo, link_block_f(mu, par, g.Vh), h, g.Vh, u);
}

// ---------------------------------------------------------------- fp64 action sums
__global__ void __launch_bounds__(FB) k_plaquette(Geom g, LinkPtrs L, double* partial) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (idx < 2LL * g.Vh) {
        const int par = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
        int x[4];
        link_coords(g, par, h, x);
        for (int mu = 0; mu < 4; ++mu) {
            int xpm[4] = {x[0], x[1], x[2], x[3]};
            step(g, xpm, mu, +1);
            Su3<double> umu = LinkFetch<double, FMT_F64>::get(L, mu, par, h, g.Vh);
            for (int nu = mu + 1; nu < 4; ++nu) {
                int xpn[4] = {x[0], x[1], x[2], x[3]};
                step(g, xpn, nu, +1);
                Su3<double> a = LinkFetch<double, FMT_F64>::get(L, nu, 1 - par, hidx(g, xpm), g.Vh);
                Su3<double> b = LinkFetch<double, FMT_F64>::get(L, mu, 1 - par, hidx(g, xpn), g.Vh);
                Su3<double> c = LinkFetch<double, FMT_F64>::get(L, nu, par, h, g.Vh);
                Su3<double> p = mul_nd(mul_nd(mul(umu, a), b), c);
                v[0] += p.e[0][0].re + p.e[1][1].re + p.e[2][2].re;
            }
        }
    }
    block_sum<1>(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v[0];
}

__global__ void __launch_bounds__(256) k_sumsq(size_t n, const double* __restrict__ a, double* partial) {
    double v[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v[0] += a[i] * a[i];
    block_sum<1>(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v[0];
}

__global__ void k_axpy_mom(size_t n, double* m, const double* __restrict__ f, double c) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) m[i] += c * f[i];
}

// ---------------------------------------------------------------- random draws
// momenta: link (mu, s) [s lexicographic] uses blocks 2*(mu*V + s) + j, j = 0, 1,
// whose four Box-Muller normals are p_{4j..4j+3}
__global__ void k_draw_momenta(Geom g, double* mom, uint64_t seed, uint64_t counter) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4LL * g.V) return;
    const int mu = (int)(idx / g.V), s = (int)(idx % g.V);
    int x = s % g.L[0], r = s / g.L[0];
    int y = r % g.L[1]; r /= g.L[1];
    int z = r % g.L[2], t = r / g.L[2];
    const int par = (x + y + z + t) & 1, h = s >> 1;
    double* o = mom + ((size_t)(2 * mu + par) * 8) * g.Vh + h;
    for (int j = 0; j < 2; ++j) {
        Philox4 w = philox_block(seed, RNG_STREAM_MOMENTA, 2ULL * (uint64_t)idx + j, counter);
        double u0 = philox_uniform(w.v[0]), u1 = philox_uniform(w.v[1]);
        double u2 = philox_uniform(w.v[2]), u3 = philox_uniform(w.v[3]);
        double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
        double s1, c1, s3, c3;
        sincospi(2.0 * u1, &s1, &c1);
        sincospi(2.0 * u3, &s3, &c3);
        o[(size_t)(4 * j + 0) * g.Vh] = r0 * c1;
        o[(size_t)(4 * j + 1) * g.Vh] = r0 * s1;
        o[(size_t)(4 * j + 2) * g.Vh] = r1 * c3;
        o[(size_t)(4 * j + 3) * g.Vh] = r1 * s3;
    }
}

// sources: even site h uses blocks 2h + j of stream base+k; the first six normals,
// times sqrt(1/2), are (Re, Im) of colours 0..2 (density exp(-xi^dag xi))
__global__ void k_draw_sources(Geom g, double2* xi, int n, uint64_t seed, uint64_t counter, uint64_t stream0) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * g.Vh) return;
    const int k = (int)(idx / g.Vh), h = (int)(idx % g.Vh);
    double gs[8];
    for (int j = 0; j < 2; ++j) {
        Philox4 w = philox_block(seed, stream0 + k, 2ULL * h + j, counter);
        double u0 = philox_uniform(w.v[0]), u1 = philox_uniform(w.v[1]);
        double u2 = philox_uniform(w.v[2]), u3 = philox_uniform(w.v[3]);
        double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
        double s1, c1, s3, c3;
        sincospi(2.0 * u1, &s1, &c1);
        sincospi(2.0 * u3, &s3, &c3);
        gs[4 * j + 0] = r0 * c1; gs[4 * j + 1] = r0 * s1;
        gs[4 * j + 2] = r1 * c3; gs[4 * j + 3] = r1 * s3;
    }
    const double sq = 0.70710678118654752;
    for (int c = 0; c < 3; ++c)
        xi[((size_t)k * 3 + c) * g.Vh + h] = make_double2(sq * gs[2 * c], sq * gs[2 * c + 1]);
}

stag_status sum_partials(stag_ctx* ctx, int nb, double* out) {
    std::vector<double> part(nb);
    CK(cudaMemcpyAsync(part.data(), ctx->red, nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[i];
    *out = s;
    return STAG_OK;
}
}  // namespace

// ---------------------------------------------------------------- host launchers
stag_status fermion_force_from_solutions(stag_ctx* ctx, stag_prec prec, int nsrc, int nshift, const double* alpha,
                                         const void* x, const void* y, double* out, double coef, int mode) {
    if (nshift > 60) return STAG_ERR_ARG;
    CKS(stage_upload(ctx, ctx->scal, alpha, nshift * sizeof(double)));
    long long n = 8LL * ctx->g.Vh;
    LinkPtrs L = link_ptrs(ctx);
    if (prec == STAG_FP64)
        k_fermion_force<double, FMT_F64><<<nblocks(n, FB), FB, 0, ctx->stream>>>(
            ctx->g, L, nsrc, nshift, ctx->scal, (const double2*)x, (const double2*)y, out, coef, mode);
    else
        k_fermion_force<float, FMT_F32_18><<<nblocks(n, FB), FB, 0, ctx->stream>>>(
            ctx->g, L, nsrc, nshift, ctx->scal, (const float2*)x, (const float2*)y, out, coef, mode);
    CKL();
    return STAG_OK;
}

stag_status gauge_force_launch(stag_ctx* ctx, stag_prec prec, double beta, double* out, double coef, int mode) {
    long long n = 8LL * ctx->g.Vh;
    LinkPtrs L = link_ptrs(ctx);
    if (prec == STAG_FP64)
        k_gauge_force<double, FMT_F64><<<nblocks(n, FB), FB, 0, ctx->stream>>>(ctx->g, L, beta, out, coef, mode);
    else
        k_gauge_force<float, FMT_F32_18><<<nblocks(n, FB), FB, 0, ctx->stream>>>(ctx->g, L, beta, out, coef, mode);
    CKL();
    return STAG_OK;
}

stag_status update_links(stag_ctx* ctx, const double* mom, double eps, stag_prec prec) {
    long long n = 8LL * ctx->g.Vh;
    if (prec == STAG_FP64)
        k_update_links<double, FMT_F64, 14><<<nblocks(n, FB), FB, 0, ctx->stream>>>(ctx->g, ctx->ghi, ctx->glo, mom,
                                                                                    eps);
    else
        k_update_links<float, FMT_F32_18, 8><<<nblocks(n, FB), FB, 0, ctx->stream>>>(ctx->g, ctx->ghi, ctx->glo, mom,
                                                                                     eps);
    CKL();
    ctx->b16_stale = true;
    ctx->asq_stale = true;
    return STAG_OK;
}

stag_status reunitarize(stag_ctx* ctx) {
    long long n = 8LL * ctx->g.Vh;
    k_reunitarize<<<nblocks(n, FB), FB, 0, ctx->stream>>>(ctx->g, ctx->ghi, ctx->glo);
    CKL();
    ctx->b16_stale = true;
    ctx->asq_stale = true;
    return STAG_OK;
}

stag_status plaquette_sum(stag_ctx* ctx, double* out) {
    long long n = 2LL * ctx->g.Vh;
    int nb = nblocks(n, FB);
    k_plaquette<<<nb, FB, 0, ctx->stream>>>(ctx->g, link_ptrs(ctx), ctx->red);
    CKL();
    return sum_partials(ctx, nb, out);
}

stag_status kinetic_sum(stag_ctx* ctx, const double* mom, double* out) {
    size_t n = (size_t)64 * ctx->g.Vh;
    int nb = 1024;
    k_sumsq<<<nb, 256, 0, ctx->stream>>>(n, mom, ctx->red);
    CKL();
    double s;
    CKS(sum_partials(ctx, nb, &s));
    *out = 0.5 * s;
    return STAG_OK;
}

stag_status mom_axpy(stag_ctx* ctx, double* mom, const double* f, double c) {
    size_t n = (size_t)64 * ctx->g.Vh;
    k_axpy_mom<<<nblocks((long long)n, 256), 256, 0, ctx->stream>>>(n, mom, f, c);
    CKL();
    return STAG_OK;
}

stag_status draw_momenta(stag_ctx* ctx, double* mom, unsigned long long seed, unsigned long long counter) {
    long long n = 4LL * ctx->g.V;
    k_draw_momenta<<<nblocks(n, 128), 128, 0, ctx->stream>>>(ctx->g, mom, seed, counter);
    CKL();
    return STAG_OK;
}

stag_status draw_sources(stag_ctx* ctx, double2* xi, int n, unsigned long long seed, unsigned long long counter,
                         int stream_base) {
    long long m = (long long)n * ctx->g.Vh;
    k_draw_sources<<<nblocks(m, 128), 128, 0, ctx->stream>>>(ctx->g, xi, n, seed, counter,
                                                              RNG_STREAM_SOURCES + (uint64_t)stream_base);
    CKL();
    return STAG_OK;
}

extern "C" stag_status stag_gauge_force(stag_ctx* ctx, double beta, double* force) {
    if (!ctx || !force) return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    return gauge_force_launch(ctx, STAG_FP64, beta, force, 1.0, 0);
}

extern "C" stag_status stag_plaquette(stag_ctx* ctx, double* plaq) {
    if (!ctx || !plaq) return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    double s;
    CKS(plaquette_sum(ctx, &s));
    *plaq = s / (18.0 * ctx->g.V);
    return STAG_OK;
}

extern "C" stag_status stag_draw_momenta(stag_ctx* ctx, unsigned long long seed, unsigned long long counter,
                                         double* mom) {
    if (!ctx || !mom) return STAG_ERR_ARG;
    return draw_momenta(ctx, mom, seed, counter);
}

extern "C" stag_status stag_draw_sources(stag_ctx* ctx, unsigned long long seed, unsigned long long counter,
                                         int stream, int n, void* xi) {
    if (!ctx || !xi || n < 1 || stream < 0) return STAG_ERR_ARG;
    return draw_sources(ctx, (double2*)xi, n, seed, counter, stream);
}
