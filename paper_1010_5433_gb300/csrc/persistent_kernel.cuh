// The persistent multi-shift CG kernel (Sec. 6; Jegerlehner's recurrences),
// instantiated per link format in persistent_<format>.cu: one
// cooperative launch runs the whole solve (convergence, max_iter or a NaN).
// Every iteration has three phases over the even/odd half lattices,
// separated by grid-wide barriers:
//   1  t = D_oe (r + beta p)                            (odd sites)
//   2  p = r + beta p;  q = c0 p - D_eo D_oe p;  (p, q)  (even sites)
//   3  r -= alpha q;  (r, r);  the deferred updates of the shifts whose window closes
// After phases 2 and 3 every block sums the per-block partials in the same
// fixed order and advances its own shared-memory copy of the scalar
// recurrences, so all blocks hold bit-identical scalars without a further
// barrier; block 0 writes them back to the device state when the loop ends.
// This replaces three kernel launches per iteration by three barriers, which
// is what small lattices (all data in L2) are limited by.
//
// Deferred shift updates.  The shifted directions and solutions follow
//   p_i <- zeta_i r + b_i p_i,   x_i <- x_i + a_i p_i
// once per iteration; neither feeds back into the base iteration.  Over a
// window of WIN iterations both are linear in the window's residuals
// r_0 .. r_{WIN-1} and in p_i, x_i at the window's start:
//   p_i = sum_l wp_l r_l + wd p_i(start),  x_i = x_i(start) + sum_l wx_l r_l + wf p_i(start)
// with scalar coefficients that the alpha step advances (the same algebra,
// reassociated).  The residuals of a window stay in a ring of WIN + 1
// fields, and p_i, x_i are read and written once per window instead of once
// per iteration: the 4 spinor passes per live shift of every iteration
// become 4 per window.  The windows are staggered: shift i's closes at the
// iterations k with (k + i) mod WIN = WIN - 1, so every iteration applies
// about n_shift / WIN of them, and phase 3 issues all its loads (r, q, the
// ring, those shifts' p_i and x_i) in one round trip to L2, which is what
// the phase waits on at these sizes.
//
// Mixed solves replace the residual inside the launch (Sec. 6 reliable
// updates): when ||r|| has fallen by the factor the host set, the fp32
// solutions are added into their fp64 accumulators and zeroed, and
// r = b - (m^2 + sigma_0 - D_eo D_oe) x_0 is recomputed from the fp64 base
// solution with the fp64 operator (float-float arithmetic on the two-float
// link store) in three further phases, without returning to the host.
//
// Every grid-barrier wait is bounded: after BAR_SPIN_LIMIT polls the block
// sets an error word, leaves the loop, and the host reports STAG_ERR_TIMEOUT.
#pragma once
#include <cmath>
#include <cstring>
#include <type_traits>

#include "internal.h"
#include "solver_state.cuh"
#include "grid_barrier.cuh"

namespace {

constexpr int WIN = 4;          // iterations per window of deferred shift updates
constexpr int RING = WIN + 1;   // residual fields kept: the window's and the next
constexpr int FG = 3;           // closing shifts per group of phase 3 (loads in flight vs registers)

// Block-local copy of the scalar recurrences (identical in every block), in
// float-float: the scalar warp advances them on the fp32 pipes (GB300's fp64
// pipe runs a warp's fp64 instruction at a small fraction of the fp32 rate,
// and a division is a dependent chain of them).  The device state keeps
// doubles; a launch converts them on entry and exit.  float-float carries a
// 48-bit significand, far below what the Krylov recurrences need.
struct Scal {
    DF zeta[STAG_MAX_RHS][STAG_MAX_SHIFTS], zeta_prev[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    DF zeta_next[STAG_MAX_RHS][STAG_MAX_SHIFTS], zratio[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    DF cx[STAG_MAX_RHS][STAG_MAX_SHIFTS], cpr[STAG_MAX_RHS][STAG_MAX_SHIFTS], cpp[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    DF dsig[STAG_MAX_SHIFTS];
    DF rr[STAG_MAX_RHS], bb[STAG_MAX_RHS], rr_ref[STAG_MAX_RHS];
    DF alpha[STAG_MAX_RHS], alpha_prev[STAG_MAX_RHS], beta_prev[STAG_MAX_RHS], beta[STAG_MAX_RHS];
    DF c0, tol2, delta2;
    double k4_units;
    int units[STAG_MAX_RHS];
    int live[STAG_MAX_RHS][STAG_MAX_SHIFTS], iters_at[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    int rhs_live[STAG_MAX_RHS], left[STAG_MAX_RHS];
    int k, halt, status, need_reliable, nrhs, nshift, max_iter, mixed, base, n_reliable;
    // the alpha step's shift ratio zeta_{k+1} / zeta_k = zF pq / (zE + zF pq), with
    // zF = zeta_{k-1} alpha_{k-1} and zE = (r, r) (beta_{k-1} (zeta_{k-1} - zeta_k)
    // + zF (sigma_i - sigma_0)) known before (p, A p): the ratio's division no
    // longer waits for alpha's; inv_rr = 1 / (r, r) serves the next beta step
    DF zE[STAG_MAX_RHS][STAG_MAX_SHIFTS], zF[STAG_MAX_RHS][STAG_MAX_SHIFTS], inv_rr[STAG_MAX_RHS];
    // deferred shift updates: shift s of source q has accumulated wj of its
    // window's iterations (shift index fastest: the lanes of a warp, one per
    // shift, touch consecutive words)
    DF wp[STAG_MAX_RHS][WIN][STAG_MAX_SHIFTS], wx[STAG_MAX_RHS][WIN][STAG_MAX_SHIFTS];
    DF wd[STAG_MAX_RHS][STAG_MAX_SHIFTS], wf[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    int touched[STAG_MAX_RHS][STAG_MAX_SHIFTS], wj[STAG_MAX_RHS][STAG_MAX_SHIFTS];
};

// a coefficient in the arithmetic of the iteration: the float part for fp32
// fields, the float-float pair for float-float fields (no conversion per thread)
template <typename R> __device__ __forceinline__ R coef(const DF& d);
template <> __device__ __forceinline__ float coef<float>(const DF& d) { return d.hi; }
template <> __device__ __forceinline__ DF coef<DF>(const DF& d) { return d; }

// float-float helpers of the scalar recurrences: conversions from and to
// double (integer operations in, one fp64 add out), a division by one
// correction step of the fp32 quotient (Dekker's long division), and sign tests
__device__ __forceinline__ DF dfv(double x) { return df_split(x); }
__device__ __forceinline__ double dbl(const DF& v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ DF df_div(const DF& a, const DF& b) {
    const float q1 = a.hi / b.hi;
    const DF r = a - b * DF(q1);
    const float q2 = r.hi / b.hi;
    return df_two_sum(q1, q2);
}
__device__ __forceinline__ bool df_le(const DF& a, const DF& b) { return (a - b).hi <= 0.f; }
__device__ __forceinline__ bool df_lt(const DF& a, const DF& b) { return (a - b).hi < 0.f; }
__device__ __forceinline__ bool df_finite(const DF& a) { return isfinite(a.hi); }

// shift s's window closes at iteration k
__device__ __forceinline__ bool window_closes(int k, int s) { return (k + s) % WIN == WIN - 1; }

__device__ void load_scal(Scal& S, const SolverState* st) {
    const int t = threadIdx.x;
    for (int i = t; i < STAG_MAX_RHS * STAG_MAX_SHIFTS; i += blockDim.x) {
        const int q = i / STAG_MAX_SHIFTS, s = i % STAG_MAX_SHIFTS;
        S.zeta[q][s] = dfv(st->zeta[q][s]);
        S.zeta_prev[q][s] = dfv(st->zeta_prev[q][s]);
        S.zeta_next[q][s] = dfv(st->zeta_next[q][s]);
        S.zratio[q][s] = dfv(st->zratio[q][s]);
        S.cx[q][s] = dfv(st->cx[q][s]);
        S.cpr[q][s] = dfv(st->cpr[q][s]);
        S.cpp[q][s] = dfv(st->cpp[q][s]);
        S.live[q][s] = st->live[q][s];
        S.iters_at[q][s] = st->iters_at[q][s];
    }
    if (t < STAG_MAX_SHIFTS) S.dsig[t] = dfv(st->dsig[t]);
    if (t < STAG_MAX_RHS) {
        S.rr[t] = dfv(st->rr[t]);
        S.bb[t] = dfv(st->bb[t]);
        S.rr_ref[t] = dfv(st->rr_ref[t]);
        S.alpha[t] = dfv(st->alpha[t]);
        S.alpha_prev[t] = dfv(st->alpha_prev[t]);
        S.beta_prev[t] = dfv(st->beta_prev[t]);
        S.beta[t] = dfv(st->beta[t]);
        S.rhs_live[t] = st->rhs_live[t];
    }
    if (t == 0) {
        S.k4_units = st->k4_units;
        S.c0 = dfv(st->c0);
        S.tol2 = dfv(st->tol2);
        S.delta2 = dfv(st->delta2);
        S.k = st->k;
        S.halt = st->halt;
        S.status = st->status;
        S.need_reliable = st->need_reliable;
        S.nrhs = st->nrhs;
        S.nshift = st->nshift;
        S.max_iter = st->max_iter;
        S.mixed = st->mixed;
        S.base = st->base;
        S.n_reliable = st->n_reliable;
    }
    __syncthreads();
}

__device__ void store_scal(const Scal& S, SolverState* st) {
    const int t = threadIdx.x;
    for (int i = t; i < STAG_MAX_RHS * STAG_MAX_SHIFTS; i += blockDim.x) {
        const int q = i / STAG_MAX_SHIFTS, s = i % STAG_MAX_SHIFTS;
        st->zeta[q][s] = dbl(S.zeta[q][s]);
        st->zeta_prev[q][s] = dbl(S.zeta_prev[q][s]);
        st->zeta_next[q][s] = dbl(S.zeta_next[q][s]);
        st->zratio[q][s] = dbl(S.zratio[q][s]);
        st->cx[q][s] = dbl(S.cx[q][s]);
        st->cpr[q][s] = dbl(S.cpr[q][s]);
        st->cpp[q][s] = dbl(S.cpp[q][s]);
        st->live[q][s] = S.live[q][s];
        st->iters_at[q][s] = S.iters_at[q][s];
    }
    if (t < STAG_MAX_RHS) {
        st->rr[t] = dbl(S.rr[t]);
        st->rr_ref[t] = dbl(S.rr_ref[t]);
        st->alpha[t] = dbl(S.alpha[t]);
        st->alpha_prev[t] = dbl(S.alpha_prev[t]);
        st->beta_prev[t] = dbl(S.beta_prev[t]);
        st->beta[t] = dbl(S.beta[t]);
        st->rhs_live[t] = S.rhs_live[t];
    }
    if (t == 0) {
        st->k4_units = S.k4_units;
        st->k = S.k;
        st->halt = S.halt;
        st->status = S.status;
        st->need_reliable = S.need_reliable;
        st->n_reliable = S.n_reliable;
    }
}

// An empty window for shift s of source q: p_i = p_i(start), x_i = x_i(start)
__device__ __forceinline__ void window_reset_one(Scal& S, int q, int s) {
#pragma unroll
    for (int l = 0; l < WIN; ++l) S.wp[q][l][s] = S.wx[q][l][s] = DF(0.f);
    S.wd[q][s] = DF(1.f);
    S.wf[q][s] = DF(0.f);
    S.touched[q][s] = 0;
    S.wj[q][s] = 0;
}
__device__ void window_reset(Scal& S) {
    for (int i = threadIdx.x; i < STAG_MAX_RHS * STAG_MAX_SHIFTS; i += blockDim.x)
        window_reset_one(S, i / STAG_MAX_SHIFTS, i % STAG_MAX_SHIFTS);
}

// zE, zF and 1 / (r, r) from the current recurrences (after every change of
// (r, r), zeta or alpha_prev): lane s of warp q for shift s of source q
__device__ void prep_alpha(Scal& S) {
    const int q = threadIdx.x >> 5, s = threadIdx.x & 31;
    if (q < S.nrhs && S.rhs_live[q]) {
        if (s < S.nshift) {
            const DF zf = S.zeta_prev[q][s] * S.alpha_prev[q];
            S.zF[q][s] = zf;
            S.zE[q][s] = S.rr[q] * (S.beta_prev[q] * (S.zeta_prev[q][s] - S.zeta[q][s]) + zf * S.dsig[s]);
        }
        if (s == 0) S.inv_rr[q] = df_div(DF(1.f), S.rr[q]);
    }
}


// Per-thread and per-warp sums of a block in float-float on the fp32 pipes
// (each thread's term is an fp32 or float-float dot product), the warps'
// sums then added in fp64 in a fixed order: the block's partial is an fp64
// sum without an fp64 operation per thread.  Result in thread 0.
template <typename R> __device__ __forceinline__ DF dot_df(const Vec3<R>& a, const Vec3<R>& b);
template <> __device__ __forceinline__ DF dot_df<float>(const Vec3<float>& a, const Vec3<float>& b) {
    DF s(0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s = s + DF(a.c[c].re) * DF(b.c[c].re);
        s = s + DF(a.c[c].im) * DF(b.c[c].im);
    }
    return s;
}
template <> __device__ __forceinline__ DF dot_df<DF>(const Vec3<DF>& a, const Vec3<DF>& b) {
    DF s(0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) s = s + a.c[c].re * b.c[c].re + a.c[c].im * b.c[c].im;
    return s;
}
template <int N>
__device__ __forceinline__ void block_sum_df(DF (&v)[N], double (&out)[N]) {
    __shared__ double sm[N][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] = v[k] + __shfl_xor_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sm[k][warp] = (double)v[k].hi + (double)v[k].lo;
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sm[k][w];
            out[k] = t;
        }
}

// Warp q of every block: the sum of source q's per-block fp64 partials
// partial[off + q][0..nb) in float-float (lane l adds the partials l, l + 32,
// ..., then a fixed butterfly), so every block gets the same bits.
__device__ __forceinline__ DF warp_partial_sum(const double* partial, int nb, int off, int q) {
    const int lane = threadIdx.x & 31;
    const double* p = partial + (size_t)(off + q) * nb;
    DF v(0.f);
    for (int i0 = lane; i0 < nb; i0 += 32 * 8) {
        double t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) t[k] = (i0 + 32 * k < nb) ? __ldcg(p + i0 + 32 * k) : 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (i0 + 32 * k < nb) v = v + dfv(t[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = v + __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// alpha = (r, r) / (p, A p) of every source and the shifted-system
// coefficients (Jegerlehner's zeta recurrence), warp q for source q with
// lane s for shift s (STAG_MAX_SHIFTS = 32); the shift's window coefficients
// take this iteration's update; one block barrier at the end
__device__ void alpha_step(Scal& S, const double* partial, int nb, int off, unsigned long long* fine) {
    static_assert(STAG_MAX_SHIFTS <= 32, "a lane per shift");
    const int q = threadIdx.x >> 5, s = threadIdx.x & 31;
    const int j = (q < STAG_MAX_RHS) ? S.wj[q][s] : 0;   // this iteration's place in the shift's window
    unsigned long long tf = fine ? gtimer() : 0;
    if (q < S.nrhs && S.rhs_live[q]) {
        const DF pq = warp_partial_sum(partial, nb, off, q);
        if (fine) {
            const unsigned long long t = gtimer();
            fine[0] += t - tf;
            tf = t;
        }
        DF a = df_div(S.rr[q], pq);
        const bool bad = !df_finite(a) || !(pq.hi > 0.f);
        if (bad) a = DF(0.f);
        if (s < S.nshift && S.live[q][s]) {
            // zeta_{k+1} / zeta_k = zeta_{k-1} alpha_{k-1} / (alpha beta_{k-1} (zeta_{k-1} - zeta_k)
            //   + zeta_{k-1} alpha_{k-1} (1 + alpha dsig)), numerator and denominator times pq / alpha
            const DF zfp = S.zF[q][s] * pq;
            const DF zr = df_div(zfp, S.zE[q][s] + zfp);
            const DF ax = bad ? DF(0.f) : a * zr;
            S.zeta_next[q][s] = S.zeta[q][s] * zr;
            S.zratio[q][s] = zr;
            S.cx[q][s] = ax;
            // p_i <- zeta r_j + b p_i;  x_i <- x_i + ax p_i  in window-coefficient form
            const DF b = S.cpp[q][s], zeta = S.cpr[q][s], axd = ax;
            DF wd = S.wd[q][s] * b, wf = S.wf[q][s];
#pragma unroll
            for (int l = 0; l < WIN; ++l) {
                if (l > j) break;
                const DF wp = l < j ? S.wp[q][l][s] * b : zeta;
                S.wp[q][l][s] = wp;
                S.wx[q][l][s] = S.wx[q][l][s] + axd * wp;
            }
            wf = wf + axd * wd;
            S.wd[q][s] = wd;
            S.wf[q][s] = wf;
            S.touched[q][s] = 1;
        }
        if (fine) {
            const unsigned long long t = gtimer();
            fine[1] += t - tf;
            tf = t;
        }
        if (s == 0) {
            S.alpha[q] = a;
            if (bad) {
                S.status = STAG_ERR_NAN;
                S.halt = 1;
            }
        }
    }
    if (q < S.nrhs && s < S.nshift) S.wj[q][s] = j + 1;   // every source's and shift's window counts the iteration
    __syncthreads();
    if (fine) fine[2] += gtimer() - tf;
}

// beta = (r', r') / (r, r), the shift coefficients of the next search
// directions, per-shift convergence and the solver's halt conditions; warp q
// for source q with lane s for shift s, then thread 0 for the whole solve
__device__ void beta_step(Scal& S, const double* partial, int nb, int off, unsigned long long* fine) {
    const int q = threadIdx.x >> 5, s = threadIdx.x & 31;
    const bool closed = window_closes(S.k, s);   // phase 3 has just applied shift s's window
    unsigned long long tf = fine ? gtimer() : 0;
    if (q < S.nrhs && S.rhs_live[q]) {
        const DF rn = warp_partial_sum(partial, nb, off, q);
        if (fine) {
            const unsigned long long t = gtimer();
            fine[3] += t - tf;
            tf = t;
        }
        const DF bt = rn * S.inv_rr[q];
        const bool on = s < S.nshift && S.live[q][s];
        const int n_live = __popc(__ballot_sync(0xffffffffu, on));
        bool still = false;
        if (on) {
            const DF zn = S.zeta_next[q][s], z = S.zeta[q][s];
            const DF zr = S.zratio[q][s];
            S.cpr[q][s] = zn;
            S.cpp[q][s] = bt * zr * zr;
            S.zeta_prev[q][s] = z;
            S.zeta[q][s] = zn;
            if (df_le(zn * zn * rn, S.tol2 * S.bb[q])) {
                S.live[q][s] = 0;
                S.iters_at[q][s] = S.k + 1;
            } else {
                still = true;
            }
        }
        const bool left = __ballot_sync(0xffffffffu, still) != 0;
        __syncwarp();
        if (s == 0) {
            if (!df_finite(rn)) {
                S.status = STAG_ERR_NAN;
                S.halt = 1;
            }
            S.units[q] = 72 + 96 * n_live;
            S.beta[q] = bt;
            S.alpha_prev[q] = S.alpha[q];
            S.beta_prev[q] = bt;
            S.rr[q] = rn;
            S.left[q] = left;
            if (!left) S.rhs_live[q] = 0;
            else if (S.mixed && df_lt(rn, S.delta2 * S.rr_ref[q])) S.need_reliable = 1;
        }
    } else if (q < S.nrhs && s == 0) {
        S.left[q] = 0;
        S.units[q] = 0;
    }
    // the warp's own entries, before the block waits: its closed windows
    // reset, and zE, zF, 1 / (r, r) of the next alpha step from what lane 0
    // has just written
    __syncwarp();
    if (closed && q < STAG_MAX_RHS) window_reset_one(S, q, s);
    prep_alpha(S);
    __syncthreads();
    if (fine) {
        const unsigned long long t = gtimer();
        fine[4] += t - tf;
        tf = t;
    }
    if (threadIdx.x == 0) {
        int any = 0;
        int units = 0;
        for (int j = 0; j < S.nrhs; ++j) {
            any |= S.left[j];
            units += S.units[j];
        }
        S.k4_units += (double)units;
        S.k += 1;
        if (!any) S.halt = 1;
        else if (S.k >= S.max_iter) { S.halt = 1; S.status = STAG_ERR_NOT_CONVERGED; }
    }
    __syncthreads();
    if (fine) fine[5] += gtimer() - tf;
}

// p_i and x_i of shift s of source j at site h from its window's
// coefficients and the window's n residuals rl[0..n) (rl[l] = r_{k0 + l})
template <typename R>
__device__ __forceinline__ void window_apply(const Scal& S, int j, int s, int n, const Vec3<R> (&rl)[WIN],
                                             Vec3<R>& pv, Vec3<R>& xv) {
    const R wd = coef<R>(S.wd[j][s]), wf = coef<R>(S.wf[j][s]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xv.c[c].re += wf * pv.c[c].re;
        xv.c[c].im += wf * pv.c[c].im;
        pv.c[c].re = wd * pv.c[c].re;
        pv.c[c].im = wd * pv.c[c].im;
    }
#pragma unroll
    for (int l = 0; l < WIN; ++l) {
        // past the shift's last update in the window the coefficients are zero,
        // and for a source that stopped the ring slot may never have been written
        if (l >= n || (S.wp[j][l][s].hi == 0.f && S.wx[j][l][s].hi == 0.f)) continue;
        const R cp = coef<R>(S.wp[j][l][s]), cx = coef<R>(S.wx[j][l][s]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pv.c[c].re += cp * rl[l].c[c].re;
            pv.c[c].im += cp * rl[l].c[c].im;
            xv.c[c].re += cx * rl[l].c[c].re;
            xv.c[c].im += cx * rl[l].c[c].im;
        }
    }
}

// Phase 3's share of the deferred updates at site h, source j, iteration k:
// the shifts whose window closes now (s = c, c + WIN, ...), whose windows
// all end at r_k (rk, already loaded) and begin at most WIN - 1 iterations
// earlier.  The older residuals and FG shifts' p_i, x_i are loaded together.
template <typename R>
__device__ __forceinline__ void flush_closing(const Scal& S, int j, int ns, size_t rs, int h, int Vh,
                                              const typename V2T<R>::T* ring, size_t rstride, int k,
                                              const Vec3<R>& rk, typename V2T<R>::T* __restrict__ ps,
                                              typename V2T<R>::T* __restrict__ x) {
    const int c0 = (2 * WIN - 1 - k % WIN) % WIN;     // the first closing shift
    if (c0 >= ns) return;
    // rl[l] = r_{k - (WIN - 1) + l}: the last WIN residuals (a shorter window uses the tail)
    Vec3<R> rl[WIN];
#pragma unroll
    for (int l = 0; l < WIN - 1; ++l) {
        const int it = k - (WIN - 1) + l;
        if (it >= 0) rl[l] = load_vec_cg<R>(ring + (size_t)(it % RING) * rstride + (size_t)j * rs, h, Vh);
        else zero(rl[l]);
    }
    rl[WIN - 1] = rk;
    for (int s0 = c0; s0 < ns; s0 += FG * WIN) {
        Vec3<R> pv[FG], xv[FG];
        bool on[FG];
#pragma unroll
        for (int u = 0; u < FG; ++u) {
            const int s = s0 + u * WIN;
            on[u] = s < ns && S.touched[j][s];
            if (on[u]) {
                pv[u] = load_vec_cg<R>(ps + ((size_t)j * ns + s) * rs, h, Vh);
                xv[u] = load_vec_cg<R>(x + ((size_t)j * ns + s) * rs, h, Vh);
            }
        }
#pragma unroll
        for (int u = 0; u < FG; ++u) {
            if (!on[u]) continue;
            const int s = s0 + u * WIN;
            const int n = S.wj[j][s];
            // the window's residuals r_{k-n+1} .. r_k sit at the end of rl
            Vec3<R> rw[WIN];
#pragma unroll
            for (int l = 0; l < WIN; ++l) {
                if (l < n) rw[l] = rl[WIN - n + l];
                else zero(rw[l]);
            }
            window_apply<R>(S, j, s, n, rw, pv[u], xv[u]);
            store_vec<R>(x + ((size_t)j * ns + s) * rs, h, Vh, xv[u]);
            store_vec<R>(ps + ((size_t)j * ns + s) * rs, h, Vh, pv[u]);
        }
    }
}

// fp64 data of the in-launch reliable updates (mixed solves)
struct RelPtrs {
    const double2* b64;   // [rhs][3][Vh]   the right-hand sides
    double2* x64;         // [rhs][shift][3][Vh]  fp64 accumulators of the solutions
    double2* t64;         // [rhs][3][Vh]   D_oe x_0 (odd sites)
};

// every pending window's updates at every site of the block (the loop
// ended, or a reliable update follows), then empty windows; S.k counts
// the iterations done, so a window of n iterations began at S.k - n
template <typename R>
__device__ __noinline__ void flush_block(Scal& S, int h0, int h1, int PB, size_t rs, int Vh,
                                         const typename V2T<R>::T* ring, size_t rstride, typename V2T<R>::T* ps,
                                         typename V2T<R>::T* x) {
    for (int h = h0 + (int)threadIdx.x; h < h1; h += PB)
        for (int j = 0; j < S.nrhs; ++j)
            for (int s = 0; s < S.nshift; ++s) {
                const int n = S.wj[j][s];
                if (!S.touched[j][s] || n == 0) continue;
                Vec3<R> rl[WIN];
#pragma unroll
                for (int l = 0; l < WIN; ++l) {
                    if (l < n) rl[l] = load_vec_cg<R>(ring + (size_t)((S.k - n + l) % RING) * rstride + (size_t)j * rs,
                                                      h, Vh);
                    else zero(rl[l]);
                }
                Vec3<R> pv = load_vec_cg<R>(ps + ((size_t)j * S.nshift + s) * rs, h, Vh);
                Vec3<R> xv = load_vec_cg<R>(x + ((size_t)j * S.nshift + s) * rs, h, Vh);
                window_apply<R>(S, j, s, n, rl, pv, xv);
                store_vec<R>(x + ((size_t)j * S.nshift + s) * rs, h, Vh, xv);
                store_vec<R>(ps + ((size_t)j * S.nshift + s) * rs, h, Vh, pv);
            }
    __syncthreads();
    window_reset(S);
    __syncthreads();
}

// The in-launch reliable update of a mixed solve, after the beta step that
// asked for it: the pending window's updates, x64_i += x_i and x_i = 0 for
// every shift, t = D_oe x64_0 (odd sites), r = b - (c0 x64_0 - 1/4 D_eo t)
// with fp64 sums (even sites), (r, r) = rr = rr_ref.  Three grid barriers.
// The fp64 operator runs in float-float on the two-float link store, as the
// standalone fp64 A does.  false if a barrier wait gave up.
template <typename R, bool ASQ>
__device__ __noinline__ bool reliable_update(Scal& S, GridSync& gs, const Geom& g, const LinkPtrs& L, const AsqLinks& A,
                                int h0, int h1, int PB,
                                typename V2T<R>::T* ring, size_t rstride, typename V2T<R>::T* ps,
                                typename V2T<R>::T* x, const RelPtrs& rp, double* partial, unsigned int nb) {
    const size_t rs = (size_t)3 * g.Vh;
    const int nrhs = S.nrhs, ns = S.nshift;
    flush_block<R>(S, h0, h1, PB, rs, g.Vh, ring, rstride, ps, x);
    // R1: x64_i += x_i, x_i = 0 (the shifts of every source still iterating)
    for (int h = h0 + (int)threadIdx.x; h < h1; h += PB)
        for (int j = 0; j < nrhs; ++j) {
            if (!S.rhs_live[j]) continue;
            for (int s = 0; s < ns; ++s) {
                const size_t off = ((size_t)j * ns + s) * rs;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const size_t i = off + (size_t)c * g.Vh + h;
                    const float2 a = ((const float2*)x)[i];
                    double2 d = rp.x64[i];
                    d.x += (double)a.x;
                    d.y += (double)a.y;
                    rp.x64[i] = d;
                    ((float2*)x)[i] = make_float2(0.f, 0.f);
                }
            }
        }
    if (!grid_sync(gs)) return false;
    // R2: t = 1/2 hops of x64_0 (odd sites)
    for (int h = h0 + (int)threadIdx.x; h < h1; h += PB)
        for (int j = 0; j < nrhs; ++j) {
            if (!S.rhs_live[j]) continue;
            SrcD2DFcg src{rp.x64 + ((size_t)j * ns + S.base) * rs};
            Vec3<DF> acc[1];
            if constexpr (ASQ) dslash_site_asq<DF, FMT_F64, 1, 1>(g, 1, A, src, 0, 1, h, 0, acc);
            else dslash_site<DF, FMT_F64, 1, 1>(g, 1, L, src, 0, 1, h, 0, acc);
            double2* o = rp.t64 + (size_t)j * rs;
            const DF half(0.5f);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                o[(size_t)c * g.Vh + h] = make_double2(df_join(half * acc[0].c[c].re), df_join(half * acc[0].c[c].im));
        }
    if (!grid_sync(gs)) return false;
    // R3: r = b - (c0 x_0 - 1/2 hops of t) (even sites), (r, r)
    double nrm[STAG_MAX_RHS];
#pragma unroll
    for (int j = 0; j < STAG_MAX_RHS; ++j) nrm[j] = 0.0;
    const DF c0 = S.c0, half(0.5f);
    typename V2T<R>::T* rcur = ring + (size_t)(S.k % RING) * rstride;
    for (int h = h0 + (int)threadIdx.x; h < h1; h += PB)
#pragma unroll
        for (int j = 0; j < STAG_MAX_RHS; ++j) {
            if (j >= nrhs || !S.rhs_live[j]) continue;
            SrcD2DFcg src{rp.t64 + (size_t)j * rs};
            Vec3<DF> acc[1];
            if constexpr (ASQ) dslash_site_asq<DF, FMT_F64, 1, 1>(g, 0, A, src, 0, 1, h, 0, acc);
            else dslash_site<DF, FMT_F64, 1, 1>(g, 0, L, src, 0, 1, h, 0, acc);
            const double2* xb = rp.x64 + ((size_t)j * ns + S.base) * rs;
            const double2* bb = rp.b64 + (size_t)j * rs;
            float2* ro = (float2*)rcur + (size_t)j * rs;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t i = (size_t)c * g.Vh + h;
                const double2 xd = xb[i], bd = bb[i];
                const double ar = df_join(c0 * df_split(xd.x) - half * acc[0].c[c].re);
                const double ai = df_join(c0 * df_split(xd.y) - half * acc[0].c[c].im);
                const double re = bd.x - ar, im = bd.y - ai;
                ro[i] = make_float2((float)re, (float)im);
                nrm[j] += re * re + im * im;
            }
        }
    block_sum<STAG_MAX_RHS>(nrm);
    if (threadIdx.x == 0)
        for (int j = 0; j < nrhs; ++j) partial[(size_t)(2 * STAG_MAX_RHS + j) * nb + blockIdx.x] = nrm[j];
    if (!grid_sync(gs)) return false;
    {
        const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (q < nrhs && S.rhs_live[q]) {
            const DF rr = warp_partial_sum(partial, nb, 2 * STAG_MAX_RHS, q);
            if (lane == 0) {
                S.rr[q] = rr;
                S.rr_ref[q] = rr;
                if (!df_finite(rr)) {
                    S.status = STAG_ERR_NAN;
                    S.halt = 1;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        S.need_reliable = 0;
        S.n_reliable += 1;
    }
    __syncthreads();
    prep_alpha(S);
    __syncthreads();
    return true;
}

// ASQ: the improved operator (asqtad.cuh): every hop through the fat link
// plus a third-neighbour hop through the Naik link, A holding both stores.
// NRP: sources per pass of the Dslash phases; ND: sources the per-thread sums
// and the update phase cover (1 and 1 for one source, 2 and 2 for two -- a
// flavour split over two pseudo-fermions --, 4 and STAG_MAX_RHS otherwise);
// PB: threads per block.  r is a ring of RING residual fields, rstride
// elements apart.
template <typename R, int FMT, bool ASQ, int NRP, int ND, int PB>
__global__ void __launch_bounds__(PB) k_ms_persistent(Geom g, LinkPtrs L, AsqLinks A, SolverState* st,
                                                      typename V2T<R>::T* ring, size_t rstride,
                                                      typename V2T<R>::T* p, typename V2T<R>::T* q,
                                                      typename V2T<R>::T* t, typename V2T<R>::T* ps,
                                                      typename V2T<R>::T* x, RelPtrs rp,
                                                      double* partial, GridBar* bar, unsigned long long* ptime) {
    typedef typename V2T<R>::T V;
    static_assert(PB >= 32 * STAG_MAX_RHS, "the reductions take a warp per source");
    __shared__ Scal S;
    // profiling: block 0 accumulates ns spent in phase 1, barrier 1, phase 2,
    // barrier 2, alpha step, phase 3, barrier 3, beta step, reliable updates
    const bool timing = ptime && blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long tp[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, t_last = timing ? gtimer() : 0;
    // inside the scalar steps: partial sums, alpha arithmetic, block barrier; partial sums,
    // beta arithmetic, thread 0 and window resets
    unsigned long long fine[6] = {0, 0, 0, 0, 0, 0};
#define PHASE_MARK(i)                               \
    if (timing) {                                   \
        unsigned long long t_now = gtimer();        \
        tp[i] += t_now - t_last;                    \
        t_last = t_now;                             \
    }
    load_scal(S, st);
    window_reset(S);
    __syncthreads();
    prep_alpha(S);
    __syncthreads();
    const unsigned int nb = gridDim.x;
    GridSync gs{bar, nb, 0u};
    // this block's sites: a contiguous range, the half lattice split evenly
    // over the grid in multiples of 8 sites (a 32-byte sector of an fp32
    // field component), so every block of the grid has work
    const int per = (int)((((size_t)g.Vh + nb - 1) / nb + 7) & ~(size_t)7);
    const int h0 = min(g.Vh, (int)blockIdx.x * per), h1 = min(g.Vh, h0 + per);
    const size_t rs = (size_t)3 * g.Vh;
    const int nrhs = S.nrhs, ns = S.nshift;
    static_assert(ND % NRP == 0 && ND <= STAG_MAX_RHS, "sources per pass divide the sources covered");
    // float-float hops are long (compensated products): unrolled over the four
    // directions the kernel outgrows the instruction cache, so they loop
    // (and so do the improved operator's sixteen hops)
    constexpr int MU_UNROLL = (std::is_same<R, DF>::value || ASQ) ? 1 : 4;
    bool ok = true;
    while (!S.halt && ok) {
        const V* r = ring + (size_t)(S.k % RING) * rstride;          // r_k
        V* r_next = ring + (size_t)((S.k + 1) % RING) * rstride;     // r_{k+1}
        // ---- phase 1: t = D_oe (r + beta p), without the 1/2
        for (int h = h0 + (int)threadIdx.x; h < h1; h += PB) {
            Nbr n;
            site_neighbours(g, h, 1, n);
            Nbr3 m3;
            if constexpr (ASQ) site_neighbours3(g, n, m3);
            for (int r0 = 0; r0 < nrhs; r0 += NRP) {
                Vec3<R> acc[NRP];
                R bt[NRP];
#pragma unroll
                for (int j = 0; j < NRP; ++j) {
                    zero(acc[j]);
                    bt[j] = (r0 + j < nrhs) ? coef<R>(S.beta[r0 + j]) : (R)0;
                }
#pragma unroll MU_UNROLL
                for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
                    for (int dir = 0; dir < 2; ++dir) {
#pragma unroll
                        for (int hop = 0; hop < (ASQ ? 2 : 1); ++hop) {
                        const int nb_h = hop == 0 ? (dir == 0 ? n.fwd[mu] : n.bwd[mu]) : (dir == 0 ? m3.fwd[mu] : m3.bwd[mu]);
                        const LinkPtrs& LH = ASQ ? (hop == 0 ? A.fat : A.lng) : L;
                        Su3<R> u = dir == 0 ? LinkFetch<R, FMT>::get(LH, mu, 1, h, g.Vh)
                                            : LinkFetch<R, FMT>::get(LH, mu, 0, nb_h, g.Vh);
                        const float sgn = hop == 0 ? (dir == 0 ? n.sf[mu] : -n.sb[mu]) : (dir == 0 ? m3.sf[mu] : -m3.sb[mu]);
#pragma unroll
                        for (int j = 0; j < NRP; ++j) {
                            if (r0 + j >= nrhs) continue;
                            const size_t off = (size_t)(r0 + j) * rs;
                            Vec3<R> a = load_vec_cg<R>(r + off, nb_h, g.Vh);
                            Vec3<R> b = load_vec_cg<R>(p + off, nb_h, g.Vh);
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                a.c[c].re += bt[j] * b.c[c].re;
                                a.c[c].im += bt[j] * b.c[c].im;
                            }
                            if (dir == 0) mac_uv(acc[j], (R)sgn, u, a);
                            else mac_udv(acc[j], (R)sgn, u, a);
                        }
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < NRP; ++j)
                    if (r0 + j < nrhs) store_vec<R>(t + (size_t)(r0 + j) * rs, h, g.Vh, acc[j]);
            }
        }
        PHASE_MARK(0)
        if (!(ok = grid_sync(gs))) break;
        PHASE_MARK(1)
        // ---- phase 2: p = r + beta p; q = c0 p - 1/4 (hops of t); (p, q)
        DF dots[ND];
#pragma unroll
        for (int j = 0; j < ND; ++j) dots[j] = DF(0.f);
        const R c0 = coef<R>(S.c0);
        for (int h = h0 + (int)threadIdx.x; h < h1; h += PB) {
            Nbr n;
            site_neighbours(g, h, 0, n);
            Nbr3 m3;
            if constexpr (ASQ) site_neighbours3(g, n, m3);
#pragma unroll
            for (int r0 = 0; r0 < ND; r0 += NRP) {
                if (r0 >= nrhs) break;
                Vec3<R> acc[NRP];
#pragma unroll
                for (int j = 0; j < NRP; ++j) zero(acc[j]);
#pragma unroll MU_UNROLL
                for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
                    for (int dir = 0; dir < 2; ++dir) {
#pragma unroll
                        for (int hop = 0; hop < (ASQ ? 2 : 1); ++hop) {
                        const int nb_h = hop == 0 ? (dir == 0 ? n.fwd[mu] : n.bwd[mu]) : (dir == 0 ? m3.fwd[mu] : m3.bwd[mu]);
                        const LinkPtrs& LH = ASQ ? (hop == 0 ? A.fat : A.lng) : L;
                        Su3<R> u = dir == 0 ? LinkFetch<R, FMT>::get(LH, mu, 0, h, g.Vh)
                                            : LinkFetch<R, FMT>::get(LH, mu, 1, nb_h, g.Vh);
                        const float sgn = hop == 0 ? (dir == 0 ? n.sf[mu] : -n.sb[mu]) : (dir == 0 ? m3.sf[mu] : -m3.sb[mu]);
#pragma unroll
                        for (int j = 0; j < NRP; ++j) {
                            if (r0 + j >= nrhs) continue;
                            Vec3<R> a = load_vec_cg<R>(t + (size_t)(r0 + j) * rs, nb_h, g.Vh);
                            if (dir == 0) mac_uv(acc[j], (R)sgn, u, a);
                            else mac_udv(acc[j], (R)sgn, u, a);
                        }
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < NRP; ++j) {
                    if (r0 + j >= nrhs) continue;
                    const size_t off = (size_t)(r0 + j) * rs;
                    const R bt = coef<R>(S.beta[r0 + j]);
                    Vec3<R> pv = load_vec_cg<R>(p + off, h, g.Vh);
                    Vec3<R> rv = load_vec_cg<R>(r + off, h, g.Vh);
                    Vec3<R> o;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        pv.c[c].re = rv.c[c].re + bt * pv.c[c].re;
                        pv.c[c].im = rv.c[c].im + bt * pv.c[c].im;
                        o.c[c].re = c0 * pv.c[c].re - (R)0.25 * acc[j].c[c].re;
                        o.c[c].im = c0 * pv.c[c].im - (R)0.25 * acc[j].c[c].im;
                    }
                    store_vec<R>(p + off, h, g.Vh, pv);
                    store_vec<R>(q + off, h, g.Vh, o);
                    dots[r0 + j] = dots[r0 + j] + dot_df<R>(pv, o);
                }
            }
        }
        double dsum[ND];
        block_sum_df<ND>(dots, dsum);
        if (threadIdx.x == 0)
            for (int j = 0; j < nrhs && j < ND; ++j) partial[(size_t)j * nb + blockIdx.x] = dsum[j];
        PHASE_MARK(2)
        if (!(ok = grid_sync(gs))) break;
        PHASE_MARK(3)
        alpha_step(S, partial, nb, 0, timing ? fine : nullptr);
        PHASE_MARK(4)
        // ---- phase 3: r_{k+1} = r_k - alpha q with (r, r); the closing windows' shift updates
        DF nrm[ND];
#pragma unroll
        for (int j = 0; j < ND; ++j) nrm[j] = DF(0.f);
        for (int h = h0 + (int)threadIdx.x; h < h1; h += PB) {
#pragma unroll
            for (int j = 0; j < ND; ++j) {
                if (j >= nrhs) continue;
                const bool live = S.rhs_live[j];
                const size_t off = (size_t)j * rs;
                Vec3<R> rv = load_vec_cg<R>(r + off, h, g.Vh);
                Vec3<R> qv;
                if (live) qv = load_vec_cg<R>(q + off, h, g.Vh);
                // a source that stopped still owes its shifts' pending updates
                flush_closing<R>(S, j, ns, rs, h, g.Vh, ring, rstride, S.k, rv, ps, x);
                if (!live) continue;
                const R a = coef<R>(S.alpha[j]);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    rv.c[c].re -= a * qv.c[c].re;
                    rv.c[c].im -= a * qv.c[c].im;
                }
                store_vec<R>(r_next + off, h, g.Vh, rv);
                nrm[j] = nrm[j] + dot_df<R>(rv, rv);
            }
        }
        double nsum[ND];
        block_sum_df<ND>(nrm, nsum);
        if (threadIdx.x == 0)
            for (int j = 0; j < nrhs && j < ND; ++j) partial[(size_t)(STAG_MAX_RHS + j) * nb + blockIdx.x] = nsum[j];
        PHASE_MARK(5)
        if (!(ok = grid_sync(gs))) break;
        PHASE_MARK(6)
        beta_step(S, partial, nb, STAG_MAX_RHS, timing ? fine : nullptr);
        PHASE_MARK(7)
        if constexpr (std::is_same<R, float>::value) {
            if (S.need_reliable && !S.halt) {
                ok = reliable_update<R, ASQ>(S, gs, g, L, A, h0, h1, PB, ring, rstride, ps, x, rp, partial, nb);
                PHASE_MARK(8)
            }
        }
    }
#undef PHASE_MARK
    if (ok) flush_block<R>(S, h0, h1, PB, rs, g.Vh, ring, rstride, ps, x);
    if (timing) {
        for (int i = 0; i < 9; ++i) ptime[24 + i] += tp[i];
        for (int i = 0; i < 6; ++i) ptime[33 + i] += fine[i];
    }
    if (!ok && threadIdx.x == 0) {
        S.halt = 1;
        S.status = STAG_ERR_TIMEOUT;
    }
    __syncthreads();
    if (blockIdx.x == 0) store_scal(S, st);
}

template <typename R, int FMT, bool ASQ, int NRP, int ND, int PB>
stag_status launch_persistent_pb(stag_ctx* ctx, void* ring, size_t rstride, void* p, void* q, void* t, void* ps,
                                 void* x, RelPtrs rp) {
    typedef typename V2T<R>::T V;
    auto kern = k_ms_persistent<R, FMT, ASQ, NRP, ND, PB>;
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PB, 0));
    if (per_sm < 1) return STAG_ERR_ARG;
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // one site per thread where the lattice allows (or at least persist_sites
    // sites per block), never more blocks than co-reside
    const long long spb = ctx->persist_sites > 0 ? ctx->persist_sites : PB;
    long long want = ((long long)ctx->g.Vh + spb - 1) / spb;
    long long cap = (long long)nsm * per_sm;
    int grid = (int)(want < cap ? want : cap);
    if (grid < 1) grid = 1;
    // partial sums: (p, A p), (r, r) and the reliable update's (r, r), per source and block
    if ((size_t)3 * STAG_MAX_RHS * grid > ctx->red_doubles) return STAG_ERR_ARG;
    CK(cudaMemsetAsync(ctx->bar, 0, sizeof(GridBar), ctx->stream));
    Geom g = ctx->g;
    LinkPtrs L = link_ptrs(ctx);
    AsqLinks A{};
    if (ASQ) A = asq_links(ctx);
    SolverState* st = ctx->st;
    V *vr = (V*)ring, *vp = (V*)p, *vq = (V*)q, *vt = (V*)t, *vps = (V*)ps, *vx = (V*)x;
    double* part = ctx->red;
    GridBar* bar = (GridBar*)ctx->bar;
    unsigned long long* pt = ctx->prof.on ? (unsigned long long*)ctx->ptime : nullptr;
    void* args[] = {&g, &L, &A, &st, &vr, &rstride, &vp, &vq, &vt, &vps, &vx, &rp, &part, &bar, &pt};
    CK(cudaLaunchCooperativeKernel((const void*)kern, grid, PB, args, 0, ctx->stream));
    ++ctx->launches;
    return STAG_OK;
}
// One link format's solve: the kernel variant by the number of sources
template <typename R, int FMT, bool ASQ = false>
stag_status launch_persistent_fmt(stag_ctx* ctx, int nrhs, void* ring, size_t rstride, void* p, void* q, void* t,
                                  void* ps, void* x, const double2* b64, double2* x64, double2* t64) {
    RelPtrs rp{b64, x64, t64};
    // 256 threads per block: one block per SM at these register counts
    if (nrhs == 1) return launch_persistent_pb<R, FMT, ASQ, 1, 1, 256>(ctx, ring, rstride, p, q, t, ps, x, rp);
    if (nrhs == 2) return launch_persistent_pb<R, FMT, ASQ, 2, 2, 256>(ctx, ring, rstride, p, q, t, ps, x, rp);
    return launch_persistent_pb<R, FMT, ASQ, 4, STAG_MAX_RHS, 256>(ctx, ring, rstride, p, q, t, ps, x, rp);
}
}  // namespace
