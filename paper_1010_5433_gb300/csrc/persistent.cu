// Persistent multi-shift CG (Sec. 6; Jegerlehner's recurrences): one
// cooperative launch runs solver iterations until the solve halts
// (convergence, a due reliable update, max_iter or a NaN).  Every iteration
// has three phases over the even/odd half lattices, separated by grid-wide
// barriers:
//   1  t = D_oe (r + beta p)                            (odd sites)
//   2  p = r + beta p;  q = c0 p - D_eo D_oe p;  (p, q)  (even sites)
//   3  p_i = zeta r + beta_i p_i;  x_i += alpha_i p_i;  r -= alpha q;  (r, r)
// After phases 2 and 3 every block sums the per-block partials in the same
// fixed order and advances its own shared-memory copy of the scalar
// recurrences, so all blocks hold bit-identical scalars without a further
// barrier; block 0 writes them back to the device state when the loop ends.
// This replaces three kernel launches per iteration by three barriers, which
// is what small lattices (all data in L2) are limited by.
//
// Every grid-barrier wait is bounded: after BAR_SPIN_LIMIT polls the block
// sets an error word, leaves the loop, and the host reports STAG_ERR_TIMEOUT.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "internal.h"
#include "solver_state.cuh"
#include "grid_barrier.cuh"

namespace {

// Block-local copy of the scalar recurrences (identical in every block).
struct Scal {
    double zeta[STAG_MAX_RHS][STAG_MAX_SHIFTS], zeta_prev[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    double zeta_next[STAG_MAX_RHS][STAG_MAX_SHIFTS], zratio[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    double cx[STAG_MAX_RHS][STAG_MAX_SHIFTS], cpr[STAG_MAX_RHS][STAG_MAX_SHIFTS], cpp[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    double dsig[STAG_MAX_SHIFTS];
    double rr[STAG_MAX_RHS], bb[STAG_MAX_RHS], rr_ref[STAG_MAX_RHS];
    double alpha[STAG_MAX_RHS], alpha_prev[STAG_MAX_RHS], beta_prev[STAG_MAX_RHS], beta[STAG_MAX_RHS];
    double sums[STAG_MAX_RHS], units[STAG_MAX_RHS];
    double k4_units, c0, tol2, delta2;
    int live[STAG_MAX_RHS][STAG_MAX_SHIFTS], iters_at[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    int rhs_live[STAG_MAX_RHS], left[STAG_MAX_RHS];
    int k, halt, status, need_reliable, nrhs, nshift, max_iter, mixed;
};

__device__ void load_scal(Scal& S, const SolverState* st) {
    const int t = threadIdx.x;
    for (int i = t; i < STAG_MAX_RHS * STAG_MAX_SHIFTS; i += blockDim.x) {
        const int q = i / STAG_MAX_SHIFTS, s = i % STAG_MAX_SHIFTS;
        S.zeta[q][s] = st->zeta[q][s];
        S.zeta_prev[q][s] = st->zeta_prev[q][s];
        S.zeta_next[q][s] = st->zeta_next[q][s];
        S.cx[q][s] = st->cx[q][s];
        S.cpr[q][s] = st->cpr[q][s];
        S.cpp[q][s] = st->cpp[q][s];
        S.live[q][s] = st->live[q][s];
        S.iters_at[q][s] = st->iters_at[q][s];
    }
    if (t < STAG_MAX_SHIFTS) S.dsig[t] = st->dsig[t];
    if (t < STAG_MAX_RHS) {
        S.rr[t] = st->rr[t];
        S.bb[t] = st->bb[t];
        S.rr_ref[t] = st->rr_ref[t];
        S.alpha[t] = st->alpha[t];
        S.alpha_prev[t] = st->alpha_prev[t];
        S.beta_prev[t] = st->beta_prev[t];
        S.beta[t] = st->beta[t];
        S.rhs_live[t] = st->rhs_live[t];
    }
    if (t == 0) {
        S.k4_units = st->k4_units;
        S.c0 = st->c0;
        S.tol2 = st->tol2;
        S.delta2 = st->delta2;
        S.k = st->k;
        S.halt = st->halt;
        S.status = st->status;
        S.need_reliable = st->need_reliable;
        S.nrhs = st->nrhs;
        S.nshift = st->nshift;
        S.max_iter = st->max_iter;
        S.mixed = st->mixed;
    }
    __syncthreads();
}

__device__ void store_scal(const Scal& S, SolverState* st) {
    const int t = threadIdx.x;
    for (int i = t; i < STAG_MAX_RHS * STAG_MAX_SHIFTS; i += blockDim.x) {
        const int q = i / STAG_MAX_SHIFTS, s = i % STAG_MAX_SHIFTS;
        st->zeta[q][s] = S.zeta[q][s];
        st->zeta_prev[q][s] = S.zeta_prev[q][s];
        st->zeta_next[q][s] = S.zeta_next[q][s];
        st->cx[q][s] = S.cx[q][s];
        st->cpr[q][s] = S.cpr[q][s];
        st->cpp[q][s] = S.cpp[q][s];
        st->live[q][s] = S.live[q][s];
        st->iters_at[q][s] = S.iters_at[q][s];
    }
    if (t < STAG_MAX_RHS) {
        st->rr[t] = S.rr[t];
        st->alpha[t] = S.alpha[t];
        st->alpha_prev[t] = S.alpha_prev[t];
        st->beta_prev[t] = S.beta_prev[t];
        st->beta[t] = S.beta[t];
        st->rhs_live[t] = S.rhs_live[t];
    }
    if (t == 0) {
        st->k4_units = S.k4_units;
        st->k = S.k;
        st->halt = S.halt;
        st->status = S.status;
        st->need_reliable = S.need_reliable;
    }
}

// Warp q of every block: the sum of source q's per-block partials
// partial[off + q][0..nb) (lane l adds the partials l, l + 32, ..., then a
// fixed shuffle tree), so every block gets the same bits, broadcast to the
// warp's lanes.
__device__ __forceinline__ double warp_partial_sum(const double* partial, int nb, int off, int q) {
    const int lane = threadIdx.x & 31;
    double v = lane_strided_sum(partial + (size_t)(off + q) * nb, nb, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// alpha = (r, r) / (p, A p) of every source and the shifted-system
// coefficients (Jegerlehner's zeta recurrence), warp q for source q with
// lane s for shift s (STAG_MAX_SHIFTS = 32), one block barrier at the end
__device__ void alpha_step(Scal& S, const double* partial, int nb, int off) {
    static_assert(STAG_MAX_SHIFTS <= 32, "a lane per shift");
    const int q = threadIdx.x >> 5, s = threadIdx.x & 31;
    if (q < S.nrhs && S.rhs_live[q]) {
        const double pq = warp_partial_sum(partial, nb, off, q);
        double a = S.rr[q] / pq;
        const bool bad = !isfinite(a) || !(pq > 0.0);
        if (bad) a = 0.0;
        if (s < S.nshift && S.live[q][s]) {
            const double ap = S.alpha_prev[q], bp = S.beta_prev[q];
            const double z = S.zeta[q][s], zp = S.zeta_prev[q][s];
            // one division: zeta_{k+1} / zeta_k = zeta_{k-1} alpha_{k-1} / den
            const double den = a * bp * (zp - z) + zp * ap * (1.0 + S.dsig[s] * a);
            const double zr = zp * ap / den;
            S.zeta_next[q][s] = z * zr;
            S.zratio[q][s] = zr;
            S.cx[q][s] = a * zr;
        }
        if (s == 0) {
            S.sums[q] = pq;
            S.alpha[q] = a;
            if (bad) {
                S.status = STAG_ERR_NAN;
                S.halt = 1;
            }
        }
    }
    __syncthreads();
}

// beta = (r', r') / (r, r), the shift coefficients of the next search
// directions, per-shift convergence and the solver's halt conditions; warp q
// for source q with lane s for shift s, then thread 0 for the whole solve
__device__ void beta_step(Scal& S, const double* partial, int nb, int off) {
    const int q = threadIdx.x >> 5, s = threadIdx.x & 31;
    if (q < S.nrhs && S.rhs_live[q]) {
        const double rn = warp_partial_sum(partial, nb, off, q);
        const double bt = rn / S.rr[q];
        const bool on = s < S.nshift && S.live[q][s];
        const int n_live = __popc(__ballot_sync(0xffffffffu, on));
        bool still = false;
        if (on) {
            const double zn = S.zeta_next[q][s], z = S.zeta[q][s];
            const double zr = S.zratio[q][s];
            S.cpr[q][s] = zn;
            S.cpp[q][s] = bt * zr * zr;
            S.zeta_prev[q][s] = z;
            S.zeta[q][s] = zn;
            if (zn * zn * rn <= S.tol2 * S.bb[q]) {
                S.live[q][s] = 0;
                S.iters_at[q][s] = S.k + 1;
            } else {
                still = true;
            }
        }
        const bool left = __ballot_sync(0xffffffffu, still) != 0;
        __syncwarp();
        if (s == 0) {
            if (!isfinite(rn)) {
                S.status = STAG_ERR_NAN;
                S.halt = 1;
            }
            S.units[q] = 72.0 + 96.0 * n_live;
            S.sums[q] = rn;
            S.beta[q] = bt;
            S.alpha_prev[q] = S.alpha[q];
            S.beta_prev[q] = bt;
            S.rr[q] = rn;
            S.left[q] = left;
            if (!left) S.rhs_live[q] = 0;
            else if (S.mixed && rn < S.delta2 * S.rr_ref[q]) S.need_reliable = 1;
        }
    } else if (q < S.nrhs && s == 0) {
        S.left[q] = 0;
        S.units[q] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int j = 0; j < S.nrhs; ++j) {
            any |= S.left[j];
            S.k4_units += S.units[j];
        }
        S.k += 1;
        if (!any) S.halt = 1;
        else if (S.k >= S.max_iter) { S.halt = 1; S.status = STAG_ERR_NOT_CONVERGED; }
        if (S.need_reliable) S.halt = 1;
    }
    __syncthreads();
}

// p_i = zeta r + beta_i p_i; x_i += alpha_i p_i for the live shifts of source j at
// site h, four shifts at a time: all their loads are issued before any store.
template <typename R>
__device__ __forceinline__ void shift_updates(const Scal& S, int j, int ns, size_t rs, int h, int Vh,
                                              const Vec3<R>& rv, typename V2T<R>::T* __restrict__ ps,
                                              typename V2T<R>::T* __restrict__ x) {
    typedef typename V2T<R>::T V;
    for (int s0 = 0; s0 < ns; s0 += 4) {
        Vec3<R> pv[4], xv[4];
        bool on[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int s = s0 + u;
            on[u] = s < ns && S.live[j][s];
            if (on[u]) {
                pv[u] = load_vec_cg<R>(ps + ((size_t)j * ns + s) * rs, h, Vh);
                xv[u] = load_vec_cg<R>(x + ((size_t)j * ns + s) * rs, h, Vh);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!on[u]) continue;
            const int s = s0 + u;
            const R cx = (R)S.cx[j][s], cpr = (R)S.cpr[j][s], cpp = (R)S.cpp[j][s];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                pv[u].c[c].re = cpr * rv.c[c].re + cpp * pv[u].c[c].re;
                pv[u].c[c].im = cpr * rv.c[c].im + cpp * pv[u].c[c].im;
                xv[u].c[c].re += cx * pv[u].c[c].re;
                xv[u].c[c].im += cx * pv[u].c[c].im;
            }
            store_vec<R>(x + ((size_t)j * ns + s) * rs, h, Vh, xv[u]);
            store_vec<R>(ps + ((size_t)j * ns + s) * rs, h, Vh, pv[u]);
        }
    }
}


// NRP: sources per pass of the Dslash phases (1, or 4 for multi-source solves);
// PB: threads per block
template <typename R, int FMT, int NRP, int PB>
__global__ void __launch_bounds__(PB) k_ms_persistent(Geom g, LinkPtrs L, SolverState* st,
                                                      typename V2T<R>::T* r, typename V2T<R>::T* p,
                                                      typename V2T<R>::T* q, typename V2T<R>::T* t,
                                                      typename V2T<R>::T* ps, typename V2T<R>::T* x,
                                                      double* partial, GridBar* bar, unsigned long long* ptime) {
    typedef typename V2T<R>::T V;
    static_assert(PB >= 32 * STAG_MAX_RHS, "the reductions take a warp per source");
    __shared__ Scal S;
    // profiling: block 0 accumulates ns spent in phase 1, barrier 1, phase 2,
    // barrier 2 + alpha step, phase 3, barrier 3 + beta step
    const bool timing = ptime && blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long tp[7] = {0, 0, 0, 0, 0, 0, 0}, t_last = timing ? gtimer() : 0;
#define PHASE_MARK(i)                               \
    if (timing) {                                   \
        unsigned long long t_now = gtimer();        \
        tp[i] += t_now - t_last;                    \
        t_last = t_now;                             \
    }
    load_scal(S, st);
    const unsigned int nb = gridDim.x;
    GridSync gs{bar, nb, 0u};
    // this block's sites: a contiguous range, the half lattice split evenly
    // over the grid in multiples of 8 sites (a 32-byte sector of an fp32
    // field component), so every block of the grid has work
    const int per = (int)((((size_t)g.Vh + nb - 1) / nb + 7) & ~(size_t)7);
    const int h0 = min(g.Vh, (int)blockIdx.x * per), h1 = min(g.Vh, h0 + per);
    const size_t rs = (size_t)3 * g.Vh;
    const int nrhs = S.nrhs, ns = S.nshift;
    constexpr int ND = NRP == 1 ? 1 : STAG_MAX_RHS;   // per-thread sums kept
    // float-float hops are long (compensated products): unrolled over the four
    // directions the kernel outgrows the instruction cache, so they loop
    constexpr int MU_UNROLL = std::is_same<R, DF>::value ? 1 : 4;
    bool ok = true;
    while (!S.halt && ok) {
        // ---- phase 1: t = D_oe (r + beta p), without the 1/2
        for (int h = h0 + (int)threadIdx.x; h < h1; h += PB) {
            Nbr n;
            site_neighbours(g, h, 1, n);
            for (int r0 = 0; r0 < nrhs; r0 += NRP) {
                Vec3<R> acc[NRP];
                R bt[NRP];
#pragma unroll
                for (int j = 0; j < NRP; ++j) {
                    zero(acc[j]);
                    bt[j] = (r0 + j < nrhs) ? (R)S.beta[r0 + j] : (R)0;
                }
#pragma unroll MU_UNROLL
                for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
                    for (int dir = 0; dir < 2; ++dir) {
                        const int nb_h = dir == 0 ? n.fwd[mu] : n.bwd[mu];
                        Su3<R> u = dir == 0 ? LinkFetch<R, FMT>::get(L, mu, 1, h, g.Vh)
                                            : LinkFetch<R, FMT>::get(L, mu, 0, nb_h, g.Vh);
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
                            if (dir == 0) mac_uv(acc[j], (R)n.sf[mu], u, a);
                            else mac_udv(acc[j], -(R)n.sb[mu], u, a);
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
        double dots[ND];
#pragma unroll
        for (int j = 0; j < ND; ++j) dots[j] = 0.0;
        const R c0 = (R)S.c0;
        for (int h = h0 + (int)threadIdx.x; h < h1; h += PB) {
            Nbr n;
            site_neighbours(g, h, 0, n);
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
                        const int nb_h = dir == 0 ? n.fwd[mu] : n.bwd[mu];
                        Su3<R> u = dir == 0 ? LinkFetch<R, FMT>::get(L, mu, 0, h, g.Vh)
                                            : LinkFetch<R, FMT>::get(L, mu, 1, nb_h, g.Vh);
#pragma unroll
                        for (int j = 0; j < NRP; ++j) {
                            if (r0 + j >= nrhs) continue;
                            Vec3<R> a = load_vec_cg<R>(t + (size_t)(r0 + j) * rs, nb_h, g.Vh);
                            if (dir == 0) mac_uv(acc[j], (R)n.sf[mu], u, a);
                            else mac_udv(acc[j], -(R)n.sb[mu], u, a);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < NRP; ++j) {
                    if (r0 + j >= nrhs) continue;
                    const size_t off = (size_t)(r0 + j) * rs;
                    const R bt = (R)S.beta[r0 + j];
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
                    dots[r0 + j] += re_dot(pv, o);
                }
            }
        }
        block_sum<ND>(dots);
        if (threadIdx.x == 0)
            for (int j = 0; j < nrhs && j < ND; ++j) partial[(size_t)j * nb + blockIdx.x] = dots[j];
        PHASE_MARK(2)
        if (!(ok = grid_sync(gs))) break;
        alpha_step(S, partial, nb, 0);
        PHASE_MARK(3)
        // ---- phase 3: shift updates and r -= alpha q with (r, r)
        double nrm[ND];
#pragma unroll
        for (int j = 0; j < ND; ++j) nrm[j] = 0.0;
        for (int h = h0 + (int)threadIdx.x; h < h1; h += PB) {
#pragma unroll
            for (int j = 0; j < ND; ++j) {
                if (j >= nrhs || !S.rhs_live[j]) continue;
                const size_t off = (size_t)j * rs;
                Vec3<R> rv = load_vec_cg<R>(r + off, h, g.Vh);
                shift_updates<R>(S, j, ns, rs, h, g.Vh, rv, ps, x);
                const R a = (R)S.alpha[j];
                Vec3<R> qv = load_vec_cg<R>(q + off, h, g.Vh);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    rv.c[c].re -= a * qv.c[c].re;
                    rv.c[c].im -= a * qv.c[c].im;
                }
                store_vec<R>(r + off, h, g.Vh, rv);
                nrm[j] += norm2(rv);
            }
        }
        block_sum<ND>(nrm);
        if (threadIdx.x == 0)
            for (int j = 0; j < nrhs && j < ND; ++j) partial[(size_t)(STAG_MAX_RHS + j) * nb + blockIdx.x] = nrm[j];
        PHASE_MARK(4)
        if (!(ok = grid_sync(gs))) break;
        beta_step(S, partial, nb, STAG_MAX_RHS);
        PHASE_MARK(5)
    }
#undef PHASE_MARK
    if (timing)
        for (int i = 0; i < 6; ++i) ptime[i] += tp[i];
    if (!ok && threadIdx.x == 0) {
        S.halt = 1;
        S.status = STAG_ERR_TIMEOUT;
    }
    __syncthreads();
    if (blockIdx.x == 0) store_scal(S, st);
}

template <typename R, int FMT, int NRP, int PB>
stag_status launch_persistent_pb(stag_ctx* ctx, void* r, void* p, void* q, void* t, void* ps, void* x) {
    typedef typename V2T<R>::T V;
    auto kern = k_ms_persistent<R, FMT, NRP, PB>;
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
    if ((size_t)2 * STAG_MAX_RHS * grid > ctx->red_doubles) return STAG_ERR_ARG;
    CK(cudaMemsetAsync(ctx->bar, 0, sizeof(GridBar), ctx->stream));
    Geom g = ctx->g;
    LinkPtrs L = link_ptrs(ctx);
    SolverState* st = ctx->st;
    V *vr = (V*)r, *vp = (V*)p, *vq = (V*)q, *vt = (V*)t, *vps = (V*)ps, *vx = (V*)x;
    double* part = ctx->red;
    GridBar* bar = (GridBar*)ctx->bar;
    unsigned long long* pt = ctx->prof.on ? (unsigned long long*)ctx->ptime : nullptr;
    void* args[] = {&g, &L, &st, &vr, &vp, &vq, &vt, &vps, &vx, &part, &bar, &pt};
    CK(cudaLaunchCooperativeKernel((const void*)kern, grid, PB, args, 0, ctx->stream));
    ++ctx->launches;
    return STAG_OK;
}
}  // namespace

bool persistent_fits(stag_ctx* ctx) {
    // small lattices, where launch and loop overhead dominate the iteration
    return ctx->use_persistent && ctx->g.Vh <= (1 << 18);
}

template <typename R, int FMT, int NRP>
stag_status launch_persistent_t(stag_ctx* ctx, void* r, void* p, void* q, void* t, void* ps, void* x) {
    // 256 threads per block: one block per SM at these register counts
    return launch_persistent_pb<R, FMT, NRP, 256>(ctx, r, p, q, t, ps, x);
}

template <int NRP>
stag_status launch_persistent_n(stag_ctx* ctx, stag_prec prec, void* r, void* p, void* q, void* t, void* ps, void* x) {
    switch (prec) {
        case STAG_FP64: return launch_persistent_t<DF, FMT_F64, NRP>(ctx, r, p, q, t, ps, x);
        case STAG_FP32: return launch_persistent_t<float, FMT_F32_18, NRP>(ctx, r, p, q, t, ps, x);
        case STAG_FP32_12: return launch_persistent_t<float, FMT_F32_12, NRP>(ctx, r, p, q, t, ps, x);
        default: return launch_persistent_t<float, FMT_BF16_12, NRP>(ctx, r, p, q, t, ps, x);
    }
}

stag_status launch_persistent(stag_ctx* ctx, stag_prec prec, int nrhs, void* r, void* p, void* q, void* t, void* ps,
                              void* x) {
    if (!ctx->bar) CKS(dev_alloc(ctx, &ctx->bar, sizeof(GridBar)));
    if (!ctx->ptime) {
        CKS(dev_alloc(ctx, &ctx->ptime, PTIME_WORDS * sizeof(unsigned long long)));
        CK(cudaMemsetAsync(ctx->ptime, 0, PTIME_WORDS * sizeof(unsigned long long), ctx->stream));
    }
    if (nrhs == 1) return launch_persistent_n<1>(ctx, prec, r, p, q, t, ps, x);
    return launch_persistent_n<4>(ctx, prec, r, p, q, t, ps, x);
}

extern "C" stag_status stag_profile_phases(stag_ctx* ctx, double* us) {
    if (!ctx || !us) return STAG_ERR_ARG;
    unsigned long long t[8] = {0};
    if (ctx->ptime) {
        CK(cudaMemcpyAsync(t, ctx->ptime, sizeof(t), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    for (int i = 0; i < 6; ++i) us[i] = t[i] * 1e-3;
    return STAG_OK;
}

// ---- self-test of the bounded grid barrier: two blocks, only block 0
// arrives, so its wait can only end by giving up after spin_limit polls
namespace {
__global__ void k_barrier_timeout_probe(GridBar* bar, long long spin_limit, int* status) {
    if (blockIdx.x != 0) return;              // the block that never arrives
    GridSync gs{bar, gridDim.x, 0u};
    const bool met = grid_sync(gs, spin_limit);
    if (threadIdx.x == 0) *status = met ? STAG_OK : STAG_ERR_TIMEOUT;
}
}  // namespace

extern "C" stag_status stag_selftest_barrier_timeout(stag_ctx* ctx, long long spin_limit) {
    if (!ctx || spin_limit < 1 || spin_limit > BAR_SPIN_LIMIT) return STAG_ERR_ARG;
    if (!ctx->bar) CKS(dev_alloc(ctx, &ctx->bar, sizeof(GridBar)));
    int* d_status;
    CKS(ws_get(ctx, WS_MISC, sizeof(int), (void**)&d_status));
    CK(cudaMemsetAsync(ctx->bar, 0, sizeof(GridBar), ctx->stream));
    k_barrier_timeout_probe<<<2, 32, 0, ctx->stream>>>((GridBar*)ctx->bar, spin_limit, d_status);
    CKL();
    int st = -1;
    CK(cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemsetAsync(ctx->bar, 0, sizeof(GridBar), ctx->stream));
    return (stag_status)st;
}
