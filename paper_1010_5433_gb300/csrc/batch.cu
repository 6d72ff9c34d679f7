// Several independent multi-shift solves -- one per context, each on its own
// lattice of any size -- iterated by ONE persistent cooperative launch.  The
// workload is a set of independent Markov chains of uneven volumes (8^4 to
// 16^4): a single small lattice leaves most of the 152 SMs idle and pays a
// grid barrier per phase for a few thousand sites, while the chains together
// fill the GPU and share every barrier.
//
// Work queue: in every phase the sites of all chains still iterating form one
// concatenated range, dealt out round-robin to all threads of the grid
// (thread i takes the sites congruent to i), so the chains are load-balanced
// whatever their sizes.  Each chain keeps its own scalar recurrences
// (Jegerlehner's, Sec. 6) in shared memory, advanced redundantly by every
// block from the per-block partial sums of all chains, summed in one fixed
// order; a chain that converges or needs a reliable update halts by itself
// (its convergence flag) while the others continue.  The launch ends when
// every chain has halted; the host then makes the fp64 reliable updates of
// the chains that asked for one and launches again.  One source per chain
// (n_rhs = 1); every wait on a grid barrier is bounded.  The launch shape
// (threads per block, blocks per SM) is chosen per precision by timing the
// candidates on the first segments of real solves.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "internal.h"
#include "solver_state.cuh"
#include "grid_barrier.cuh"

namespace {

constexpr int MAXC = STAG_MAX_BATCH;
constexpr int NS = STAG_MAX_SHIFTS;

struct ChainArgs {
    Geom g;
    LinkPtrs L;
    SolverState* st;
    void *r, *p, *q, *t, *ps, *x;
};
struct BatchArgs {
    int n;
    ChainArgs c[MAXC];
};

// one chain's scalar recurrences (one source), with float-float copies of
// the coefficients every thread applies, made once per block when they
// change: a per-thread fp64 load and conversion per site and shift runs on
// GB300's slow fp64 pipe
struct ScalM {
    double zeta[NS], zeta_prev[NS], zeta_next[NS], zratio[NS], cx[NS], cpr[NS], cpp[NS], dsig[NS];
    double rr, bb, rr_ref, alpha, alpha_prev, beta_prev, beta, sum, k4_units, c0, tol2, delta2;
    DF cxD[NS], cprD[NS], cppD[NS], alphaD, betaD, c0D;
    int live[NS], iters_at[NS];
    int rhs_live, k, halt, status, need_reliable, nshift, max_iter, mixed, left, nan;
};

// a coefficient in the arithmetic of the iteration: the float part for fp32
// fields, the float-float pair for float-float fields
template <typename R> __device__ __forceinline__ R coef(const DF& d);
template <> __device__ __forceinline__ float coef<float>(const DF& d) { return d.hi; }
template <> __device__ __forceinline__ DF coef<DF>(const DF& d) { return d; }

__device__ void load_scal_m(ScalM* S, const ChainArgs* C, int nc) {
    const int t = threadIdx.x;
    for (int i = t; i < nc * NS; i += blockDim.x) {
        const int c = i / NS, s = i % NS;
        const SolverState* st = C[c].st;
        S[c].zeta[s] = st->zeta[0][s];
        S[c].zeta_prev[s] = st->zeta_prev[0][s];
        S[c].zeta_next[s] = st->zeta_next[0][s];
        S[c].cx[s] = st->cx[0][s];
        S[c].cpr[s] = st->cpr[0][s];
        S[c].cpp[s] = st->cpp[0][s];
        S[c].cxD[s] = DF(st->cx[0][s]);
        S[c].cprD[s] = DF(st->cpr[0][s]);
        S[c].cppD[s] = DF(st->cpp[0][s]);
        S[c].dsig[s] = st->dsig[s];
        S[c].live[s] = st->live[0][s];
        S[c].iters_at[s] = st->iters_at[0][s];
    }
    if (t < nc) {
        const SolverState* st = C[t].st;
        ScalM& s = S[t];
        s.rr = st->rr[0];
        s.bb = st->bb[0];
        s.rr_ref = st->rr_ref[0];
        s.alpha = st->alpha[0];
        s.alphaD = DF(st->alpha[0]);
        s.alpha_prev = st->alpha_prev[0];
        s.beta_prev = st->beta_prev[0];
        s.beta = st->beta[0];
        s.betaD = DF(st->beta[0]);
        s.k4_units = st->k4_units;
        s.c0 = st->c0;
        s.c0D = DF(st->c0);
        s.tol2 = st->tol2;
        s.delta2 = st->delta2;
        s.rhs_live = st->rhs_live[0];
        s.k = st->k;
        s.halt = st->halt;
        s.status = st->status;
        s.need_reliable = st->need_reliable;
        s.nshift = st->nshift;
        s.max_iter = st->max_iter;
        s.mixed = st->mixed;
        s.nan = 0;
    }
    __syncthreads();
}

__device__ void store_scal_m(const ScalM* S, const ChainArgs* C, int nc) {
    const int t = threadIdx.x;
    for (int i = t; i < nc * NS; i += blockDim.x) {
        const int c = i / NS, s = i % NS;
        SolverState* st = C[c].st;
        st->zeta[0][s] = S[c].zeta[s];
        st->zeta_prev[0][s] = S[c].zeta_prev[s];
        st->zeta_next[0][s] = S[c].zeta_next[s];
        st->cx[0][s] = S[c].cx[s];
        st->cpr[0][s] = S[c].cpr[s];
        st->cpp[0][s] = S[c].cpp[s];
        st->live[0][s] = S[c].live[s];
        st->iters_at[0][s] = S[c].iters_at[s];
    }
    if (t < nc) {
        SolverState* st = C[t].st;
        const ScalM& s = S[t];
        st->rr[0] = s.rr;
        st->alpha[0] = s.alpha;
        st->alpha_prev[0] = s.alpha_prev;
        st->beta_prev[0] = s.beta_prev;
        st->beta[0] = s.beta;
        st->rhs_live[0] = s.rhs_live;
        st->k4_units = s.k4_units;
        st->k = s.k;
        st->halt = s.halt;
        st->status = s.status;
        st->need_reliable = s.need_reliable;
    }
}

// every block: S[c].sum = sum over blocks of partial[base + c][.] for all
// chains, warp c summing chain c (lane l adds the partials l, l + 32, ...,
// then a fixed shuffle tree), so every block gets the same bits
__device__ void sum_partials_m(ScalM* S, const double* partial, int nb, int nc, int base) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < nc) {
        double v = lane_strided_sum(partial + (size_t)(base + warp) * nb, nb, lane);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) S[warp].sum = v;
    }
    __syncthreads();
}

// The (chain, shift) pairs of the scalar steps, packed densely: pair i belongs
// to chain c with base[c] <= i < base[c + 1] (fp64 is slow on GB300, so only
// real shifts issue its instructions).
struct Pairs {
    int base[MAXC + 1];
};
__device__ __forceinline__ void pair_of(const Pairs& P, int nc, int i, int& c, int& s) {
    c = 0;
    while (c + 1 < nc && i >= P.base[c + 1]) ++c;
    s = i - P.base[c];
}

// alpha_k = (r, r) / (p, A p) and the shifted zeta_{k+1}, alpha_{i,k}
__device__ void alpha_step_m(ScalM* S, int nc, const Pairs& P) {
    const int t = threadIdx.x;
    if (t < nc && !S[t].halt) {
        double a = S[t].rr / S[t].sum;
        if (!isfinite(a) || !(S[t].sum > 0.0)) {
            S[t].status = STAG_ERR_NAN;
            S[t].halt = 1;
            a = 0.0;
        }
        S[t].alpha = a;
        S[t].alphaD = DF(a);
    }
    __syncthreads();
    for (int i = t; i < P.base[nc]; i += blockDim.x) {
        int c, s;
        pair_of(P, nc, i, c, s);
        ScalM& C = S[c];
        if (C.halt || !C.live[s]) continue;
        const double a = C.alpha, ap = C.alpha_prev, bp = C.beta_prev;
        const double z = C.zeta[s], zp = C.zeta_prev[s];
        // one division: zeta_{k+1} / zeta_k = zeta_{k-1} alpha_{k-1} / den
        const double den = a * bp * (zp - z) + zp * ap * (1.0 + C.dsig[s] * a);
        const double zr = zp * ap / den;
        C.zeta_next[s] = z * zr;
        C.zratio[s] = zr;
        C.cx[s] = a * zr;
        C.cxD[s] = DF(C.cx[s]);
    }
    __syncthreads();
}

// beta_k = (r', r') / (r, r), the shifted beta_{i,k}, per-shift convergence,
// and the chain's halt: converged, reliable update due, max_iter or NaN
__device__ void beta_step_m(ScalM* S, int nc, const Pairs& P) {
    const int t = threadIdx.x;
    __shared__ double s_beta[MAXC];
    __shared__ int active[MAXC];
    if (t < nc) {
        active[t] = !S[t].halt;
        S[t].left = 0;
        if (active[t]) {
            const double rn = S[t].sum;
            if (!isfinite(rn)) S[t].nan = 1;
            s_beta[t] = rn / S[t].rr;
            int n_live = 0;
            for (int s = 0; s < S[t].nshift; ++s) n_live += S[t].live[s];
            S[t].k4_units += 72.0 + 96.0 * n_live;
        }
    }
    __syncthreads();
    for (int i = t; i < P.base[nc]; i += blockDim.x) {
        int c, s;
        pair_of(P, nc, i, c, s);
        ScalM& C = S[c];
        if (!active[c] || !C.live[s]) continue;
        const double zn = C.zeta_next[s], z = C.zeta[s];
        const double zr = C.zratio[s];
        C.cpr[s] = zn;
        C.cpp[s] = s_beta[c] * zr * zr;
        C.cprD[s] = DF(zn);
        C.cppD[s] = DF(C.cpp[s]);
        C.zeta_prev[s] = z;
        C.zeta[s] = zn;
        if (zn * zn * C.sum <= C.tol2 * C.bb) {
            C.live[s] = 0;
            C.iters_at[s] = C.k + 1;
        } else {
            atomicOr(&C.left, 1);
        }
    }
    __syncthreads();
    if (t < nc && active[t]) {
        ScalM& C = S[t];
        C.beta = s_beta[t];
        C.betaD = DF(s_beta[t]);
        C.alpha_prev = C.alpha;
        C.beta_prev = s_beta[t];
        C.rr = C.sum;
        C.k += 1;
        if (C.nan) {
            C.status = STAG_ERR_NAN;
            C.halt = 1;
        } else if (!C.left) {
            C.rhs_live = 0;
            C.halt = 1;
        } else {
            if (C.mixed && C.sum < C.delta2 * C.rr_ref) C.need_reliable = 1;
            if (C.k >= C.max_iter) {
                C.halt = 1;
                C.status = STAG_ERR_NOT_CONVERGED;
            }
            if (C.need_reliable) C.halt = 1;
        }
    }
    __syncthreads();
}

// first site of this thread in a chain whose sites start at `off` in the
// concatenated range (round-robin over all threads of the grid)
__device__ __forceinline__ int first_site(long long tid, long long off, long long nthreads) {
    long long d = (tid - off) % nthreads;
    return (int)(d < 0 ? d + nthreads : d);
}

// phase 1 at odd site h: t = D_oe (r + beta p), without the 1/2 (the
// float-float hops loop over the directions: unrolled, the kernel outgrows
// the instruction cache)
template <typename R, int FMT>
__device__ __forceinline__ void site_doe(const Geom& g, const LinkPtrs& L, int h, const typename V2T<R>::T* r,
                                         const typename V2T<R>::T* p, typename V2T<R>::T* t, R bt) {
    Nbr n;
    site_neighbours(g, h, 1, n);
    Vec3<R> acc;
    zero(acc);
#pragma unroll (std::is_same<R, DF>::value ? 1 : 4)
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            const int nb_h = dir == 0 ? n.fwd[mu] : n.bwd[mu];
            Su3<R> u = dir == 0 ? LinkFetch<R, FMT>::get(L, mu, 1, h, g.Vh) : LinkFetch<R, FMT>::get(L, mu, 0, nb_h, g.Vh);
            Vec3<R> a = load_vec_cg<R>(r, nb_h, g.Vh);
            Vec3<R> b = load_vec_cg<R>(p, nb_h, g.Vh);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a.c[c].re += bt * b.c[c].re;
                a.c[c].im += bt * b.c[c].im;
            }
            if (dir == 0) mac_uv(acc, (R)n.sf[mu], u, a);
            else mac_udv(acc, -(R)n.sb[mu], u, a);
        }
    }
    store_vec<R>(t, h, g.Vh, acc);
}

// phase 2 at even site h: p = r + beta p; q = c0 p - 1/4 (hops of t); returns (p, q)
template <typename R, int FMT>
__device__ __forceinline__ double site_a(const Geom& g, const LinkPtrs& L, int h, const typename V2T<R>::T* t,
                                         typename V2T<R>::T* p, const typename V2T<R>::T* r,
                                         typename V2T<R>::T* q, R bt, R c0) {
    Nbr n;
    site_neighbours(g, h, 0, n);
    Vec3<R> acc;
    zero(acc);
#pragma unroll (std::is_same<R, DF>::value ? 1 : 4)
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            const int nb_h = dir == 0 ? n.fwd[mu] : n.bwd[mu];
            Su3<R> u = dir == 0 ? LinkFetch<R, FMT>::get(L, mu, 0, h, g.Vh) : LinkFetch<R, FMT>::get(L, mu, 1, nb_h, g.Vh);
            Vec3<R> a = load_vec_cg<R>(t, nb_h, g.Vh);
            if (dir == 0) mac_uv(acc, (R)n.sf[mu], u, a);
            else mac_udv(acc, -(R)n.sb[mu], u, a);
        }
    }
    Vec3<R> pv = load_vec_cg<R>(p, h, g.Vh);
    Vec3<R> rv = load_vec_cg<R>(r, h, g.Vh);
    Vec3<R> o;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        pv.c[c].re = rv.c[c].re + bt * pv.c[c].re;
        pv.c[c].im = rv.c[c].im + bt * pv.c[c].im;
        o.c[c].re = c0 * pv.c[c].re - (R)0.25 * acc.c[c].re;
        o.c[c].im = c0 * pv.c[c].im - (R)0.25 * acc.c[c].im;
    }
    store_vec<R>(p, h, g.Vh, pv);
    store_vec<R>(q, h, g.Vh, o);
    return re_dot(pv, o);
}

// phase 3 at even site h: p_i = zeta r + beta_i p_i; x_i += alpha_i p_i for
// the live shifts (four at a time, loads before stores); r -= alpha q; returns (r, r)
template <typename R>
__device__ __forceinline__ double site_update(const ScalM& S, int h, int Vh, typename V2T<R>::T* r,
                                              const typename V2T<R>::T* q, typename V2T<R>::T* ps,
                                              typename V2T<R>::T* x) {
    const size_t rs = (size_t)3 * Vh;
    Vec3<R> rv = load_vec_cg<R>(r, h, Vh);
    const int ns = S.nshift;
    for (int s0 = 0; s0 < ns; s0 += 4) {
        Vec3<R> pv[4], xv[4];
        bool on[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int s = s0 + u;
            on[u] = s < ns && S.live[s];
            if (on[u]) {
                pv[u] = load_vec_cg<R>(ps + (size_t)s * rs, h, Vh);
                xv[u] = load_vec_cg<R>(x + (size_t)s * rs, h, Vh);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!on[u]) continue;
            const int s = s0 + u;
            const R cx = coef<R>(S.cxD[s]), cpr = coef<R>(S.cprD[s]), cpp = coef<R>(S.cppD[s]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                pv[u].c[c].re = cpr * rv.c[c].re + cpp * pv[u].c[c].re;
                pv[u].c[c].im = cpr * rv.c[c].im + cpp * pv[u].c[c].im;
                xv[u].c[c].re += cx * pv[u].c[c].re;
                xv[u].c[c].im += cx * pv[u].c[c].im;
            }
            store_vec<R>(x + (size_t)s * rs, h, Vh, xv[u]);
            store_vec<R>(ps + (size_t)s * rs, h, Vh, pv[u]);
        }
    }
    const R a = coef<R>(S.alphaD);
    Vec3<R> qv = load_vec_cg<R>(q, h, Vh);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        rv.c[c].re -= a * qv.c[c].re;
        rv.c[c].im -= a * qv.c[c].im;
    }
    store_vec<R>(r, h, Vh, rv);
    return norm2(rv);
}

// add v into slot c of a register array without dynamic register indexing
__device__ __forceinline__ void add_slot(double (&a)[MAXC], int c, double v) {
#pragma unroll
    for (int j = 0; j < MAXC; ++j)
        if (j == c) a[j] += v;
}

// PB threads per block, MB blocks per SM requested of the register allocator
template <typename R, int FMT, int PB, int MB>
__global__ void __launch_bounds__(PB, MB) k_ms_persistent_batch(BatchArgs A, double* partial, GridBar* bar,
                                                                 unsigned long long* ptime) {
    typedef typename V2T<R>::T V;
    // profiling: block 0 accumulates ns in phase 1, barrier 1, phase 2,
    // barrier 2, alpha step (with the partial sums), phase 3, barrier 3, beta step
    const bool timing = ptime && blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long tp[8] = {0, 0, 0, 0, 0, 0, 0, 0}, t_last = timing ? gtimer() : 0;
#define PHASE_MARK(i)                               \
    if (timing) {                                   \
        unsigned long long t_now = gtimer();        \
        tp[i] += t_now - t_last;                    \
        t_last = t_now;                             \
    }
    __shared__ ScalM S[MAXC];
    __shared__ ChainArgs C[MAXC];
    const int nc = A.n;
    if (threadIdx.x < nc) C[threadIdx.x] = A.c[threadIdx.x];
    __syncthreads();
    load_scal_m(S, C, nc);
    __shared__ Pairs P;
    if (threadIdx.x == 0) {
        P.base[0] = 0;
        for (int c = 0; c < nc; ++c) P.base[c + 1] = P.base[c] + S[c].nshift;
    }
    __syncthreads();
    const unsigned int nb = gridDim.x;
    GridSync gs{bar, nb, 0u};
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = true;
    for (;;) {
        int any = 0;
        for (int c = 0; c < nc; ++c) any |= !S[c].halt;
        if (!any) break;
        // ---- phase 1: t = D_oe (r + beta p) on every iterating chain
        long long off = 0;
        for (int c = 0; c < nc; ++c) {
            if (S[c].halt) continue;
            const Geom g = C[c].g;
            const LinkPtrs L = C[c].L;
            const R bt = coef<R>(S[c].betaD);
            const V *r = (const V*)C[c].r, *p = (const V*)C[c].p;
            V* t = (V*)C[c].t;
            for (int h = first_site(tid, off, nthreads); h < g.Vh; h += (int)nthreads)
                site_doe<R, FMT>(g, L, h, r, p, t, bt);
            off += g.Vh;
        }
        PHASE_MARK(0)
        if (!(ok = grid_sync(gs))) break;
        PHASE_MARK(1)
        // ---- phase 2: p = r + beta p; q = (A + s0) p; (p, q)
        double dots[MAXC];
#pragma unroll
        for (int j = 0; j < MAXC; ++j) dots[j] = 0.0;
        off = 0;
        for (int c = 0; c < nc; ++c) {
            if (S[c].halt) continue;
            const Geom g = C[c].g;
            const LinkPtrs L = C[c].L;
            const R bt = coef<R>(S[c].betaD), c0 = coef<R>(S[c].c0D);
            const V *t = (const V*)C[c].t, *r = (const V*)C[c].r;
            V *p = (V*)C[c].p, *q = (V*)C[c].q;
            double d = 0.0;
            for (int h = first_site(tid, off, nthreads); h < g.Vh; h += (int)nthreads)
                d += site_a<R, FMT>(g, L, h, t, p, r, q, bt, c0);
            add_slot(dots, c, d);
            off += g.Vh;
        }
        block_sum<MAXC>(dots);
        if (threadIdx.x == 0)
            for (int j = 0; j < nc; ++j) partial[(size_t)j * nb + blockIdx.x] = dots[j];
        PHASE_MARK(2)
        if (!(ok = grid_sync(gs))) break;
        PHASE_MARK(3)
        sum_partials_m(S, partial, nb, nc, 0);
        alpha_step_m(S, nc, P);
        PHASE_MARK(4)
        // ---- phase 3: shift updates, r -= alpha q, (r, r)
        double nrm[MAXC];
#pragma unroll
        for (int j = 0; j < MAXC; ++j) nrm[j] = 0.0;
        off = 0;
        for (int c = 0; c < nc; ++c) {
            if (S[c].halt) continue;   // halted by its alpha step (NaN)
            const int Vh = C[c].g.Vh;
            V *r = (V*)C[c].r, *ps = (V*)C[c].ps, *x = (V*)C[c].x;
            const V* q = (const V*)C[c].q;
            double d = 0.0;
            for (int h = first_site(tid, off, nthreads); h < Vh; h += (int)nthreads)
                d += site_update<R>(S[c], h, Vh, r, q, ps, x);
            add_slot(nrm, c, d);
            off += Vh;
        }
        block_sum<MAXC>(nrm);
        if (threadIdx.x == 0)
            for (int j = 0; j < nc; ++j) partial[(size_t)(MAXC + j) * nb + blockIdx.x] = nrm[j];
        PHASE_MARK(5)
        if (!(ok = grid_sync(gs))) break;
        PHASE_MARK(6)
        sum_partials_m(S, partial, nb, nc, MAXC);
        beta_step_m(S, nc, P);
        PHASE_MARK(7)
    }
#undef PHASE_MARK
    if (timing)
        for (int i = 0; i < 8; ++i) ptime[8 + 8 * (sizeof(R) == 4 ? 0 : 1) + i] += tp[i];
    if (!ok && threadIdx.x < nc && !S[threadIdx.x].halt) {
        S[threadIdx.x].halt = 1;
        S[threadIdx.x].status = STAG_ERR_TIMEOUT;
    }
    __syncthreads();
    if (blockIdx.x == 0) store_scal_m(S, C, nc);
}

template <typename R, int FMT, int PB, int MB>
stag_status launch_batch_pb(stag_ctx* ctx, const BatchArgs& A, long long sites, double* partial,
                            size_t partial_doubles, GridBar* bar) {
    auto kern = k_ms_persistent_batch<R, FMT, PB, MB>;
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PB, 0));
    if (per_sm < 1) return STAG_ERR_ARG;
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // the fewest blocks that give no thread more sites per phase than the
    // largest co-resident grid would: the same phase time, fewer blocks
    // meeting at every barrier
    const long long cap = (long long)nsm * per_sm;
    const long long per_thread = (sites + cap * PB - 1) / (cap * PB);
    long long want = (sites + per_thread * PB - 1) / (per_thread * PB);
    int grid = (int)(want < cap ? want : cap);
    if (grid < 1) grid = 1;
    if ((size_t)2 * MAXC * grid > partial_doubles) return STAG_ERR_ARG;
    CK(cudaMemsetAsync(bar, 0, sizeof(GridBar), ctx->stream));
    BatchArgs a = A;
    unsigned long long* pt = ctx->prof.on ? (unsigned long long*)ctx->ptime : nullptr;
    void* args[] = {&a, &partial, &bar, &pt};
    CK(cudaLaunchCooperativeKernel((const void*)kern, grid, PB, args, 0, ctx->stream));
    ++ctx->launches;
    return STAG_OK;
}

// launch shapes (threads per block, blocks per SM) the tuner chooses among;
// float-float keeps the first only (its registers allow no second block)
constexpr int N_SHAPES = 3;
constexpr int SHAPE_PB[N_SHAPES] = {256, 384, 320};
static_assert(256 >= 32 * MAXC, "sum_partials_m needs a warp per chain");
constexpr int SHAPE_MB[N_SHAPES] = {1, 1, 1};

template <typename R, int FMT>
stag_status launch_batch_t(stag_ctx* ctx, int shape, const BatchArgs& A, long long sites, double* partial, size_t pd,
                           GridBar* bar) {
    switch (shape) {
        case 1: return launch_batch_pb<R, FMT, 384, 1>(ctx, A, sites, partial, pd, bar);
        case 2: return launch_batch_pb<R, FMT, 320, 1>(ctx, A, sites, partial, pd, bar);
        default: return launch_batch_pb<R, FMT, 256, 1>(ctx, A, sites, partial, pd, bar);
    }
}

int n_shapes(stag_prec prec) { return prec == STAG_FP64 ? 1 : N_SHAPES; }

stag_status launch_batch(stag_ctx* ctx, stag_prec prec, int shape, const BatchArgs& A, long long sites,
                         double* partial, size_t pd, GridBar* bar) {
    switch (prec) {
        case STAG_FP64: return launch_batch_pb<DF, FMT_F64, 256, 1>(ctx, A, sites, partial, pd, bar);
        case STAG_FP32: return launch_batch_t<float, FMT_F32_18>(ctx, shape, A, sites, partial, pd, bar);
        case STAG_FP32_12: return launch_batch_t<float, FMT_F32_12>(ctx, shape, A, sites, partial, pd, bar);
        default: return launch_batch_t<float, FMT_BF16_12>(ctx, shape, A, sites, partial, pd, bar);
    }
}
}  // namespace

stag_status ms_core_multi(MsRun* runs, int n, MsStats* stats, stag_status* per_chain) {
    if (n < 1 || n > MAXC || !runs) return STAG_ERR_ARG;
    stag_ctx* lead = runs[0].ctx;
    for (int i = 0; i < n; ++i) {
        if (runs[i].nrhs != 1 || runs[i].prec != runs[0].prec || runs[i].ctx->stream != lead->stream)
            return STAG_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (runs[j].ctx == runs[i].ctx) return STAG_ERR_ARG;
    }
    stag_ctx* ctx = lead;   // error reporting of the CK macros
    for (int i = 0; i < n; ++i) CKS(ms_setup(runs[i]));
    if (!lead->bar) CKS(dev_alloc(lead, &lead->bar, sizeof(GridBar)));
    if (!lead->ptime) {
        CKS(dev_alloc(lead, &lead->ptime, PTIME_WORDS * sizeof(unsigned long long)));
        CK(cudaMemsetAsync(lead->ptime, 0, PTIME_WORDS * sizeof(unsigned long long), lead->stream));
    }
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t pd = (size_t)2 * MAXC * nsm * 8;   // up to 8 co-resident blocks per SM
    void* partial;
    CKS(ws_get(lead, WS_BATCH_RED, pd * sizeof(double), &partial));
    std::vector<int> active(n, 1);
    std::vector<stag_status> st(n, STAG_OK);
    cudaEvent_t pe0 = nullptr, pe1 = nullptr;
    double launch_ms = 0.0;
    if (lead->prof.on) {
        CK(cudaEventCreate(&pe0));
        CK(cudaEventCreate(&pe1));
    }
    const bool profiling = lead->prof.on;
    int max_iter = 0;
    for (int i = 0; i < n; ++i) max_iter = std::max(max_iter, runs[i].max_iter);
    const int max_segments = 64 + max_iter;
    for (int seg = 0;; ++seg) {
        BatchArgs A;
        std::memset(&A, 0, sizeof(A));
        long long sites = 0;
        std::vector<int> idx;
        for (int i = 0; i < n; ++i) {
            if (!active[i]) continue;
            stag_ctx* c = runs[i].ctx;
            ChainArgs& a = A.c[A.n++];
            a.g = c->g;
            a.L = link_ptrs(c);
            a.st = c->st;
            a.r = runs[i].r;
            a.p = runs[i].p;
            a.q = runs[i].q;
            a.t = runs[i].tmp;
            a.ps = runs[i].ps;
            a.x = runs[i].x;
            sites += c->g.Vh;
            idx.push_back(i);
        }
        if (A.n == 0) break;
        if (seg > max_segments) {
            for (int i : idx) { st[i] = STAG_ERR_TIMEOUT; active[i] = 0; }
            break;
        }
        // launch shape: the tuned one, or the next candidate while tuning
        BatchTune& tu = lead->batch_tune[runs[0].prec];
        const int ns_prec = n_shapes(runs[0].prec);
        int shape = tu.chosen;
        if (shape < 0) {
            if (lead->batch_shape_force >= 0) shape = tu.chosen = std::min(lead->batch_shape_force, ns_prec - 1);
            else shape = tu.tried % ns_prec;
        }
        const bool timed = pe0 || tu.chosen < 0;
        if (timed && !pe0) {
            CK(cudaEventCreate(&pe0));
            CK(cudaEventCreate(&pe1));
        }
        int k_before = 0;
        for (int i : idx) k_before = std::max(k_before, runs[i].ctx->st_host->k);
        if (timed) CK(cudaEventRecord(pe0, lead->stream));
        CKS(launch_batch(lead, runs[0].prec, shape, A, sites, (double*)partial, pd, (GridBar*)lead->bar));
        if (timed) CK(cudaEventRecord(pe1, lead->stream));
        for (int i : idx) CKS(ms_pull_control_async(runs[i].ctx));
        CK(cudaStreamSynchronize(lead->stream));
        if (timed) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, pe0, pe1));
            if (lead->prof.on) launch_ms += ms;
            if (tu.chosen < 0) {
                // microseconds per batched iteration of this segment, for its shape
                int k_after = 0;
                for (int i : idx) k_after = std::max(k_after, runs[i].ctx->st_host->k);
                if (k_after > k_before) {
                    tu.us[shape] += 1e3 * ms;
                    tu.iters[shape] += k_after - k_before;
                    tu.tried += 1;
                }
                if (tu.tried >= 2 * ns_prec) {
                    int best = 0;
                    for (int v = 1; v < ns_prec; ++v)
                        if (tu.us[v] / std::max(1, tu.iters[v]) < tu.us[best] / std::max(1, tu.iters[best])) best = v;
                    tu.chosen = best;
                }
            }
        }
        for (int i : idx) {
            const SolverState* hs = runs[i].ctx->st_host;
            if (!hs->halt) { st[i] = STAG_ERR_TIMEOUT; active[i] = 0; continue; }
            if (hs->status != STAG_OK) { st[i] = (stag_status)hs->status; active[i] = 0; continue; }
            if (hs->need_reliable) { CKS(ms_reliable_update(runs[i])); continue; }
            active[i] = 0;   // converged
        }
    }
    long long kmax = 0;
    double bytes = 0.0;
    for (int i = 0; i < n; ++i) {
        CKS(ms_pull_state(runs[i].ctx));
        const SolverState* hs = runs[i].ctx->st_host;
        const double S = 3.0 * (double)(runs[i].mixed ? sizeof(float2) : sizeof(double2));   // one spinor at a site
        const double Vh = runs[i].ctx->g.Vh;
        // as the single-lattice persistent solver: both Dslash phases and the updates
        bytes += (double)hs->k * Vh * (2.0 * link_bytes_site(runs[i].prec) + 8.0 * S) +
                 hs->k4_units * Vh * (runs[i].mixed ? 1.0 : 2.0);
        kmax = std::max(kmax, (long long)hs->k);
        CKS(ms_finish(runs[i]));
        if (stats) ms_stats(runs[i], &stats[i]);
        if (per_chain) per_chain[i] = st[i];
    }
    if (profiling) {
        ProfData& pf = lead->prof;
        pf.bytes_total[PK_BATCH] += bytes;
        pf.launches[PK_BATCH] += kmax;
        pf.batch_ms += launch_ms;
        pf.batch_iters += kmax;
    }
    if (pe0) cudaEventDestroy(pe0);
    if (pe1) cudaEventDestroy(pe1);
    return STAG_OK;
}

extern "C" int stag_batch_shape(stag_ctx* ctx, stag_prec prec, int* threads_per_block, int* blocks_per_sm) {
    if (!ctx || prec < STAG_FP64 || prec > STAG_BF16_12) return -1;
    const int c = ctx->batch_tune[prec].chosen;
    if (c >= 0) {
        if (threads_per_block) *threads_per_block = SHAPE_PB[c];
        if (blocks_per_sm) *blocks_per_sm = SHAPE_MB[c];
    }
    return c;
}

extern "C" stag_status stag_profile_batch_phases(stag_ctx* ctx, stag_prec prec, double* us) {
    if (!ctx || !us) return STAG_ERR_ARG;
    unsigned long long t[PTIME_WORDS] = {0};
    if (ctx->ptime) {
        CK(cudaMemcpyAsync(t, ctx->ptime, sizeof(t), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    const int base = 8 + 8 * (prec == STAG_FP64 ? 1 : 0);
    for (int i = 0; i < 8; ++i) us[i] = t[base + i] * 1e-3;
    return STAG_OK;
}
