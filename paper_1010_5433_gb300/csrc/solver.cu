// Multi-shift CG (Sec. 6 of the paper; B. Jegerlehner, hep-lat/9612014) for
//   (A + sigma_i) x_i = b,   A = m^2 - D_eo D_oe,
// with nrhs independent sources iterated together, so every Dslash is a
// multi-RHS Dslash that loads each link once for all of them.
//
// One iteration is four kernels:
//   K1  t  = D_oe p                                     (multi-RHS Dslash)
//   K2  q  = (m^2 + sigma_0) p - D_eo t,  (p, q)        (multi-RHS Dslash, A epilogue)
//       last block: alpha = (r,r)/(p,q), zeta_{k+1}, alpha_i for every live shift
//   K3  r -= alpha q,  (r, r)
//       last block: beta, beta_i, shift convergence, loop control
//   K4  x_i += alpha_i p_i;  p_i = zeta_{k+1} r + beta_i p_i;  p = r + beta p
// All sums are fp64 in a fixed order; the scalar recurrences run on the device,
// so the host only polls a halt flag every chunk of iterations.
//
// Mixed precision (fp32 or bf16 Dslash, fp32 vectors): the recursive residual of
// the base system is replaced by the true one, b - (A + sigma_0) x_0 computed
// with the fp64 operator, whenever it fell by delta since the last replacement
// (reliable updates, van der Vorst & Ye; Clark et al. 2010).  x_0 is then
// accumulated in fp64.  The paper argues that a shifted solver cannot restart
// (Sec. 6); replacing the base residual keeps the shifted residuals collinear
// only approximately, which is why every shift's true residual is reported.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "solver_state.cuh"

namespace {

constexpr int VB = 256;   // block of the vector kernels

// ---------------------------------------------------------------- init
template <typename R>
__global__ void k_ms_init(SolverState* st, int Vh, const typename V2T<R>::T* __restrict__ b,
                          typename V2T<R>::T* r, typename V2T<R>::T* p, typename V2T<R>::T* ps,
                          typename V2T<R>::T* x, double* partial, unsigned int* counter) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const int ns = st->nshift;
    const size_t rs = (size_t)3 * Vh;
    double v[1] = {0.0};
    if (h < Vh) {
        Vec3<R> bv = load_vec<R>(b + rhs * rs, h, Vh);
        store_vec<R>(r + rhs * rs, h, Vh, bv);
        store_vec<R>(p + rhs * rs, h, Vh, bv);
        Vec3<R> z;
        zero(z);
        for (int s = 0; s < ns; ++s) {
            store_vec<R>(ps + ((size_t)rhs * ns + s) * rs, h, Vh, bv);
            store_vec<R>(x + ((size_t)rhs * ns + s) * rs, h, Vh, z);
        }
        v[0] = norm2(bv);
    }
    block_sum<1>(v);
    if (threadIdx.x == 0) partial[(size_t)rhs * gridDim.x + blockIdx.x] = v[0];
    if (elect_last_block(counter, gridDim.x * gridDim.y)) {
        __shared__ double sums[STAG_MAX_RHS];
        for (int q = 0; q < st->nrhs; ++q) {
            double s = block_sum_array(partial + (size_t)q * gridDim.x, gridDim.x);
            if (threadIdx.x == 0) sums[q] = s;
        }
        if (threadIdx.x == 0) {
            st->k = 0;
            st->halt = 0;
            st->status = STAG_OK;
            st->need_reliable = 0;
            st->n_reliable = 0;
            st->k4_units = 0.0;
            int any = 0;
            for (int q = 0; q < st->nrhs; ++q) {
                double bb = sums[q];
                st->bb[q] = bb;
                st->rr[q] = bb;
                st->rr_ref[q] = bb;
                st->alpha_prev[q] = 1.0;
                st->beta_prev[q] = 0.0;
                st->beta[q] = 0.0;
                int live = (bb > 0.0) && isfinite(bb);
                if (!isfinite(bb)) st->status = STAG_ERR_NAN;
                st->rhs_live[q] = live;
                any |= live;
                for (int s = 0; s < st->nshift; ++s) {
                    st->zeta[q][s] = 1.0;
                    st->zeta_prev[q][s] = 1.0;
                    st->zeta_next[q][s] = 1.0;
                    st->zratio[q][s] = 1.0;
                    st->live[q][s] = live;
                    st->iters_at[q][s] = 0;
                    st->cx[q][s] = 0.0;
                    st->cpr[q][s] = 1.0;    // p_i = zeta_0 r_0 + 0 = b in the first update
                    st->cpp[q][s] = 0.0;
                }
            }
            if (!any) st->halt = 1;
        }
    }
}

// ---------------------------------------------------------------- K1
// t = D_oe p_k without the 1/2, where the base direction p_k = r_k + beta_{k-1} p_{k-1}
// is formed on the fly at every neighbour (it is stored only by K2).
template <typename R> struct SrcRp {
    const typename V2T<R>::T* r;
    const typename V2T<R>::T* p;
    const SolverState* st;
    R beta[4];
    template <int NR> __device__ __forceinline__ void prepare(int r0, int nrhs) {
#pragma unroll
        for (int q = 0; q < NR; ++q) beta[q] = (r0 + q < nrhs) ? (R)st->beta[r0 + q] : (R)0;
    }
    __device__ __forceinline__ Vec3<R> load(int slot, int rhs, int h, int Vh) const {
        Vec3<R> a = load_vec_cg<R>(r + (size_t)rhs * 3 * Vh, h, Vh);
        Vec3<R> b = load_vec_cg<R>(p + (size_t)rhs * 3 * Vh, h, Vh);
        const R bt = beta[slot];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.c[c].re += bt * b.c[c].re;
            a.c[c].im += bt * b.c[c].im;
        }
        return a;
    }
};

template <typename R> struct EpiMsOdd {
    typename V2T<R>::T* out;
    SolverState* st;
    cudaGraphConditionalHandle cond;       // loop condition of the solver graph
    int use_cond;
    __device__ __forceinline__ bool halted() const {
        // inside the solver graph the loop continues only if the update kernel
        // of this iteration explicitly says so
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return *(volatile int*)&st->halt != 0;
    }
    template <int NR>
    __device__ __forceinline__ void finish(const Geom& g, int h, bool valid, int r0, int nrhs, Vec3<R> (&acc)[NR]) {
        if (!valid) return;
        const size_t rs = (size_t)3 * g.Vh;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r0 + r < nrhs) store_vec<R>(out + (size_t)(r0 + r) * rs, h, g.Vh, acc[r]);
    }
};

// ---------------------------------------------------------------- K2
// The scalar step once (p, A p) is known, by the whole last block: alpha per
// source, then the shifted zeta recurrence with one thread per (source, shift).
__device__ void ms_alpha_step(SolverState* st, const double* pap) {
    __shared__ double s_alpha[STAG_MAX_RHS];
    const int t = threadIdx.x;
    if (t < st->nrhs) {
        double alpha = 0.0;
        if (st->rhs_live[t]) {
            alpha = st->rr[t] / pap[t];
            if (!isfinite(alpha) || !(pap[t] > 0.0)) {
                st->status = STAG_ERR_NAN;
                st->halt = 1;
                alpha = 0.0;
            }
            st->alpha[t] = alpha;
        }
        s_alpha[t] = alpha;
    }
    __syncthreads();
    for (int idx = t; idx < st->nrhs * STAG_MAX_SHIFTS; idx += blockDim.x) {
        const int q = idx / STAG_MAX_SHIFTS, s = idx % STAG_MAX_SHIFTS;
        if (s >= st->nshift || !st->rhs_live[q] || !st->live[q][s]) continue;
        const double alpha = s_alpha[q];
        const double ap = st->alpha_prev[q], bp = st->beta_prev[q];
        const double z = st->zeta[q][s], zp = st->zeta_prev[q][s];
        // one division: zeta_{k+1} / zeta_k = zeta_{k-1} alpha_{k-1} / den
        const double den = alpha * bp * (zp - z) + zp * ap * (1.0 + st->dsig[s] * alpha);
        const double zr = zp * ap / den;
        st->zeta_next[q][s] = z * zr;
        st->zratio[q][s] = zr;
        st->cx[q][s] = alpha * zr;
    }
}

// p_k = r_k + beta_{k-1} p_{k-1} stored at the own site; q = c0 p_k - D_eo D_oe p_k;
// (p_k, q) per source; the last block runs the alpha step.
template <typename R> struct EpiMsA {
    typename V2T<R>::T* q;
    typename V2T<R>::T* p;
    const typename V2T<R>::T* r;
    SolverState* st;
    double* partial;
    unsigned int* counter;
    __device__ __forceinline__ bool halted() const { return *(volatile int*)&st->halt != 0; }
    template <int NR>
    __device__ __forceinline__ void finish(const Geom& g, int h, bool valid, int r0, int nrhs, Vec3<R> (&acc)[NR]) {
        const size_t rs = (size_t)3 * g.Vh;
        const R c0 = (R)st->c0;
        double d[NR];
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
            d[rr] = 0.0;
            if (valid && r0 + rr < nrhs) {
                const size_t off = (size_t)(r0 + rr) * rs;
                const R bt = (R)st->beta[r0 + rr];
                Vec3<R> pv = load_vec_cg<R>(p + off, h, g.Vh);
                Vec3<R> rv = load_vec_cg<R>(r + off, h, g.Vh);
                Vec3<R> o;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    pv.c[c].re = rv.c[c].re + bt * pv.c[c].re;
                    pv.c[c].im = rv.c[c].im + bt * pv.c[c].im;
                    // t = 2 D_oe p, so D_eo D_oe p = 1/4 (sum of hops of t)
                    o.c[c].re = c0 * pv.c[c].re - (R)0.25 * acc[rr].c[c].re;
                    o.c[c].im = c0 * pv.c[c].im - (R)0.25 * acc[rr].c[c].im;
                }
                store_vec<R>(p + off, h, g.Vh, pv);
                store_vec<R>(q + off, h, g.Vh, o);
                d[rr] = re_dot(pv, o);
            }
        }
        block_sum<NR>(d);
        const int nchunk = (nrhs + NR - 1) / NR;
        const int sblock = blockIdx.x / nchunk, nsb = gridDim.x / nchunk;
        if (threadIdx.x == 0) {
#pragma unroll
            for (int rr = 0; rr < NR; ++rr)
                if (r0 + rr < nrhs) partial[(size_t)(r0 + rr) * nsb + sblock] = d[rr];
        }
        if (elect_last_block(counter, gridDim.x)) {
            __shared__ double sums[STAG_MAX_RHS];
            for (int rr = 0; rr < nrhs; ++rr) {
                double s = block_sum_array(partial + (size_t)rr * nsb, nsb);
                if (threadIdx.x == 0) sums[rr] = s;
            }
            __syncthreads();
            ms_alpha_step(st, sums);
        }
    }
};

// ---------------------------------------------------------------- K3
// The scalar step once (r_{k+1}, r_{k+1}) is known, by the whole last block:
// beta, beta_i = beta (zeta_{k+1}/zeta_k)^2, shift convergence, loop control.
__device__ void ms_beta_step(SolverState* st, const double* rrn, cudaGraphConditionalHandle cond, int use_cond) {
    __shared__ double s_beta[STAG_MAX_RHS], s_rrn[STAG_MAX_RHS];
    __shared__ int s_left[STAG_MAX_RHS], s_any;
    const int t = threadIdx.x;
    if (t == 0) s_any = 0;
    if (t < st->nrhs) {
        s_left[t] = 0;
        if (st->rhs_live[t]) {
            const double rr_new = rrn[t];
            if (!isfinite(rr_new)) {
                st->status = STAG_ERR_NAN;
                st->halt = 1;
            }
            s_rrn[t] = rr_new;
            s_beta[t] = rr_new / st->rr[t];
            int n_live = 0;
            for (int s = 0; s < st->nshift; ++s) n_live += st->live[t][s];
            atomicAdd(&st->k4_units, 72.0 + 96.0 * n_live);
        }
    }
    __syncthreads();
    for (int idx = t; idx < st->nrhs * STAG_MAX_SHIFTS; idx += blockDim.x) {
        const int q = idx / STAG_MAX_SHIFTS, s = idx % STAG_MAX_SHIFTS;
        if (s >= st->nshift || !st->rhs_live[q] || !st->live[q][s]) continue;
        const double zn = st->zeta_next[q][s], z = st->zeta[q][s];
        const double zr = st->zratio[q][s];
        st->cpr[q][s] = zn;                     // p_i = zeta_{k+1} r + beta_i p_i in the next update
        st->cpp[q][s] = s_beta[q] * zr * zr;
        st->zeta_prev[q][s] = z;
        st->zeta[q][s] = zn;
        if (zn * zn * s_rrn[q] <= st->tol2 * st->bb[q]) {
            st->live[q][s] = 0;
            st->iters_at[q][s] = st->k + 1;
        } else {
            atomicOr(&s_left[q], 1);
        }
    }
    __syncthreads();
    if (t < st->nrhs && st->rhs_live[t]) {
        st->beta[t] = s_beta[t];
        st->alpha_prev[t] = st->alpha[t];
        st->beta_prev[t] = s_beta[t];
        st->rr[t] = s_rrn[t];
        if (!s_left[t]) st->rhs_live[t] = 0;
        else {
            atomicOr(&s_any, 1);
            if (st->mixed && s_rrn[t] < st->delta2 * st->rr_ref[t]) st->need_reliable = 1;
        }
    }
    __syncthreads();
    if (t == 0) {
        st->k += 1;
        if (!s_any) st->halt = 1;
        else if (st->k >= st->max_iter) { st->halt = 1; st->status = STAG_ERR_NOT_CONVERGED; }
        if (st->need_reliable) st->halt = 1;
        if (use_cond) cudaGraphSetConditional(cond, st->halt ? 0u : 1u);
    }
}

// Fused update of iteration k at every site of every live source:
//   p_i = zeta_k r_k + beta_{i,k-1} p_i ;  x_i += alpha_{i,k} p_i   (live shifts)
//   r_{k+1} = r_k - alpha_k q ;  (r_{k+1}, r_{k+1})
// A block covers VB/G sites; the G thread groups of a site share its shifts
// (group g takes shifts g, g+G, ...), and the block synchronises before group 0
// overwrites r_k, which every group reads.
template <typename R, int G>
__global__ void __launch_bounds__(VB) k_ms_update(SolverState* st, int Vh, typename V2T<R>::T* r,
                                                  const typename V2T<R>::T* __restrict__ q, typename V2T<R>::T* ps,
                                                  typename V2T<R>::T* x, double* partial, unsigned int* counter,
                                                  cudaGraphConditionalHandle cond, int use_cond) {
    if (*(volatile int*)&st->halt) return;
    constexpr int SPB = VB / G;
    const int rhs = blockIdx.y;
    const int grp = threadIdx.x / SPB;
    const int h = blockIdx.x * SPB + threadIdx.x % SPB;
    const int ns = st->nshift;
    const size_t rs = (size_t)3 * Vh;
    const bool work = st->rhs_live[rhs] && h < Vh;
    double v[1] = {0.0};
    Vec3<R> rv;
    zero(rv);
    if (work) {
        rv = load_vec_cg<R>(r + rhs * rs, h, Vh);
        // shifts grp, grp+G, ... in batches of 4: all loads of a batch before its stores
        for (int s0 = grp; s0 < ns; s0 += 4 * G) {
            Vec3<R> pv[4], xv[4];
            bool on[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int s = s0 + u * G;
                on[u] = s < ns && st->live[rhs][s];
                if (on[u]) {
                    pv[u] = load_vec_cg<R>(ps + ((size_t)rhs * ns + s) * rs, h, Vh);
                    xv[u] = load_vec_cg<R>(x + ((size_t)rhs * ns + s) * rs, h, Vh);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!on[u]) continue;
                const int s = s0 + u * G;
                const R cx = (R)st->cx[rhs][s], cpr = (R)st->cpr[rhs][s], cpp = (R)st->cpp[rhs][s];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    pv[u].c[c].re = cpr * rv.c[c].re + cpp * pv[u].c[c].re;
                    pv[u].c[c].im = cpr * rv.c[c].im + cpp * pv[u].c[c].im;
                    xv[u].c[c].re += cx * pv[u].c[c].re;
                    xv[u].c[c].im += cx * pv[u].c[c].im;
                }
                store_vec<R>(x + ((size_t)rhs * ns + s) * rs, h, Vh, xv[u]);
                store_vec<R>(ps + ((size_t)rhs * ns + s) * rs, h, Vh, pv[u]);
            }
        }
    }
    __syncthreads();
    if (work && grp == 0) {
        const R a = (R)st->alpha[rhs];
        Vec3<R> qv = load_vec_cg<R>(q + rhs * rs, h, Vh);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rv.c[c].re -= a * qv.c[c].re;
            rv.c[c].im -= a * qv.c[c].im;
        }
        store_vec<R>(r + rhs * rs, h, Vh, rv);
        v[0] = norm2(rv);
    }
    block_sum<1>(v);
    if (threadIdx.x == 0) partial[(size_t)rhs * gridDim.x + blockIdx.x] = v[0];
    if (elect_last_block(counter, gridDim.x * gridDim.y)) {
        __shared__ double sums[STAG_MAX_RHS];
        for (int q2 = 0; q2 < st->nrhs; ++q2) {
            double s = block_sum_array(partial + (size_t)q2 * gridDim.x, gridDim.x);
            if (threadIdx.x == 0) sums[q2] = s;
        }
        __syncthreads();
        ms_beta_step(st, sums, cond, use_cond);
    }
}

// ---------------------------------------------------------------- reliable update kernels
// Windowed accumulation: x64_i += x_i (fp32), x_i = 0 for every shift of every
// rhs still iterating, so fp32 rounding only ever touches one residual decade.
__global__ void k_rel_accumulate(const SolverState* st, int Vh, double2* x64, float2* x) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh || !st->rhs_live[rhs]) return;
    const size_t rs = (size_t)3 * Vh;
    for (int s = 0; s < st->nshift; ++s) {
        const size_t off = ((size_t)rhs * st->nshift + s) * rs;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            size_t i = off + (size_t)c * Vh + h;
            float2 a = x[i];
            double2 d = x64[i];
            d.x += (double)a.x;
            d.y += (double)a.y;
            x64[i] = d;
            x[i] = make_float2(0.f, 0.f);
        }
    }
}

// gather the base shift's fp64 solution of every rhs into xb64 [rhs][3][Vh]
__global__ void k_rel_gather_base(const SolverState* st, int Vh, const double2* x64, double2* xb64) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    const size_t rs = (size_t)3 * Vh;
    const size_t off = ((size_t)rhs * st->nshift + st->base) * rs;
#pragma unroll
    for (int c = 0; c < 3; ++c) xb64[rhs * rs + (size_t)c * Vh + h] = x64[off + (size_t)c * Vh + h];
}

// r = b - Ax (fp64), stored in fp32; new rr / rr_ref for the rhs still iterating
__global__ void __launch_bounds__(VB) k_rel_finish(SolverState* st, int Vh, const double2* __restrict__ b64,
                                                   const double2* __restrict__ ax, float2* r, double* partial,
                                                   unsigned int* counter) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t rs = (size_t)3 * Vh;
    double v[1] = {0.0};
    if (h < Vh && st->rhs_live[rhs]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            size_t i = rhs * rs + (size_t)c * Vh + h;
            double2 bb = b64[i], a = ax[i];
            double re = bb.x - a.x, im = bb.y - a.y;
            r[i] = make_float2((float)re, (float)im);
            v[0] += re * re + im * im;
        }
    }
    block_sum<1>(v);
    if (threadIdx.x == 0) partial[(size_t)rhs * gridDim.x + blockIdx.x] = v[0];
    if (elect_last_block(counter, gridDim.x * gridDim.y)) {
        __shared__ double sums[STAG_MAX_RHS];
        for (int q = 0; q < st->nrhs; ++q) {
            double s = block_sum_array(partial + (size_t)q * gridDim.x, gridDim.x);
            if (threadIdx.x == 0) sums[q] = s;
        }
        if (threadIdx.x == 0) {
            for (int q = 0; q < st->nrhs; ++q) {
                if (!st->rhs_live[q]) continue;
                st->rr[q] = sums[q];
                st->rr_ref[q] = sums[q];
                if (!isfinite(sums[q])) st->status = STAG_ERR_NAN;
            }
            st->need_reliable = 0;
            st->n_reliable += 1;
        }
    }
}

// x_i = (float)(x64_i + x_i) for every shift at the end of a mixed solve
__global__ void k_rel_output(const SolverState* st, int Vh, const double2* x64, float2* x) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    const size_t rs = (size_t)3 * Vh;
    for (int s = 0; s < st->nshift; ++s) {
        const size_t off = ((size_t)rhs * st->nshift + s) * rs;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            size_t i = off + (size_t)c * Vh + h;
            float2 a = x[i];
            double2 d = x64[i];
            x[i] = make_float2((float)(d.x + (double)a.x), (float)(d.y + (double)a.y));
        }
    }
}

// x64_i += x_i (fp32) for every shift: the fp64 result of a mixed solve
__global__ void k_acc_final(const SolverState* st, int Vh, double2* x64, const float2* x) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    const size_t rs = (size_t)3 * Vh;
    for (int s = 0; s < st->nshift; ++s) {
        const size_t off = ((size_t)rhs * st->nshift + s) * rs;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            size_t i = off + (size_t)c * Vh + h;
            float2 a = x[i];
            double2 d = x64[i];
            d.x += (double)a.x;
            d.y += (double)a.y;
            x64[i] = d;
        }
    }
}

// g[rhs] = x[rhs][s]  (fp64 gather of one shift)
__global__ void k_gather_shift(int Vh, int nshift, int s, const double2* x, double2* g) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    const size_t rs = (size_t)3 * Vh;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        g[rhs * rs + (size_t)c * Vh + h] = x[((size_t)rhs * nshift + s) * rs + (size_t)c * Vh + h];
}

// x[rhs][s] += e[rhs]
__global__ void k_scatter_add_shift(int Vh, int nshift, int s, const double2* e, double2* x) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    const size_t rs = (size_t)3 * Vh;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        size_t i = ((size_t)rhs * nshift + s) * rs + (size_t)c * Vh + h;
        double2 a = x[i], d = e[rhs * rs + (size_t)c * Vh + h];
        x[i] = make_double2(a.x + d.x, a.y + d.y);
    }
}

// r = b - ax - shift * x (fp64), r32 = (float) r, per-rhs partials of |r|^2 and |b|^2
__global__ void __launch_bounds__(VB) k_residual(int Vh, double shift, const double2* __restrict__ b,
                                                 const double2* __restrict__ ax, const double2* __restrict__ x,
                                                 double2* r, float2* r32, double* partial) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t rs = (size_t)3 * Vh;
    double v[2] = {0.0, 0.0};
    if (h < Vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            size_t i = rhs * rs + (size_t)c * Vh + h;
            double re = b[i].x - ax[i].x - shift * x[i].x;
            double im = b[i].y - ax[i].y - shift * x[i].y;
            if (r) r[i] = make_double2(re, im);
            if (r32) r32[i] = make_float2((float)re, (float)im);
            v[0] += re * re + im * im;
            v[1] += b[i].x * b[i].x + b[i].y * b[i].y;
        }
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
        partial[(size_t)(2 * rhs) * gridDim.x + blockIdx.x] = v[0];
        partial[(size_t)(2 * rhs + 1) * gridDim.x + blockIdx.x] = v[1];
    }
}

__global__ void k_d2df(size_t n, const double2* a, float4* b) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = a[i];
    b[i] = f4_of(mk(DF(v.x), DF(v.y)));
}

__global__ void k_df2d(size_t n, const float4* a, double2* b) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Cx<DF> v = cx_of(a[i]);
    b[i] = make_double2((double)v.re, (double)v.im);
}

__global__ void k_d2f(size_t n, const double2* a, float2* b) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}


}  // namespace


// ---------------------------------------------------------------- host driver
// five consecutive events of the profiling pool (created on first use)
static stag_status prof_events(stag_ctx* ctx, int* ev) {
    ProfData& pf = ctx->prof;
    if (pf.used + 4 > 50000) { pf.on = false; return STAG_OK; }
    while (pf.pool.size() < pf.used + 4) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        pf.pool.push_back(e);
    }
    for (int k = 0; k < 4; ++k) ev[k] = (int)(pf.used + k);
    pf.used += 4;
    return STAG_OK;
}
// the two Dslash launches of one iteration for a given link format, sources
// per thread and threads per site
template <typename R, int FMT, int NR, int TPS>
static void ms_dslash_pair(cudaStream_t stream, int grid, const Geom& g, const LinkPtrs& L, const SrcRp<R>& s1,
                           const SrcPlain<R>& s2, const EpiMsOdd<R>& e1, const EpiMsA<R>& e2, int nrhs, int nchunk,
                           cudaEvent_t mid) {
    const int bs = STAG_DSLASH_BLOCK;
    k_dslash<R, FMT, NR, TPS, SrcRp<R>, EpiMsOdd<R>><<<grid, bs, 0, stream>>>(g, 1, L, s1, nrhs, nchunk, e1);
    if (mid) cudaEventRecord(mid, stream);
    k_dslash<R, FMT, NR, TPS, SrcPlain<R>, EpiMsA<R>><<<grid, bs, 0, stream>>>(g, 0, L, s2, nrhs, nchunk, e2);
}

// the same pair for the improved operator (fat and Naik links)
template <typename R, int FMT, int NR, int TPS>
static void ms_dslash_pair_asq(cudaStream_t stream, int grid, const Geom& g, const AsqLinks& A, const SrcRp<R>& s1,
                               const SrcPlain<R>& s2, const EpiMsOdd<R>& e1, const EpiMsA<R>& e2, int nrhs,
                               int nchunk, cudaEvent_t mid) {
    const int bs = STAG_DSLASH_BLOCK;
    k_dslash_asq<R, FMT, NR, TPS, SrcRp<R>, EpiMsOdd<R>><<<grid, bs, 0, stream>>>(g, 1, A, s1, nrhs, nchunk, e1);
    if (mid) cudaEventRecord(mid, stream);
    k_dslash_asq<R, FMT, NR, TPS, SrcPlain<R>, EpiMsA<R>><<<grid, bs, 0, stream>>>(g, 0, A, s2, nrhs, nchunk, e2);
}

template <typename R, int FMT, int NR>
static void ms_dslash_asq_tps(int tps, cudaStream_t stream, int grid, const Geom& g, const AsqLinks& A,
                              const SrcRp<R>& s1, const SrcPlain<R>& s2, const EpiMsOdd<R>& e1, const EpiMsA<R>& e2,
                              int nrhs, int nchunk, cudaEvent_t mid) {
    switch (tps) {
        case 8: ms_dslash_pair_asq<R, FMT, NR, 8>(stream, grid, g, A, s1, s2, e1, e2, nrhs, nchunk, mid); break;
        case 4: ms_dslash_pair_asq<R, FMT, NR, 4>(stream, grid, g, A, s1, s2, e1, e2, nrhs, nchunk, mid); break;
        case 2: ms_dslash_pair_asq<R, FMT, NR, 2>(stream, grid, g, A, s1, s2, e1, e2, nrhs, nchunk, mid); break;
        default: ms_dslash_pair_asq<R, FMT, NR, 1>(stream, grid, g, A, s1, s2, e1, e2, nrhs, nchunk, mid); break;
    }
}

template <typename R, int FMT>
static void ms_dslash_asq(int nr, int tps, cudaStream_t stream, int grid, const Geom& g, const AsqLinks& A,
                          const SrcRp<R>& s1, const SrcPlain<R>& s2, const EpiMsOdd<R>& e1, const EpiMsA<R>& e2,
                          int nrhs, int nchunk, cudaEvent_t mid) {
    if (nr == 4) ms_dslash_asq_tps<R, FMT, 4>(tps, stream, grid, g, A, s1, s2, e1, e2, nrhs, nchunk, mid);
    else ms_dslash_asq_tps<R, FMT, 1>(tps, stream, grid, g, A, s1, s2, e1, e2, nrhs, nchunk, mid);
}

template <typename R, int FMT, int NR>
static void ms_dslash_tps(int tps, cudaStream_t stream, int grid, const Geom& g, const LinkPtrs& L,
                          const SrcRp<R>& s1, const SrcPlain<R>& s2, const EpiMsOdd<R>& e1, const EpiMsA<R>& e2,
                          int nrhs, int nchunk, cudaEvent_t mid) {
    switch (tps) {
        case 8: ms_dslash_pair<R, FMT, NR, 8>(stream, grid, g, L, s1, s2, e1, e2, nrhs, nchunk, mid); break;
        case 4: ms_dslash_pair<R, FMT, NR, 4>(stream, grid, g, L, s1, s2, e1, e2, nrhs, nchunk, mid); break;
        case 2: ms_dslash_pair<R, FMT, NR, 2>(stream, grid, g, L, s1, s2, e1, e2, nrhs, nchunk, mid); break;
        default: ms_dslash_pair<R, FMT, NR, 1>(stream, grid, g, L, s1, s2, e1, e2, nrhs, nchunk, mid); break;
    }
}

template <typename R, int FMT>
static void ms_dslash(int nr, int tps, cudaStream_t stream, int grid, const Geom& g, const LinkPtrs& L,
                      const SrcRp<R>& s1, const SrcPlain<R>& s2, const EpiMsOdd<R>& e1, const EpiMsA<R>& e2,
                      int nrhs, int nchunk, cudaEvent_t mid) {
    if (nr == 4) ms_dslash_tps<R, FMT, 4>(tps, stream, grid, g, L, s1, s2, e1, e2, nrhs, nchunk, mid);
    else ms_dslash_tps<R, FMT, 1>(tps, stream, grid, g, L, s1, s2, e1, e2, nrhs, nchunk, mid);
}

constexpr int UPDATE_GROUPS = 4;

template <typename R>
static stag_status ms_iterations(stag_ctx* ctx, cudaStream_t stream, stag_prec prec, int nrhs, int chunk, void* tmp,
                                 void* r, void* p, void* q, void* ps, void* x, bool sample,
                                 cudaGraphConditionalHandle cond, int use_cond) {
    typedef typename V2T<R>::T V;
    const Geom& g = ctx->g;
    const int nr = dslash_nr_for(nrhs);
    const int tps = ctx->asqtad ? asq_tps(ctx) : dslash_tps(ctx, prec, nr);
    const int nchunk = (nrhs + nr - 1) / nr;
    const int grid_d = nblocks(g.Vh, STAG_DSLASH_BLOCK / tps) * nchunk;
    dim3 grid_u(nblocks(g.Vh, VB / UPDATE_GROUPS), nrhs);
    LinkPtrs L = link_ptrs(ctx);
    SrcRp<R> src1{(const V*)r, (const V*)p, ctx->st, {}};
    SrcPlain<R> src2{(const V*)tmp};
    EpiMsOdd<R> e1{(V*)tmp, ctx->st, cond, use_cond};
    EpiMsA<R> e2{(V*)q, (V*)p, (const V*)r, ctx->st, ctx->red, ctx->counters + 0};
    ProfData& pf = ctx->prof;
    for (int it = 0; it < chunk; ++it) {
        const bool smp = sample && pf.on;
        int ev[4];
        if (smp) {
            CKS(prof_events(ctx, ev));
            CK(cudaEventRecord(pf.pool[ev[0]], stream));
        }
        cudaEvent_t mid = smp ? pf.pool[ev[1]] : nullptr;
        if (ctx->asqtad) {
            const AsqLinks A = asq_links(ctx);
            if constexpr (sizeof(R) == 8) ms_dslash_asq<R, FMT_F64>(nr, tps, stream, grid_d, g, A, src1, src2, e1, e2, nrhs, nchunk, mid);
            else ms_dslash_asq<R, FMT_F32_18>(nr, tps, stream, grid_d, g, A, src1, src2, e1, e2, nrhs, nchunk, mid);
        } else if constexpr (sizeof(R) == 8) {
            ms_dslash<R, FMT_F64>(nr, tps, stream, grid_d, g, L, src1, src2, e1, e2, nrhs, nchunk, mid);
        } else {
            if (prec == STAG_FP32) ms_dslash<R, FMT_F32_18>(nr, tps, stream, grid_d, g, L, src1, src2, e1, e2, nrhs, nchunk, mid);
            else if (prec == STAG_FP32_12) ms_dslash<R, FMT_F32_12>(nr, tps, stream, grid_d, g, L, src1, src2, e1, e2, nrhs, nchunk, mid);
            else ms_dslash<R, FMT_BF16_12>(nr, tps, stream, grid_d, g, L, src1, src2, e1, e2, nrhs, nchunk, mid);
        }
        if (smp) CK(cudaEventRecord(pf.pool[ev[2]], stream));
        k_ms_update<R, UPDATE_GROUPS><<<grid_u, VB, 0, stream>>>(ctx->st, g.Vh, (V*)r, (const V*)q, (V*)ps, (V*)x,
                                                                 ctx->red, ctx->counters + 1, cond, use_cond);
        if (smp) {
            CK(cudaEventRecord(pf.pool[ev[3]], stream));
            for (int k = 0; k < 3; ++k) pf.marks[k].push_back({ev[k], ev[k + 1]});
        }
    }
    if (!use_cond) ctx->launches += 3LL * chunk;
    CK(cudaGetLastError());
    return STAG_OK;
}

static size_t rsize(stag_prec p) { return p == STAG_FP64 ? sizeof(double) : sizeof(float); }

// One solver iteration as the body of a WHILE conditional node: the graph
// replays iterations on the device until the r-update's last block stops it
// (convergence, a due reliable update, max_iter or a NaN), so the host waits
// once per segment instead of launching four kernels per iteration.

static stag_status solver_graph(stag_ctx* ctx, stag_prec prec, int nrhs, void* tmp, void* r, void* p, void* q,
                                void* ps, void* x, cudaGraphExec_t* out) {
    const void* key[8] = {tmp, r, p, q, ps, x, ctx->st, ctx->red};
    const int pkey = (int)prec + (ctx->asqtad ? 16 : 0);    // the operator is part of the captured launches
    auto& cache = ctx->graphs;
    for (auto& e : cache) {
        if (e.prec == pkey && e.nrhs == nrhs && std::memcmp(e.key, key, sizeof(key)) == 0) {
            *out = e.exec;
            return STAG_OK;
        }
    }
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    SolverGraphEntry sg = {};
    std::memcpy(sg.key, key, sizeof(key));
    sg.prec = pkey;
    sg.nrhs = nrhs;
    CK(cudaGraphCreate(&sg.graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, sg.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, sg.graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    stag_status s;
    if (prec == STAG_FP64) s = ms_iterations<DF>(ctx, ctx->cap_stream, prec, nrhs, 1, tmp, r, p, q, ps, x, false, h, 1);
    else s = ms_iterations<float>(ctx, ctx->cap_stream, prec, nrhs, 1, tmp, r, p, q, ps, x, false, h, 1);
    cudaGraph_t captured;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &captured);
    if (s != STAG_OK) return s;
    CK(e);
    CK(cudaGraphInstantiate(&sg.exec, sg.graph, 0));
    if (cache.size() >= 12) {      // a few live configurations are enough
        cudaGraphExecDestroy(cache.front().exec);
        cudaGraphDestroy(cache.front().graph);
        cache.erase(cache.begin());
    }
    cache.push_back(sg);
    *out = sg.exec;
    return STAG_OK;
}

void destroy_solver_graphs(stag_ctx* ctx) {
    for (auto& e : ctx->graphs) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        if (e.graph) cudaGraphDestroy(e.graph);
    }
    ctx->graphs.clear();
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    ctx->cap_stream = nullptr;
}

static stag_status pull_state(stag_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(SolverState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return STAG_OK;
}

// the loop-control words only (k .. k4_units)
static stag_status pull_control(stag_ctx* ctx) {
    const size_t off = offsetof(SolverState, k);
    const size_t len = offsetof(SolverState, rhs_live) - off;
    CK(cudaMemcpyAsync((char*)ctx->st_host + off, (const char*)ctx->st + off, len, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return STAG_OK;
}

stag_status ms_setup(MsRun& R) {
    stag_ctx* ctx = R.ctx;
    const Geom& g = ctx->g;
    R.mixed = R.prec != STAG_FP64;
    if (R.nrhs < 1 || R.nrhs > STAG_MAX_RHS || R.nshift < 1 || R.nshift > STAG_MAX_SHIFTS) return STAG_ERR_ARG;
    if (ctx->asqtad && R.prec != STAG_FP64 && R.prec != STAG_FP32) return STAG_ERR_ARG;
    CKS(asq_ensure(ctx));
    if (R.mixed && R.reliable && (!R.b64 || !R.x64)) return STAG_ERR_ARG;
    // the bf16 copy must follow every link update before a bf16 iteration
    if (R.prec == STAG_BF16_12 && ctx->b16_stale) CKS(refresh_bf16(ctx));
    R.base = 0;
    for (int s = 0; s < R.nshift; ++s)
        if (R.shifts[s] < R.shifts[R.base]) R.base = s;
    const size_t vbytes = (size_t)R.nrhs * 3 * g.Vh * 2 * rsize(R.prec);
    CKS(ws_get(ctx, WS_TMP_ODD, vbytes, &R.tmp));
    // the persistent solver keeps a ring of residuals (slot 0 here, where the
    // other paths keep their only one)
    CKS(ws_get(ctx, WS_R, vbytes * persistent_ring_slots(), &R.r));
    R.rstride = (size_t)R.nrhs * 3 * g.Vh;
    CKS(ws_get(ctx, WS_P, vbytes, &R.p));
    CKS(ws_get(ctx, WS_Q, vbytes, &R.q));
    CKS(ws_get(ctx, WS_PS, vbytes * R.nshift, &R.ps));
    const size_t v64 = (size_t)R.nrhs * 3 * g.Vh * sizeof(double2);
    R.use_rel = R.mixed && R.reliable;
    if (R.use_rel) {
        CKS(ws_get(ctx, WS_R64, v64, &R.ax64));
        CKS(ws_get(ctx, WS_T64, v64, &R.t64));
        CKS(ws_get(ctx, WS_U64, v64, &R.xb64));
    }
    if (R.mixed && R.x64) CK(cudaMemsetAsync(R.x64, 0, v64 * R.nshift, ctx->stream));
    // fp64 solves iterate in float-float (Sec. 5: the two-float representation
    // used directly): b and x are double on the outside, float-float inside
    R.b_user = R.b;
    R.x_user = R.x;
    if (!R.mixed) {
        void *bdf, *xdf;
        CKS(ws_get(ctx, WS_B_DF, v64, &bdf));
        CKS(ws_get(ctx, WS_X_DF, v64 * R.nshift, &xdf));
        k_d2df<<<nblocks((long long)R.nrhs * 3 * g.Vh, 256), 256, 0, ctx->stream>>>(
            (size_t)R.nrhs * 3 * g.Vh, (const double2*)R.b_user, (float4*)bdf);
        CKL();
        R.b = bdf;
        R.x = xdf;
    }
    SolverState* hs = ctx->st_host;
    std::memset(hs, 0, sizeof(SolverState));
    hs->nrhs = R.nrhs;
    hs->nshift = R.nshift;
    hs->base = R.base;
    hs->max_iter = R.max_iter;
    hs->mixed = R.use_rel ? 1 : 0;
    hs->tol2 = R.tol * R.tol;
    hs->c0 = R.mass * R.mass + R.shifts[R.base];
    hs->delta2 = 0.01;   // replace the residual after every factor 10 in ||r||
    for (int s = 0; s < R.nshift; ++s) hs->dsig[s] = R.shifts[s] - R.shifts[R.base];
    // staged: with deferred solves the host fills hs for the next solve before this copy has run
    static_assert(sizeof(SolverState) <= STAGE_SLOT_BYTES, "the solver state fits a staging slot");
    CKS(stage_upload(ctx, ctx->st, hs, sizeof(SolverState)));
    dim3 grid_v(nblocks(g.Vh, VB), R.nrhs);
    if (R.mixed)
        k_ms_init<float><<<grid_v, VB, 0, ctx->stream>>>(ctx->st, g.Vh, (const float2*)R.b, (float2*)R.r,
                                                         (float2*)R.p, (float2*)R.ps, (float2*)R.x, ctx->red,
                                                         ctx->counters + 2);
    else
        k_ms_init<DF><<<grid_v, VB, 0, ctx->stream>>>(ctx->st, g.Vh, (const float4*)R.b, (float4*)R.r,
                                                      (float4*)R.p, (float4*)R.ps, (float4*)R.x, ctx->red,
                                                      ctx->counters + 2);
    CKL();
    return STAG_OK;
}

// fp64 accumulation of every shift, then the true base residual
// b - (A + s0) x0 with the fp64 operator replaces the recursive one; the
// solve may then continue (halt cleared)
stag_status ms_reliable_update(MsRun& R) {
    stag_ctx* ctx = R.ctx;
    const Geom& g = ctx->g;
    dim3 grid_v(nblocks(g.Vh, VB), R.nrhs);
    SolverState* hs = ctx->st_host;
    k_rel_accumulate<<<grid_v, VB, 0, ctx->stream>>>(ctx->st, g.Vh, R.x64, (float2*)R.x);
    k_rel_gather_base<<<grid_v, VB, 0, ctx->stream>>>(ctx->st, g.Vh, R.x64, (double2*)R.xb64);
    CKS(launch_apply_a(ctx, hs->c0, STAG_FP64, R.nrhs, R.xb64, R.ax64, R.t64));
    k_rel_finish<<<grid_v, VB, 0, ctx->stream>>>(ctx->st, g.Vh, R.b64, (const double2*)R.ax64, (float2*)R.r,
                                                 ctx->red, ctx->counters + 3);
    ctx->launches += 3;
    CK(cudaGetLastError());
    hs->halt = 0;
    CK(cudaMemcpyAsync(&ctx->st->halt, &hs->halt, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    return STAG_OK;
}

// the solutions in the caller's format once the iteration has stopped
stag_status ms_finish(MsRun& R) {
    stag_ctx* ctx = R.ctx;
    const Geom& g = ctx->g;
    dim3 grid_v(nblocks(g.Vh, VB), R.nrhs);
    if (!R.mixed) {
        const size_t n = (size_t)R.nrhs * R.nshift * 3 * g.Vh;
        k_df2d<<<nblocks((long long)n, 256), 256, 0, ctx->stream>>>(n, (const float4*)R.x, (double2*)R.x_user);
        CKL();
        R.x = R.x_user;
        R.b = R.b_user;
    }
    if (R.mixed && R.x64) {
        if (R.finish_to_f64) k_acc_final<<<grid_v, VB, 0, ctx->stream>>>(ctx->st, g.Vh, R.x64, (const float2*)R.x);
        else k_rel_output<<<grid_v, VB, 0, ctx->stream>>>(ctx->st, g.Vh, R.x64, (float2*)R.x);
        CKL();
    }
    return STAG_OK;
}

void ms_stats(const MsRun& R, MsStats* stats) {
    if (!stats) return;
    const SolverState* hs = R.ctx->st_host;
    stats->iterations = hs->k;
    stats->reliable = hs->n_reliable;
    for (int s = 0; s < R.nshift; ++s) {
        int it = 0;
        for (int q2 = 0; q2 < R.nrhs; ++q2) it = hs->iters_at[q2][s] > it ? hs->iters_at[q2][s] : it;
        stats->shift_iterations[s] = it;
    }
}

stag_status ms_pull_state(stag_ctx* ctx) { return pull_state(ctx); }

// ---------------------------------------------------------------- deferred solves
// After a persistent launch, on the device: what ms_core would otherwise
// read on the host (iterations, residual replacements, the algorithmic bytes
// of the profile, and whether the launch halted with a usable status).
__global__ void k_solve_note(const SolverState* st, SolveNote* note, int w, double vh, double bytes_iter,
                             double unit_scale) {
    const long long k = st->k;
    note->iters[w] += k;
    note->reliable += st->n_reliable;
    note->bytes[w] += (double)k * vh * bytes_iter + st->k4_units * vh * unit_scale;
    note->solves += 1;
    if (note->err == 0) {
        if (!st->halt) note->err = STAG_ERR_TIMEOUT;
        else if (st->status != STAG_OK && st->status != STAG_ERR_NOT_CONVERGED) note->err = st->status;
    }
}

stag_status defer_begin(stag_ctx* ctx) {
    CK(cudaMemsetAsync(ctx->note, 0, sizeof(SolveNote), ctx->stream));
    ctx->defer = persistent_fits(ctx);
    return STAG_OK;
}

stag_status defer_end(stag_ctx* ctx, long long* iters, long long* reliable) {
    if (!ctx->defer) return STAG_OK;
    ctx->defer = false;
    SolveNote n;
    CK(cudaMemcpyAsync(&n, ctx->note, sizeof(n), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (iters) *iters += n.iters[0] + n.iters[1];
    if (reliable) *reliable += n.reliable;
    ProfData& pf = ctx->prof;
    for (int w = 0; w < 2; ++w) {
        double ms = 0.0;
        for (auto& e : ctx->deferred_ev[w]) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, e.first, e.second) == cudaSuccess) ms += t;
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        const bool timed = !ctx->deferred_ev[w].empty();
        ctx->deferred_ev[w].clear();
        if (pf.on && timed) {
            const int kind = w == 0 ? PK_PERSISTENT : PK_PERSISTENT_FF;
            pf.bytes_total[kind] += n.bytes[w];
            pf.launches[kind] += n.iters[w];
            pf.persist_ms[w] += ms;
            pf.persist_iters[w] += n.iters[w];
        }
    }
    cudaGetLastError();
    return n.err ? (stag_status)n.err : STAG_OK;
}
stag_status ms_pull_control_async(stag_ctx* ctx) {
    const size_t off = offsetof(SolverState, k);
    const size_t len = offsetof(SolverState, rhs_live) - off;
    CK(cudaMemcpyAsync((char*)ctx->st_host + off, (const char*)ctx->st + off, len, cudaMemcpyDeviceToHost,
                       ctx->stream));
    return STAG_OK;
}

stag_status ms_core(stag_ctx* ctx, double mass, int nshift, const double* shifts, stag_prec prec, int nrhs,
                    const void* b, const double2* b64, void* x, double2* x64, double tol, int max_iter,
                    bool reliable, bool finish_to_f64, MsStats* stats) {
    const Geom& g = ctx->g;
    MsRun R;
    R.ctx = ctx;
    R.mass = mass;
    R.nshift = nshift;
    R.shifts = shifts;
    R.prec = prec;
    R.nrhs = nrhs;
    R.b = b;
    R.b64 = b64;
    R.x = x;
    R.x64 = x64;
    R.tol = tol;
    R.max_iter = max_iter;
    R.reliable = reliable;
    R.finish_to_f64 = finish_to_f64;
    CKS(ms_setup(R));
    const bool mixed = R.mixed;
    SolverState* hs = ctx->st_host;
    stag_status status = STAG_OK;
    cudaGraphExec_t gexec = nullptr;
    const bool persistent = persistent_fits(ctx);
    bool deferred = false;
    if (!persistent) {
        if (!ctx->asqtad) dslash_tps(ctx, prec, dslash_nr_for(nrhs));   // tune before any capture
        if (ctx->use_graphs) CKS(solver_graph(ctx, prec, nrhs, R.tmp, R.r, R.p, R.q, R.ps, R.x, &gexec));
    }
    cudaEvent_t pe0 = nullptr, pe1 = nullptr;
    double persist_ms = 0.0;
    if (persistent && ctx->prof.on) {
        CK(cudaEventCreate(&pe0));
        CK(cudaEventCreate(&pe1));
    }
    // every segment either ends the solve or makes a reliable update (at most
    // one per decade of the residual), so the number of segments is bounded
    const int max_segments = ctx->use_graphs ? 64 + max_iter / 4 : 64 + max_iter;
    const int chunk = 16;
    for (int seg = 0;; ++seg) {
        if (seg > max_segments) { status = STAG_ERR_TIMEOUT; break; }
        if (persistent) {
            // one launch runs the whole solve, reliable updates included
            if (pe0) CK(cudaEventRecord(pe0, ctx->stream));
            CKS(launch_persistent(ctx, prec, nrhs, R.r, R.rstride, R.p, R.q, R.tmp, R.ps, R.x,
                                  R.use_rel ? R.b64 : nullptr, R.use_rel ? R.x64 : nullptr,
                                  R.use_rel ? (double2*)R.t64 : nullptr));
            if (pe1) CK(cudaEventRecord(pe1, ctx->stream));
            if (ctx->defer) {
                // no host read: the note takes the iterations, the algorithmic
                // bytes and the first error; the events wait for defer_end
                const double S = 3.0 * (double)(mixed ? sizeof(float2) : sizeof(double2));
                k_solve_note<<<1, 1, 0, ctx->stream>>>(ctx->st, ctx->note, mixed ? 0 : 1, (double)g.Vh,
                                                       2.0 * op_link_bytes_site(ctx, prec) + 8.0 * S * nrhs,
                                                       mixed ? 1.0 : 2.0);
                CKL();
                if (pe0) {
                    ctx->deferred_ev[mixed ? 0 : 1].push_back({pe0, pe1});
                    pe0 = pe1 = nullptr;
                }
                deferred = true;
                break;
            }
            CKS(pull_control(ctx));
            if (pe0) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, pe0, pe1));
                persist_ms += ms;
            }
            if (!hs->halt) { status = STAG_ERR_TIMEOUT; break; }   // the loop only ends by halting
            if (hs->status != STAG_OK) status = (stag_status)hs->status;
            break;
        }
        // sampled timing: a few plainly launched iterations at the start of every segment
        if (ctx->prof.on) {
            if (mixed) CKS(ms_iterations<float>(ctx, ctx->stream, prec, nrhs, 4, R.tmp, R.r, R.p, R.q, R.ps, R.x,
                                                true, 0, 0));
            else CKS(ms_iterations<DF>(ctx, ctx->stream, prec, nrhs, 4, R.tmp, R.r, R.p, R.q, R.ps, R.x, true, 0, 0));
        }
        if (gexec) {
            CK(cudaGraphLaunch(gexec, ctx->stream));
            ++ctx->launches;
        } else if (mixed) {
            CKS(ms_iterations<float>(ctx, ctx->stream, prec, nrhs, chunk, R.tmp, R.r, R.p, R.q, R.ps, R.x, false, 0,
                                     0));
        } else {
            CKS(ms_iterations<DF>(ctx, ctx->stream, prec, nrhs, chunk, R.tmp, R.r, R.p, R.q, R.ps, R.x, false, 0, 0));
        }
        CKS(pull_control(ctx));
        if (!hs->halt) continue;
        if (hs->status != STAG_OK) { status = (stag_status)hs->status; break; }
        if (hs->need_reliable) {
            CKS(ms_reliable_update(R));
            continue;
        }
        break;   // converged
    }
    if (deferred) {
        CKS(ms_finish(R));
        if (stats) std::memset(stats, 0, sizeof(*stats));   // the note has them; defer_end reads it
        return STAG_OK;
    }
    CKS(pull_state(ctx));
    if (pe0) cudaEventDestroy(pe0);
    if (pe1) cudaEventDestroy(pe1);
    if (gexec) ctx->launches += 3LL * hs->k;   // kernels the graph ran
    if (persistent && ctx->prof.on) {
        ProfData& pf = ctx->prof;
        // bytes of one spinor (3 colours) at a site
        const double S = 3.0 * (double)(mixed ? sizeof(float2) : sizeof(double2));
        // one iteration: both Dslash phases (links twice; r, p in, t out / t, p, r in,
        // p, q out) and the updates (r, q in, r out and 96 B per live shift: k4_units)
        const int kind = mixed ? PK_PERSISTENT : PK_PERSISTENT_FF;
        pf.bytes_total[kind] += (double)hs->k * g.Vh * (2.0 * op_link_bytes_site(ctx, prec) + 8.0 * S * nrhs) +
                                hs->k4_units * g.Vh * (mixed ? 1.0 : 2.0);
        pf.launches[kind] += hs->k;
        pf.persist_ms[mixed ? 0 : 1] += persist_ms;
        pf.persist_iters[mixed ? 0 : 1] += hs->k;
    } else if (ctx->prof.on) {
        ProfData& pf = ctx->prof;
        const double S = 3.0 * (double)(mixed ? sizeof(float2) : sizeof(double2));   // one spinor at a site
        // K1 reads r and p (the direction is formed on the fly) and writes t;
        // K2 reads t, r, p and writes p, q
        const double lb = op_link_bytes_site(ctx, prec);
        pf.bytes_total[PK_DSLASH_OE] += (double)hs->k * g.Vh * (lb + 3.0 * S * nrhs);
        pf.bytes_total[PK_DSLASH_EO_A] += (double)hs->k * g.Vh * (lb + 5.0 * S * nrhs);
        for (int kk = PK_DSLASH_OE; kk <= PK_UPDATE; ++kk) pf.launches[kk] += hs->k;
    }
    CKS(ms_finish(R));
    if (ctx->prof.on && !persistent) ctx->prof.bytes_total[PK_UPDATE] += hs->k4_units * g.Vh * (mixed ? 1.0 : 2.0);
    ms_stats(R, stats);
    return status;
}

// ||b - (A + s) x_s|| / ||b|| for every rhs of one shift, fp64 (x fp64, all shifts).
// Leaves the fp64 residual in WS_REF_R64 and its fp32 copy in WS_REF_B32.
static stag_status shift_residuals(stag_ctx* ctx, double mass, int nshift, int s, double shift, int nrhs,
                                   const double2* b, const double2* x, double* rel_out) {
    const Geom& g = ctx->g;
    const size_t v64 = (size_t)nrhs * 3 * g.Vh * sizeof(double2);
    void *gx, *ax, *t, *r64, *r32;
    CKS(ws_get(ctx, WS_REF_G, v64, &gx));
    CKS(ws_get(ctx, WS_REF_AX, v64, &ax));
    CKS(ws_get(ctx, WS_REF_T, v64, &t));
    CKS(ws_get(ctx, WS_REF_R64, v64, &r64));
    CKS(ws_get(ctx, WS_REF_B32, v64 / 2, &r32));
    dim3 grid_v(nblocks(g.Vh, VB), nrhs);
    k_gather_shift<<<grid_v, VB, 0, ctx->stream>>>(g.Vh, nshift, s, x, (double2*)gx);
    CKS(launch_apply_a(ctx, mass * mass, STAG_FP64, nrhs, gx, ax, t));
    k_residual<<<grid_v, VB, 0, ctx->stream>>>(g.Vh, shift, b, (const double2*)ax, (const double2*)gx,
                                               (double2*)r64, (float2*)r32, ctx->red);
    ctx->launches += 2;
    CK(cudaGetLastError());
    std::vector<double> part((size_t)2 * nrhs * grid_v.x);
    CK(cudaMemcpyAsync(part.data(), ctx->red, part.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < nrhs; ++q) {
        double num = 0.0, den = 0.0;
        for (unsigned i = 0; i < grid_v.x; ++i) {
            num += part[(size_t)(2 * q) * grid_v.x + i];
            den += part[(size_t)(2 * q + 1) * grid_v.x + i];
        }
        rel_out[q] = den > 0 ? std::sqrt(num / den) : 0.0;
    }
    return STAG_OK;
}

// Per-shift refinement of fp64 solutions: while a shift's true residual is
// above tol, solve (A + s) e = r with a single-shift fp32 CG whose residual is
// replaced in fp64 every decade (reliable updates; with one shift the solver
// can restart, unlike the multi-shift one, Sec. 6), then x_s += e.
static stag_status refine_shifts(stag_ctx* ctx, double mass, int nshift, const double* shifts, int nrhs,
                                 const double2* b, double2* x, double tol, int max_iter, int* extra_iters,
                                 int* n_reliable, double* final_res) {
    const Geom& g = ctx->g;
    const size_t v64 = (size_t)nrhs * 3 * g.Vh * sizeof(double2);
    void *e32, *e64;
    CKS(ws_get(ctx, WS_REF_E32, v64 / 2, &e32));
    CKS(ws_get(ctx, WS_REF_E64, v64, &e64));
    dim3 grid_v(nblocks(g.Vh, VB), nrhs);
    for (int s = 0; s < nshift; ++s) {
        double rel[STAG_MAX_RHS];
        double worst = 0.0;
        for (int round = 0; round < 6; ++round) {
            CKS(shift_residuals(ctx, mass, nshift, s, shifts[s], nrhs, b, x, rel));
            worst = 0.0;
            double ratio = 1e300;
            for (int q = 0; q < nrhs; ++q) {
                worst = rel[q] > worst ? rel[q] : worst;
                if (rel[q] > 0) ratio = std::min(ratio, tol / rel[q]);
            }
            if (worst <= tol) break;
            double tol_in = std::min(0.5, std::max(0.5 * ratio, 1e-12));
            MsStats st;
            void *r64, *r32;
            CKS(ws_get(ctx, WS_REF_R64, v64, &r64));
            CKS(ws_get(ctx, WS_REF_B32, v64 / 2, &r32));
            stag_status rs = ms_core(ctx, mass, 1, &shifts[s], STAG_FP32, nrhs, r32, (const double2*)r64, e32,
                                     (double2*)e64, tol_in, max_iter, true, true, &st);
            if (rs != STAG_OK && rs != STAG_ERR_NOT_CONVERGED) return rs;
            *extra_iters += st.iterations;
            *n_reliable += st.reliable;
            k_scatter_add_shift<<<grid_v, VB, 0, ctx->stream>>>(g.Vh, nshift, s, (const double2*)e64, x);
            CKL();
        }
        final_res[s] = worst;
    }
    return STAG_OK;
}

static stag_status ms_api_batch(stag_ctx* ctx, double mass, int nshift, const double* shifts, stag_prec prec,
                                int nrhs, const double2* b, double2* x, double tol, int max_iter,
                                stag_solve_info* info) {
    const Geom& g = ctx->g;
    MsStats st;
    std::memset(&st, 0, sizeof(st));
    stag_status status;
    int extra = 0, nrel = 0;
    double res[STAG_MAX_SHIFTS] = {0};
    if (prec == STAG_FP64) {
        status = ms_core(ctx, mass, nshift, shifts, prec, nrhs, b, nullptr, x, nullptr, tol, max_iter, false, true,
                         &st);
        if (status != STAG_OK && status != STAG_ERR_NOT_CONVERGED) return status;
        for (int s = 0; s < nshift; ++s) {
            double rel[STAG_MAX_RHS];
            CKS(shift_residuals(ctx, mass, nshift, s, shifts[s], nrhs, b, x, rel));
            for (int q = 0; q < nrhs; ++q) res[s] = rel[q] > res[s] ? rel[q] : res[s];
        }
    } else {
        const size_t n = (size_t)nrhs * 3 * g.Vh;
        void *b32, *x32;
        CKS(ws_get(ctx, WS_B32, n * sizeof(float2), &b32));
        CKS(ws_get(ctx, WS_X32, n * nshift * sizeof(float2), &x32));
        k_d2f<<<nblocks((long long)n, 256), 256, 0, ctx->stream>>>(n, b, (float2*)b32);
        CKL();
        // residual replacement keeps the shifted recurrences consistent only when
        // the iteration operator is the fp32 one; the bf16 operator iterates plainly
        const bool rel = prec != STAG_BF16_12;
        status = ms_core(ctx, mass, nshift, shifts, prec, nrhs, b32, b, x32, x, tol, max_iter, rel, true, &st);
        if (status != STAG_OK && status != STAG_ERR_NOT_CONVERGED) return status;
        // refinement only follows a converged multi-shift stage
        if (status == STAG_OK) CKS(refine_shifts(ctx, mass, nshift, shifts, nrhs, b, x, tol, max_iter, &extra, &nrel, res));
    }
    if (info) {
        info->iterations = st.iterations + extra;
        info->reliable_updates = st.reliable + nrel;
        for (int s = 0; s < nshift; ++s) {
            info->shift_iterations[s] = st.shift_iterations[s];
            info->true_residual[s] = res[s];
        }
    }
    return status;
}

extern "C" stag_status stag_multishift_solve(stag_ctx* ctx, double mass, int nshift, const double* shifts,
                                             stag_prec prec, int nrhs, const void* b, void* x, double tol,
                                             int max_iter, stag_solve_info* info) {
    if (!ctx || !shifts || !b || !x || nshift < 1 || nshift > STAG_MAX_SHIFTS || nrhs < 1 || max_iter < 1 ||
        !(tol > 0.0))
        return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    if (prec < STAG_FP64 || prec > STAG_BF16_12) return STAG_ERR_ARG;
    if (prec == STAG_BF16_12 && ctx->b16_stale) CKS(refresh_bf16(ctx));
    for (int s = 0; s < nshift; ++s)
        if (!(mass * mass + shifts[s] > 0.0)) return STAG_ERR_ARG;
    const size_t per_rhs = (size_t)3 * ctx->g.Vh;
    stag_solve_info acc;
    std::memset(&acc, 0, sizeof(acc));
    stag_status worst = STAG_OK;
    for (int r0 = 0; r0 < nrhs; r0 += STAG_MAX_RHS) {
        int n = nrhs - r0 < STAG_MAX_RHS ? nrhs - r0 : STAG_MAX_RHS;
        stag_solve_info one;
        std::memset(&one, 0, sizeof(one));
        stag_status s = ms_api_batch(ctx, mass, nshift, shifts, prec, n, (const double2*)b + r0 * per_rhs,
                                     (double2*)x + (size_t)r0 * nshift * per_rhs, tol, max_iter, &one);
        if (s != STAG_OK && s != STAG_ERR_NOT_CONVERGED) return s;
        if (s != STAG_OK) worst = s;
        acc.iterations = std::max(acc.iterations, one.iterations);
        acc.reliable_updates += one.reliable_updates;
        for (int k = 0; k < nshift; ++k) {
            acc.shift_iterations[k] = std::max(acc.shift_iterations[k], one.shift_iterations[k]);
            acc.true_residual[k] = std::max(acc.true_residual[k], one.true_residual[k]);
        }
    }
    if (info) *info = acc;
    return worst;
}

extern "C" stag_status stag_profile_begin(stag_ctx* ctx, int sample_every) {
    if (!ctx || sample_every < 0) return STAG_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    ProfData& pf = ctx->prof;
    pf.on = sample_every > 0;
    pf.every = sample_every > 0 ? sample_every : 1;
    pf.iter = 0;
    pf.used = 0;
    for (int k = 0; k < PK_COUNT; ++k) {
        pf.marks[k].clear();
        pf.bytes_total[k] = 0.0;
        pf.launches[k] = 0;
    }
    pf.persist_ms[0] = pf.persist_ms[1] = 0.0;
    pf.persist_iters[0] = pf.persist_iters[1] = 0;
    pf.batch_ms = 0.0;
    pf.batch_iters = 0;
    if (ctx->ptime) CK(cudaMemsetAsync(ctx->ptime, 0, PTIME_WORDS * sizeof(unsigned long long), ctx->stream));
    return STAG_OK;
}

extern "C" stag_status stag_profile_read(stag_ctx* ctx, int kind, stag_kernel_profile* out) {
    if (!ctx || !out || kind < 0 || kind >= PK_COUNT) return STAG_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    ProfData& pf = ctx->prof;
    double ms = 0.0;
    for (auto& m : pf.marks[kind]) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, pf.pool[m.first], pf.pool[m.second]));
        ms += t;
    }
    out->launches = pf.launches[kind];
    out->sampled = (int)pf.marks[kind].size();
    out->sampled_ms = ms;
    if (kind == PK_PERSISTENT || kind == PK_PERSISTENT_FF) {   // every launch is timed; units are iterations
        const int w = kind == PK_PERSISTENT ? 0 : 1;
        out->sampled = (int)pf.persist_iters[w];
        out->sampled_ms = pf.persist_ms[w];
    }
    if (kind == PK_BATCH) {
        out->sampled = (int)pf.batch_iters;
        out->sampled_ms = pf.batch_ms;
    }
    out->bytes_per_launch = pf.launches[kind] ? pf.bytes_total[kind] / pf.launches[kind] : 0.0;
    return STAG_OK;
}

extern "C" long long stag_launch_count(stag_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" stag_status stag_multishift_solve_batch(stag_ctx* const* ctxs, int n, double mass, int nshift,
                                                   const double* shifts, stag_prec prec, const void* const* b,
                                                   void* const* x, double tol, int max_iter, stag_solve_info* info) {
    if (!ctxs || !shifts || !b || !x || n < 1 || n > STAG_MAX_BATCH || nshift < 1 || nshift > STAG_MAX_SHIFTS ||
        max_iter < 1 || !(tol > 0.0) || prec < STAG_FP64 || prec > STAG_BF16_12)
        return STAG_ERR_ARG;
    for (int s = 0; s < nshift; ++s)
        if (!(mass * mass + shifts[s] > 0.0)) return STAG_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !b[i] || !x[i]) return STAG_ERR_ARG;
        if (!ctxs[i]->has_gauge) return STAG_ERR_NO_GAUGE;
        if (ctxs[i]->asqtad) return STAG_ERR_ARG;   // batched solves run the unimproved operator
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return STAG_ERR_ARG;
    }
    stag_ctx* ctx = ctxs[0];
    std::vector<std::pair<stag_ctx*, cudaStream_t>> saved;
    for (int i = 0; i < n; ++i) saved.push_back({ctxs[i], ctxs[i]->stream});
    struct Restore {
        std::vector<std::pair<stag_ctx*, cudaStream_t>>& s;
        ~Restore() {
            for (auto& e : s) e.first->stream = e.second;
        }
    } restore{saved};
    for (int i = 1; i < n; ++i) {
        if (ctxs[i]->stream == ctx->stream) continue;
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, ctxs[i]->stream));
        CK(cudaStreamWaitEvent(ctx->stream, ev, 0));
        cudaEventDestroy(ev);
        ctxs[i]->stream = ctx->stream;
    }
    std::vector<MsRun> runs(n);
    for (int i = 0; i < n; ++i) {
        stag_ctx* c = ctxs[i];
        MsRun& R = runs[i];
        R.ctx = c;
        R.mass = mass;
        R.nshift = nshift;
        R.shifts = shifts;
        R.prec = prec;
        R.nrhs = 1;
        R.tol = tol;
        R.max_iter = max_iter;
        if (prec == STAG_FP64) {
            R.b = b[i];
            R.x = x[i];
            R.finish_to_f64 = true;
        } else {
            const size_t nc = (size_t)3 * c->g.Vh;
            void *b32, *x32;
            CKS(ws_get(c, WS_B32, nc * sizeof(float2), &b32));
            CKS(ws_get(c, WS_X32, nc * nshift * sizeof(float2), &x32));
            k_d2f<<<nblocks((long long)nc, 256), 256, 0, c->stream>>>(nc, (const double2*)b[i], (float2*)b32);
            ++c->launches;
            CK(cudaGetLastError());
            R.b = b32;
            R.b64 = (const double2*)b[i];
            R.x = x32;
            R.x64 = (double2*)x[i];
            R.reliable = prec != STAG_BF16_12;
            R.finish_to_f64 = true;
        }
    }
    std::vector<MsStats> st(n);
    std::vector<stag_status> ok(n);
    CKS(ms_core_multi(runs.data(), n, st.data(), ok.data()));
    stag_status worst = STAG_OK;
    for (int i = 0; i < n; ++i) {
        stag_ctx* c = ctxs[i];
        if (ok[i] != STAG_OK && ok[i] != STAG_ERR_NOT_CONVERGED) return ok[i];
        if (ok[i] != STAG_OK) worst = ok[i];
        int extra = 0, nrel = 0;
        double res[STAG_MAX_SHIFTS] = {0};
        if (prec == STAG_FP64) {
            for (int s = 0; s < nshift; ++s)
                CKS(shift_residuals(c, mass, nshift, s, shifts[s], 1, (const double2*)b[i], (const double2*)x[i],
                                    &res[s]));
        } else if (ok[i] == STAG_OK) {
            CKS(refine_shifts(c, mass, nshift, shifts, 1, (const double2*)b[i], (double2*)x[i], tol, max_iter, &extra,
                              &nrel, res));
        }
        if (info) {
            stag_solve_info& in = info[i];
            std::memset(&in, 0, sizeof(in));
            in.iterations = st[i].iterations + extra;
            in.reliable_updates = st[i].reliable + nrel;
            for (int s = 0; s < nshift; ++s) {
                in.shift_iterations[s] = st[i].shift_iterations[s];
                in.true_residual[s] = res[s];
            }
        }
    }
    return worst;
}
