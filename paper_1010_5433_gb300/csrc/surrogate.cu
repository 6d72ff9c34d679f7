// Learned fermion-force surrogate (a workload of this build; the paper has
// none).  Per link (x, mu):
//   staples S_k, k = 8 i + j over the three nu != mu (i) and eight loops (j):
//     j = 0, 1  plaquette up / down
//     j = 2..5  2mu x nu rectangles: up with the link first / second, down first / second
//     j = 6, 7  mu x 2nu rectangles up / down
//   features   f_k = Re tr(U S_k) / 3                (gauge invariant)
//   MLP        w = W3 tanh(W2 tanh(W1 f + b1) + b2) + b3   (24-32-32-24) on the
//              tensor cores: bf16 weights and bf16 inputs to every product
//              (f, h1, h2), fp32 accumulation in TMEM, fp32 biases and tanh
//   force      F^_a = Re tr(i T_a sum_k w_k U S_k)    (gauge covariant)
// Training minimises the mean over links of |F^ - F|^2 against exact fermion
// forces with Adam on fp32 master weights; its forward, backward and
// weight-gradient products run on the tensor cores as well.
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "internal.h"

namespace {
constexpr int SB = 128;   // threads per block of the per-link kernels

__device__ __forceinline__ Su3<float> dagm(const Su3<float>& a) {
    Su3<float> d;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) d.e[i][j] = conj(a.e[j][i]);
    return d;
}

struct LinkAt {
    const Geom& g;
    const LinkPtrs& L;
    int x[4], mu, nu;
    // U_dir at x + a mu_hat + b nu_hat
    __device__ __forceinline__ Su3<float> operator()(int dir, int a, int b) const {
        int c[4] = {x[0], x[1], x[2], x[3]};
        c[mu] += a;
        c[nu] += b;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (c[i] < 0) c[i] += g.L[i];
            if (c[i] >= g.L[i]) c[i] -= g.L[i];
        }
        const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
        const int h = (c[0] >> 1) + g.Lxh * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
        return LinkFetch<float, FMT_F32_18>::get(L, dir, par, h, g.Vh);
    }
};

__device__ Su3<float> staple(const LinkAt& U, int j) {
    const int m = U.mu, n = U.nu;
    switch (j) {
        case 0: return mul(mul(U(n, 1, 0), dagm(U(m, 0, 1))), dagm(U(n, 0, 0)));
        case 1: return mul(mul(dagm(U(n, 1, -1)), dagm(U(m, 0, -1))), U(n, 0, -1));
        case 2: return mul(mul(mul(mul(U(m, 1, 0), U(n, 2, 0)), dagm(U(m, 1, 1))), dagm(U(m, 0, 1))), dagm(U(n, 0, 0)));
        case 3: return mul(mul(mul(mul(U(n, 1, 0), dagm(U(m, 0, 1))), dagm(U(m, -1, 1))), dagm(U(n, -1, 0))), U(m, -1, 0));
        case 4: return mul(mul(mul(mul(U(m, 1, 0), dagm(U(n, 2, -1))), dagm(U(m, 1, -1))), dagm(U(m, 0, -1))), U(n, 0, -1));
        case 5: return mul(mul(mul(mul(dagm(U(n, 1, -1)), dagm(U(m, 0, -1))), dagm(U(m, -1, -1))), U(n, -1, -1)), U(m, -1, 0));
        case 6: return mul(mul(mul(mul(U(n, 1, 0), U(n, 1, 1)), dagm(U(m, 0, 2))), dagm(U(n, 0, 1))), dagm(U(n, 0, 0)));
        default: return mul(mul(mul(mul(dagm(U(n, 1, -1)), dagm(U(n, 1, -2))), dagm(U(m, 0, -2))), U(n, 0, -2)), U(n, 0, -1));
    }
}

// Re tr(i T_a W) for the eight Gell-Mann generators T_a = lambda_a / 2
__device__ __forceinline__ void gen_coeffs(const Su3<float>& w, float (&f)[8]) {
    f[0] = -0.5f * (w.e[1][0].im + w.e[0][1].im);
    f[1] = -0.5f * (w.e[0][1].re - w.e[1][0].re);
    f[2] = -0.5f * (w.e[0][0].im - w.e[1][1].im);
    f[3] = -0.5f * (w.e[2][0].im + w.e[0][2].im);
    f[4] = -0.5f * (w.e[0][2].re - w.e[2][0].re);
    f[5] = -0.5f * (w.e[2][1].im + w.e[1][2].im);
    f[6] = -0.5f * (w.e[1][2].re - w.e[2][1].re);
    f[7] = -(w.e[0][0].im + w.e[1][1].im - 2.f * w.e[2][2].im) * 0.28867513459481287f;
}

__device__ __forceinline__ void link_of(const Geom& g, long long l, int& mu, int& par, int& h, int x[4]) {
    const int blk = (int)(l / g.Vh);
    h = (int)(l % g.Vh);
    mu = blk >> 1;
    par = blk & 1;
    int xh = h % g.Lxh, r = h / g.Lxh;
    x[1] = r % g.L[1]; r /= g.L[1];
    x[2] = r % g.L[2]; x[3] = r / g.L[2];
    x[0] = 2 * xh + ((x[1] + x[2] + x[3] + par) & 1);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void __launch_bounds__(SB) k_sur_features(Geom g, LinkPtrs L, float* f, float* G, long long stride) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 8LL * g.Vh) return;
    int mu, par, h, x[4];
    link_of(g, l, mu, par, h, x);
    const Su3<float> u = LinkFetch<float, FMT_F32_18>::get(L, mu, par, h, g.Vh);
    int i = 0;
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        LinkAt U{g, L, {x[0], x[1], x[2], x[3]}, mu, nu};
        for (int j = 0; j < 8; ++j) {
            const int k = 8 * i + j;
            Su3<float> w = mul(u, staple(U, j));
            f[(size_t)k * stride + l] = (w.e[0][0].re + w.e[1][1].re + w.e[2][2].re) * (1.f / 3.f);
            float c[8];
            gen_coeffs(w, c);
#pragma unroll
            for (int a = 0; a < 8; ++a) G[((size_t)k * 8 + a) * stride + l] = c[a];
        }
        ++i;
    }
}

// ---- the MLP on the 5th-generation tensor cores (tcgen05): 128 links per
// block, one link per thread.  Layer l: D_l [128 x 32] = A_l [128 x 32] . W_l^T,
// A_l the bf16 inputs of the 128 links (features zero-padded 24 -> 32, then
// h1, h2), W_l [32 x 32] bf16 (W3's 24 rows zero-padded), fp32 accumulators
// in tensor memory (TMEM), three 32-column accumulators.  One thread issues
// the MMAs; each thread reads back its own row (its link), adds the bias and
// applies tanh, and writes the next layer's bf16 row.
namespace tc {
constexpr int M = 128, K = 32, N = 32;
constexpr int TMEM_COLS = 128;                 // three accumulators of 32 columns
constexpr long long WAIT_LIMIT = 1LL << 24;    // polls of the MMA-completion barrier

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, no-swizzle layout of a [rows x 32] bf16 operand: 8 x 8 core matrices
// (8 rows x 16 bytes, contiguous), core (r/8, k/8) at ((r/8)*4 + k/8) * 128 bytes;
// so 128 bytes between core matrices along K (LBO) and 512 along rows (SBO)
__device__ __forceinline__ int op_index(int r, int k) { return ((r >> 3) * 4 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }
constexpr uint32_t LBO = 128, SBO = 512;

// [rows x 128] operands whose K is the 128 links of a tile: 16 core matrices
// per 8-row group, so 2048 bytes between 8-row groups
__device__ __forceinline__ int op_index128(int r, int k) {
    return ((r >> 3) * 16 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}
constexpr uint32_t SBO128 = 2048;

// shared-memory matrix descriptor: start, LBO, SBO (>> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo = SBO) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((LBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both K-major, n, M
__host__ __device__ constexpr uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t IDESC = idesc(N);

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, int accumulate,
                                    uint32_t id = IDESC) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate));
}
// D (M x n) [+]= A (M x k) B^T with both operands K-major in shared memory, k a
// multiple of 16 (one MMA per 16 columns: 2 core matrices = 2 x LBO further on)
__device__ __forceinline__ void mma_k(uint32_t d, uint32_t a_addr, uint32_t a_sbo, uint32_t b_addr, uint32_t b_sbo,
                                      int k, int n, int accumulate) {
    for (int s = 0; s < k / 16; ++s)
        mma(d, smem_desc(a_addr + s * 2 * LBO, a_sbo), smem_desc(b_addr + s * 2 * LBO, b_sbo),
            (accumulate || s > 0) ? 1 : 0, idesc(n));
}
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void load_row(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void load_row16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
}  // namespace tc

// Surrogate force of every link: out = coef F^ (mode 0) or out += coef F^ (mode 1),
// momentum layout.  Staples are formed twice (features, then the weighted sum)
// so that no per-staple state is kept in registers; the MLP between the two
// passes runs on the tensor cores.  A failed wait sets *err and the block
// stops issuing (the host reports STAG_ERR_TIMEOUT).
__global__ void __launch_bounds__(SB) k_sur_force(Geom g, LinkPtrs L, const float* __restrict__ params, double* out,
                                                  double coef, int mode, unsigned int* err) {
    __shared__ __align__(1024) __nv_bfloat16 sA[tc::M * tc::K];        // the layer's inputs, 8 KB
    __shared__ __align__(1024) __nv_bfloat16 sW[3][tc::N * tc::K];     // W1, W2, W3 (padded), 6 KB
    __shared__ float sb[3][tc::N];                                      // b1, b2, b3 (padded)
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    const int t = threadIdx.x, warp = t >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&s_tmem)),
                     "r"(tc::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_u32(&s_mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights as bf16 operands (they hold bf16 values already), biases
    for (int i = t; i < 3 * tc::N * tc::K; i += blockDim.x) {
        const int layer = i / (tc::N * tc::K), q = i % (tc::N * tc::K), n = q / tc::K, k = q % tc::K;
        float v = 0.f;
        if (layer == 0 && k < SUR_NF) v = params[SUR_W1 + n * SUR_NF + k];
        if (layer == 1) v = params[SUR_W2 + n * SUR_NH + k];
        if (layer == 2 && n < SUR_NF) v = params[SUR_W3 + n * SUR_NH + k];
        sW[layer][tc::op_index(n, k)] = __float2bfloat16_rn(v);
    }
    if (t < tc::N) {
        sb[0][t] = params[SUR_B1 + t];
        sb[1][t] = params[SUR_B2 + t];
        sb[2][t] = t < SUR_NF ? params[SUR_B3 + t] : 0.f;
    }
    const long long l = (long long)blockIdx.x * blockDim.x + t;
    const bool valid = l < 8LL * g.Vh;
    int mu = 0, par = 0, h = 0, x[4] = {0, 0, 0, 0};
    Su3<float> u;
    float fv[SUR_NF];
#pragma unroll
    for (int k = 0; k < SUR_NF; ++k) fv[k] = 0.f;
    if (valid) {
        link_of(g, l, mu, par, h, x);
        u = LinkFetch<float, FMT_F32_18>::get(L, mu, par, h, g.Vh);
        int i = 0;
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            LinkAt U{g, L, {x[0], x[1], x[2], x[3]}, mu, nu};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                Su3<float> wk = mul(u, staple(U, j));
                fv[8 * i + j] = (wk.e[0][0].re + wk.e[1][1].re + wk.e[2][2].re) * (1.f / 3.f);
            }
            ++i;
        }
    }
#pragma unroll
    for (int k = 0; k < tc::K; ++k) sA[tc::op_index(t, k)] = __float2bfloat16_rn(k < SUR_NF ? fv[k] : 0.f);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t mbar = tc::smem_u32(&s_mbar);
    const uint32_t a_addr = tc::smem_u32(sA);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;     // this warp's TMEM lanes
    float w[tc::N];
    bool ok = true;
    for (int layer = 0; layer < 3; ++layer) {
        const uint32_t d = tmem + (uint32_t)(layer * tc::N);
        if (t == 0 && ok) {
            const uint32_t b_addr = tc::smem_u32(sW[layer]);
            // K = 32 as two K = 16 steps: the next 16 columns are two core matrices (2 x LBO) on
            tc::mma(d, tc::smem_desc(a_addr), tc::smem_desc(b_addr), 0);
            tc::mma(d, tc::smem_desc(a_addr + 2 * tc::LBO), tc::smem_desc(b_addr + 2 * tc::LBO), 1);
            tc::commit(mbar);
        }
        __syncthreads();
        if (!ok || !tc::wait_phase(mbar, (uint32_t)(layer & 1))) {
            ok = false;
            if (t == 0) atomicExch(err, 1u);
        }
        tc::fence_after();
        float z[32];
        tc::load_row(tmem + lane_base + (uint32_t)(layer * tc::N), z);
        if (layer < 2) {
#pragma unroll
            for (int k = 0; k < tc::K; ++k) sA[tc::op_index(t, k)] = __float2bfloat16_rn(tanhf(z[k] + sb[layer][k]));
            tc::fence_async_smem();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
        } else {
#pragma unroll
            for (int k = 0; k < tc::N; ++k) w[k] = z[k] + sb[2][k];
        }
    }
    // weighted staple sum with the network's 24 weights
    if (valid && ok) {
        Su3<float> m;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) m.e[a][b] = mk(0.f, 0.f);
        int i = 0;
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            LinkAt U{g, L, {x[0], x[1], x[2], x[3]}, mu, nu};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const Su3<float> s = staple(U, j);
                const float wk = w[8 * i + j];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        m.e[a][b].re += wk * s.e[a][b].re;
                        m.e[a][b].im += wk * s.e[a][b].im;
                    }
            }
            ++i;
        }
        float c[8];
        gen_coeffs(mul(u, m), c);
        double* o = out + ((size_t)(2 * mu + par) * 8) * g.Vh + h;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            if (mode) o[(size_t)a * g.Vh] += coef * (double)c[a];
            else o[(size_t)a * g.Vh] = coef * (double)c[a];
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc::TMEM_COLS));
}

// exact forces [4][2][8][Vh] (double) -> dataset slot [8][nl] (float)
__global__ void k_sur_target(Geom g, const double* __restrict__ F, float* out, long long stride) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 8LL * g.Vh) return;
    const int blk = (int)(l / g.Vh), h = (int)(l % g.Vh);
#pragma unroll
    for (int a = 0; a < 8; ++a) out[(size_t)a * stride + l] = (float)F[((size_t)blk * 8 + a) * g.Vh + h];
}

// Training pass on the tensor cores: loss and parameter gradients over the
// dataset, every block persistent over tiles of 128 links (one per thread).
// Per tile:
//   forward   D1..D3 as in k_sur_force (fq, h1q, h2q the bf16 product inputs)
//   loss      e_a = sum_k w_k G_ka - F_a, dw_k = (2/n) sum_a e_a G_ka   (CUDA cores)
//   backward  dh2 = dw W3, dz2 = dh2 (1 - h2^2), dh1 = dz2 W2, dz1 = dh1 (1 - h1^2)
//             as MMAs against transposed weight tiles (dw, dz2 rounded to bf16)
//   weights   dW3 += dw^T h2q, dW2 += dz2^T h1q, dW1 += dz1^T fq: M = 128 (rows
//             beyond the layer width zero) x K = the tile's 128 links, accumulated
//             in TMEM over all tiles of the block; a row of ones (zero for links
//             past the end) in each transposed input gives the bias gradients
// Each block writes its partial gradient (SUR_NP floats) and loss sum.
constexpr int TT = 128;
constexpr int TMEM_TRAIN = 256;
// TMEM columns: D1 / D4 at 0, D2 / D5 at 32, D3 at 64, dW3 (48) at 96, dW2 (48) at 160, dW1 (32) at 224
constexpr int C_DW3 = 96, C_DW2 = 160, C_DW1 = 224;
// dynamic shared memory (bytes): operands first, each 1024-aligned
constexpr int SM_A = 0;                          // [128 x 32] bf16: forward / backward rows, 8 KB
constexpr int SM_AT = SM_A + 8192;               // [128 x 128] bf16: dw^T, dz2^T, dz1^T, 32 KB
constexpr int SM_BT1 = SM_AT + 32768;            // [32 x 128] bf16: fq^T, ones row 24, 8 KB
constexpr int SM_BT2 = SM_BT1 + 8192;            // [48 x 128] bf16: h1q^T, ones row 32, 12 KB
constexpr int SM_BT3 = SM_BT2 + 12288;           // [48 x 128] bf16: h2q^T, ones row 32, 12 KB
constexpr int SM_W = SM_BT3 + 12288;             // 5 x [32 x 32] bf16: W1, W2, W3, W3^T, W2^T, 10 KB
constexpr int SM_BIAS = SM_W + 5 * 2048;         // 3 x 32 floats
constexpr int SM_TRAIN = SM_BIAS + 3 * 32 * 4;

__global__ void __launch_bounds__(TT, 1) k_sur_train(long long nl, const float* __restrict__ f,
                                                     const float* __restrict__ G, const float* __restrict__ F,
                                                     long long stride, const float* __restrict__ params, float sc,
                                                     float* grad_part, double* loss_part, unsigned int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __nv_bfloat16* sA = (__nv_bfloat16*)(smem + SM_A);
    __nv_bfloat16* sAt = (__nv_bfloat16*)(smem + SM_AT);
    __nv_bfloat16* sBt1 = (__nv_bfloat16*)(smem + SM_BT1);
    __nv_bfloat16* sBt2 = (__nv_bfloat16*)(smem + SM_BT2);
    __nv_bfloat16* sBt3 = (__nv_bfloat16*)(smem + SM_BT3);
    __nv_bfloat16* sW = (__nv_bfloat16*)(smem + SM_W);    // 5 tiles of 1024 elements
    float* sb = (float*)(smem + SM_BIAS);
    __shared__ __align__(8) unsigned long long s_mbar;
    __shared__ uint32_t s_tmem;
    const int t = threadIdx.x, warp = t >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&s_tmem)),
                     "r"(TMEM_TRAIN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_u32(&s_mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // operands that stay: transposed inputs zero (their padding rows stay zero), weights
    for (int i = t; i < (SM_W - SM_AT) / 2; i += TT) sAt[i] = __float2bfloat16_rn(0.f);   // At, Bt1..Bt3
    for (int i = t; i < 5 * 1024; i += TT) {
        const int tile = i / 1024, q = i % 1024, n = q / 32, k = q % 32;
        float v = 0.f;
        if (tile == 0 && k < SUR_NF) v = params[SUR_W1 + n * SUR_NF + k];              // W1 [hidden][feature]
        if (tile == 1) v = params[SUR_W2 + n * SUR_NH + k];                             // W2
        if (tile == 2 && n < SUR_NF) v = params[SUR_W3 + n * SUR_NH + k];              // W3 [output][hidden]
        if (tile == 3 && k < SUR_NF) v = params[SUR_W3 + k * SUR_NH + n];              // W3^T [hidden][output]
        if (tile == 4) v = params[SUR_W2 + k * SUR_NH + n];                             // W2^T
        sW[tile * 1024 + tc::op_index(n, k)] = __float2bfloat16_rn(v);
    }
    if (t < 32) {
        sb[t] = params[SUR_B1 + t];
        sb[32 + t] = params[SUR_B2 + t];
        sb[64 + t] = t < SUR_NF ? params[SUR_B3 + t] : 0.f;
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem, mbar = tc::smem_u32(&s_mbar);
    const uint32_t aA = tc::smem_u32(sA), aAt = tc::smem_u32(sAt);
    const uint32_t aB1 = tc::smem_u32(sBt1), aB2 = tc::smem_u32(sBt2), aB3 = tc::smem_u32(sBt3);
    const uint32_t aW = tc::smem_u32(sW);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t parity = 0;
    bool ok = true;
    // operands written by the threads -> visible to the tensor cores; then one
    // thread issues the MMAs of `issue`, and everyone waits for their completion
    auto run = [&](auto issue) {
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (t == 0 && ok) {
            issue();
            tc::commit(mbar);
        }
        if (ok && !tc::wait_phase(mbar, parity)) {
            ok = false;
            atomicExch(err, 1u);
        }
        parity ^= 1u;
        tc::fence_after();
    };
    auto put_row = [&](const float* v, int n) {      // this link's row of the [128 x 32] operand
#pragma unroll
        for (int k = 0; k < 32; ++k) sA[tc::op_index(t, k)] = __float2bfloat16_rn(k < n ? v[k] : 0.f);
    };
    double loss_acc = 0.0;
    int acc = 0;                                  // weight-gradient accumulators hold data
    const long long ntiles = (nl + TT - 1) / TT;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long l = tile * TT + t;
        const bool valid = l < nl;
        const float one = valid ? 1.f : 0.f;
        float fq[SUR_NF];
#pragma unroll
        for (int k = 0; k < SUR_NF; ++k) fq[k] = valid ? bf16r(f[(size_t)k * stride + l]) : 0.f;
        put_row(fq, SUR_NF);
#pragma unroll
        for (int k = 0; k < SUR_NF; ++k) sBt1[tc::op_index128(k, t)] = __float2bfloat16_rn(fq[k]);
        sBt1[tc::op_index128(SUR_NF, t)] = __float2bfloat16_rn(one);
        float z[32], h1[32], h2[32];
        // ---- forward
        run([&] { tc::mma_k(tmem + 0, aA, tc::SBO, aW + 0 * 2048, tc::SBO, 32, 32, 0); });
        tc::load_row(tmem + lane_base + 0, z);
#pragma unroll
        for (int k = 0; k < 32; ++k) h1[k] = tanhf(z[k] + sb[k]), z[k] = bf16r(h1[k]);
        put_row(z, 32);
#pragma unroll
        for (int k = 0; k < 32; ++k) sBt2[tc::op_index128(k, t)] = __float2bfloat16_rn(z[k]);
        sBt2[tc::op_index128(32, t)] = __float2bfloat16_rn(one);
        run([&] { tc::mma_k(tmem + 32, aA, tc::SBO, aW + 1 * 2048, tc::SBO, 32, 32, 0); });
        tc::load_row(tmem + lane_base + 32, z);
#pragma unroll
        for (int k = 0; k < 32; ++k) h2[k] = tanhf(z[k] + sb[32 + k]), z[k] = bf16r(h2[k]);
        put_row(z, 32);
#pragma unroll
        for (int k = 0; k < 32; ++k) sBt3[tc::op_index128(k, t)] = __float2bfloat16_rn(z[k]);
        sBt3[tc::op_index128(32, t)] = __float2bfloat16_rn(one);
        run([&] { tc::mma_k(tmem + 64, aA, tc::SBO, aW + 2 * 2048, tc::SBO, 32, 32, 0); });
        tc::load_row(tmem + lane_base + 64, z);
        // ---- loss and dL/dw for this link
        float dw[SUR_NF];
#pragma unroll
        for (int k = 0; k < SUR_NF; ++k) dw[k] = 0.f;
        if (valid) {
            float e[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) e[a] = -F[(size_t)a * stride + l];
            for (int k = 0; k < SUR_NF; ++k) {
                const float wk = z[k] + sb[64 + k];
#pragma unroll
                for (int a = 0; a < 8; ++a) e[a] = fmaf(wk, G[((size_t)k * 8 + a) * stride + l], e[a]);
            }
            float ls = 0.f;
#pragma unroll
            for (int a = 0; a < 8; ++a) ls = fmaf(e[a], e[a], ls);
            loss_acc += ls;
            for (int k = 0; k < SUR_NF; ++k) {
                float sum = 0.f;
#pragma unroll
                for (int a = 0; a < 8; ++a) sum = fmaf(e[a], G[((size_t)k * 8 + a) * stride + l], sum);
                dw[k] = bf16r(sc * sum);
            }
        }
        // ---- backward: dh2 = dw W3 (D4), dW3 += dw^T h2q
        put_row(dw, SUR_NF);
#pragma unroll
        for (int k = 0; k < 32; ++k) sAt[tc::op_index128(k, t)] = __float2bfloat16_rn(k < SUR_NF ? dw[k] : 0.f);
        run([&] {
            tc::mma_k(tmem + 0, aA, tc::SBO, aW + 3 * 2048, tc::SBO, 32, 32, 0);
            tc::mma_k(tmem + C_DW3, aAt, tc::SBO128, aB3, tc::SBO128, 128, 48, acc);
        });
        tc::load_row(tmem + lane_base + 0, z);
#pragma unroll
        for (int k = 0; k < 32; ++k) z[k] = bf16r(z[k] * (1.f - h2[k] * h2[k]));    // dz2
        // ---- dh1 = dz2 W2 (D5), dW2 += dz2^T h1q
        put_row(z, 32);
#pragma unroll
        for (int k = 0; k < 32; ++k) sAt[tc::op_index128(k, t)] = __float2bfloat16_rn(z[k]);
        run([&] {
            tc::mma_k(tmem + 32, aA, tc::SBO, aW + 4 * 2048, tc::SBO, 32, 32, 0);
            tc::mma_k(tmem + C_DW2, aAt, tc::SBO128, aB2, tc::SBO128, 128, 48, acc);
        });
        tc::load_row(tmem + lane_base + 32, z);
#pragma unroll
        for (int k = 0; k < 32; ++k) z[k] = bf16r(z[k] * (1.f - h1[k] * h1[k]));    // dz1
        // ---- dW1 += dz1^T fq
#pragma unroll
        for (int k = 0; k < 32; ++k) sAt[tc::op_index128(k, t)] = __float2bfloat16_rn(z[k]);
        run([&] { tc::mma_k(tmem + C_DW1, aAt, tc::SBO128, aB1, tc::SBO128, 128, 32, acc); });
        acc = 1;
    }
    // ---- this block's gradient: rows 0..31 of the accumulators are TMEM lanes 0..31 (warp 0)
    float* gp = grad_part + (size_t)blockIdx.x * SUR_NP;
    if (warp == 0) {
        float a[32], b[16];
        const uint32_t lb = 0;
        // dW3 rows 0..23 (output k), columns 0..31 (hidden) and the bias column 32
        tc::load_row(tmem + lb + C_DW3, a);
        tc::load_row16(tmem + lb + C_DW3 + 32, b);
        if (t < SUR_NF) {
#pragma unroll
            for (int n = 0; n < 32; ++n) gp[SUR_W3 + t * SUR_NH + n] = acc ? a[n] : 0.f;
            gp[SUR_B3 + t] = acc ? b[0] : 0.f;
        }
        tc::load_row(tmem + lb + C_DW2, a);
        tc::load_row16(tmem + lb + C_DW2 + 32, b);
#pragma unroll
        for (int n = 0; n < 32; ++n) gp[SUR_W2 + t * SUR_NH + n] = acc ? a[n] : 0.f;
        gp[SUR_B2 + t] = acc ? b[0] : 0.f;
        tc::load_row(tmem + lb + C_DW1, a);
#pragma unroll
        for (int k = 0; k < SUR_NF; ++k) gp[SUR_W1 + t * SUR_NF + k] = acc ? a[k] : 0.f;
        gp[SUR_B1 + t] = acc ? a[SUR_NF] : 0.f;
    }
    double lv[1] = {loss_acc};
    block_sum<1>(lv);
    if (t == 0) loss_part[blockIdx.x] = lv[0];
    tc::fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_TRAIN));
}

// fixed-order sum of the per-block gradients
__global__ void k_sur_reduce(int nb, const float* __restrict__ part, double* grad) {
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= SUR_NP) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * SUR_NP + pi];
    grad[pi] = s;
}

float bf16_round_host(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}
}  // namespace

// device copy: weights rounded to bf16, biases fp32
static stag_status upload_params(stag_ctx* ctx) {
    if (!ctx->sur_w) CKS(dev_alloc(ctx, (void**)&ctx->sur_w, SUR_NP * sizeof(float)));
    std::vector<float> dev(SUR_NP);
    for (int i = 0; i < SUR_NP; ++i) {
        const bool is_w = (i < SUR_B1) || (i >= SUR_W2 && i < SUR_B2) || (i >= SUR_W3 && i < SUR_B3);
        const float v = (float)ctx->sur_master[i];
        dev[i] = is_w ? bf16_round_host(v) : v;
    }
    CK(cudaMemcpyAsync(ctx->sur_w, dev.data(), SUR_NP * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->sur_loaded = true;
    return STAG_OK;
}

// Shared memory reserved per block of k_sur_force beyond its own ~15 KB, so
// that at most 3 blocks share an SM: 3 x 128 TMEM columns stay within the
// SM's 512 and no block ever waits in its TMEM allocation.
constexpr int SUR_FORCE_RESERVE = 60 * 1024;

stag_status surrogate_force_launch(stag_ctx* ctx, double* out, double coef, int mode) {
    if (!ctx->sur_loaded) return STAG_ERR_ARG;
    if (!ctx->sur_err) {
        CKS(dev_alloc(ctx, (void**)&ctx->sur_err, sizeof(unsigned int)));
        CK(cudaMemsetAsync(ctx->sur_err, 0, sizeof(unsigned int), ctx->stream));
    }
    static bool attr_set = false;
    if (!attr_set) {
        CK(cudaFuncSetAttribute(k_sur_force, cudaFuncAttributeMaxDynamicSharedMemorySize, SUR_FORCE_RESERVE));
        attr_set = true;
    }
    const long long n = 8LL * ctx->g.Vh;
    k_sur_force<<<nblocks(n, SB), SB, SUR_FORCE_RESERVE, ctx->stream>>>(ctx->g, link_ptrs(ctx), ctx->sur_w, out,
                                                                          coef, mode, ctx->sur_err);
    CKL();
    return STAG_OK;
}

// STAG_ERR_TIMEOUT (and the word cleared) if a surrogate launch gave up a wait
stag_status surrogate_check(stag_ctx* ctx) {
    if (!ctx->sur_err) return STAG_OK;
    unsigned int e = 0;
    CK(cudaMemcpyAsync(&e, ctx->sur_err, sizeof(e), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (!e) return STAG_OK;
    CK(cudaMemsetAsync(ctx->sur_err, 0, sizeof(unsigned int), ctx->stream));
    return STAG_ERR_TIMEOUT;
}

// the training store with capacity for exactly cap samples, keeping those held
static stag_status surrogate_resize(stag_ctx* ctx, long long cap) {
    const long long nl = 8LL * ctx->g.Vh;
    const long long per = (long long)(SUR_NF + SUR_NF * 8 + 8);
    {
        float* nb = nullptr;
        CKS(dev_alloc(ctx, (void**)&nb, (size_t)cap * nl * per * sizeof(float)));
        if (ctx->sur_data) {
            // component-major layout [component][sample][link]: copy component by component
            for (long long c = 0; c < per; ++c)
                CK(cudaMemcpyAsync(nb + (size_t)c * cap * nl, ctx->sur_data + (size_t)c * ctx->sur_cap * nl,
                                   (size_t)ctx->sur_count * nl * sizeof(float), cudaMemcpyDeviceToDevice,
                                   ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            CK(cudaFree(ctx->sur_data));
            ctx->dev_bytes -= (size_t)ctx->sur_cap * nl * per * sizeof(float);
        }
        ctx->sur_data = nb;
        ctx->sur_cap = cap;
    }
    return STAG_OK;
}

// append (features, generators, exact force) of the current field to the dataset
stag_status surrogate_append(stag_ctx* ctx, const double* exact_force) {
    const long long nl = 8LL * ctx->g.Vh;
    // grow by doubling unless the caller reserved the capacity
    if (ctx->sur_count >= ctx->sur_cap) CKS(surrogate_resize(ctx, ctx->sur_cap ? 2 * ctx->sur_cap : 4));
    const long long stride = ctx->sur_cap * nl;     // one component over all samples
    const long long base = ctx->sur_count * nl;
    float* f = ctx->sur_data + base;
    float* G = ctx->sur_data + (size_t)SUR_NF * stride + base;
    float* F = ctx->sur_data + (size_t)(SUR_NF + SUR_NF * 8) * stride + base;
    k_sur_features<<<nblocks(nl, SB), SB, 0, ctx->stream>>>(ctx->g, link_ptrs(ctx), f, G, stride);
    CKL();
    k_sur_target<<<nblocks(nl, 256), 256, 0, ctx->stream>>>(ctx->g, exact_force, F, stride);
    CKL();
    ctx->sur_count += 1;
    return STAG_OK;
}

// loss and gradient over every stored sample with the current weights
static stag_status loss_grad(stag_ctx* ctx, double* loss, std::vector<double>& grad) {
    if (ctx->sur_count < 1) return STAG_ERR_ARG;
    const long long nl1 = 8LL * ctx->g.Vh;
    const long long stride = ctx->sur_cap * nl1;
    const long long nl = ctx->sur_count * nl1;
    // persistent blocks: as many as share the SMs two by two (shared memory
    // and TMEM: 2 x 256 columns), never more than there are tiles
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const long long ntiles = (nl + TT - 1) / TT;
    const int nb = (int)std::min<long long>(ntiles, 2LL * nsm);
    void *gp, *lp, *gd;
    CKS(ws_get(ctx, WS_SUR_GRAD_PART, (size_t)nb * SUR_NP * sizeof(float), &gp));
    CKS(ws_get(ctx, WS_SUR_LOSS_PART, (size_t)nb * sizeof(double), &lp));
    CKS(ws_get(ctx, WS_SUR_GRAD, SUR_NP * sizeof(double), &gd));
    if (!ctx->sur_err) {
        CKS(dev_alloc(ctx, (void**)&ctx->sur_err, sizeof(unsigned int)));
        CK(cudaMemsetAsync(ctx->sur_err, 0, sizeof(unsigned int), ctx->stream));
    }
    CK(cudaFuncSetAttribute(k_sur_train, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_TRAIN));
    const float* d = ctx->sur_data;
    k_sur_train<<<nb, TT, SM_TRAIN, ctx->stream>>>(nl, d, d + (size_t)SUR_NF * stride,
                                                   d + (size_t)(SUR_NF + SUR_NF * 8) * stride, stride, ctx->sur_w,
                                                   (float)(2.0 / (double)nl), (float*)gp, (double*)lp, ctx->sur_err);
    CKL();
    CKS(surrogate_check(ctx));
    k_sur_reduce<<<nblocks(SUR_NP, 256), 256, 0, ctx->stream>>>(nb, (const float*)gp, (double*)gd);
    CKL();
    grad.resize(SUR_NP);
    std::vector<double> lpart(nb);
    CK(cudaMemcpyAsync(grad.data(), gd, SUR_NP * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(lpart.data(), lp, nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double s = 0.0;
    for (double v : lpart) s += v;
    *loss = s / (double)nl;
    return STAG_OK;
}

extern "C" stag_status stag_surrogate_load(stag_ctx* ctx, const float* params) {
    if (!ctx || !params) return STAG_ERR_ARG;
    ctx->sur_master.assign(params, params + SUR_NP);
    ctx->adam_m.assign(SUR_NP, 0.0);
    ctx->adam_v.assign(SUR_NP, 0.0);
    ctx->adam_t = 0;
    return upload_params(ctx);
}

extern "C" stag_status stag_surrogate_store(stag_ctx* ctx, float* params) {
    if (!ctx || !params || ctx->sur_master.size() != SUR_NP) return STAG_ERR_ARG;
    for (int i = 0; i < SUR_NP; ++i) params[i] = (float)ctx->sur_master[i];
    return STAG_OK;
}

extern "C" stag_status stag_surrogate_force(stag_ctx* ctx, double* force) {
    if (!ctx || !force) return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    CKS(surrogate_force_launch(ctx, force, 1.0, 0));
    return surrogate_check(ctx);
}

extern "C" stag_status stag_surrogate_add_force_sample(stag_ctx* ctx, const double* exact_force) {
    if (!ctx || !exact_force) return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    return surrogate_append(ctx, exact_force);
}

extern "C" long long stag_surrogate_samples(stag_ctx* ctx) { return ctx ? ctx->sur_count : 0; }

extern "C" stag_status stag_surrogate_reserve(stag_ctx* ctx, long long n_samples) {
    if (!ctx || n_samples < 1 || n_samples < ctx->sur_count) return STAG_ERR_ARG;
    if (n_samples == ctx->sur_cap) return STAG_OK;
    return surrogate_resize(ctx, n_samples);
}

extern "C" stag_status stag_surrogate_loss_grad(stag_ctx* ctx, double* loss, double* grad) {
    if (!ctx || !loss || !ctx->sur_loaded) return STAG_ERR_ARG;
    std::vector<double> g;
    CKS(loss_grad(ctx, loss, g));
    if (grad) std::memcpy(grad, g.data(), SUR_NP * sizeof(double));
    return STAG_OK;
}

// Adam (Kingma & Ba) on the fp32 master weights, the device copy re-rounded
// to bf16 after every step.
extern "C" stag_status stag_surrogate_train(stag_ctx* ctx, int steps, double lr, double* loss_first,
                                            double* loss_last) {
    if (!ctx || steps < 1 || !(lr > 0) || !ctx->sur_loaded) return STAG_ERR_ARG;
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    std::vector<double> g;
    for (int s = 0; s < steps; ++s) {
        double loss;
        CKS(loss_grad(ctx, &loss, g));
        if (!std::isfinite(loss)) return STAG_ERR_NAN;
        if (s == 0 && loss_first) *loss_first = loss;
        if (loss_last) *loss_last = loss;
        ctx->adam_t += 1;
        const double c1 = 1.0 - std::pow(b1, ctx->adam_t), c2 = 1.0 - std::pow(b2, ctx->adam_t);
        for (int i = 0; i < SUR_NP; ++i) {
            ctx->adam_m[i] = b1 * ctx->adam_m[i] + (1 - b1) * g[i];
            ctx->adam_v[i] = b2 * ctx->adam_v[i] + (1 - b2) * g[i] * g[i];
            ctx->sur_master[i] -= lr * (ctx->adam_m[i] / c1) / (std::sqrt(ctx->adam_v[i] / c2) + eps);
        }
        CKS(upload_params(ctx));
    }
    return STAG_OK;
}
