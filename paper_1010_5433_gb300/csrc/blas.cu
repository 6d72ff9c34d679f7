// Small vector kernels on half-lattice fields: fp64 norms and dot products
// (fixed-order sums), the rational combination a0 phi + sum_i alpha_i X_i,
// precision conversion.
#include <vector>

#include "internal.h"

namespace {
constexpr int BB = 256;

template <typename R>
__global__ void __launch_bounds__(BB) k_norm2(int Vh, const typename V2T<R>::T* __restrict__ v, double* partial) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    double s[1] = {0.0};
    if (h < Vh) {
        Vec3<R> a = load_vec<R>(v + (size_t)rhs * 3 * Vh, h, Vh);
        for (int c = 0; c < 3; ++c) s[0] += (double)a.c[c].re * a.c[c].re + (double)a.c[c].im * a.c[c].im;
    }
    block_sum<1>(s);
    if (threadIdx.x == 0) partial[(size_t)rhs * gridDim.x + blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(BB) k_dot_re(int Vh, const double2* __restrict__ a, const double2* __restrict__ b,
                                               double* partial) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    double s[1] = {0.0};
    if (h < Vh) {
        for (int c = 0; c < 3; ++c) {
            size_t i = ((size_t)rhs * 3 + c) * Vh + h;
            s[0] += a[i].x * b[i].x + a[i].y * b[i].y;
        }
    }
    block_sum<1>(s);
    if (threadIdx.x == 0) partial[(size_t)rhs * gridDim.x + blockIdx.x] = s[0];
}

// out[r] = a0 phi[r] + sum_i alpha_i x[r][i]
__global__ void k_combine(int Vh, int nshift, double a0, const double2* __restrict__ phi,
                          const double* __restrict__ alpha, const double2* __restrict__ x, double2* out) {
    const int rhs = blockIdx.y;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    const size_t rs = (size_t)3 * Vh;
    for (int c = 0; c < 3; ++c) {
        size_t i = rhs * rs + (size_t)c * Vh + h;
        double re = a0 * phi[i].x, im = a0 * phi[i].y;
        for (int s = 0; s < nshift; ++s) {
            double2 v = x[((size_t)rhs * nshift + s) * rs + (size_t)c * Vh + h];
            re += alpha[s] * v.x;
            im += alpha[s] * v.y;
        }
        out[i] = make_double2(re, im);
    }
}

__global__ void k_convert(size_t n, const void* src, int sd, void* dst, int dd) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double re, im;
    if (sd) { double2 a = ((const double2*)src)[i]; re = a.x; im = a.y; }
    else { float2 a = ((const float2*)src)[i]; re = a.x; im = a.y; }
    if (dd) ((double2*)dst)[i] = make_double2(re, im);
    else ((float2*)dst)[i] = make_float2((float)re, (float)im);
}

stag_status fetch_sums(stag_ctx* ctx, int nrhs, int nb, double* out) {
    std::vector<double> part((size_t)nrhs * nb);
    CK(cudaMemcpyAsync(part.data(), ctx->red, part.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < nrhs; ++r) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += part[(size_t)r * nb + i];
        out[r] = s;
    }
    return STAG_OK;
}
}  // namespace

stag_status blas_norm2(stag_ctx* ctx, stag_prec prec, int nrhs, const void* v, double* out_host) {
    dim3 grid(nblocks(ctx->g.Vh, BB), nrhs);
    if (prec == STAG_FP64) k_norm2<double><<<grid, BB, 0, ctx->stream>>>(ctx->g.Vh, (const double2*)v, ctx->red);
    else k_norm2<float><<<grid, BB, 0, ctx->stream>>>(ctx->g.Vh, (const float2*)v, ctx->red);
    CKL();
    return fetch_sums(ctx, nrhs, grid.x, out_host);
}

stag_status blas_dot_re(stag_ctx* ctx, int nrhs, const double2* a, const double2* b, double* out_host) {
    dim3 grid(nblocks(ctx->g.Vh, BB), nrhs);
    k_dot_re<<<grid, BB, 0, ctx->stream>>>(ctx->g.Vh, a, b, ctx->red);
    CKL();
    return fetch_sums(ctx, nrhs, grid.x, out_host);
}

stag_status blas_combine(stag_ctx* ctx, int nrhs, double a0, const double2* phi, int nshift, const double* alpha,
                         const double2* x, double2* out) {
    // coefficients through the small scalar area
    if (nshift > 60) return STAG_ERR_ARG;
    CKS(stage_upload(ctx, ctx->scal, alpha, nshift * sizeof(double)));
    dim3 grid(nblocks(ctx->g.Vh, BB), nrhs);
    k_combine<<<grid, BB, 0, ctx->stream>>>(ctx->g.Vh, nshift, a0, phi, ctx->scal, x, out);
    CKL();
    return STAG_OK;
}

stag_status blas_convert(stag_ctx* ctx, size_t n, const void* src, int sd, void* dst, int dd) {
    if (n == 0) return STAG_OK;
    k_convert<<<nblocks((long long)n, 256), 256, 0, ctx->stream>>>(n, src, sd, dst, dd);
    CKL();
    return STAG_OK;
}
