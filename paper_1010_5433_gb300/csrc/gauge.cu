// Gauge-field store: conversion between the host layout and the two-float
// structure-of-arrays store (Sec. 5, Fig. 2), the bf16 copy, field copies.
#include "internal.h"

// staging[(mu*V + s)*18 + k], k = 2*(3i+j) + {re, im}  ->  hi/lo planes
__global__ void k_pack_gauge(Geom g, const double* __restrict__ stage, float* hi, float* lo) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4LL * g.V) return;
    int mu = (int)(idx / g.V);
    int s = (int)(idx % g.V);
    int x = s % g.L[0], r = s / g.L[0];
    int y = r % g.L[1]; r /= g.L[1];
    int z = r % g.L[2], t = r / g.L[2];
    int par = (x + y + z + t) & 1;
    int h = s >> 1;
    size_t blk = link_block_f(mu, par, g.Vh);
    float vh[18], vl[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) {
        double a = stage[(size_t)idx * 18 + k];
        float b = (float)a;                 // most significant part  (Sec. 5)
        float c = (float)(a - (double)b);   // least significant part
        hl_canonical(b, c);
        vh[k] = b;
        vl[k] = c;
    }
    float4* h4 = reinterpret_cast<float4*>(hi + blk);
    float4* l4 = reinterpret_cast<float4*>(lo + blk);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h4[(size_t)k * g.Vh + h] = make_float4(vh[4 * k], vh[4 * k + 1], vh[4 * k + 2], vh[4 * k + 3]);
        l4[(size_t)k * g.Vh + h] = make_float4(vl[4 * k], vl[4 * k + 1], vl[4 * k + 2], vl[4 * k + 3]);
    }
    reinterpret_cast<float2*>(hi + blk + 16 * (size_t)g.Vh)[h] = make_float2(vh[16], vh[17]);
    reinterpret_cast<float2*>(lo + blk + 16 * (size_t)g.Vh)[h] = make_float2(vl[16], vl[17]);
}

__global__ void k_unpack_gauge(Geom g, const float* __restrict__ hi, const float* __restrict__ lo, double* stage) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4LL * g.V) return;
    int mu = (int)(idx / g.V);
    int s = (int)(idx % g.V);
    int x = s % g.L[0], r = s / g.L[0];
    int y = r % g.L[1]; r /= g.L[1];
    int z = r % g.L[2], t = r / g.L[2];
    int par = (x + y + z + t) & 1;
    int h = s >> 1;
    Su3<double> u = load_link_d(hi, lo, link_block_f(mu, par, g.Vh), h, g.Vh);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        stage[(size_t)idx * 18 + 2 * k] = u.e[k / 3][k % 3].re;
        stage[(size_t)idx * 18 + 2 * k + 1] = u.e[k / 3][k % 3].im;
    }
}

__device__ __forceinline__ uint32_t pack_bf2(float re, float im) {
    __nv_bfloat16 a = __float2bfloat16_rn(re);
    __nv_bfloat16 b = __float2bfloat16_rn(im);
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// bf16 copy of rows 0 and 1 of every link, from the hi words
__global__ void k_make_bf16(Geom g, const float* __restrict__ hi, uint16_t* b16) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4LL * g.V) return;
    int blk_id = (int)(idx / g.Vh);       // 2*mu + par
    int h = (int)(idx % g.Vh);
    const float* blk = hi + (size_t)blk_id * 18 * g.Vh;
    const float4* p4 = reinterpret_cast<const float4*>(blk);
    float4 a = p4[h], b = p4[g.Vh + h], c = p4[2 * (size_t)g.Vh + h];
    uint16_t* ob = b16 + (size_t)blk_id * 12 * g.Vh;
    reinterpret_cast<uint4*>(ob)[h] = make_uint4(pack_bf2(a.x, a.y), pack_bf2(a.z, a.w),
                                                 pack_bf2(b.x, b.y), pack_bf2(b.z, b.w));
    reinterpret_cast<uint2*>(ob + 8 * (size_t)g.Vh)[h] = make_uint2(pack_bf2(c.x, c.y), pack_bf2(c.z, c.w));
}

stag_status refresh_bf16(stag_ctx* ctx) {
    long long n = 4LL * ctx->g.V;
    k_make_bf16<<<nblocks(n, 256), 256, 0, ctx->stream>>>(ctx->g, ctx->ghi, ctx->g16);
    CKL();
    ctx->b16_stale = false;
    return STAG_OK;
}

stag_status gauge_copy(stag_ctx* ctx, float* dh, float* dl, const float* sh, const float* sl) {
    size_t bytes = (size_t)4 * 2 * 18 * ctx->g.Vh * sizeof(float);
    CK(cudaMemcpyAsync(dh, sh, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dl, sl, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    return STAG_OK;
}

stag_status unpack_links(stag_ctx* ctx, const float* hi, const float* lo, double* stage) {
    long long n = 4LL * ctx->g.V;
    k_unpack_gauge<<<nblocks(n, 128), 128, 0, ctx->stream>>>(ctx->g, hi, lo, stage);
    CKL();
    return STAG_OK;
}

static stag_status pack_from_device(stag_ctx* ctx, const double* dev_u) {
    long long n = 4LL * ctx->g.V;
    k_pack_gauge<<<nblocks(n, 128), 128, 0, ctx->stream>>>(ctx->g, dev_u, ctx->ghi, ctx->glo);
    CKL();
    ctx->has_gauge = true;
    ctx->asq_stale = true;
    return refresh_bf16(ctx);
}

extern "C" stag_status stag_load_gauge(stag_ctx* ctx, const double* host_u) {
    if (!ctx || !host_u) return STAG_ERR_ARG;
    size_t bytes = (size_t)4 * ctx->g.V * 18 * sizeof(double);
    void* stage;
    CKS(ws_get(ctx, WS_STAGE, bytes, &stage));
    CK(cudaMemcpyAsync(stage, host_u, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CKS(pack_from_device(ctx, (const double*)stage));
    CK(cudaStreamSynchronize(ctx->stream));
    return STAG_OK;
}

extern "C" stag_status stag_load_gauge_device(stag_ctx* ctx, const double* dev_u) {
    if (!ctx || !dev_u) return STAG_ERR_ARG;
    return pack_from_device(ctx, dev_u);
}

extern "C" stag_status stag_store_gauge(stag_ctx* ctx, double* host_u) {
    if (!ctx || !host_u) return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    size_t bytes = (size_t)4 * ctx->g.V * 18 * sizeof(double);
    void* stage;
    CKS(ws_get(ctx, WS_STAGE, bytes, &stage));
    long long n = 4LL * ctx->g.V;
    k_unpack_gauge<<<nblocks(n, 128), 128, 0, ctx->stream>>>(ctx->g, ctx->ghi, ctx->glo, (double*)stage);
    CKL();
    CK(cudaMemcpyAsync(host_u, stage, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return STAG_OK;
}
