// Host side of the persistent multi-shift CG (persistent_kernel.cuh): the
// choice of the solver path, the dispatch to the link formats' instances
// (compiled in parallel, one translation unit each), the phase timers and
// the self-test of the bounded grid barrier.
#include "persistent_kernel.cuh"


bool persistent_fits(stag_ctx* ctx) {
    // every volume: measured on GB300, one persistent launch per solve beats
    // the three-kernel iteration at 16^4 (launch- and latency-bound) and at
    // 32^4 and 48^4 alike (fp32-12: 194 against 429 us and 990 against 2062 us
    // per iteration), the deferred shift updates moving a third of the bytes
    return ctx->use_persistent;
}

int persistent_ring_slots() { return RING; }

stag_status launch_persistent(stag_ctx* ctx, stag_prec prec, int nrhs, void* ring, size_t rstride, void* p, void* q,
                              void* t, void* ps, void* x, const double2* b64, double2* x64, double2* t64) {
    if (!ctx->bar) CKS(dev_alloc(ctx, &ctx->bar, sizeof(GridBar)));
    if (!ctx->ptime) {
        CKS(dev_alloc(ctx, &ctx->ptime, PTIME_WORDS * sizeof(unsigned long long)));
        CK(cudaMemsetAsync(ctx->ptime, 0, PTIME_WORDS * sizeof(unsigned long long), ctx->stream));
    }
    if (ctx->asqtad) {
        if (prec == STAG_FP64) return launch_persistent_asq_ff(ctx, nrhs, ring, rstride, p, q, t, ps, x, b64, x64, t64);
        return launch_persistent_asq_f32(ctx, nrhs, ring, rstride, p, q, t, ps, x, b64, x64, t64);
    }
    switch (prec) {
        case STAG_FP64: return launch_persistent_ff(ctx, nrhs, ring, rstride, p, q, t, ps, x, b64, x64, t64);
        case STAG_FP32: return launch_persistent_f32_18(ctx, nrhs, ring, rstride, p, q, t, ps, x, b64, x64, t64);
        case STAG_FP32_12: return launch_persistent_f32_12(ctx, nrhs, ring, rstride, p, q, t, ps, x, b64, x64, t64);
        default: return launch_persistent_bf16_12(ctx, nrhs, ring, rstride, p, q, t, ps, x, b64, x64, t64);
    }
}

extern "C" stag_status stag_profile_phases(stag_ctx* ctx, double* us) {
    if (!ctx || !us) return STAG_ERR_ARG;
    unsigned long long t[PTIME_WORDS] = {0};
    if (ctx->ptime) {
        CK(cudaMemcpyAsync(t, ctx->ptime, sizeof(t), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    for (int i = 0; i < 15; ++i) us[i] = t[24 + i] * 1e-3;
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
