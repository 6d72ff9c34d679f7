// Context management and error plumbing of the C ABI.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"
#include "solver_state.cuh"

stag_status cuda_fail(stag_ctx* c, cudaError_t e, const char* where) {
    if (c) {
        c->last_err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    cudaGetLastError();   // a non-sticky error must not leak into the next call
    return STAG_ERR_CUDA;
}

stag_status dev_alloc(stag_ctx* ctx, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        ctx->last_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        cudaGetLastError();
        *p = nullptr;
        return STAG_ERR_ALLOC;
    }
    ctx->dev_bytes += bytes;
    return STAG_OK;
}

stag_status ws_get(stag_ctx* ctx, int slot, size_t bytes, void** out) {
    if (slot < 0 || slot >= WS_COUNT) return STAG_ERR_ARG;
    if (ctx->ws_bytes[slot] < bytes) {
        if (ctx->ws[slot]) {
            // the old buffer may still be read by queued work
            CK(cudaStreamSynchronize(ctx->stream));
            CK(cudaFree(ctx->ws[slot]));
            ctx->dev_bytes -= ctx->ws_bytes[slot];
            ctx->ws[slot] = nullptr;
            ctx->ws_bytes[slot] = 0;
        }
        void* p;
        CKS(dev_alloc(ctx, &p, bytes));
        ctx->ws[slot] = p;
        ctx->ws_bytes[slot] = bytes;
    }
    *out = ctx->ws[slot];
    return STAG_OK;
}

stag_status stage_upload(stag_ctx* ctx, void* dst, const void* src, size_t bytes) {
    if (bytes > STAGE_SLOT_BYTES || !ctx->stage_host) return STAG_ERR_ARG;
    const int slot = ctx->stage_next;
    ctx->stage_next = (slot + 1) % STAGE_SLOTS;
    // the slot's previous copy has run (long ago, normally: 64 uploads back)
    CK(cudaEventSynchronize(ctx->stage_ev[slot]));
    char* h = ctx->stage_host + (size_t)slot * STAGE_SLOT_BYTES;
    std::memcpy(h, src, bytes);
    CK(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaEventRecord(ctx->stage_ev[slot], ctx->stream));
    return STAG_OK;
}

extern "C" const char* stag_strerror(stag_status s) {
    switch (s) {
        case STAG_OK: return "ok";
        case STAG_ERR_ARG: return "invalid argument";
        case STAG_ERR_ALLOC: return "allocation failed";
        case STAG_ERR_CUDA: return "CUDA error";
        case STAG_ERR_NOT_CONVERGED: return "solver did not converge";
        case STAG_ERR_TIMEOUT: return "device wait timed out";
        case STAG_ERR_NAN: return "NaN or Inf in a reduction";
        case STAG_ERR_NO_GAUGE: return "no gauge field loaded";
    }
    return "unknown status";
}

extern "C" const char* stag_last_cuda_error(stag_ctx* ctx) { return ctx ? ctx->last_err.c_str() : ""; }

extern "C" stag_status stag_set_stream(stag_ctx* ctx, void* s) {
    if (!ctx) return STAG_ERR_ARG;
    ctx->stream = (cudaStream_t)s;
    return STAG_OK;
}

extern "C" size_t stag_device_bytes(stag_ctx* ctx) { return ctx ? ctx->dev_bytes : 0; }

extern "C" size_t stag_abi_sizeof(int which) {
    switch (which) {
        case 0: return sizeof(stag_lattice);
        case 1: return sizeof(stag_rational);
        case 2: return sizeof(stag_solve_info);
        case 3: return sizeof(stag_flavour);
        case 4: return sizeof(stag_hmc);
        case 5: return sizeof(stag_traj);
        case 6: return sizeof(stag_kernel_profile);
    }
    return 0;
}

extern "C" void stag_destroy(stag_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    destroy_solver_graphs(ctx);
    for (int i = 0; i < WS_COUNT; ++i)
        if (ctx->ws[i]) cudaFree(ctx->ws[i]);
    if (ctx->ghi) cudaFree(ctx->ghi);
    if (ctx->glo) cudaFree(ctx->glo);
    if (ctx->g16) cudaFree(ctx->g16);
    if (ctx->red) cudaFree(ctx->red);
    if (ctx->counters) cudaFree(ctx->counters);
    if (ctx->bar) cudaFree(ctx->bar);
    if (ctx->ptime) cudaFree(ctx->ptime);
    if (ctx->sur_w) cudaFree(ctx->sur_w);
    if (ctx->sur_err) cudaFree(ctx->sur_err);
    if (ctx->sur_data) cudaFree(ctx->sur_data);
    if (ctx->scal) cudaFree(ctx->scal);
    if (ctx->st) cudaFree(ctx->st);
    if (ctx->st_host) cudaFreeHost(ctx->st_host);
    if (ctx->note) cudaFree(ctx->note);
    for (int w = 0; w < 2; ++w)
        for (auto& e : ctx->deferred_ev[w]) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    for (int i = 0; i < STAGE_SLOTS; ++i)
        if (ctx->stage_ev[i]) cudaEventDestroy(ctx->stage_ev[i]);
    if (ctx->stage_host) cudaFreeHost(ctx->stage_host);
    delete ctx;
}

// Partial sums of every reducing kernel: at most 2 values per source per
// block of >= 64 threads.
static size_t red_doubles(int Vh) {
    size_t n = (size_t)2 * STAG_MAX_RHS * ((size_t)Vh / 64 + 2);
    return n < 65536 ? 65536 : n;
}

extern "C" stag_status stag_create(const stag_lattice* lat, stag_ctx** out) {
    if (!lat || !out) return STAG_ERR_ARG;
    *out = nullptr;
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        int L = lat->dims[mu];
        if (L < 2 || (L & 1)) return STAG_ERR_ARG;
        V *= L;
    }
    if (V > (1LL << 30)) return STAG_ERR_ARG;
    stag_ctx* ctx = new (std::nothrow) stag_ctx();
    if (!ctx) return STAG_ERR_ALLOC;
    for (int mu = 0; mu < 4; ++mu) ctx->g.L[mu] = lat->dims[mu];
    ctx->g.Lxh = lat->dims[0] / 2;
    ctx->g.V = (int)V;
    ctx->g.Vh = (int)(V / 2);
    ctx->g.apt = lat->t_antiperiodic ? 1 : 0;
    ctx->stream = (cudaStream_t)lat->cuda_stream;
    // STAG_GRAPHS=0 runs the solver loop as plain launches (same kernels),
    // e.g. under a profiler that replays single kernels
    const char* gr = std::getenv("STAG_GRAPHS");
    ctx->use_graphs = !(gr && gr[0] == '0');
    // STAG_DSLASH_TPS=1|2|4|8 fixes the threads per site instead of tuning
    const char* tp = std::getenv("STAG_DSLASH_TPS");
    ctx->tps_force = tp ? std::atoi(tp) : 0;
    const char* pe = std::getenv("STAG_PERSISTENT");
    ctx->use_persistent = !(pe && pe[0] == '0');
    // STAG_BATCH_SHAPE=0|1|2 fixes the batched solver's launch shape instead of tuning
    const char* bs = std::getenv("STAG_BATCH_SHAPE");
    ctx->batch_shape_force = bs ? std::atoi(bs) : -1;
    // STAG_PERSIST_SITES=n: the persistent solver gives every block at least n sites
    const char* ps = std::getenv("STAG_PERSIST_SITES");
    ctx->persist_sites = ps ? std::atoi(ps) : 0;
    // STAG_ASQ_FORCE=gather: the improved operator's force as the per-link
    // gather over path incidences instead of the reverse pass
    const char* af = std::getenv("STAG_ASQ_FORCE");
    ctx->asq_gather = af && std::strcmp(af, "gather") == 0;
    stag_status s = STAG_OK;
    size_t gbytes = (size_t)4 * 2 * 18 * ctx->g.Vh * sizeof(float);
    size_t bbytes = (size_t)4 * 2 * 12 * ctx->g.Vh * sizeof(uint16_t);
    ctx->red_doubles = red_doubles(ctx->g.Vh);
    if ((s = dev_alloc(ctx, (void**)&ctx->ghi, gbytes)) != STAG_OK ||
        (s = dev_alloc(ctx, (void**)&ctx->glo, gbytes)) != STAG_OK ||
        (s = dev_alloc(ctx, (void**)&ctx->g16, bbytes)) != STAG_OK ||
        (s = dev_alloc(ctx, (void**)&ctx->red, sizeof(double) * red_doubles(ctx->g.Vh))) != STAG_OK ||
        (s = dev_alloc(ctx, (void**)&ctx->counters, sizeof(unsigned int) * 16)) != STAG_OK ||
        (s = dev_alloc(ctx, (void**)&ctx->scal, sizeof(double) * 64)) != STAG_OK ||
        (s = dev_alloc(ctx, (void**)&ctx->st, sizeof(SolverState))) != STAG_OK ||
        (s = dev_alloc(ctx, (void**)&ctx->note, sizeof(SolveNote))) != STAG_OK) {
        stag_destroy(ctx);
        return s;
    }
    if (cudaMallocHost((void**)&ctx->st_host, sizeof(SolverState)) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->stage_host, (size_t)STAGE_SLOTS * STAGE_SLOT_BYTES) != cudaSuccess) {
        cudaGetLastError();
        stag_destroy(ctx);
        return STAG_ERR_ALLOC;
    }
    for (int i = 0; i < STAGE_SLOTS; ++i)
        if (cudaEventCreateWithFlags(&ctx->stage_ev[i], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            stag_destroy(ctx);
            return STAG_ERR_CUDA;
        }
    if (cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned int) * 16, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        stag_destroy(ctx);
        return STAG_ERR_CUDA;
    }
    *out = ctx;
    return STAG_OK;
}
