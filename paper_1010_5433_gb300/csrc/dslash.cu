// Host entry points for the staggered operator: D_eo / D_oe on any number of
// right-hand sides (Sec. 2, Table 2) and the even/odd operator A (Sec. 2).
#include <algorithm>
#include <map>
#include <mutex>

#include "internal.h"

// R is the arithmetic: float for the fp32 formats, float-float (DF) for the
// fp64 one, whose fields are double (SrcFor<DF> splits them on load)
template <typename R, int FMT, int NR, class Epi>
static void launch_tps(stag_ctx* ctx, cudaStream_t stream, int tps, int out_par, int nrhs, const void* in, Epi epi) {
    typedef typename SrcFor<R>::type Src;
    const int bs = STAG_DSLASH_BLOCK;
    const int nchunk = (nrhs + NR - 1) / NR;
    const int grid = nblocks(ctx->g.Vh, bs / tps) * nchunk;
    Src src{(const typename SrcFor<R>::io*)in};
    LinkPtrs L = link_ptrs(ctx);
    switch (tps) {
        case 8: k_dslash<R, FMT, NR, 8, Src, Epi><<<grid, bs, 0, stream>>>(ctx->g, out_par, L, src, nrhs, nchunk, epi); break;
        case 4: k_dslash<R, FMT, NR, 4, Src, Epi><<<grid, bs, 0, stream>>>(ctx->g, out_par, L, src, nrhs, nchunk, epi); break;
        case 2: k_dslash<R, FMT, NR, 2, Src, Epi><<<grid, bs, 0, stream>>>(ctx->g, out_par, L, src, nrhs, nchunk, epi); break;
        default: k_dslash<R, FMT, NR, 1, Src, Epi><<<grid, bs, 0, stream>>>(ctx->g, out_par, L, src, nrhs, nchunk, epi); break;
    }
}

// the same for the improved operator (asqtad.cuh): fat and Naik links
template <typename R, int FMT, int NR, class Epi>
static void launch_tps_asq(stag_ctx* ctx, cudaStream_t stream, int tps, int out_par, int nrhs, const void* in,
                           Epi epi) {
    typedef typename SrcFor<R>::type Src;
    const int bs = STAG_DSLASH_BLOCK;
    const int nchunk = (nrhs + NR - 1) / NR;
    const int grid = nblocks(ctx->g.Vh, bs / tps) * nchunk;
    Src src{(const typename SrcFor<R>::io*)in};
    const AsqLinks A = asq_links(ctx);
    switch (tps) {
        case 8: k_dslash_asq<R, FMT, NR, 8, Src, Epi><<<grid, bs, 0, stream>>>(ctx->g, out_par, A, src, nrhs, nchunk, epi); break;
        case 4: k_dslash_asq<R, FMT, NR, 4, Src, Epi><<<grid, bs, 0, stream>>>(ctx->g, out_par, A, src, nrhs, nchunk, epi); break;
        case 2: k_dslash_asq<R, FMT, NR, 2, Src, Epi><<<grid, bs, 0, stream>>>(ctx->g, out_par, A, src, nrhs, nchunk, epi); break;
        default: k_dslash_asq<R, FMT, NR, 1, Src, Epi><<<grid, bs, 0, stream>>>(ctx->g, out_par, A, src, nrhs, nchunk, epi); break;
    }
}

// out = scale * D in: the plain-store epilogue of each arithmetic
template <typename R> struct StoreEpi {
    static EpiStore<R> make(void* out, double scale) { return EpiStore<R>{(typename V2T<R>::T*)out, (R)scale}; }
};
template <> struct StoreEpi<DF> {
    static EpiStoreD2 make(void* out, double scale) { return EpiStoreD2{(double2*)out, DF(scale)}; }
};

static stag_prec prec_of(int fmt) {
    return fmt == FMT_F64 ? STAG_FP64 : fmt == FMT_F32_18 ? STAG_FP32 : fmt == FMT_F32_12 ? STAG_FP32_12 : STAG_BF16_12;
}

template <typename R, int FMT, class Epi>
static stag_status launch_t(stag_ctx* ctx, int out_par, int nrhs, const void* in, Epi epi) {
    if ((long long)nblocks(ctx->g.Vh, 16) * nrhs > 0x7fffffffLL) return STAG_ERR_ARG;
    const int nr = dslash_nr_for(nrhs);
    if constexpr (FMT == FMT_F64 || FMT == FMT_F32_18) {
        if (ctx->asqtad) {
            const int tps = asq_tps(ctx);
            if (nr == 4) launch_tps_asq<R, FMT, 4>(ctx, ctx->stream, tps, out_par, nrhs, in, epi);
            else launch_tps_asq<R, FMT, 1>(ctx, ctx->stream, tps, out_par, nrhs, in, epi);
            CKL();
            return STAG_OK;
        }
    }
    const int tps = dslash_tps(ctx, prec_of(FMT), nr);
    if (nr == 4) launch_tps<R, FMT, 4>(ctx, ctx->stream, tps, out_par, nrhs, in, epi);
    else launch_tps<R, FMT, 1>(ctx, ctx->stream, tps, out_par, nrhs, in, epi);
    CKL();
    return STAG_OK;
}

// ---------------------------------------------------------------- autotuner
// Each candidate number of threads per site is timed as a CUDA graph of 20
// launches (so host launch gaps do not enter), best of three replays, on a
// private stream; the fastest is cached in the context.
template <typename R, int FMT, int NR>
static stag_status time_candidate(stag_ctx* ctx, cudaStream_t s, int tps, int nrhs, const void* in, void* out,
                                  float* us) {
    auto e = StoreEpi<R>::make(out, 0.5);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    stag_status st = STAG_OK;
    const int reps = 20;
    float best = 1e30f;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "capture");
    for (int k = 0; k < reps; ++k) launch_tps<R, FMT, NR>(ctx, s, tps, 1, nrhs, in, e);
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture (autotune)");
    if ((ce = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess ||
        (ce = cudaEventCreate(&e0)) != cudaSuccess || (ce = cudaEventCreate(&e1)) != cudaSuccess ||
        (ce = cudaGraphLaunch(exec, s)) != cudaSuccess) {
        st = cuda_fail(ctx, ce, "autotune graph");
    } else {
        for (int t = 0; t < 3 && st == STAG_OK; ++t) {
            float ms = 0.f;
            if ((ce = cudaEventRecord(e0, s)) != cudaSuccess || (ce = cudaGraphLaunch(exec, s)) != cudaSuccess ||
                (ce = cudaEventRecord(e1, s)) != cudaSuccess || (ce = cudaEventSynchronize(e1)) != cudaSuccess ||
                (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
                st = cuda_fail(ctx, ce, "autotune timing");
            else best = std::min(best, ms * 1000.f / reps);
        }
        ctx->launches += 4LL * reps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    *us = best;
    return st;
}

template <typename R, int FMT>
static stag_status tune_fmt(stag_ctx* ctx, int nr, int* best_tps, float* best_us) {
    const int nrhs = nr;
    const size_t bytes = (size_t)nrhs * 3 * ctx->g.Vh * sizeof(typename SrcFor<R>::io);
    void *in, *out;
    CKS(ws_get(ctx, WS_TUNE_IN, bytes, &in));
    CKS(ws_get(ctx, WS_TUNE_OUT, bytes, &out));
    CK(cudaMemsetAsync(in, 0, bytes, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    *best_tps = 1;
    *best_us = 1e30f;
    for (int tps = 1; tps <= 8; tps *= 2) {
        if (tps > 1 && (long long)ctx->g.Vh * tps > (1LL << 22)) break;   // enough threads already
        float us;
        stag_status st = nr == 4 ? time_candidate<R, FMT, 4>(ctx, ctx->cap_stream, tps, nrhs, in, out, &us)
                                 : time_candidate<R, FMT, 1>(ctx, ctx->cap_stream, tps, nrhs, in, out, &us);
        if (st != STAG_OK) return st;
        if (us < *best_us) { *best_us = us; *best_tps = tps; }
    }
    return STAG_OK;
}

// Tuned choices are kept for the whole process, per device, lattice shape and
// precision: every context on the same lattice then uses the same threads per
// site, so its sums run in the same order and its results are reproducible
// from context to context (the candidates' timings can be close enough for
// separate tunings to disagree).
namespace {
struct TuneKey {
    int dev, L[4], prec;
    bool operator<(const TuneKey& o) const {
        if (dev != o.dev) return dev < o.dev;
        for (int i = 0; i < 4; ++i)
            if (L[i] != o.L[i]) return L[i] < o.L[i];
        return prec < o.prec;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, float>> g_tuned;

bool tune_key(const stag_ctx* ctx, stag_prec prec, TuneKey* k) {
    if (cudaGetDevice(&k->dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    for (int i = 0; i < 4; ++i) k->L[i] = ctx->g.L[i];
    k->prec = prec;
    return true;
}
}  // namespace

int dslash_tps(stag_ctx* ctx, stag_prec prec, int nr) {
    if (ctx->tps_force == 1 || ctx->tps_force == 2 || ctx->tps_force == 4 || ctx->tps_force == 8)
        return ctx->tps_force;
    // one choice per precision, tuned with one source per thread, so that an
    // n-source launch sums every site in the same order as n single launches
    (void)nr;
    const int slot = 0;
    int& c = ctx->tps_cache[prec][slot];
    if (c) return c;
    TuneKey key;
    const bool keyed = tune_key(ctx, prec, &key);
    if (keyed) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            ctx->tps_us[prec][slot] = it->second.second;
            return c = it->second.first;
        }
    }
    if (ctx->no_alloc_call) return 1;   // tuning would allocate its test fields
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!ctx->has_gauge || cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return 1;    // no tuning possible now: one thread per site
    }
    int best = 1;
    float us = 0.f;
    stag_status s;
    switch (prec) {
        case STAG_FP64: s = tune_fmt<DF, FMT_F64>(ctx, 1, &best, &us); break;
        case STAG_FP32: s = tune_fmt<float, FMT_F32_18>(ctx, 1, &best, &us); break;
        case STAG_FP32_12: s = tune_fmt<float, FMT_F32_12>(ctx, 1, &best, &us); break;
        default:
            if (ctx->b16_stale) refresh_bf16(ctx);
            s = tune_fmt<float, FMT_BF16_12>(ctx, 1, &best, &us);
            break;
    }
    if (s != STAG_OK) return 1;
    if (keyed) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto ins = g_tuned.insert({key, {best, us}});   // a concurrent tuning that finished first wins
        best = ins.first->second.first;
        us = ins.first->second.second;
    }
    c = best;
    ctx->tps_us[prec][slot] = us;
    return c;
}

extern "C" int stag_tuned_threads_per_site(stag_ctx* ctx, stag_prec prec, int nrhs, double* us_per_launch) {
    if (!ctx || prec < STAG_FP64 || prec > STAG_BF16_12 || nrhs < 1) return 0;
    const int t = dslash_tps(ctx, prec, dslash_nr_for(nrhs));
    if (us_per_launch) *us_per_launch = ctx->tps_us[prec][0];
    return t;
}

static stag_status check_prec(stag_ctx* ctx, stag_prec prec) {
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    if (prec == STAG_BF16_12 && ctx->b16_stale) CKS(refresh_bf16(ctx));
    if (prec < STAG_FP64 || prec > STAG_BF16_12) return STAG_ERR_ARG;
    if (ctx->asqtad && prec != STAG_FP64 && prec != STAG_FP32) return STAG_ERR_ARG;   // fat links are not unitary
    return STAG_OK;
}

stag_status launch_dslash(stag_ctx* ctx, int out_par, stag_prec prec, int nrhs, const void* in, void* out,
                          double scale) {
    CKS(check_prec(ctx, prec));
    switch (prec) {
        case STAG_FP64: {
            EpiStoreD2 e{(double2*)out, DF(scale)};
            return launch_t<DF, FMT_F64>(ctx, out_par, nrhs, in, e);
        }
        case STAG_FP32: {
            EpiStore<float> e{(float2*)out, (float)scale};
            return launch_t<float, FMT_F32_18>(ctx, out_par, nrhs, in, e);
        }
        case STAG_FP32_12: {
            EpiStore<float> e{(float2*)out, (float)scale};
            return launch_t<float, FMT_F32_12>(ctx, out_par, nrhs, in, e);
        }
        case STAG_BF16_12: {
            EpiStore<float> e{(float2*)out, (float)scale};
            return launch_t<float, FMT_BF16_12>(ctx, out_par, nrhs, in, e);
        }
    }
    return STAG_ERR_ARG;
}

stag_status launch_apply_a(stag_ctx* ctx, double c0, stag_prec prec, int nrhs, const void* in, void* out,
                           void* tmp) {
    CKS(launch_dslash(ctx, 1, prec, nrhs, in, tmp, 0.5));   // tmp = D_oe in
    switch (prec) {
        case STAG_FP64: {
            EpiAopD2 e{(double2*)out, (const double2*)in, DF(c0)};
            return launch_t<DF, FMT_F64>(ctx, 0, nrhs, tmp, e);
        }
        case STAG_FP32: {
            EpiAop<float> e{(float2*)out, (const float2*)in, (float)c0};
            return launch_t<float, FMT_F32_18>(ctx, 0, nrhs, tmp, e);
        }
        case STAG_FP32_12: {
            EpiAop<float> e{(float2*)out, (const float2*)in, (float)c0};
            return launch_t<float, FMT_F32_12>(ctx, 0, nrhs, tmp, e);
        }
        case STAG_BF16_12: {
            EpiAop<float> e{(float2*)out, (const float2*)in, (float)c0};
            return launch_t<float, FMT_BF16_12>(ctx, 0, nrhs, tmp, e);
        }
    }
    return STAG_ERR_ARG;
}

static size_t real_size(stag_prec p) { return p == STAG_FP64 ? sizeof(double) : sizeof(float); }

extern "C" stag_status stag_dslash(stag_ctx* ctx, int out_parity, stag_prec prec, int nrhs, const void* in,
                                   void* out) {
    if (!ctx || !in || !out || nrhs < 1 || (out_parity != 0 && out_parity != 1)) return STAG_ERR_ARG;
    CKS(asq_ensure(ctx));
    return launch_dslash(ctx, out_parity, prec, nrhs, in, out, 0.5);
}

extern "C" stag_status stag_apply_a(stag_ctx* ctx, double mass, double shift, stag_prec prec, int nrhs,
                                    const void* in, void* out) {
    if (!ctx || !in || !out || nrhs < 1) return STAG_ERR_ARG;
    CKS(asq_ensure(ctx));
    void* tmp;
    CKS(ws_get(ctx, WS_APPLY_TMP, (size_t)nrhs * 3 * ctx->g.Vh * 2 * real_size(prec), &tmp));
    return launch_apply_a(ctx, mass * mass + shift, prec, nrhs, in, out, tmp);
}
