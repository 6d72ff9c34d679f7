// Host entry points for the staggered operator: D_eo / D_oe on any number of
// right-hand sides (Sec. 2, Table 2) and the even/odd operator A (Sec. 2).
#include "internal.h"

template <typename R, int FMT, class Epi>
static stag_status launch_t(stag_ctx* ctx, int out_par, int nrhs, const void* in, Epi epi) {
    const int bs = 128;
    int nr = dslash_nr_for(nrhs);
    int nchunk = (nrhs + nr - 1) / nr;
    long long grid = (long long)nblocks(ctx->g.Vh, bs) * nchunk;
    if (grid > 0x7fffffffLL) return STAG_ERR_ARG;
    SrcPlain<R> src{(const typename V2T<R>::T*)in};
    LinkPtrs L = link_ptrs(ctx);
    switch (nr) {
        case 4: k_dslash<R, FMT, 4, SrcPlain<R>, Epi><<<(int)grid, bs, 0, ctx->stream>>>(ctx->g, out_par, L, src, nrhs, nchunk, epi); break;
        case 2: k_dslash<R, FMT, 2, SrcPlain<R>, Epi><<<(int)grid, bs, 0, ctx->stream>>>(ctx->g, out_par, L, src, nrhs, nchunk, epi); break;
        default: k_dslash<R, FMT, 1, SrcPlain<R>, Epi><<<(int)grid, bs, 0, ctx->stream>>>(ctx->g, out_par, L, src, nrhs, nchunk, epi); break;
    }
    CKL();
    return STAG_OK;
}

static stag_status check_prec(stag_ctx* ctx, stag_prec prec) {
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    if (prec == STAG_BF16_12 && ctx->b16_stale) CKS(refresh_bf16(ctx));
    if (prec < STAG_FP64 || prec > STAG_BF16_12) return STAG_ERR_ARG;
    return STAG_OK;
}

stag_status launch_dslash(stag_ctx* ctx, int out_par, stag_prec prec, int nrhs, const void* in, void* out,
                          double scale) {
    CKS(check_prec(ctx, prec));
    switch (prec) {
        case STAG_FP64: {
            EpiStore<double> e{(double2*)out, scale};
            return launch_t<double, FMT_F64>(ctx, out_par, nrhs, in, e);
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
            EpiAop<double> e{(double2*)out, (const double2*)in, c0};
            return launch_t<double, FMT_F64>(ctx, 0, nrhs, tmp, e);
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
    return launch_dslash(ctx, out_parity, prec, nrhs, in, out, 0.5);
}

extern "C" stag_status stag_apply_a(stag_ctx* ctx, double mass, double shift, stag_prec prec, int nrhs,
                                    const void* in, void* out) {
    if (!ctx || !in || !out || nrhs < 1) return STAG_ERR_ARG;
    void* tmp;
    CKS(ws_get(ctx, WS_APPLY_TMP, (size_t)nrhs * 3 * ctx->g.Vh * 2 * real_size(prec), &tmp));
    return launch_apply_a(ctx, mass * mass + shift, prec, nrhs, in, out, tmp);
}
