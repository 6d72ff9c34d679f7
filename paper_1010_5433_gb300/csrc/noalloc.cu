// stag_apply_a_noalloc: the even/odd operator A for callers that must not
// allocate device memory.
//
// stag_apply_a keeps its intermediate odd field (D_oe applied to the input)
// in a workspace that the context allocates with cudaMalloc the first time it
// is needed, and grows (cudaFree + cudaMalloc) when a larger call comes.  Some
// callers cannot let that happen: a program whose device memory is handed out
// by its own pool with no headroom left, or a loop that may not take the
// device-wide synchronisation that cudaFree implies.  This entry point does
// the same computation with the same kernels, but the intermediate field
// lives in the fixed array below, part of the library's device image, so the
// call itself allocates nothing.
#include <mutex>

#include "internal.h"

// 32 MiB: enough for the odd field of nrhs * Vh <= 1,398,101 sites in fp32
// (24 bytes per site and source) or 699,050 in fp64 (48 bytes), e.g. one
// source on 40^4 in fp32 or on 32^4 in fp64.  Every GPU that loads the
// library holds this array until the process exits.
#define STAG_NOALLOC_SCRATCH_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[STAG_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
// Device address of the array, per device ordinal, looked up once and kept
// for the process: valid while the caller's current device is the context's
// device and the device is not reset (a reset reloads the module, and the
// kept address would then be stale).
void* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// In host code the array's name is only a host-side stand-in; its device
// address is looked up once per device, with that device current.
stag_status scratch_address(stag_ctx* ctx, void** out) {
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        ctx->last_err = "stag_apply_a_noalloc: device ordinal out of range";
        return STAG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return STAG_OK;
}
}  // namespace

extern "C" stag_status stag_apply_a_noalloc(stag_ctx* ctx, double mass, double shift, stag_prec prec, int nrhs,
                                            const void* in, void* out) {
    if (!ctx || !in || !out || nrhs < 1) return STAG_ERR_ARG;
    if (prec < STAG_FP64 || prec > STAG_BF16_12) return STAG_ERR_ARG;
    const size_t need = (size_t)nrhs * 3 * ctx->g.Vh * 2 * (prec == STAG_FP64 ? sizeof(double) : sizeof(float));
    if (need > STAG_NOALLOC_SCRATCH_BYTES) {
        ctx->last_err = "stag_apply_a_noalloc: the odd field needs " + std::to_string(need) +
                        " bytes of scratch, more than the fixed " + std::to_string(STAG_NOALLOC_SCRATCH_BYTES) +
                        " bytes; use stag_apply_a or fewer sources";
        return STAG_ERR_ARG;
    }
    void* tmp = nullptr;
    CKS(scratch_address(ctx, &tmp));
    // D_oe overwrites all nrhs*3*Vh entries of the scratch before D_eo reads
    // them, so nothing left there by an earlier call needs clearing.  The
    // flag keeps the Dslash autotuner (which allocates test fields) from
    // running inside this call; an untuned precision uses one thread per site.
    CKS(asq_ensure(ctx));   // the improved operator's links, if due: a kernel, no allocation
    ctx->no_alloc_call = true;
    stag_status s = launch_apply_a(ctx, mass * mass + shift, prec, nrhs, in, out, tmp);
    ctx->no_alloc_call = false;
    return s;
}
