// The persistent multi-shift CG for bf16 links, 12 reals.
#include "persistent_kernel.cuh"

stag_status launch_persistent_bf16_12(stag_ctx* ctx, int nrhs, void* ring, size_t rstride, void* p, void* q, void* t, void* ps,
        void* x, const double2* b64, double2* x64, double2* t64) {
    return launch_persistent_fmt<float, FMT_BF16_12>(ctx, nrhs, ring, rstride, p, q, t, ps, x, b64, x64, t64);
}
