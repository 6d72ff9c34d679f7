// The persistent multi-shift CG for fp32 links, 18 reals.
#include "persistent_kernel.cuh"

stag_status launch_persistent_f32_18(stag_ctx* ctx, int nrhs, void* ring, size_t rstride, void* p, void* q, void* t, void* ps,
        void* x, const double2* b64, double2* x64, double2* t64) {
    return launch_persistent_fmt<float, FMT_F32_18>(ctx, nrhs, ring, rstride, p, q, t, ps, x, b64, x64, t64);
}
