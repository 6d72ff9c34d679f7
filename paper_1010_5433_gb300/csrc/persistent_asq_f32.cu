// The persistent multi-shift CG of the improved (asqtad) operator, fp32 fat and Naik links.
#include "persistent_kernel.cuh"

stag_status launch_persistent_asq_f32(stag_ctx* ctx, int nrhs, void* ring, size_t rstride, void* p, void* q, void* t,
        void* ps, void* x, const double2* b64, double2* x64, double2* t64) {
    return launch_persistent_fmt<float, FMT_F32_18, true>(ctx, nrhs, ring, rstride, p, q, t, ps, x, b64, x64, t64);
}
