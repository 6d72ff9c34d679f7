// Grid-wide barrier of the persistent (cooperative) solver kernels, with
// every wait bounded: after BAR_SPIN_LIMIT polls a block sets the error word
// and every block leaves its loop, so a launch that cannot meet its barrier
// ends instead of hanging; the host reports STAG_ERR_TIMEOUT.
#pragma once

namespace {

constexpr long long BAR_SPIN_LIMIT = 1LL << 26;   // ~0.1-1 s of polling

struct GridBar {
    unsigned int count;
    unsigned int gen;
    unsigned int err;
    unsigned int pad;
};

// Generation barrier over all blocks of a cooperative launch, with gpu-scope
// release/acquire atomics: a block's writes are released by its arrival and
// acquired by every block that sees the generation advance.
__device__ __forceinline__ unsigned int atom_add_release(unsigned int* a, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(a), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* a) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned int nblocks, long long spin_limit = BAR_SPIN_LIMIT) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int g0 = ld_acquire(&b->gen);
        const unsigned int arrived = atom_add_release(&b->count, 1u);
        if (arrived == nblocks - 1) {
            // everyone has arrived (and released); reset, then open the next generation
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(&b->count), "r"(0u) : "memory");
            atom_add_release(&b->gen, 1u);
        } else {
            long long spins = 0;
            while (ld_acquire(&b->gen) == g0 && ld_acquire(&b->err) == 0) {
                if (++spins > spin_limit) {
                    atomicExch(&b->err, 1u);
                    break;
                }
            }
        }
    }
    __syncthreads();
    return *(volatile unsigned int*)&b->err == 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace
