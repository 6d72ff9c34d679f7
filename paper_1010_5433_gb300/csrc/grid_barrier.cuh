// Grid-wide barrier of the persistent (cooperative) solver kernels, with
// every wait bounded: after BAR_SPIN_LIMIT polls a block sets the error word
// and leaves its loop, every other block sees the word while it polls and
// leaves too, so a launch that cannot meet its barrier ends instead of
// hanging; the host reports STAG_ERR_TIMEOUT.
#pragma once

namespace {

constexpr long long BAR_SPIN_LIMIT = 1LL << 26;   // ~0.1-1 s of polling

struct GridBar {
    unsigned int count;   // arrivals since the launch began
    unsigned int err;     // set by a block whose wait gave up
    unsigned int pad[2];
};

// Counting barrier over all blocks of a cooperative launch.  The counter only
// grows within a launch (the host zeroes it before each one): every block
// adds 1 with a gpu-scope release at each barrier and waits, with acquire
// loads, until the counter reaches nblocks x (barriers it has passed), so a
// block's writes before the barrier are visible to every block after it.
// One fire-and-forget arrival and the polls are the whole cost: no read of a
// generation word before arriving, no reset by the last block, no read of the
// error word once the barrier is met.
__device__ __forceinline__ void red_add_release(unsigned int* a, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* a) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int* a) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

// one per block, in registers: the barrier, the grid size, and the counter
// value that ends the block's next wait
struct GridSync {
    GridBar* b;
    unsigned int nblocks;
    unsigned int target;
};

// false when the wait gave up (after spin_limit polls, this block sets the
// error word) or another block had given up: the caller leaves its loop
__device__ __forceinline__ bool grid_sync(GridSync& s, long long spin_limit = BAR_SPIN_LIMIT) {
    __shared__ int s_met;
    __syncthreads();
    s.target += s.nblocks;
    if (threadIdx.x == 0) {
        red_add_release(&s.b->count, 1u);
        int met = 1;
        long long spins = 0;
        while ((int)(ld_acquire(&s.b->count) - s.target) < 0) {
            if (++spins > spin_limit) {
                atomicExch(&s.b->err, 1u);
                met = 0;
                break;
            }
            if ((spins & 31) == 0 && ld_relaxed(&s.b->err) != 0) {
                met = 0;
                break;
            }
        }
        s_met = met;
    }
    __syncthreads();
    return s_met != 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace
