// Host-side context and the launchers each translation unit provides.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "dslash.cuh"
#include "asqtad.cuh"

// Device state of one multi-shift solve (see solver.cu).
struct SolverState;

enum WsSlot {
    WS_STAGE = 0,      // host-layout gauge staging (load/store)
    WS_TMP_ODD,        // D_oe p (odd), solver
    WS_R, WS_P, WS_Q, WS_PS,   // solver vectors (real type of the solve)
    WS_B64, WS_X64, WS_R64, WS_T64, WS_U64,  // fp64 vectors for reliable updates
    WS_APPLY_TMP,      // stag_apply_a scratch
    WS_FORCE_X, WS_FORCE_Y,    // fermion force: solutions and D_oe solutions
    WS_PHI, WS_XI, WS_HB,      // trajectory: pseudo-fermions, sources, heatbath output
    WS_FORCE,          // trajectory: force accumulator
    WS_SAVE_HI, WS_SAVE_LO,    // saved gauge field for Metropolis rejection
    WS_MOM,            // momenta
    WS_MISC,
    WS_B32, WS_X32,    // multishift API: fp32 copy of b, fp32 iteration solutions
    WS_REF_G, WS_REF_AX, WS_REF_T, WS_REF_R64, WS_REF_B32, WS_REF_E32, WS_REF_E64,  // refinement
    WS_FORCE_X64,      // fermion force: fp64 accumulation of the mixed solutions
    WS_FORCE_B32,      // fermion force: fp32 copy of phi
    WS_TUNE_IN, WS_TUNE_OUT,   // autotuner fields
    WS_B_DF, WS_X_DF,  // fp64 solves: float-float copies of b and x
    WS_SUR_GRAD_PART, WS_SUR_LOSS_PART, WS_SUR_GRAD,   // surrogate training
    WS_BATCH_RED,      // batched solves: per-block partial sums of all chains
    WS_ASQ_LINKS,      // improved staggered: fat and Naik links (two-float stores)
    WS_ASQ_X,          // improved staggered force: the outer-product fields of V and W
    WS_ASQ_F,          // improved staggered force: the staple and cotangent fields of the reverse pass
    WS_COUNT
};

// Sampled CUDA-event timing of the solver kernels (stag_profile_*).
enum ProfKind { PK_DSLASH_OE = 0, PK_DSLASH_EO_A, PK_UPDATE, PK_PERSISTENT, PK_BATCH, PK_PERSISTENT_FF, PK_COUNT };
struct ProfData {
    bool on = false;
    int every = 16;
    long long iter = 0;                          // solver iterations launched while on
    std::vector<cudaEvent_t> pool;               // created lazily, reused
    size_t used = 0;
    std::vector<std::pair<int, int>> marks[PK_COUNT];
    double bytes_total[PK_COUNT] = {};           // algorithmic bytes over all launches
    long long launches[PK_COUNT] = {};
    double persist_ms[2] = {};                   // persistent solver (fp32 / float-float): event time
    long long persist_iters[2] = {};             // of all launches and the iterations they ran
    double batch_ms = 0.0;                       // batched solver (this context leading): launch time
    long long batch_iters = 0;                   // and batched iterations
};

// surrogate MLP parameters: W1 (32x24), b1, W2 (32x32), b2, W3 (24x32), b3
#define SUR_NF 24
#define SUR_NH 32
#define SUR_W1 0
#define SUR_B1 (SUR_W1 + SUR_NH * SUR_NF)
#define SUR_W2 (SUR_B1 + SUR_NH)
#define SUR_B2 (SUR_W2 + SUR_NH * SUR_NH)
#define SUR_W3 (SUR_B2 + SUR_NH)
#define SUR_B3 (SUR_W3 + SUR_NF * SUR_NH)
#define SUR_NP (SUR_B3 + SUR_NF)

#define PTIME_WORDS 40   // [0,8) unused, [8,16) batched fp32, [16,24) batched float-float, [24,39) single lattice

// Launch-shape tuning of the batched solver, per precision: while chosen < 0
// the candidate shapes take turns on real segments, timed per iteration.
struct BatchTune {
    int chosen = -1;
    int tried = 0;
    double us[4] = {};
    int iters[4] = {};
};

// What the host would read after each solve, kept on the device while the
// MD evolution enqueues solve after solve without waiting (SolveNote's
// deferred mode); read once after the evolution.
struct SolveNote {
    long long iters[2];       // iterations of the persistent solves: [fp32, float-float]
    long long reliable;       // in-launch residual replacements
    double bytes[2];          // their algorithmic bytes (the profile's units)
    int err;                  // first status other than OK / NOT_CONVERGED; TIMEOUT if a launch did not halt
    int solves;
};
// pinned staging slots for host-to-device uploads the host does not wait for
#define STAGE_SLOTS 64
#define STAGE_SLOT_BYTES 32768

struct SolverGraphEntry {
    const void* key[8];
    int prec, nrhs;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};
void destroy_solver_graphs(stag_ctx* ctx);

struct stag_ctx {
    Geom g;
    cudaStream_t stream = nullptr;
    float* ghi = nullptr;
    float* glo = nullptr;
    uint16_t* g16 = nullptr;
    bool has_gauge = false;
    bool b16_stale = true;
    // reductions
    double* red = nullptr;            // partial sums of the reducing kernels
    size_t red_doubles = 0;
    unsigned int* counters = nullptr; // 16 counters, zero between launches
    double* scal = nullptr;           // small device scalar area (64 doubles)
    SolverState* st = nullptr;        // device
    SolverState* st_host = nullptr;   // pinned
    // workspace
    void* ws[WS_COUNT] = {};
    size_t ws_bytes[WS_COUNT] = {};
    std::string last_err;
    size_t dev_bytes = 0;
    long long launches = 0;           // kernels launched by this context
    ProfData prof;
    bool use_graphs = true;           // solver iterations as a device-side WHILE graph
    int tps_cache[4][2] = {};         // autotuned threads per site, [prec][nr == 4]
    float tps_us[4][2] = {};          // the winner's time per launch (us)
    int tps_force = 0;                // STAG_DSLASH_TPS: force a value (0 = tune)
    bool no_alloc_call = false;       // inside stag_apply_a_noalloc: nothing may allocate
    // improved (asqtad) operator: fat and Naik links rebuilt after every change of the thin links
    bool asqtad = false;
    bool asq_stale = true;
    int asq_built = 0;                // arithmetic of the current fat links: 1 fp32, 2 float-float
    bool asq_fp32_build = false;      // set while fp32 MD forces run: their solves take fp32-built fat links
    bool asq_gather = false;          // STAG_ASQ_FORCE=gather: the force as a per-link gather over path incidences
    double asq_coef[6] = {};          // 1-link, 3-, 5-, 7-staple, Lepage, Naik
    float* asq_store = nullptr;       // fat hi, fat lo, Naik hi, Naik lo (WS_ASQ_LINKS)
    bool use_persistent = true;       // persistent cooperative solver (STAG_PERSISTENT=0: the three-kernel path)
    void* bar = nullptr;              // grid-barrier words of the persistent solver
    void* ptime = nullptr;            // per-phase ns counters of the persistent kernels while profiling
                                      // ([8,16) batched fp32, [16,24) batched float-float, [24,39) single lattice)
    BatchTune batch_tune[4];          // batched solver launch shape per precision (this context leading)
    int batch_shape_force = -1;       // STAG_BATCH_SHAPE=0|1|2: fixed shape, no tuning
    int persist_sites = 0;            // STAG_PERSIST_SITES=n: at least n sites per block of the persistent solver (0: the default)
    // force surrogate
    float* sur_w = nullptr;           // device parameters (weights rounded to bf16)
    unsigned int* sur_err = nullptr;  // set by a tensor-core surrogate launch that gave up a wait
    bool sur_loaded = false;
    std::vector<double> sur_master, adam_m, adam_v;   // fp32-valued master weights, Adam moments
    long long adam_t = 0;
    float* sur_data = nullptr;        // training samples, component-major [224][capacity x links]
    long long sur_cap = 0, sur_count = 0;
    cudaStream_t cap_stream = nullptr;
    std::vector<SolverGraphEntry> graphs;
    // deferred solves (inside the MD evolution): no host read between them
    bool defer = false;
    SolveNote* note = nullptr;        // device
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> deferred_ev[2];   // profiled persistent launches
    // staging ring of small uploads (SolverState, coefficients)
    char* stage_host = nullptr;
    cudaEvent_t stage_ev[STAGE_SLOTS] = {};
    int stage_next = 0;
};

// a single kernel launch: count it and check the launch
#define CKL()                                   \
    do {                                        \
        ++ctx->launches;                        \
        CK(cudaGetLastError());                 \
    } while (0)
// bytes of the eight links of one site in a Dslash of this precision
inline double link_bytes_site(stag_prec p) {
    return p == STAG_FP64 ? 1152.0 : p == STAG_FP32 ? 576.0 : p == STAG_FP32_12 ? 384.0 : 192.0;
}
// the same for the context's operator: the improved one reads a fat and a Naik link per hop
inline double op_link_bytes_site(const stag_ctx* ctx, stag_prec p) {
    return (ctx->asqtad ? 2.0 : 1.0) * link_bytes_site(p);
}

// error plumbing
stag_status cuda_fail(stag_ctx* c, cudaError_t e, const char* where);
#define CK(call)                                                        \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call);        \
    } while (0)
#define CKS(call)                                                       \
    do {                                                                \
        stag_status _s = (call);                                        \
        if (_s != STAG_OK) return _s;                                   \
    } while (0)

stag_status ws_get(stag_ctx* ctx, int slot, size_t bytes, void** out);
// bytes (<= STAGE_SLOT_BYTES) from host memory to dst on the context's
// stream, through a pinned slot that is reused only after its copy has run:
// the caller may change src as soon as this returns, without a sync
stag_status stage_upload(stag_ctx* ctx, void* dst, const void* src, size_t bytes);
// deferred solves: begin (the note cleared), end (one sync: the note read,
// the profile updated, the first error returned)
stag_status defer_begin(stag_ctx* ctx);
stag_status defer_end(stag_ctx* ctx, long long* iters, long long* reliable);
stag_status dev_alloc(stag_ctx* ctx, void** p, size_t bytes);

inline LinkPtrs link_ptrs(const stag_ctx* c) { return LinkPtrs{c->ghi, c->glo, c->g16}; }
inline int nblocks(long long n, int bs) { return (int)((n + bs - 1) / bs); }

// gauge.cu
stag_status refresh_bf16(stag_ctx* ctx);
stag_status gauge_copy(stag_ctx* ctx, float* dst_hi, float* dst_lo, const float* src_hi, const float* src_lo);

// asqtad.cu: the improved operator.  asq_ensure rebuilds the fat and Naik
// links if the thin links changed since (a no-op for the unimproved operator);
// the force accumulates the outer products of every term, then one pass
// through the paths writes (mode 0) or adds (mode 1) the force into out.
AsqLinks asq_links(const stag_ctx* ctx);
int asq_tps(const stag_ctx* ctx);
stag_status asq_ensure(stag_ctx* ctx);
stag_status asq_outer_begin(stag_ctx* ctx, stag_prec prec);
stag_status asq_outer_add(stag_ctx* ctx, stag_prec prec, int nsrc, int nshift, const double* alpha, const void* x,
                          const void* y, double coef);
stag_status asq_force_finish(stag_ctx* ctx, stag_prec prec, double* out, int mode);
// gauge.cu: a two-float link store to the host layout (double, [mu][site][3][3] complex) on the device
stag_status unpack_links(stag_ctx* ctx, const float* hi, const float* lo, double* stage);

// dslash.cu: threads per site for a Dslash of this precision and sources per
// thread, autotuned on first use (never call it first inside a stream capture)
int dslash_tps(stag_ctx* ctx, stag_prec prec, int nr);
// out = scale * D_{out_par} in  (no reductions)
stag_status launch_dslash(stag_ctx* ctx, int out_par, stag_prec prec, int nrhs, const void* in, void* out,
                          double scale);
// out = c0 * aux - 1/2 D_eo tmp  with tmp = D_oe in  computed into ws
stag_status launch_apply_a(stag_ctx* ctx, double c0, stag_prec prec, int nrhs, const void* in, void* out,
                           void* tmp_odd);

// solver.cu
// Core multi-shift iteration in the arithmetic of prec.  b, x: [nrhs][3][Vh] and
// [nrhs][nshift][3][Vh] in the real type of prec (x overwritten).  For mixed
// precisions with reliable updates, b64 (fp64 source) and x64 (fp64
// accumulator, same shape as x) are required; finish_to_f64 selects whether
// the result ends in x64 (x64 += x) or in x (x = (float)(x64 + x)).
struct MsStats {
    int iterations;
    int reliable;
    int shift_iterations[STAG_MAX_SHIFTS];
};
stag_status ms_core(stag_ctx* ctx, double mass, int nshift, const double* shifts, stag_prec prec, int nrhs,
                    const void* b, const double2* b64, void* x, double2* x64, double tol, int max_iter,
                    bool reliable, bool finish_to_f64, MsStats* stats);

// The pieces of ms_core, for solves of several contexts iterated by one
// launch (batch.cu): one MsRun per solve, arguments as for ms_core.
struct MsRun {
    stag_ctx* ctx = nullptr;
    double mass = 0.0;
    int nshift = 0;
    const double* shifts = nullptr;
    stag_prec prec = STAG_FP32;
    int nrhs = 1;
    const void* b = nullptr;
    const double2* b64 = nullptr;
    void* x = nullptr;
    double2* x64 = nullptr;
    double tol = 0.0;
    int max_iter = 0;
    bool reliable = false, finish_to_f64 = false;
    // set by ms_setup
    bool mixed = false, use_rel = false;
    int base = 0;
    void *tmp = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *ps = nullptr;   // iteration vectors
    size_t rstride = 0;             // elements between the persistent solver's residual ring slots
    void *ax64 = nullptr, *t64 = nullptr, *xb64 = nullptr;                         // reliable-update scratch
    const void* b_user = nullptr;   // fp64 solves: the caller's arrays (the iteration runs on float-float copies)
    void* x_user = nullptr;
};
stag_status ms_setup(MsRun& R);                 // workspace, solver state, initial vectors (stream-ordered)
stag_status ms_reliable_update(MsRun& R);       // after a halt with need_reliable: fp64 residual, halt cleared
stag_status ms_finish(MsRun& R);                // solutions into the caller's format
void ms_stats(const MsRun& R, MsStats* stats);  // from the host copy of the state (after ms_pull_state)
stag_status ms_pull_state(stag_ctx* ctx);       // whole state to the host copy, synchronous
stag_status ms_pull_control_async(stag_ctx* ctx);   // loop-control words to the host copy, no sync

// batch.cu: solves of up to STAG_MAX_BATCH contexts (one source each, same
// prec, all on one stream) iterated together by persistent cooperative
// launches; per-chain statuses in per_chain, stats (n entries) may be NULL
stag_status ms_core_multi(MsRun* runs, int n, MsStats* stats, stag_status* per_chain);

// persistent.cu: the whole iteration loop in one cooperative launch
bool persistent_fits(stag_ctx* ctx);
int persistent_ring_slots();        // residual fields the persistent solver cycles through
// the link formats' instances of the persistent solver (persistent_<format>.cu)
#define STAG_PERSISTENT_ARGS stag_ctx* ctx, int nrhs, void* ring, size_t rstride, void* p, void* q, void* t, \
    void* ps, void* x, const double2* b64, double2* x64, double2* t64
stag_status launch_persistent_f32_18(STAG_PERSISTENT_ARGS);
stag_status launch_persistent_f32_12(STAG_PERSISTENT_ARGS);
stag_status launch_persistent_bf16_12(STAG_PERSISTENT_ARGS);
stag_status launch_persistent_ff(STAG_PERSISTENT_ARGS);
stag_status launch_persistent_asq_f32(STAG_PERSISTENT_ARGS);
stag_status launch_persistent_asq_ff(STAG_PERSISTENT_ARGS);
stag_status launch_persistent(stag_ctx* ctx, stag_prec prec, int nrhs, void* ring, size_t rstride, void* p, void* q,
                              void* t, void* ps, void* x, const double2* b64, double2* x64, double2* t64);

// force.cu
// force kernels write out = coef F (mode 0) or add out += coef F (mode 1)
stag_status fermion_force_from_solutions(stag_ctx* ctx, stag_prec prec, int nsrc, int nshift, const double* alpha,
                                         const void* x, const void* y, double* out, double coef, int mode);
stag_status gauge_force_launch(stag_ctx* ctx, stag_prec prec, double beta, double* out, double coef, int mode);
stag_status update_links(stag_ctx* ctx, const double* mom, double eps, stag_prec prec);
stag_status reunitarize(stag_ctx* ctx);
stag_status plaquette_sum(stag_ctx* ctx, double* out_host);
stag_status kinetic_sum(stag_ctx* ctx, const double* mom, double* out_host);
stag_status mom_axpy(stag_ctx* ctx, double* mom, const double* f, double c);
stag_status draw_momenta(stag_ctx* ctx, double* mom, unsigned long long seed, unsigned long long counter);
stag_status draw_sources(stag_ctx* ctx, double2* xi, int n, unsigned long long seed, unsigned long long counter,
                         int stream_base);

// surrogate.cu
stag_status surrogate_force_launch(stag_ctx* ctx, double* out, double coef, int mode);
stag_status surrogate_check(stag_ctx* ctx);   // STAG_ERR_TIMEOUT if a launch gave up a wait (synchronises)
stag_status surrogate_append(stag_ctx* ctx, const double* exact_force);

// blas.cu
stag_status blas_norm2(stag_ctx* ctx, stag_prec prec, int nrhs, const void* v, double* out_host);
stag_status blas_dot_re(stag_ctx* ctx, int nrhs, const double2* a, const double2* b, double* out_host);
stag_status blas_combine(stag_ctx* ctx, int n, double a0, const double2* phi, int nshift, const double* alpha,
                         const double2* x, double2* out);
stag_status blas_convert(stag_ctx* ctx, size_t ncomplex, const void* src, int src_double, void* dst, int dst_double);
