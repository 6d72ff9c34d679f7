/*
 * stag.h -- C ABI of libstag, a GB300 (sm_103a) implementation of the
 * all-on-GPU RHMC hot path for unimproved staggered fermions described in
 * Bonati, Cossu, D'Elia, Di Giacomo, "Staggered fermions simulations on GPUs"
 * (Lattice 2010).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice: dims = {Lx, Ly, Lz, Lt}, all even and >= 2; V = Lx Ly Lz Lt,
 *   Vh = V / 2.  Lexicographic site index s = x + Lx*(y + Ly*(z + Lz*t)).
 *   Parity p(s) = (x+y+z+t) mod 2, 0 = even.  Within one parity a site has
 *   the half index h = s >> 1 (a bijection onto [0, Vh) because Lx is even).
 * Operator (Sec. 2: unimproved staggered, even/odd preconditioned):
 *   D psi(x) = 1/2 sum_mu eta_mu(x) [U_mu(x) psi(x+mu) - U_mu(x-mu)^dag psi(x-mu)]
 *   eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z),
 *   times -1 on t-links leaving the last time slice when t_antiperiodic.
 *   D_eo maps odd -> even fields, D_oe even -> odd;  A = m^2 - D_eo D_oe.
 * Spinor fields (caller-owned DEVICE memory): half-lattice, structure of
 *   arrays, [nrhs][colour 3][Vh] complex, i.e. element (r, c, h) at
 *   ((r*3 + c)*Vh + h), each complex stored (re, im).  Real type: double for
 *   STAG_FP64, float for every other precision.  16-byte aligned.
 * Momenta and forces (caller-owned DEVICE memory, always double):
 *   [mu 4][parity 2][a 8][Vh]: coefficient a of sum_a p_a lambda_a/2 on link
 *   (x, mu), x of the given parity with half index h.
 * Host gauge layout (load/store): double complex U[mu][s][3][3] row-major,
 *   i.e. 4*V*18 doubles, ((mu*V + s)*9 + 3*i + j)*2 + {0 re, 1 im}.
 *
 * Every call returns a stag_status and never aborts the process.  Calls are
 * ordered on the context's stream; only those that return host scalars, and
 * stag_store_gauge, synchronise it.  Device memory the context allocates is
 * freed by stag_destroy.  A context is not thread-safe.
 */
#ifndef STAG_H
#define STAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stag_ctx stag_ctx;

typedef enum {
    STAG_OK = 0,
    STAG_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, ...) */
    STAG_ERR_ALLOC = 2,          /* device or pinned-host allocation failed */
    STAG_ERR_CUDA = 3,           /* a CUDA runtime call failed (see stag_last_cuda_error) */
    STAG_ERR_NOT_CONVERGED = 4,  /* solver hit max_iter; partial results are valid */
    STAG_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    STAG_ERR_NAN = 6,            /* a NaN/Inf appeared in a reduction */
    STAG_ERR_NO_GAUGE = 7        /* no gauge field loaded yet */
} stag_status;

/* Arithmetic of a Dslash / solver call (Sec. 4 and Sec. 5, Fig. 2):
 *  STAG_FP64     links rebuilt as hi + lo from the two-float store, fp64 math
 *  STAG_FP32     fp32 links (the hi words), 18 reals, fp32 math
 *  STAG_FP32_12  fp32 links, first two rows only, third row rebuilt (Sec. 5)
 *  STAG_BF16_12  bf16 copies of the first two rows, fp32 spinors and math   */
typedef enum { STAG_FP64 = 0, STAG_FP32 = 1, STAG_FP32_12 = 2, STAG_BF16_12 = 3 } stag_prec;

typedef struct {
    int dims[4];          /* Lx, Ly, Lz, Lt: even, >= 2 */
    int t_antiperiodic;   /* 1: antiperiodic fermion boundary in time */
    void* cuda_stream;    /* cudaStream_t the context launches on (NULL = legacy default) */
} stag_lattice;

/* r(x) = a0 + sum_i alpha[i] / (x + beta[i]), n <= STAG_MAX_SHIFTS (Sec. 2). */
#define STAG_MAX_SHIFTS 32
/* independent chains (contexts) advanced together by stag_md_trajectory_batch */
#define STAG_MAX_BATCH 8
typedef struct {
    int n;
    double a0;
    const double* alpha;  /* host array of n */
    const double* beta;   /* host array of n, all > -m^2 */
} stag_rational;

/* ---- context and gauge field (Sec. 3: the configuration is copied to the
 *      device once and the whole update runs there) ---------------------- */

/* Creates a context for one lattice.  *out receives the handle.  The
 * context reads these environment variables once, here (none is needed):
 *   STAG_GRAPHS=0          the large-lattice solver loop as plain launches
 *                          instead of a CUDA-graph WHILE loop
 *   STAG_PERSISTENT=0      no persistent solver kernel: every solve takes the
 *                          three-kernel iteration (CUDA-graph WHILE loop)
 *   STAG_DSLASH_TPS=n      threads per site of the standalone Dslash (1, 2,
 *                          4 or 8) instead of the tuned value
 *   STAG_BATCH_SHAPE=k     launch shape k (0, 1, 2) of the batched solver
 *                          instead of the tuned one
 *   STAG_PERSIST_SITES=n   at least n sites per block of the persistent
 *                          solver (default: one site per thread)
 *   STAG_ASQ_FORCE=gather  the improved operator's force as a per-link gather
 *                          over the path incidences instead of the reverse
 *                          pass through the nested staples (same sum, other order) */
stag_status stag_create(const stag_lattice* lat, stag_ctx** out);
/* Frees every device and pinned buffer of the context (NULL is a no-op);
 * the caller's buffers are untouched.  Synchronises the context's stream. */
void        stag_destroy(stag_ctx* ctx);
/* Static text naming a status code. */
const char* stag_strerror(stag_status s);
/* Text of the last CUDA error seen by this context ("" if none). */
const char* stag_last_cuda_error(stag_ctx* ctx);
/* Later calls are ordered on cuda_stream (a cudaStream_t; NULL = legacy
 * default stream); work already issued stays on the previous stream. */
stag_status stag_set_stream(stag_ctx* ctx, void* cuda_stream);
/* Device bytes the context currently holds. */
size_t      stag_device_bytes(stag_ctx* ctx);

/* Copy a host gauge field (host layout above; the caller keeps ownership)
 * into the device two-float store of Sec. 5, Fig. 2: every real a is kept
 * as b = (float)a and c = (float)(a - b); fp32 kernels read b, fp64 kernels
 * rebuild b + c.  Also refreshes the bf16 copy.  Synchronous. */
stag_status stag_load_gauge(stag_ctx* ctx, const double* host_u);
/* Same, from a DEVICE buffer in the host layout (stream-ordered). */
stag_status stag_load_gauge_device(stag_ctx* ctx, const double* dev_u);
/* Copy the device gauge field (b + c) back to a caller-allocated host
 * buffer of 4*V*18 doubles.  Synchronous. */
stag_status stag_store_gauge(stag_ctx* ctx, double* host_u);

/* ---- operator (Sec. 2, Sec. 5 Table 2) ---------------------------------- */

/* out = D_{out_parity, 1-out_parity} in for nrhs right-hand sides: each link
 * is loaded once per site and applied to every right-hand side.
 * in: [nrhs][3][Vh] on parity 1-out_parity; out: same shape on out_parity. */
stag_status stag_dslash(stag_ctx* ctx, int out_parity, stag_prec prec, int nrhs,
                        const void* in, void* out);

/* out = (m^2 + shift) in - D_eo D_oe in on even fields, nrhs right-hand sides. */
stag_status stag_apply_a(stag_ctx* ctx, double mass, double shift, stag_prec prec,
                         int nrhs, const void* in, void* out);

/* Same result as stag_apply_a, for callers that must not allocate device
 * memory (a program whose device memory belongs to its own pool with no room
 * left, or a loop that may not take the device-wide synchronisation of
 * cudaFree).  No counterpart in the paper.  The intermediate odd field
 * D_oe in lives in a fixed 32 MiB array in the library's device image instead
 * of a workspace the context would allocate, so this call allocates nothing.
 * Limit: nrhs * 3 * Vh * (16 bytes fp64, 8 bytes otherwise) <= 32 MiB, else
 * STAG_ERR_ARG with the sizes in stag_last_cuda_error.  The first call on a
 * device looks up the array's device address with that device current (make
 * that first call before any stream capture) and keeps it for the process:
 * call with the context's device current, and do not reset the device
 * (cudaDeviceReset) while the library is in use.  All calls share the one
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it. */
stag_status stag_apply_a_noalloc(stag_ctx* ctx, double mass, double shift, stag_prec prec,
                                 int nrhs, const void* in, void* out);

/* ---- improved staggered fermions (not in the paper: its Sec. 2 runs the
 *      unimproved operator; the improved one is the asqtad action of Lepage,
 *      PRD 59 (1999) 074502, and Orginos, Toussaint, Sugar, PRD 60 (1999) 054503) */

typedef enum { STAG_ACTION_UNIMPROVED = 0, STAG_ACTION_ASQTAD = 1 } stag_action;

/* Selects the fermion operator every later call of this context uses
 * (stag_dslash, stag_apply_a, stag_apply_a_noalloc, stag_multishift_solve,
 * stag_fermion_force, stag_md_trajectory).  STAG_ACTION_UNIMPROVED (the
 * default) is the paper's operator.  STAG_ACTION_ASQTAD replaces each hop by
 * a fat link V (1-link 5/8, 6 three-link staples 1/16 u0^-2, 24 five-link
 * staples 1/64 u0^-4, 48 seven-link staples 1/384 u0^-6, 6 Lepage paths
 * -1/16 u0^-4) and adds a third-neighbour hop through the Naik link
 * W = -1/24 u0^-2 U_mu(x) U_mu(x+mu) U_mu(x+2mu):
 *   D psi(x) = 1/2 sum_mu eta_mu(x) [V_mu(x) psi(x+mu) - V_mu(x-mu)^dag psi(x-mu)
 *                                  + W_mu(x) psi(x+3mu) - W_mu(x-3mu)^dag psi(x-3mu)],
 * A = m^2 - D_eo D_oe as before; its spectrum lies in [m^2, m^2 + (4 sum |c|)^2]
 * (58.8 + m^2 at u0 = 1).  u0: tadpole factor, 0 < u0 <= 1 (1: tree level).
 * The fat and Naik links are rebuilt on the device (float-float arithmetic
 * from the two-float store) before the first use after every change of the
 * thin links.  With the improved operator, prec must be STAG_FP64 or
 * STAG_FP32 (the fat links are not unitary, so no 12-real or bf16 copy), and
 * the batched calls and the force surrogate return STAG_ERR_ARG.  fp32
 * forces (the MD) build the fat links in fp32 from the thin links' hi words;
 * every other use builds them in float-float.  The gauge action stays
 * Wilson's.
 * Allocates the two link stores (2 x 4 V x 18 x 8 bytes) on the first switch. */
stag_status stag_set_action(stag_ctx* ctx, stag_action action, double u0);

/* Fat and Naik links of the current gauge field (after the rebuild, if one is
 * due) into caller-allocated host buffers of 4*V*18 doubles each, in the host
 * layout of stag_store_gauge, without eta or boundary signs.  STAG_ERR_ARG
 * unless the context uses STAG_ACTION_ASQTAD.  Synchronous. */
stag_status stag_asqtad_links(stag_ctx* ctx, double* host_fat, double* host_naik);

/* ---- solvers (Sec. 6; multi-shift CG after Jegerlehner, hep-lat/9612014) --- */

typedef struct {
    int iterations;                       /* Krylov iterations of the base system */
    int shift_iterations[STAG_MAX_SHIFTS]; /* iteration at which each shift froze */
    double true_residual[STAG_MAX_SHIFTS]; /* max over rhs of ||b-(A+s)x||/||b||, fp64 */
    int reliable_updates;                 /* fp64 residual replacements made */
} stag_solve_info;

/* Solve (A + shift_i) x_i = b for nshift shifts and nrhs independent sources,
 * one Krylov space per source, the sources iterated together (every Dslash
 * is a multi-RHS Dslash).  I/O is always fp64: b [nrhs][3][Vh] and
 * x [nrhs][nshift][3][Vh] double complex (x caller-owned, overwritten).
 * prec selects the arithmetic of the iteration:
 *   STAG_FP64   fp64 throughout (the paper's Metropolis/heatbath inversions).
 *   fp32 / fp32-12: fp32 vectors, fp64 sums, and the base residual replaced
 *     by b - (A+s0)x0 from the fp64 operator after every decade (reliable
 *     updates); every shift's solution is accumulated in fp64 per decade.
 *   bf16-12: bf16-link iteration without residual replacement.
 *   For the three mixed precisions each shift whose fp64 true residual is
 *   still above tol is then refined by single-shift fp32 CG with fp64
 *   reliable updates, warm-started at x_i (a single shift may restart;
 *   the multi-shift solver may not, Sec. 6).
 * Convergence: shift i stops when |zeta_i| ||r|| <= tol ||b||; on return the
 * fp64 true residual of every shift is reported in info (may be NULL).
 * Returns STAG_ERR_NOT_CONVERGED after max_iter iterations of a stage, with
 * the partial solutions in x. */
stag_status stag_multishift_solve(stag_ctx* ctx, double mass, int nshift, const double* shifts,
                                  stag_prec prec, int nrhs, const void* b, void* x,
                                  double tol, int max_iter, stag_solve_info* info);

/* The same solve for n independent lattices at once (1 <= n <= STAG_MAX_BATCH,
 * one source each, one mass and shift set; no counterpart in the paper):
 * ctxs[i] with source b[i] [3][Vh_i] and solutions x[i] [nshift][3][Vh_i],
 * fp64 device arrays, info[i] per lattice (may be NULL).  One persistent
 * cooperative launch iterates every lattice whose solve has not converged;
 * each stops on its own convergence flag; reliable updates and the per-shift
 * refinement of mixed solves are made per lattice between launches.  Runs on
 * ctxs[0]'s stream (after the work queued on the other contexts' streams);
 * the contexts must be distinct.  Returns STAG_ERR_NOT_CONVERGED if any
 * lattice did not converge. */
stag_status stag_multishift_solve_batch(stag_ctx* const* ctxs, int n, double mass, int nshift, const double* shifts,
                                        stag_prec prec, const void* const* b, void* const* x, double tol,
                                        int max_iter, stag_solve_info* info);

/* ---- forces and actions (Sec. 2, Sec. 4) -------------------------------- */

/* Force of S_f = sum_k phi_k^dag r(A) phi_k over n_pf pseudo-fermions:
 *   F_a(x,mu) = sum_i alpha_i eps(x) eta_mu(x) Re tr[i T_a U_mu(x) Z_i(x+mu) Z_i(x)^dag]
 * with Z_i = X_i on even and D_oe X_i on odd sites, X_i = (A+beta_i)^-1 phi,
 * eps = +1/-1 on even/odd sites (dS/domega_a for U -> exp(i omega T_a) U).
 * phi: [n_pf][3][Vh] even fields, fp64 complex; prec is the arithmetic of
 * the inversions (fp32 ones get fp64 reliable updates) and of the force sum.
 * force: momentum layout, written (not accumulated). */
stag_status stag_fermion_force(stag_ctx* ctx, double mass, const stag_rational* r, stag_prec prec,
                               int n_pf, const void* phi, double* force, double tol, int max_iter,
                               stag_solve_info* info);

/* Wilson gauge force F_a = -(beta/3) Re tr(i T_a U_mu(x) Sigma_mu(x)),
 * Sigma the sum of the six staples; force in momentum layout. */
stag_status stag_gauge_force(stag_ctx* ctx, double beta, double* force);

/* Mean plaquette <Re tr U_P / 3> in fp64 (synchronous). */
stag_status stag_plaquette(stag_ctx* ctx, double* plaq);

/* ---- random draws: counter-based Philox4x64-10 (Salmon et al., SC'11) ----
 * Block (key = (seed, stream), counter = (index, counter, 0, 0)) gives four
 * uniforms u = ((w >> 11) + 1/2) 2^-53 and, by Box-Muller on (u0, u1) and
 * (u2, u3), four normals sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), ...
 * Momenta (stream 1): link (mu, s), s lexicographic, uses blocks
 *   2 (mu V + s) + j, j = 0, 1, for p_{4j..4j+3}; output in momentum layout.
 * Sources (stream 0x100 + stream + k for source k): even site h uses blocks
 *   2h + j; normals 0..5 times sqrt(1/2) are (Re, Im) of colours 0..2, so the
 *   density is exp(-xi^dag xi).  Output [n][3][Vh] fp64 complex.
 * The trajectory draws its momenta with seed/counter of stag_hmc and the
 * sources of flavour f with stream 16 f; the Metropolis uniform is word 0
 * of block (seed, stream 3, index 0, counter). */
/* Writes 8 x 4V momentum coefficients to the caller's DEVICE buffer mom. */
stag_status stag_draw_momenta(stag_ctx* ctx, unsigned long long seed, unsigned long long counter,
                              double* mom);
/* Writes n Gaussian sources ([n][3][Vh] fp64 complex, even sites) to the
 * caller's DEVICE buffer xi. */
stag_status stag_draw_sources(stag_ctx* ctx, unsigned long long seed, unsigned long long counter,
                              int stream, int n, void* xi);

/* ---- the RHMC trajectory (Sec. 2, Sec. 4) -------------------------------- */

#define STAG_MAX_FLAVOURS 2
/* One fermion term of the action: a flavour at its mass with n_pf
 * pseudo-fermions (Sec. 2: multiple pseudo-fermions), or one term of a
 * Hasenbusch mass split, det(A)^s = det(A_h)^s det(A / A_h)^s: the heavy term
 * is an ordinary flavour at m_h, the ratio term one at m whose rationals
 * approximate ((x + m_h^2 - m^2) / x)^s (heatbath: its power -1/2) -- the
 * same multi-shift solves and force formula with other coefficients.
 * level 0 puts the term's force on the outer integration level; level 1 on
 * a middle level of n_mid minimum-norm steps per outer half step around the
 * gauge level (stag_hmc.n_mid >= 1), where a split puts its heavy term
 * (large force, cheap solves).  Zero-initialised structs give level 0. */
typedef struct {
    double mass;
    int n_pf;                   /* pseudo-fermions of this flavour */
    int level;                  /* 0: outer level; 1: middle level (no counterpart in the paper) */
    stag_rational hb;           /* heatbath rational, ~ x^(+s/2)             */
    stag_rational md;           /* MD-force rational, ~ x^(-s)               */
    stag_rational met;          /* Metropolis rational, ~ x^(-s), tighter    */
} stag_flavour;

typedef struct {
    double beta;                /* Wilson coupling */
    double tau;                 /* trajectory length */
    int n_outer;                /* minimum-norm steps of the fermion level */
    int n_gauge;                /* gauge substeps per fermion half step */
    int n_flavours;
    stag_flavour flavour[STAG_MAX_FLAVOURS];
    double tol_md, tol_met;     /* relative residuals of MD and heatbath/Metropolis solves */
    int max_iter;
    stag_prec md_prec;          /* arithmetic of the MD force solves and link update:
                                   STAG_FP64 (plain fp64 path) or fp32 variants
                                   (mixed path: fp32 update, fp64 reunitarisation,
                                   fp64 heatbath and Metropolis, Sec. 4) */
    unsigned long long seed;    /* Philox4x64 key word 0 */
    unsigned long long counter; /* trajectory counter (Philox counter words 1-2) */
    const double* ext_mom;      /* optional DEVICE momenta (momentum layout) instead of drawn ones */
    const void* ext_xi;         /* optional DEVICE sources, [flavour][pf][3][Vh] fp64 complex */
    const void* ext_phi;        /* optional DEVICE pseudo-fermions (same layout) used instead of
                                   the heatbath; H at the start then uses phi^dag r_met(A) phi */
    double ext_uniform;         /* used for the accept test when ext_mom is set */
    int no_metropolis;          /* 1: always keep the new field (tests, reversibility) */
    int flip_momenta;           /* 1: start from -P (reversibility test) */
    int use_surrogate;          /* 1: three levels -- exact remainder F - F^ on the outer level,
                                   the loaded surrogate F^ on n_mid minimum-norm steps per outer
                                   half step, the gauge level inside (needs stag_surrogate_load) */
    int n_mid;                  /* minimum-norm steps of the middle level per outer half step
                                   (the surrogate and the level-1 flavour terms); >= 1 when used */
} stag_hmc;

typedef struct {
    double dH, H0, H1;          /* Hamiltonian change and its ends */
    double plaq;                /* mean plaquette after the trajectory */
    int accepted;
    long long cg_iterations;    /* Krylov iterations summed over all solves */
    int reliable_updates;
    double seconds;             /* device time of the trajectory */
    double t_heatbath;          /* device time of the heatbath inversions (s) */
    double t_fermion;           /* of the fermion-force kicks: MD inversions + force */
    double t_gauge;             /* of the gauge levels: Wilson force + link updates */
    double t_metropolis;        /* of the final fermion action (Metropolis inversions) */
} stag_traj;

/* One RHMC trajectory: heatbath, two-level minimum-norm MD, Metropolis with a
 * host-side uniform, restore of the old field on rejection. */
stag_status stag_md_trajectory(stag_ctx* ctx, const stag_hmc* p, stag_traj* out);

/* One trajectory of each of n independent chains (1 <= n <= STAG_MAX_BATCH),
 * advanced together (Sec. 2 algorithm per chain; the batching has no
 * counterpart in the paper).  ctxs[i] holds chain i's lattice (any size) and
 * field; p[i] and out[i] are its parameters and record, with the same
 * integrator schedule for all chains (n_outer, n_gauge, tau, md_prec,
 * flavours and pseudo-fermions per flavour, surrogate use, supplied phi or
 * not; seeds, counters, masses, rationals and supplied fields may differ).
 * Every multi-shift solve of the trajectories -- heatbath, each fermion force,
 * Metropolis -- is one solve over all chains: a persistent cooperative launch
 * that iterates every chain still converging, each with its own convergence
 * flag, one pseudo-fermion at a time.  The work runs on ctxs[0]'s stream,
 * after the work already queued on the other contexts' streams; the contexts
 * must be distinct and must not be used by other threads during the call.
 * out[i].seconds and the phase times are those of the whole batch.  Returns
 * the first error; with n == 1 it is stag_md_trajectory. */
stag_status stag_md_trajectory_batch(stag_ctx* const* ctxs, int n, const stag_hmc* p, stag_traj* out);

/* Momenta of the last trajectory (device, momentum layout, read-only). */
const double* stag_momenta(stag_ctx* ctx);

/* ---- learned fermion-force surrogate (a workload of this build; the paper has
 *      none).  Per link: 24 loop features f_k = Re tr(U S_k)/3 over the 6
 *      plaquette and 18 rectangle staples S_k through the link; an MLP
 *      24-32-32-24 (tanh, bf16 weights, fp32 math) gives weights w_k and
 *      F^_a = Re tr(i T_a U sum_k w_k S_k).  The staples are, for each nu != mu
 *      in increasing order, j = 0..7: plaquette up, down; 2mu x nu rectangles
 *      up (link first, second), down (first, second); mu x 2nu up, down. ---- */
#define STAG_SUR_PARAMS 2648  /* W1 (32x24, row-major), b1 (32), W2 (32x32), b2 (32), W3 (24x32), b3 (24) */
/* Set the weights (host array of STAG_SUR_PARAMS floats; weights are rounded
 * to bf16 on the device, the fp32 values kept as Adam's master copy). */
stag_status stag_surrogate_load(stag_ctx* ctx, const float* params);
/* Copies the fp32 master weights to a host array of STAG_SUR_PARAMS floats. */
stag_status stag_surrogate_store(stag_ctx* ctx, float* params);
/* F^ of the loaded field (momentum layout, written). */
stag_status stag_surrogate_force(stag_ctx* ctx, double* force);
/* Training data: append the current field's features and generators with the
 * given exact force (device, momentum layout) as the target. */
stag_status stag_surrogate_add_force_sample(stag_ctx* ctx, const double* exact_force);
/* Same, with the target computed here: the exact MD fermion force of the
 * flavours of p for pseudo-fermions from the heatbath with Philox counter. */
stag_status stag_surrogate_add_sample(stag_ctx* ctx, const stag_hmc* p, unsigned long long counter);
/* Number of training samples (configurations) stored; 0 for a NULL ctx. */
long long   stag_surrogate_samples(stag_ctx* ctx);
/* Sets the training store's capacity to exactly n_samples configurations
 * (896 bytes per link each: 24 features, 24 x 8 generators, 8 target
 * components in fp32), so that a large training set is allocated once
 * instead of growing by doubling (which copies and, near the end, needs
 * twice the memory).  Keeps the samples already stored; STAG_ERR_ARG if
 * n_samples is smaller than their number, STAG_ERR_ALLOC if the device
 * cannot hold it.  No counterpart in the paper. */
stag_status stag_surrogate_reserve(stag_ctx* ctx, long long n_samples);
/* Mean over stored links of |F^ - F|^2 and its gradient (host, STAG_SUR_PARAMS doubles, may be NULL). */
stag_status stag_surrogate_loss_grad(stag_ctx* ctx, double* loss, double* grad);
/* steps full-batch Adam steps (learning rate lr); losses before the first and last step. */
stag_status stag_surrogate_train(stag_ctx* ctx, int steps, double lr, double* loss_first, double* loss_last);

/* ---- self-test (no counterpart in the paper) ------------------------------
 * The bounded grid barrier of the persistent solvers, made to run out: two
 * blocks, only one arrives, its wait gives up after spin_limit polls
 * (1 <= spin_limit <= 2^26, as the solvers' own limit) and the kernel
 * reports it.  Returns STAG_ERR_TIMEOUT when the bound works (the context
 * stays usable), STAG_OK would mean the wait ended otherwise; synchronous. */
stag_status stag_selftest_barrier_timeout(stag_ctx* ctx, long long spin_limit);

/* ---- measurement (no counterpart in the paper; used for the roofline) ---- */

/* Kernels of the multi-shift iteration, timed by sampling. */
#define STAG_PK_DSLASH_OE 0      /* t = D_oe (r + beta p), multi-RHS                             */
#define STAG_PK_DSLASH_EO_A 1    /* p = r + beta p; q = c0 p - D_eo t; (p, q) and the alpha step */
#define STAG_PK_UPDATE 2         /* p_i, x_i of the live shifts; r -= alpha q; (r, r), beta step  */
#define STAG_PK_PERSISTENT 3     /* persistent solver in fp32 arithmetic (fp32 / 12-real / bf16
                                    links; every volume): units are iterations, every launch
                                    event-timed, bytes = one whole iteration                    */
#define STAG_PK_BATCH 4          /* batched solver (stag_*_batch; profile of the first context):
                                    units are batched iterations (one iteration of every lattice
                                    still iterating), every launch event-timed, bytes = those
                                    iterations of all lattices                                   */
#define STAG_PK_PERSISTENT_FF 5  /* persistent solver in float-float (the FP64 solves: heatbath,
                                    Metropolis, the FP64 path's MD), as STAG_PK_PERSISTENT       */
typedef struct {
    long long launches;       /* launches of this kernel since stag_profile_begin */
    int sampled;              /* of which bracketed by CUDA events on the context's stream */
    double sampled_ms;        /* summed device time of the sampled launches */
    double bytes_per_launch;  /* algorithmic DRAM bytes per launch, averaged over all launches:
                                 links once + every spinor read/written once */
} stag_kernel_profile;
/* Start counting; every sample_every-th solver iteration records events
 * around its four kernels (0 stops sampling). */
stag_status stag_profile_begin(stag_ctx* ctx, int sample_every);
/* Synchronises the stream and reports kernel `kind` (STAG_PK_*). */
stag_status stag_profile_read(stag_ctx* ctx, int kind, stag_kernel_profile* out);
/* Launch shape the batched solver chose for prec on batches led by ctx (the
 * candidates are timed on the first batched solves): its index, with the
 * threads per block and the blocks per SM requested of the register
 * allocator; -1 while still tuning. */
int stag_batch_shape(stag_ctx* ctx, stag_prec prec, int* threads_per_block, int* blocks_per_sm);
/* sizeof of the ABI's structs, for a binding to check its layouts against
 * (no device needed): which = 0 stag_lattice, 1 stag_rational,
 * 2 stag_solve_info, 3 stag_flavour, 4 stag_hmc, 5 stag_traj,
 * 6 stag_kernel_profile; 0 for any other value. */
size_t stag_abi_sizeof(int which);
/* Persistent solver only: microseconds that block 0 spent since
 * stag_profile_begin in [phase 1, barrier 1, phase 2, barrier 2, alpha step,
 * phase 3, barrier 3, beta step, in-launch reliable updates], then inside the
 * scalar steps [alpha: partial sums, arithmetic, block barrier; beta: partial
 * sums, arithmetic, the rest] (15 values, us must hold 15 doubles;
 * %globaltimer). */
stag_status stag_profile_phases(stag_ctx* ctx, double* us);
/* The batched solver's launches led by ctx, for fp32-class precisions (any
 * prec but STAG_FP64) or for the float-float fp64 iteration: 8 values, us in
 * [phase 1, barrier 1, phase 2, barrier 2, alpha step, phase 3, barrier 3,
 * beta step] (the steps include summing the blocks' partial sums). */
stag_status stag_profile_batch_phases(stag_ctx* ctx, stag_prec prec, double* us);
/* Number of kernels this context has launched since its creation. */
long long stag_launch_count(stag_ctx* ctx);
/* Threads per site the Dslash of this precision and source count uses (1, 2,
 * 4 or 8), autotuned on the first need for a lattice shape: every candidate
 * is timed as a CUDA graph of 20 launches and the fastest kept for every
 * context of that shape, precision and device in the process (so that their
 * sums run in the same order); us_per_launch (may be NULL) receives its
 * time.  The environment variable STAG_DSLASH_TPS fixes the value instead.
 * Returns 0 on a bad argument. */
int stag_tuned_threads_per_site(stag_ctx* ctx, stag_prec prec, int nrhs, double* us_per_launch);

#ifdef __cplusplus
}
#endif
#endif /* STAG_H */
