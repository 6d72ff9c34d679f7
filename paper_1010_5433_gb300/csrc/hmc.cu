// The RHMC trajectory on the device (Sec. 2 and Sec. 4 of the paper; ref.
// [rhmc] Horvath, Kennedy, Sint):
//   heatbath    phi = r_hb(A) xi             fp64 multi-shift (first inversion)
//   MD          two-level 2nd-order minimum-norm integrator, fermion force on
//               the outer level, Wilson force on n_gauge substeps per half step;
//               mixed path: fp32 force inversions, fp32 link update with fp64
//               reunitarisation; fp64 path: fp64 everywhere
//   Metropolis  H = 1/2 p^2 + S_g + phi^dag r_met(A) phi, fp64 (last inversion)
// The gauge field and momenta stay on the device; the host reads back only
// the scalars of H (Sec. 3).
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "philox.cuh"

namespace {
const double LAMBDA_2MN = 0.1931833275037836;   // Omelyan, Mryglod, Folk (2002)

size_t half_c(const stag_ctx* ctx) { return (size_t)3 * ctx->g.Vh; }

struct TrajStats {
    long long iters = 0;
    int reliable = 0;
};

// One flavour's share of a fermion force: its mass, rational, pseudo-fermions.
struct ForceTerm {
    double mass;
    const stag_rational* r;
    int n;                 // pseudo-fermions
    const double2* phi;    // [n][3][Vh] fp64
};

// Solutions X_i of every term and pseudo-fermion go into one buffer x
// ([term][pf][shift][3][Vh], the real type of the force arithmetic), their
// Y_i = D_oe X_i into y.
struct ForceBufs {
    void* x = nullptr;
    void* y = nullptr;
    size_t total = 0;      // right-hand sides: sum over terms of n_pf x n_shift
};
stag_status force_buffers(stag_ctx* ctx, const ForceTerm* terms, int nterms, stag_prec prec, ForceBufs* B) {
    const size_t cs = prec == STAG_FP64 ? sizeof(double2) : sizeof(float2);
    B->total = 0;
    for (int t = 0; t < nterms; ++t) B->total += (size_t)terms[t].n * terms[t].r->n;
    if (B->total > 0x7fffffff) return STAG_ERR_ARG;
    CKS(ws_get(ctx, WS_FORCE_X, B->total * half_c(ctx) * cs, &B->x));
    CKS(ws_get(ctx, WS_FORCE_Y, B->total * half_c(ctx) * cs, &B->y));
    return STAG_OK;
}

// The solve of pseudo-fermions k0 .. k0+nb-1 of term t as an MsRun: fp64
// solves iterate directly on phi; mixed ones on an fp32 copy, with the fp64
// accumulator for reliable updates (none for bf16 links), result in fp32.
stag_status force_solve_run(stag_ctx* ctx, const ForceTerm* terms, int t, int k0, int nb, stag_prec prec,
                            double tol, int max_iter, const ForceBufs& B, MsRun* R) {
    const size_t hc = half_c(ctx);
    const size_t cs = prec == STAG_FP64 ? sizeof(double2) : sizeof(float2);
    size_t off = 0;
    for (int q = 0; q < t; ++q) off += (size_t)terms[q].n * terms[q].r->n;
    const ForceTerm& T = terms[t];
    const int ns = T.r->n;
    *R = MsRun();
    R->ctx = ctx;
    R->mass = T.mass;
    R->nshift = ns;
    R->shifts = T.r->beta;
    R->prec = prec;
    R->nrhs = nb;
    R->x = (char*)B.x + (off + (size_t)k0 * ns) * hc * cs;
    R->tol = tol;
    R->max_iter = max_iter;
    const double2* ph = T.phi + (size_t)k0 * hc;
    if (prec == STAG_FP64) {
        R->b = ph;
        R->finish_to_f64 = true;
        return STAG_OK;
    }
    void *b32, *x64 = nullptr;
    CKS(ws_get(ctx, WS_FORCE_B32, (size_t)nb * hc * sizeof(float2), &b32));
    CKS(blas_convert(ctx, (size_t)nb * hc, ph, 1, b32, 0));
    R->reliable = prec != STAG_BF16_12;
    if (R->reliable) CKS(ws_get(ctx, WS_FORCE_X64, (size_t)nb * ns * hc * sizeof(double2), &x64));
    R->b = b32;
    R->b64 = ph;
    R->x64 = (double2*)x64;
    return STAG_OK;
}

stag_status ms_run(MsRun& R, MsStats* st) {
    return ms_core(R.ctx, R.mass, R.nshift, R.shifts, R.prec, R.nrhs, R.b, R.b64, R.x, R.x64, R.tol, R.max_iter,
                   R.reliable, R.finish_to_f64, st);
}

// Y_i = D_oe X_i for every term, pseudo-fermion and shift as one n-RHS
// Dslash, then the force of each term written (mode 0) or added (mode 1)
stag_status force_from_buffers(stag_ctx* ctx, const ForceTerm* terms, int nterms, stag_prec prec,
                               const ForceBufs& B, double* out, double coef, int mode) {
    const size_t hc = half_c(ctx);
    const stag_prec py = prec == STAG_FP64 ? STAG_FP64 : STAG_FP32;
    const size_t cs = prec == STAG_FP64 ? sizeof(double2) : sizeof(float2);
    CKS(launch_dslash(ctx, 1, py, (int)B.total, B.x, B.y, 0.5));
    if (ctx->asqtad) {
        // the outer products of every term and pseudo-fermion first, then one
        // pass through the fat and Naik paths (asqtad.cu)
        CKS(asq_outer_begin(ctx, py));
        size_t off = 0;
        for (int t = 0; t < nterms; ++t) {
            const ForceTerm& T = terms[t];
            const int ns = T.r->n;
            CKS(asq_outer_add(ctx, py, T.n, ns, T.r->alpha, (const char*)B.x + off * hc * cs,
                              (const char*)B.y + off * hc * cs, coef));
            off += (size_t)T.n * ns;
        }
        return asq_force_finish(ctx, py, out, mode);
    }
    size_t off = 0;
    for (int t = 0; t < nterms; ++t) {
        const ForceTerm& T = terms[t];
        const int ns = T.r->n;
        const char* xt = (const char*)B.x + off * hc * cs;
        const char* yt = (const char*)B.y + off * hc * cs;
        CKS(fermion_force_from_solutions(ctx, py, T.n, ns, T.r->alpha, xt, yt, out, coef, (t == 0) ? mode : 1));
        off += (size_t)T.n * ns;
    }
    return STAG_OK;
}

// Force of sum over terms and pseudo-fermions of phi^dag r(A) phi, written
// (mode 0) or added (mode 1) into out with coefficient coef.  Every term's
// multi-shift solutions go into one buffer, Y_i = D_oe X_i is then one
// multi-RHS Dslash over all terms, pseudo-fermions and shifts (e.g. 60
// right-hand sides for 2+1 flavours x 2 pseudo-fermions x 15 shifts), and the
// force kernel runs once per term.
stag_status fermion_force_terms(stag_ctx* ctx, const ForceTerm* terms, int nterms, stag_prec prec, double* out,
                                double coef, int mode, double tol, int max_iter, TrajStats* ts) {
    // an fp32 force of the improved operator uses fat links built in fp32 (a
    // deterministic function of the thin links, as the MD needs); the fp64
    // solves of the heatbath and the Metropolis step use float-float ones
    struct Fp32Build {
        stag_ctx* c;
        bool old;
        ~Fp32Build() { c->asq_fp32_build = old; }
    } guard{ctx, ctx->asq_fp32_build};
    ctx->asq_fp32_build = prec != STAG_FP64;
    ForceBufs B;
    CKS(force_buffers(ctx, terms, nterms, prec, &B));
    for (int t = 0; t < nterms; ++t) {
        for (int k0 = 0; k0 < terms[t].n; k0 += STAG_MAX_RHS) {
            const int nb = std::min(STAG_MAX_RHS, terms[t].n - k0);
            MsRun R;
            CKS(force_solve_run(ctx, terms, t, k0, nb, prec, tol, max_iter, B, &R));
            MsStats st;
            std::memset(&st, 0, sizeof(st));
            stag_status s = ms_run(R, &st);
            if (s != STAG_OK && s != STAG_ERR_NOT_CONVERGED) return s;
            if (ts) { ts->iters += st.iterations; ts->reliable += st.reliable; }
        }
    }
    return force_from_buffers(ctx, terms, nterms, prec, B, out, coef, mode);
}

// One term: the force of a single flavour (stag_fermion_force).
stag_status fermion_force_core(stag_ctx* ctx, double mass, const stag_rational* r, stag_prec prec, int n,
                               const double2* phi, double* out, double coef, int mode, double tol, int max_iter,
                               TrajStats* ts) {
    ForceTerm t{mass, r, n, phi};
    return fermion_force_terms(ctx, &t, 1, prec, out, coef, mode, tol, max_iter, ts);
}

bool valid_rational(const stag_rational& r) {
    if (r.n < 1 || r.n > STAG_MAX_SHIFTS || !r.alpha || !r.beta) return false;
    for (int i = 0; i < r.n; ++i)
        if (!std::isfinite(r.alpha[i]) || !std::isfinite(r.beta[i])) return false;
    return std::isfinite(r.a0);
}

// phi = a0 xi + sum_i alpha_i (A + beta_i)^-1 xi, fp64 (n sources)
stag_status apply_rational_f64(stag_ctx* ctx, double mass, const stag_rational& r, int n, const double2* xi,
                               double2* out, double tol, int max_iter, TrajStats* ts) {
    const size_t hc = half_c(ctx);
    for (int k0 = 0; k0 < n; k0 += STAG_MAX_RHS) {
        const int nb = std::min(STAG_MAX_RHS, n - k0);
        void* x;
        CKS(ws_get(ctx, WS_HB, (size_t)nb * r.n * hc * sizeof(double2), &x));
        MsStats st;
        std::memset(&st, 0, sizeof(st));
        stag_status s = ms_core(ctx, mass, r.n, r.beta, STAG_FP64, nb, xi + k0 * hc, nullptr, x, nullptr, tol,
                                max_iter, false, true, &st);
        if (s != STAG_OK && s != STAG_ERR_NOT_CONVERGED) return s;
        if (ts) ts->iters += st.iterations;
        CKS(blas_combine(ctx, nb, r.a0, xi + k0 * hc, r.n, r.alpha, (const double2*)x, out + k0 * hc));
    }
    return STAG_OK;
}

// Events bracketing the phases of a trajectory, read after its final sync.
struct PhaseTimer {
    stag_ctx* ctx = nullptr;
    std::vector<cudaEvent_t> ev;
    std::vector<std::pair<int, int>> spans[4];   // heatbath, fermion, gauge, metropolis
    int open_at = -1;
    stag_status begin(int) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaEventCreate");
        ev.push_back(e);
        open_at = (int)ev.size() - 1;
        return cudaEventRecord(e, ctx->stream) == cudaSuccess ? STAG_OK : cuda_fail(ctx, cudaGetLastError(), "rec");
    }
    stag_status end(int kind) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaEventCreate");
        ev.push_back(e);
        spans[kind].push_back({open_at, (int)ev.size() - 1});
        return cudaEventRecord(e, ctx->stream) == cudaSuccess ? STAG_OK : cuda_fail(ctx, cudaGetLastError(), "rec");
    }
    double seconds(int kind) {
        double t = 0.0;
        for (auto& sp : spans[kind]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[sp.first], ev[sp.second]) == cudaSuccess) t += ms * 1e-3;
        }
        return t;
    }
    ~PhaseTimer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

struct Traj {
    stag_ctx* ctx = nullptr;
    const stag_hmc* p = nullptr;
    PhaseTimer* timer = nullptr;
    double* mom = nullptr;
    double2* phi = nullptr;    // [flavour][pf][3][Vh]
    double2* xi = nullptr;     // heatbath sources, same layout
    float *save_hi = nullptr, *save_lo = nullptr;
    int npf_total = 0;
    stag_prec upd = STAG_FP32; // arithmetic of the gauge force and link update
    TrajStats ts;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double kin0 = 0.0, sg0 = 0.0, sf0 = 0.0;

    Traj() = default;
    Traj(const Traj&) = delete;
    Traj& operator=(const Traj&) = delete;
    ~Traj() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }

    double2* phi_of(int f) {
        size_t off = 0;
        for (int q = 0; q < f; ++q) off += (size_t)p->flavour[q].n_pf;
        return phi + off * half_c(ctx);
    }
    double2* xi_of(int f) {
        size_t off = 0;
        for (int q = 0; q < f; ++q) off += (size_t)p->flavour[q].n_pf;
        return xi + off * half_c(ctx);
    }

    // Workspace; momenta and sources (supplied, or Philox draws); the saved
    // field for a rejection; the kinetic and gauge parts of H at the start,
    // and S_f = xi^dag xi after the heatbath (with phi supplied, phi is
    // copied in and the caller evaluates S_f = phi^dag r_met(A) phi)
    stag_status begin() {
        const Geom& g = ctx->g;
        const size_t hc = half_c(ctx);
        const size_t mom_n = (size_t)64 * g.Vh;
        upd = p->md_prec == STAG_FP64 ? STAG_FP64 : STAG_FP32;
        npf_total = 0;
        for (int f = 0; f < p->n_flavours; ++f) npf_total += p->flavour[f].n_pf;
        void *m, *sh, *sl;
        CKS(ws_get(ctx, WS_MOM, mom_n * sizeof(double), &m));
        const size_t gauge_bytes = (size_t)4 * 2 * 18 * g.Vh * sizeof(float);
        CKS(ws_get(ctx, WS_SAVE_HI, gauge_bytes, &sh));
        CKS(ws_get(ctx, WS_SAVE_LO, gauge_bytes, &sl));
        mom = (double*)m;
        save_hi = (float*)sh;
        save_lo = (float*)sl;
        if (npf_total > 0) {
            void *x, *ph;
            CKS(ws_get(ctx, WS_XI, (size_t)npf_total * hc * sizeof(double2), &x));
            CKS(ws_get(ctx, WS_PHI, (size_t)npf_total * hc * sizeof(double2), &ph));
            xi = (double2*)x;
            phi = (double2*)ph;
        }
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, ctx->stream));
        if (p->ext_mom) CK(cudaMemcpyAsync(mom, p->ext_mom, mom_n * sizeof(double), cudaMemcpyDeviceToDevice,
                                           ctx->stream));
        else CKS(draw_momenta(ctx, mom, p->seed, p->counter));
        if (p->flip_momenta) CKS(mom_axpy(ctx, mom, mom, -2.0));
        if (npf_total > 0) {
            if (p->ext_xi)
                CK(cudaMemcpyAsync(xi, p->ext_xi, (size_t)npf_total * hc * sizeof(double2), cudaMemcpyDeviceToDevice,
                                   ctx->stream));
            else
                for (int f = 0; f < p->n_flavours; ++f)
                    CKS(draw_sources(ctx, xi_of(f), p->flavour[f].n_pf, p->seed, p->counter, 16 * f));
        }
        CKS(gauge_copy(ctx, save_hi, save_lo, ctx->ghi, ctx->glo));
        CKS(kinetic_sum(ctx, mom, &kin0));
        CKS(gauge_action(&sg0));
        sf0 = 0.0;
        if (npf_total > 0 && p->ext_phi) {
            CK(cudaMemcpyAsync(phi, p->ext_phi, (size_t)npf_total * hc * sizeof(double2), cudaMemcpyDeviceToDevice,
                               ctx->stream));
        } else if (npf_total > 0) {
            std::vector<double> nn(npf_total);
            CKS(blas_norm2(ctx, STAG_FP64, npf_total, xi, nn.data()));
            for (double v : nn) sf0 += v;
        }
        return STAG_OK;
    }

    // phi = r_hb(A) xi for every flavour (the first inversion, fp64)
    stag_status heatbath() {
        if (p->ext_phi) return STAG_OK;
        for (int f = 0; f < p->n_flavours; ++f) {
            const stag_flavour& fl = p->flavour[f];
            CKS(apply_rational_f64(ctx, fl.mass, fl.hb, fl.n_pf, xi_of(f), phi_of(f), p->tol_met, p->max_iter, &ts));
        }
        return STAG_OK;
    }

    // dH with S_f = sf1 at the end (fp64 sums), the Metropolis decision
    // (restoring the saved field on rejection) and the record of the trajectory
    stag_status finish(double sf1, stag_traj* out) {
        double kin1, sg1;
        CKS(kinetic_sum(ctx, mom, &kin1));
        CKS(gauge_action(&sg1));
        const double h0 = kin0 + sg0 + sf0, h1 = kin1 + sg1 + sf1;
        const double dh = h1 - h0;
        double u;
        if (p->ext_mom) u = p->ext_uniform;
        else u = philox_uniform(philox_block(p->seed, RNG_STREAM_METROPOLIS, 0, p->counter).v[0]);
        const int accept = std::isfinite(dh) && (dh <= 0.0 || u < std::exp(-dh));
        if (!accept && !p->no_metropolis) {
            CKS(gauge_copy(ctx, ctx->ghi, ctx->glo, save_hi, save_lo));
            ctx->b16_stale = true;
            ctx->asq_stale = true;
        }
        CK(cudaEventRecord(e1, ctx->stream));
        double plaq;
        CKS(plaquette_sum(ctx, &plaq));
        float ms = 0.f;
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        out->dH = dh;
        out->H0 = h0;
        out->H1 = h1;
        out->plaq = plaq / (18.0 * ctx->g.V);
        out->accepted = accept;
        out->cg_iterations = ts.iters;
        out->reliable_updates = ts.reliable;
        out->seconds = ms * 1e-3;
        out->t_heatbath = timer->seconds(0);
        out->t_fermion = timer->seconds(1);
        out->t_gauge = timer->seconds(2);
        out->t_metropolis = timer->seconds(3);
        return std::isfinite(dh) ? STAG_OK : STAG_ERR_NAN;
    }

    // p -= c F_fermion of the flavour terms on integration level `level` (all
    // of them, and all their pseudo-fermions, in one force evaluation)
    stag_status fermion_kick(double c, int level) {
        CKS(timer->begin(1));
        ForceTerm terms[STAG_MAX_FLAVOURS];
        int nt = 0;
        for (int f = 0; f < p->n_flavours; ++f)
            if (p->flavour[f].level == level)
                terms[nt++] = ForceTerm{p->flavour[f].mass, &p->flavour[f].md, p->flavour[f].n_pf, phi_of(f)};
        if (nt > 0) CKS(fermion_force_terms(ctx, terms, nt, p->md_prec, mom, -c, 1, p->tol_md, p->max_iter, &ts));
        return timer->end(1);
    }
    bool has_middle_terms() const {
        for (int f = 0; f < p->n_flavours; ++f)
            if (p->flavour[f].level == 1) return true;
        return false;
    }
    stag_status gauge_kick(double c) { return gauge_force_launch(ctx, upd, p->beta, mom, -c, 1); }

    // n minimum-norm steps of the gauge force over h, adjacent kicks merged
    stag_status gauge_level(double h, int n) {
        const double d = h / n;
        CKS(timer->begin(2));
        CKS(gauge_kick(LAMBDA_2MN * d));
        for (int j = 0; j < n; ++j) {
            CKS(update_links(ctx, mom, d / 2, upd));
            CKS(gauge_kick((1 - 2 * LAMBDA_2MN) * d));
            CKS(update_links(ctx, mom, d / 2, upd));
            CKS(gauge_kick((j == n - 1 ? 1.0 : 2.0) * LAMBDA_2MN * d));
        }
        return timer->end(2);
    }

    // the level between fermion steps: the gauge level, or, with the surrogate
    // or flavour terms on the middle level (a Hasenbusch mass split), n_mid
    // minimum-norm steps of their force around gauge levels
    stag_status inner(double h) {
        if (!p->use_surrogate && !has_middle_terms()) return gauge_level(h, p->n_gauge);
        const int n = p->n_mid;
        const double d = h / n;
        CKS(mid_kick(LAMBDA_2MN * d));
        for (int j = 0; j < n; ++j) {
            CKS(gauge_level(d / 2, p->n_gauge));
            CKS(mid_kick((1 - 2 * LAMBDA_2MN) * d));
            CKS(gauge_level(d / 2, p->n_gauge));
            CKS(mid_kick((j == n - 1 ? 1.0 : 2.0) * LAMBDA_2MN * d));
        }
        return STAG_OK;
    }
    // p -= c (F^ + F of the middle-level flavour terms)
    stag_status mid_kick(double c) {
        if (p->use_surrogate) CKS(surrogate_force_launch(ctx, mom, -c, 1));
        if (has_middle_terms()) CKS(fermion_kick(c, 1));
        return STAG_OK;
    }
    // outer kick: p -= c F_fermion of the outer-level terms, and with the
    // surrogate p += c F^ (the exact remainder)
    stag_status outer_kick(double c) {
        CKS(fermion_kick(c, 0));
        if (p->use_surrogate) CKS(surrogate_force_launch(ctx, mom, c, 1));
        return STAG_OK;
    }

    stag_status md_evolve() {
        const double e = p->tau / p->n_outer;
        CKS(outer_kick(LAMBDA_2MN * e));
        for (int s = 0; s < p->n_outer; ++s) {
            CKS(inner(e / 2));
            CKS(outer_kick((1 - 2 * LAMBDA_2MN) * e));
            CKS(inner(e / 2));
            CKS(outer_kick((s == p->n_outer - 1 ? 1.0 : 2.0) * LAMBDA_2MN * e));
        }
        return STAG_OK;
    }

    stag_status gauge_action(double* s) {
        double plaq;
        CKS(plaquette_sum(ctx, &plaq));
        *s = p->beta * (6.0 * ctx->g.V - plaq / 3.0);
        return STAG_OK;
    }

    // sum_f,k phi^dag r_met(A) phi in fp64
    stag_status fermion_action(double* s) {
        *s = 0.0;
        const size_t hc = half_c(ctx);
        for (int f = 0; f < p->n_flavours; ++f) {
            const stag_flavour& fl = p->flavour[f];
            void* t;
            CKS(ws_get(ctx, WS_MISC, (size_t)fl.n_pf * hc * sizeof(double2), &t));
            CKS(apply_rational_f64(ctx, fl.mass, fl.met, fl.n_pf, phi_of(f), (double2*)t, p->tol_met, p->max_iter,
                                   &ts));
            std::vector<double> d(fl.n_pf);
            CKS(blas_dot_re(ctx, fl.n_pf, phi_of(f), (const double2*)t, d.data()));
            for (double v : d) *s += v;
        }
        return STAG_OK;
    }
};

stag_status check_hmc(stag_ctx* ctx, const stag_hmc* p) {
    if (!ctx || !p) return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    if (p->use_surrogate && (p->n_mid < 1 || !ctx->sur_loaded)) return STAG_ERR_ARG;
    if (ctx->asqtad && (p->use_surrogate || (p->md_prec != STAG_FP64 && p->md_prec != STAG_FP32)))
        return STAG_ERR_ARG;
    for (int f = 0; f < p->n_flavours && f < STAG_MAX_FLAVOURS; ++f)
        if (p->flavour[f].level < 0 || p->flavour[f].level > 1 || (p->flavour[f].level == 1 && p->n_mid < 1))
            return STAG_ERR_ARG;
    if (p->n_outer < 1 || p->n_gauge < 1 || !(p->tau > 0) || p->n_flavours < 0 ||
        p->n_flavours > STAG_MAX_FLAVOURS || p->max_iter < 1 || p->md_prec < STAG_FP64 ||
        p->md_prec > STAG_BF16_12 || !(p->tol_md > 0) || !(p->tol_met > 0))
        return STAG_ERR_ARG;
    for (int f = 0; f < p->n_flavours; ++f) {
        const stag_flavour& fl = p->flavour[f];
        if (fl.n_pf < 1 || !valid_rational(fl.hb) || !valid_rational(fl.md) || !valid_rational(fl.met))
            return STAG_ERR_ARG;
    }
    return STAG_OK;
}
}  // namespace

extern "C" stag_status stag_fermion_force(stag_ctx* ctx, double mass, const stag_rational* r, stag_prec prec,
                                          int n_pf, const void* phi, double* force, double tol, int max_iter,
                                          stag_solve_info* info) {
    if (!ctx || !r || !phi || !force || n_pf < 1 || !valid_rational(*r) || !(tol > 0) || max_iter < 1)
        return STAG_ERR_ARG;
    if (prec < STAG_FP64 || prec > STAG_BF16_12) return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    if (prec == STAG_BF16_12 && ctx->b16_stale) CKS(refresh_bf16(ctx));
    TrajStats ts;
    CKS(fermion_force_core(ctx, mass, r, prec, n_pf, (const double2*)phi, force, 1.0, 0, tol, max_iter, &ts));
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->iterations = (int)ts.iters;
        info->reliable_updates = ts.reliable;
    }
    return STAG_OK;
}

extern "C" const double* stag_momenta(stag_ctx* ctx) { return ctx ? (const double*)ctx->ws[WS_MOM] : nullptr; }

extern "C" stag_status stag_md_trajectory(stag_ctx* ctx, const stag_hmc* p, stag_traj* out) {
    if (!out) return STAG_ERR_ARG;
    CKS(check_hmc(ctx, p));
    std::memset(out, 0, sizeof(*out));
    PhaseTimer timer;
    timer.ctx = ctx;
    Traj T;
    T.ctx = ctx;
    T.p = p;
    T.timer = &timer;
    CKS(T.begin());
    if (T.npf_total > 0 && p->ext_phi) CKS(T.fermion_action(&T.sf0));
    CKS(timer.begin(0));
    CKS(T.heatbath());
    CKS(timer.end(0));
    // the MD evolution is enqueued without a host read between its solves
    // (their iterations and first error are read once, here)
    CKS(defer_begin(ctx));
    const stag_status md = T.md_evolve();
    long long md_iters = 0, md_rel = 0;
    const stag_status de = defer_end(ctx, &md_iters, &md_rel);
    T.ts.iters += md_iters;
    T.ts.reliable += (int)md_rel;
    CKS(md);
    CKS(de);
    double sf1 = 0.0;
    CKS(timer.begin(3));
    if (T.npf_total > 0) CKS(T.fermion_action(&sf1));
    CKS(timer.end(3));
    if (p->use_surrogate) CKS(surrogate_check(ctx));
    return T.finish(sf1, out);
}

extern "C" stag_status stag_surrogate_add_sample(stag_ctx* ctx, const stag_hmc* p, unsigned long long counter) {
    if (!ctx || !p || p->n_flavours < 1 || p->n_flavours > STAG_MAX_FLAVOURS) return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    const size_t hc = half_c(ctx);
    int npf = 0;
    for (int f = 0; f < p->n_flavours; ++f) {
        if (p->flavour[f].n_pf < 1 || !valid_rational(p->flavour[f].hb) || !valid_rational(p->flavour[f].md))
            return STAG_ERR_ARG;
        npf += p->flavour[f].n_pf;
    }
    void *xi, *phi, *force;
    CKS(ws_get(ctx, WS_XI, (size_t)npf * hc * sizeof(double2), &xi));
    CKS(ws_get(ctx, WS_PHI, (size_t)npf * hc * sizeof(double2), &phi));
    CKS(ws_get(ctx, WS_FORCE, (size_t)64 * ctx->g.Vh * sizeof(double), &force));
    ForceTerm terms[STAG_MAX_FLAVOURS];
    size_t off = 0;
    for (int f = 0; f < p->n_flavours; ++f) {
        const stag_flavour& fl = p->flavour[f];
        CKS(draw_sources(ctx, (double2*)xi + off * hc, fl.n_pf, p->seed, counter, 16 * f));
        CKS(apply_rational_f64(ctx, fl.mass, fl.hb, fl.n_pf, (const double2*)xi + off * hc, (double2*)phi + off * hc,
                               p->tol_met, p->max_iter, nullptr));
        terms[f] = ForceTerm{fl.mass, &fl.md, fl.n_pf, (const double2*)phi + off * hc};
        off += fl.n_pf;
    }
    CKS(fermion_force_terms(ctx, terms, p->n_flavours, p->md_prec, (double*)force, 1.0, 0, p->tol_md, p->max_iter,
                            nullptr));
    return surrogate_append(ctx, (const double*)force);
}

// ---------------------------------------------------------------------------
// Independent chains advanced together: every chain runs its own trajectory
// (own field, momenta, pseudo-fermions, accept/reject), in lockstep, so that
// each multi-shift solve of the trajectory -- heatbath, every fermion-force
// evaluation, Metropolis -- is one batched solve over all chains (one source
// per chain at a time, batch.cu); the gauge levels and force kernels run per
// chain on the shared stream.
namespace {

// Restores the contexts' own streams when the batch call returns.
struct StreamSwap {
    std::vector<std::pair<stag_ctx*, cudaStream_t>> saved;
    ~StreamSwap() {
        for (auto& s : saved) s.first->stream = s.second;
    }
};

bool same_schedule(const stag_hmc& a, const stag_hmc& b) {
    for (int f = 0; f < a.n_flavours; ++f)
        if (a.flavour[f].level != 0 || b.flavour[f].level != 0) return false;   // batched chains: one fermion level
    if (a.n_outer != b.n_outer || a.n_gauge != b.n_gauge || a.tau != b.tau || a.md_prec != b.md_prec ||
        a.n_flavours != b.n_flavours || a.use_surrogate != b.use_surrogate || (a.use_surrogate && a.n_mid != b.n_mid) ||
        (a.ext_phi != nullptr) != (b.ext_phi != nullptr))
        return false;
    for (int f = 0; f < a.n_flavours; ++f)
        if (a.flavour[f].n_pf != b.flavour[f].n_pf) return false;
    return true;
}

// out_i = a0 src_i + sum_k alpha_k (A + beta_k)^-1 src_i in fp64 for one
// flavour and pseudo-fermion k of every chain (hb: the heatbath; met: the
// Metropolis action, out then dotted with phi and added to sf)
stag_status batch_rational(std::vector<Traj>& T, bool met, std::vector<double>* sf) {
    const int n = (int)T.size();
    stag_ctx* ctx = T[0].ctx;
    const stag_hmc& p0 = *T[0].p;
    for (int f = 0; f < p0.n_flavours; ++f) {
        for (int k = 0; k < p0.flavour[f].n_pf; ++k) {
            std::vector<MsRun> runs(n);
            std::vector<void*> xs(n), outs(n);
            for (int i = 0; i < n; ++i) {
                Traj& t = T[i];
                const stag_flavour& fl = t.p->flavour[f];
                const stag_rational& r = met ? fl.met : fl.hb;
                const size_t hc = half_c(t.ctx);
                CKS(ws_get(t.ctx, WS_HB, (size_t)r.n * hc * sizeof(double2), &xs[i]));
                if (met) CKS(ws_get(t.ctx, WS_MISC, hc * sizeof(double2), &outs[i]));
                else outs[i] = t.phi_of(f) + (size_t)k * hc;
                MsRun& R = runs[i];
                R.ctx = t.ctx;
                R.mass = fl.mass;
                R.nshift = r.n;
                R.shifts = r.beta;
                R.prec = STAG_FP64;
                R.nrhs = 1;
                R.b = (met ? t.phi_of(f) : t.xi_of(f)) + (size_t)k * hc;
                R.x = xs[i];
                R.tol = t.p->tol_met;
                R.max_iter = t.p->max_iter;
                R.finish_to_f64 = true;
            }
            std::vector<MsStats> st(n);
            std::vector<stag_status> ok(n);
            CKS(ms_core_multi(runs.data(), n, st.data(), ok.data()));
            for (int i = 0; i < n; ++i) {
                if (ok[i] != STAG_OK && ok[i] != STAG_ERR_NOT_CONVERGED) return ok[i];
                Traj& t = T[i];
                const stag_flavour& fl = t.p->flavour[f];
                const stag_rational& r = met ? fl.met : fl.hb;
                t.ts.iters += st[i].iterations;
                CKS(blas_combine(t.ctx, 1, r.a0, (const double2*)runs[i].b, r.n, r.alpha, (const double2*)xs[i],
                                 (double2*)outs[i]));
                if (met) {
                    double d = 0.0;
                    CKS(blas_dot_re(t.ctx, 1, (const double2*)runs[i].b, (const double2*)outs[i], &d));
                    (*sf)[i] += d;
                }
            }
        }
    }
    (void)ctx;
    return STAG_OK;
}

// p_i -= c (F_i - F^_i) on every chain: the solves of each flavour and
// pseudo-fermion batched over the chains, then per chain one n-RHS D_oe and
// the force kernels
stag_status batch_outer_kick(std::vector<Traj>& T, double c) {
    const int n = (int)T.size();
    const stag_hmc& p0 = *T[0].p;
    CKS(T[0].timer->begin(1));
    if (p0.n_flavours > 0) {
        std::vector<std::vector<ForceTerm>> terms(n);
        std::vector<ForceBufs> B(n);
        for (int i = 0; i < n; ++i) {
            const stag_hmc& p = *T[i].p;
            for (int f = 0; f < p.n_flavours; ++f)
                terms[i].push_back(ForceTerm{p.flavour[f].mass, &p.flavour[f].md, p.flavour[f].n_pf, T[i].phi_of(f)});
            CKS(force_buffers(T[i].ctx, terms[i].data(), p.n_flavours, p.md_prec, &B[i]));
        }
        for (int f = 0; f < p0.n_flavours; ++f) {
            for (int k = 0; k < p0.flavour[f].n_pf; ++k) {
                std::vector<MsRun> runs(n);
                for (int i = 0; i < n; ++i)
                    CKS(force_solve_run(T[i].ctx, terms[i].data(), f, k, 1, T[i].p->md_prec, T[i].p->tol_md,
                                        T[i].p->max_iter, B[i], &runs[i]));
                std::vector<MsStats> st(n);
                std::vector<stag_status> ok(n);
                CKS(ms_core_multi(runs.data(), n, st.data(), ok.data()));
                for (int i = 0; i < n; ++i) {
                    if (ok[i] != STAG_OK && ok[i] != STAG_ERR_NOT_CONVERGED) return ok[i];
                    T[i].ts.iters += st[i].iterations;
                    T[i].ts.reliable += st[i].reliable;
                }
            }
        }
        for (int i = 0; i < n; ++i)
            CKS(force_from_buffers(T[i].ctx, terms[i].data(), T[i].p->n_flavours, T[i].p->md_prec, B[i], T[i].mom,
                                   -c, 1));
    }
    if (p0.use_surrogate)
        for (int i = 0; i < n; ++i) CKS(surrogate_force_launch(T[i].ctx, T[i].mom, c, 1));
    return T[0].timer->end(1);
}

stag_status batch_md_evolve(std::vector<Traj>& T) {
    const stag_hmc& p = *T[0].p;
    const double e = p.tau / p.n_outer;
    CKS(batch_outer_kick(T, LAMBDA_2MN * e));
    for (int s = 0; s < p.n_outer; ++s) {
        for (auto& t : T) CKS(t.inner(e / 2));
        CKS(batch_outer_kick(T, (1 - 2 * LAMBDA_2MN) * e));
        for (auto& t : T) CKS(t.inner(e / 2));
        CKS(batch_outer_kick(T, (s == p.n_outer - 1 ? 1.0 : 2.0) * LAMBDA_2MN * e));
    }
    return STAG_OK;
}
}  // namespace

extern "C" stag_status stag_md_trajectory_batch(stag_ctx* const* ctxs, int n, const stag_hmc* ps, stag_traj* outs) {
    if (!ctxs || !ps || !outs || n < 1 || n > STAG_MAX_BATCH) return STAG_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return STAG_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return STAG_ERR_ARG;
        CKS(check_hmc(ctxs[i], &ps[i]));
        if (ctxs[i]->asqtad) return STAG_ERR_ARG;   // batched chains run the unimproved operator
        if (!same_schedule(ps[0], ps[i])) return STAG_ERR_ARG;
    }
    if (n == 1) return stag_md_trajectory(ctxs[0], &ps[0], &outs[0]);
    stag_ctx* ctx = ctxs[0];
    StreamSwap swap;
    for (int i = 0; i < n; ++i) {
        swap.saved.push_back({ctxs[i], ctxs[i]->stream});
        std::memset(&outs[i], 0, sizeof(stag_traj));
    }
    // the chains' own streams may hold earlier work: the lead stream waits for it
    for (int i = 1; i < n; ++i) {
        if (ctxs[i]->stream == ctx->stream) continue;
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, ctxs[i]->stream));
        CK(cudaStreamWaitEvent(ctx->stream, ev, 0));
        cudaEventDestroy(ev);
        ctxs[i]->stream = ctx->stream;
    }
    PhaseTimer timer;
    timer.ctx = ctx;
    std::vector<Traj> T(n);
    for (int i = 0; i < n; ++i) {
        T[i].ctx = ctxs[i];
        T[i].p = &ps[i];
        T[i].timer = &timer;
        CKS(T[i].begin());
    }
    std::vector<double> sf0(n, 0.0), sf1(n, 0.0);
    if (ps[0].n_flavours > 0 && ps[0].ext_phi) {
        CKS(batch_rational(T, true, &sf0));
        for (int i = 0; i < n; ++i) T[i].sf0 = sf0[i];
    }
    CKS(timer.begin(0));
    if (ps[0].n_flavours > 0 && !ps[0].ext_phi) CKS(batch_rational(T, false, nullptr));
    CKS(timer.end(0));
    CKS(batch_md_evolve(T));
    CKS(timer.begin(3));
    if (ps[0].n_flavours > 0) CKS(batch_rational(T, true, &sf1));
    CKS(timer.end(3));
    if (ps[0].use_surrogate)
        for (int i = 0; i < n; ++i) CKS(surrogate_check(ctxs[i]));
    stag_status worst = STAG_OK;
    for (int i = 0; i < n; ++i) {
        stag_status s = T[i].finish(sf1[i], &outs[i]);
        if (s != STAG_OK && worst == STAG_OK) worst = s;
    }
    return worst;
}
