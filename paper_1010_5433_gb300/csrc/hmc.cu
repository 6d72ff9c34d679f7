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

// Force of sum over terms and pseudo-fermions of phi^dag r(A) phi, written
// (mode 0) or added (mode 1) into out with coefficient coef.  Every term's
// multi-shift solutions go into one buffer, Y_i = D_oe X_i is then one
// multi-RHS Dslash over all terms, pseudo-fermions and shifts (e.g. 60
// right-hand sides for 2+1 flavours x 2 pseudo-fermions x 15 shifts), and the
// force kernel runs once per term.
stag_status fermion_force_terms(stag_ctx* ctx, const ForceTerm* terms, int nterms, stag_prec prec, double* out,
                                double coef, int mode, double tol, int max_iter, TrajStats* ts) {
    const size_t hc = half_c(ctx);
    const bool f64 = prec == STAG_FP64;
    const size_t cs = f64 ? sizeof(double2) : sizeof(float2);
    size_t total = 0;
    for (int t = 0; t < nterms; ++t) total += (size_t)terms[t].n * terms[t].r->n;
    void *x, *y;
    CKS(ws_get(ctx, WS_FORCE_X, total * hc * cs, &x));
    CKS(ws_get(ctx, WS_FORCE_Y, total * hc * cs, &y));
    size_t off = 0;
    for (int t = 0; t < nterms; ++t) {
        const ForceTerm& T = terms[t];
        const int ns = T.r->n;
        for (int k0 = 0; k0 < T.n; k0 += STAG_MAX_RHS) {
            const int nb = std::min(STAG_MAX_RHS, T.n - k0);
            const double2* ph = T.phi + (size_t)k0 * hc;
            char* xk = (char*)x + (off + (size_t)k0 * ns) * hc * cs;
            MsStats st;
            std::memset(&st, 0, sizeof(st));
            stag_status s;
            if (f64) {
                s = ms_core(ctx, T.mass, ns, T.r->beta, STAG_FP64, nb, ph, nullptr, xk, nullptr, tol, max_iter, false,
                            true, &st);
            } else {
                void *b32, *x64 = nullptr;
                CKS(ws_get(ctx, WS_FORCE_B32, (size_t)nb * hc * sizeof(float2), &b32));
                CKS(blas_convert(ctx, (size_t)nb * hc, ph, 1, b32, 0));
                const bool rel = prec != STAG_BF16_12;
                if (rel) CKS(ws_get(ctx, WS_FORCE_X64, (size_t)nb * ns * hc * sizeof(double2), &x64));
                s = ms_core(ctx, T.mass, ns, T.r->beta, prec, nb, b32, ph, xk, (double2*)x64, tol, max_iter, rel,
                            false, &st);
            }
            if (s != STAG_OK && s != STAG_ERR_NOT_CONVERGED) return s;
            if (ts) { ts->iters += st.iterations; ts->reliable += st.reliable; }
        }
        off += (size_t)T.n * ns;
    }
    // Y_i = D_oe X_i for every term, pseudo-fermion and shift: one n-RHS Dslash
    const stag_prec py = f64 ? STAG_FP64 : STAG_FP32;
    if (total > 0x7fffffff) return STAG_ERR_ARG;
    CKS(launch_dslash(ctx, 1, py, (int)total, x, y, 0.5));
    off = 0;
    for (int t = 0; t < nterms; ++t) {
        const ForceTerm& T = terms[t];
        const int ns = T.r->n;
        const char* xt = (const char*)x + off * hc * cs;
        const char* yt = (const char*)y + off * hc * cs;
        CKS(fermion_force_from_solutions(ctx, py, T.n, ns, T.r->alpha, xt, yt, out, coef, (t == 0) ? mode : 1));
        off += (size_t)T.n * ns;
    }
    return STAG_OK;
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
    stag_ctx* ctx;
    const stag_hmc* p;
    PhaseTimer* timer = nullptr;
    double* mom;
    double* force;
    double2* phi;      // [flavour][pf][3][Vh]
    stag_prec upd;     // arithmetic of the gauge force and link update
    TrajStats ts;

    double2* phi_of(int f) {
        size_t off = 0;
        for (int q = 0; q < f; ++q) off += (size_t)p->flavour[q].n_pf;
        return phi + off * half_c(ctx);
    }

    // p -= c F_fermion (all flavours, all pseudo-fermions in one force evaluation)
    stag_status fermion_kick(double c) {
        CKS(timer->begin(1));
        ForceTerm terms[STAG_MAX_FLAVOURS];
        for (int f = 0; f < p->n_flavours; ++f)
            terms[f] = ForceTerm{p->flavour[f].mass, &p->flavour[f].md, p->flavour[f].n_pf, phi_of(f)};
        if (p->n_flavours > 0)
            CKS(fermion_force_terms(ctx, terms, p->n_flavours, p->md_prec, mom, -c, 1, p->tol_md, p->max_iter, &ts));
        return timer->end(1);
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

    // the level between fermion steps: the gauge level, or with the surrogate
    // n_mid minimum-norm steps of F^ around gauge levels
    stag_status inner(double h) {
        if (!p->use_surrogate) return gauge_level(h, p->n_gauge);
        const int n = p->n_mid;
        const double d = h / n;
        CKS(sur_kick(LAMBDA_2MN * d));
        for (int j = 0; j < n; ++j) {
            CKS(gauge_level(d / 2, p->n_gauge));
            CKS(sur_kick((1 - 2 * LAMBDA_2MN) * d));
            CKS(gauge_level(d / 2, p->n_gauge));
            CKS(sur_kick((j == n - 1 ? 1.0 : 2.0) * LAMBDA_2MN * d));
        }
        return STAG_OK;
    }
    stag_status sur_kick(double c) { return surrogate_force_launch(ctx, mom, -c, 1); }
    // outer kick: p -= c F_fermion, and with the surrogate p += c F^ (the exact remainder)
    stag_status outer_kick(double c) {
        CKS(fermion_kick(c));
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
    if (!ctx || !p || !out) return STAG_ERR_ARG;
    if (!ctx->has_gauge) return STAG_ERR_NO_GAUGE;
    if (p->use_surrogate && (p->n_mid < 1 || !ctx->sur_loaded)) return STAG_ERR_ARG;
    if (p->n_outer < 1 || p->n_gauge < 1 || !(p->tau > 0) || p->n_flavours < 0 ||
        p->n_flavours > STAG_MAX_FLAVOURS || p->max_iter < 1 || p->md_prec < STAG_FP64 ||
        p->md_prec > STAG_BF16_12 || !(p->tol_md > 0) || !(p->tol_met > 0))
        return STAG_ERR_ARG;
    int npf_total = 0;
    for (int f = 0; f < p->n_flavours; ++f) {
        const stag_flavour& fl = p->flavour[f];
        if (fl.n_pf < 1 || !valid_rational(fl.hb) || !valid_rational(fl.md) || !valid_rational(fl.met))
            return STAG_ERR_ARG;
        npf_total += fl.n_pf;
    }
    std::memset(out, 0, sizeof(*out));
    const Geom& g = ctx->g;
    const size_t hc = half_c(ctx);
    const size_t mom_n = (size_t)64 * g.Vh;
    Traj T;
    PhaseTimer timer;
    timer.ctx = ctx;
    T.timer = &timer;
    T.ctx = ctx;
    T.p = p;
    T.upd = p->md_prec == STAG_FP64 ? STAG_FP64 : STAG_FP32;
    void *mom, *save_hi, *save_lo, *xi = nullptr, *phi = nullptr;
    CKS(ws_get(ctx, WS_MOM, mom_n * sizeof(double), &mom));
    const size_t gauge_bytes = (size_t)4 * 2 * 18 * g.Vh * sizeof(float);
    CKS(ws_get(ctx, WS_SAVE_HI, gauge_bytes, &save_hi));
    CKS(ws_get(ctx, WS_SAVE_LO, gauge_bytes, &save_lo));
    if (npf_total > 0) {
        CKS(ws_get(ctx, WS_XI, (size_t)npf_total * hc * sizeof(double2), &xi));
        CKS(ws_get(ctx, WS_PHI, (size_t)npf_total * hc * sizeof(double2), &phi));
    }
    T.mom = (double*)mom;
    T.phi = (double2*)phi;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, ctx->stream));

    // momenta and pseudo-fermion sources: supplied, or Philox draws
    if (p->ext_mom) CK(cudaMemcpyAsync(mom, p->ext_mom, mom_n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    else CKS(draw_momenta(ctx, T.mom, p->seed, p->counter));
    if (p->flip_momenta) CKS(mom_axpy(ctx, T.mom, T.mom, -2.0));
    if (npf_total > 0) {
        if (p->ext_xi)
            CK(cudaMemcpyAsync(xi, p->ext_xi, (size_t)npf_total * hc * sizeof(double2), cudaMemcpyDeviceToDevice,
                               ctx->stream));
        else {
            size_t off = 0;
            for (int f = 0; f < p->n_flavours; ++f) {
                CKS(draw_sources(ctx, (double2*)xi + off * hc, p->flavour[f].n_pf, p->seed, p->counter, 16 * f));
                off += p->flavour[f].n_pf;
            }
        }
    }
    CKS(gauge_copy(ctx, (float*)save_hi, (float*)save_lo, ctx->ghi, ctx->glo));

    // H at the start: fp64 sums, S_f = xi^dag xi after the heatbath
    double kin0, sg0, sf0 = 0.0;
    CKS(kinetic_sum(ctx, T.mom, &kin0));
    CKS(T.gauge_action(&sg0));
    if (npf_total > 0 && p->ext_phi) {
        CK(cudaMemcpyAsync(phi, p->ext_phi, (size_t)npf_total * hc * sizeof(double2), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CKS(T.fermion_action(&sf0));
    } else if (npf_total > 0) {
        std::vector<double> nn(npf_total);
        CKS(blas_norm2(ctx, STAG_FP64, npf_total, xi, nn.data()));
        for (double v : nn) sf0 += v;
    }
    // heatbath (first inversion, fp64)
    CKS(timer.begin(0));
    if (!p->ext_phi) {
        size_t off = 0;
        for (int f = 0; f < p->n_flavours; ++f) {
            const stag_flavour& fl = p->flavour[f];
            CKS(apply_rational_f64(ctx, fl.mass, fl.hb, fl.n_pf, (const double2*)xi + off * hc, T.phi + off * hc,
                                   p->tol_met, p->max_iter, &T.ts));
            off += fl.n_pf;
        }
    }
    CKS(timer.end(0));
    // molecular dynamics
    CKS(T.md_evolve());
    // H at the end (last inversion, fp64)
    double kin1, sg1, sf1 = 0.0;
    CKS(kinetic_sum(ctx, T.mom, &kin1));
    CKS(T.gauge_action(&sg1));
    CKS(timer.begin(3));
    if (npf_total > 0) CKS(T.fermion_action(&sf1));
    CKS(timer.end(3));
    const double h0 = kin0 + sg0 + sf0, h1 = kin1 + sg1 + sf1;
    const double dh = h1 - h0;
    double u;
    if (p->ext_mom) u = p->ext_uniform;
    else u = philox_uniform(philox_block(p->seed, RNG_STREAM_METROPOLIS, 0, p->counter).v[0]);
    int accept = std::isfinite(dh) && (dh <= 0.0 || u < std::exp(-dh));
    if (!accept && !p->no_metropolis) {
        CKS(gauge_copy(ctx, ctx->ghi, ctx->glo, (const float*)save_hi, (const float*)save_lo));
        ctx->b16_stale = true;
    }
    CK(cudaEventRecord(e1, ctx->stream));
    double plaq;
    CKS(plaquette_sum(ctx, &plaq));
    float ms = 0.f;
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out->dH = dh;
    out->H0 = h0;
    out->H1 = h1;
    out->plaq = plaq / (18.0 * g.V);
    out->accepted = accept;
    out->cg_iterations = T.ts.iters;
    out->reliable_updates = T.ts.reliable;
    out->seconds = ms * 1e-3;
    out->t_heatbath = timer.seconds(0);
    out->t_fermion = timer.seconds(1);
    out->t_gauge = timer.seconds(2);
    out->t_metropolis = timer.seconds(3);
    return std::isfinite(dh) ? STAG_OK : STAG_ERR_NAN;
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
