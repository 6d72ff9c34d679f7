// The improved (asqtad) staggered Dslash: the paper's operator (Sec. 2) with
// the thin links replaced by fat links V and a third-neighbour Naik term W
// (Lepage, PRD 59 (1999) 074502; Orginos, Toussaint, Sugar, PRD 60 (1999)
// 054503):
//   D psi(x) = 1/2 sum_mu eta_mu(x) [ V_mu(x) psi(x+mu) - V_mu(x-mu)^dag psi(x-mu)
//                                   + W_mu(x) psi(x+3mu) - W_mu(x-3mu)^dag psi(x-3mu) ]
// V and W (path coefficients included, eta and the time boundary sign not)
// sit in two-float stores of the thin links' layout, built by asqtad.cu.
// The kernel is k_dslash's with sixteen hops per site instead of eight, so it
// takes the same sources and epilogues (plain store, A operator, the solver's).
#pragma once
#include "dslash.cuh"

struct AsqLinks {
    LinkPtrs fat, lng;
};

// x + 3 mu and x - 3 mu on the other parity, with the hop signs: eta_mu(x)
// times the product of the time-boundary signs of the three t-links crossed
struct Nbr3 {
    int fwd[4], bwd[4];
    float sf[4], sb[4];
};

__device__ __forceinline__ float asq_bc3(const Geom& g, int t0) {
    float s = 1.f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if ((t0 + k) % g.L[3] == g.L[3] - 1) s = -s;
    return s;
}

__device__ __forceinline__ void site_neighbours3(const Geom& g, const Nbr& n, Nbr3& m) {
    const int* c = n.x;
    const float e[4] = {1.f, (c[0] & 1) ? -1.f : 1.f, ((c[0] + c[1]) & 1) ? -1.f : 1.f,
                        ((c[0] + c[1] + c[2]) & 1) ? -1.f : 1.f};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int f[4] = {c[0], c[1], c[2], c[3]}, b[4] = {c[0], c[1], c[2], c[3]};
        f[mu] = (c[mu] + 3) % g.L[mu];
        b[mu] = ((c[mu] - 3) % g.L[mu] + g.L[mu]) % g.L[mu];
        m.fwd[mu] = (f[0] >> 1) + g.Lxh * (f[1] + g.L[1] * (f[2] + g.L[2] * f[3]));
        m.bwd[mu] = (b[0] >> 1) + g.Lxh * (b[1] + g.L[1] * (b[2] + g.L[2] * b[3]));
        m.sf[mu] = e[mu];
        m.sb[mu] = e[mu];
        if (mu == 3 && g.apt) {
            m.sf[3] *= asq_bc3(g, c[3]);
            m.sb[3] *= asq_bc3(g, b[3]);
        }
    }
}

// The sixteen hops of one site for NR sources, split over TPS threads as in
// dslash_site: each thread takes the fat and the Naik hop of its (mu, direction).
template <typename R, int FMT, int NR, int TPS, class Src>
__device__ __forceinline__ void dslash_site_asq(const Geom& g, int out_par, const AsqLinks& A, const Src& src,
                                                int r0, int nrhs, int h, int sub, Vec3<R> (&acc)[NR]) {
    Nbr n;
    site_neighbours(g, h, out_par, n);
    Nbr3 m;
    site_neighbours3(g, n, m);
#pragma unroll
    for (int r = 0; r < NR; ++r) zero(acc[r]);
#pragma unroll
    for (int k = 0; k < (TPS >= 4 ? 1 : 4 / TPS); ++k) {
        const int mu = TPS == 8 ? (sub >> 1) : (TPS == 4 ? sub : sub + k * TPS);
        const bool do_fwd = TPS < 8 || (sub & 1) == 0;
        const bool do_bwd = TPS < 8 || (sub & 1) == 1;
        if (do_fwd) {
            const Su3<R> v = LinkFetch<R, FMT>::get(A.fat, mu, out_par, h, g.Vh);
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (r0 + r < nrhs) mac_uv(acc[r], (R)n.sf[mu], v, src.load(r, r0 + r, n.fwd[mu], g.Vh));
            const Su3<R> w = LinkFetch<R, FMT>::get(A.lng, mu, out_par, h, g.Vh);
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (r0 + r < nrhs) mac_uv(acc[r], (R)m.sf[mu], w, src.load(r, r0 + r, m.fwd[mu], g.Vh));
        }
        if (do_bwd) {
            const Su3<R> v = LinkFetch<R, FMT>::get(A.fat, mu, 1 - out_par, n.bwd[mu], g.Vh);
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (r0 + r < nrhs) mac_udv(acc[r], -(R)n.sb[mu], v, src.load(r, r0 + r, n.bwd[mu], g.Vh));
            const Su3<R> w = LinkFetch<R, FMT>::get(A.lng, mu, 1 - out_par, m.bwd[mu], g.Vh);
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (r0 + r < nrhs) mac_udv(acc[r], -(R)m.sb[mu], w, src.load(r, r0 + r, m.bwd[mu], g.Vh));
        }
    }
}

template <typename R, int FMT, int NR, int TPS, class Src, class Epi>
__global__ void __launch_bounds__(STAG_RED_BLOCK)
k_dslash_asq(Geom g, int out_par, AsqLinks A, Src src, int nrhs, int nchunk, Epi epi) {
    if (epi.halted()) return;
    const int chunk = blockIdx.x % nchunk;
    const int sblock = blockIdx.x / nchunk;
    const int sub = TPS > 1 ? (int)(threadIdx.x % TPS) : 0;
    const int h = sblock * (blockDim.x / TPS) + threadIdx.x / TPS;
    const int r0 = chunk * NR;
    Vec3<R> acc[NR];
    const bool inside = h < g.Vh;
    src.template prepare<NR>(r0, nrhs);
    if (inside) {
        dslash_site_asq<R, FMT, NR, TPS>(g, out_par, A, src, r0, nrhs, h, sub, acc);
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) zero(acc[r]);
    }
    if (TPS > 1) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[r].c[c].re = group_sum<TPS>(acc[r].c[c].re);
                acc[r].c[c].im = group_sum<TPS>(acc[r].c[c].im);
            }
    }
    epi.template finish<NR>(g, h, inside && sub == 0, r0, nrhs, acc);
}
