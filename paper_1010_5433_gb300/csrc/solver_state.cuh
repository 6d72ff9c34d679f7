// Device-resident state of one multi-shift CG solve (Sec. 6; Jegerlehner's
// shifted recurrences).  Written by the host before a solve, then owned by the
// kernels: the scalar recurrences run in the last block of the reducing
// kernels, so the iteration needs no host round trip.
#pragma once
#include "common.cuh"

struct SolverState {
    // set by the host
    int nrhs, nshift, base, max_iter;
    int mixed;                         // 1: fp64 reliable updates of the base residual
    int pad0;
    double tol2;                       // tol^2
    double c0;                         // m^2 + sigma_0
    double delta2;                     // reliable update when rr < delta2 * rr_at_last_update
    double dsig[STAG_MAX_SHIFTS];      // sigma_i - sigma_0
    // loop control (device)
    int k;                             // iterations completed
    int halt;                          // stop after the current iteration
    int status;                        // stag_status of the solve
    int need_reliable;                 // host must replace the base residual
    int n_reliable;
    double k4_units;                   // sum over updates of (72 + 96 n_live) per rhs (fp32 bytes/site)
    // per source
    int rhs_live[STAG_MAX_RHS];
    double bb[STAG_MAX_RHS], rr[STAG_MAX_RHS], rr_ref[STAG_MAX_RHS];
    double alpha[STAG_MAX_RHS], alpha_prev[STAG_MAX_RHS], beta_prev[STAG_MAX_RHS], beta[STAG_MAX_RHS];
    // per source and shift
    double zeta[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    double zeta_prev[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    double zeta_next[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    double cx[STAG_MAX_RHS][STAG_MAX_SHIFTS];    // x_i += cx p_i      (alpha_{i,k})
    double cpr[STAG_MAX_RHS][STAG_MAX_SHIFTS];   // p_i = cpr r + cpp p_i (zeta_k, beta_{i,k-1})
    double cpp[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    int live[STAG_MAX_RHS][STAG_MAX_SHIFTS];     // not converged: updated in the next iteration
    int iters_at[STAG_MAX_RHS][STAG_MAX_SHIFTS];
    double zratio[STAG_MAX_RHS][STAG_MAX_SHIFTS]; // zeta_{k+1} / zeta_k, from the alpha to the beta step
};
