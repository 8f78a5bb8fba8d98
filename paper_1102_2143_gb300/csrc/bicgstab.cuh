// Multi-shift BiCGStab (BiCGStab-M) for non-Hermitian shifted families
// (A + sigma_s I) x_s = b: the multi-shift solver the paper names for
// non-Hermitian operators (Sec. 1, Sec. 3) without printing it. FP64,
// generic block-CSR operator, one system per launch sequence.
//
// Seed: BiCGStab on A + sigma0 (sigma0 = the smallest shift) with shadow
// residual r~ = b; per iteration
//   v = A' p, alpha = rho / (r~, v), s = r - alpha v, t = A' s,
//   omega = (t, s) / (t, t), x0 += alpha p + omega s, r' = s - omega t,
//   rho' = (r~, r'), beta = (rho' / rho)(alpha / omega), p = r' + beta (p - omega v).
// Shift s (sigma_rel = sigma_s - sigma0): the BiCG part of its residual
// polynomial is zeta_s times the seed's (CG-M's zeta recurrence with the
// seed's alpha, beta) and each stabilising factor becomes
// omega_s = omega / (1 + sigma_rel omega), so its residual is (zeta/T) r with
// T = prod (1 + sigma_rel omega):
//   zeta' = zeta zeta^- alpha^- / (alpha beta^- (zeta^- - zeta) + zeta^- alpha^- (1 + sigma_rel alpha))
//   alpha_s = alpha zeta'/zeta, T' = T (1 + sigma_rel omega)
//   x_s += alpha_s p_s + omega_s (zeta'/T) s
//   p_s = (zeta'/T') r' + beta_s (p_s - (omega_s/alpha_s)((zeta/T) r - (zeta'/T) s)),
//   beta_s = beta (zeta'/zeta)^2;
// shift s has met tol once |zeta'/T'| |r'| <= tol |b|.
#pragma once
#include "engine.h"

namespace msc {

enum : int { ST_ERR_BREAKDOWN = 6 };  // a BiCGStab denominator vanished

struct BcgSys {
    double2 rho, alpha, omega, beta, alpha_prev, beta_prev;
    double bnorm2;   // |b|^2
    double tol2;     // tol^2
    double rnorm2;   // |r|^2 after the last iteration
    double sigma0;   // seed shift, applied by the operator kernels
    int status, it, max_iter, capped;
    int S, base, freeze, pad;
};

struct BcgSlot {
    double sigma_rel;                    // sigma_s - sigma0
    double2 zeta, zeta_prev, zeta_new;
    double2 T, T_new;
    double2 a_s, o_s, b_s;               // alpha_s, omega_s, beta_s
    double2 cr, cs, crn;                 // zeta/T, zeta'/T, zeta'/T'
    int active;                          // still iterating
    int flag;                            // this iteration: 0 skip, 1 x only, 2 x and p_s
    int conv_iter;                       // iteration at which tol was met (-1)
    int pad;
};

// Vectors of one system (n complex unknowns, FP64). r[par] is the current
// residual and r[1 - par] receives the next one (par = iteration parity).
struct BcgVec {
    double2* r[2];
    const double2* rt;   // shadow residual r~ = b
    double2* p;
    double2* v;
    double2* s;
    double2* t;
    double2* x;          // [S][npad] shift solutions (the base shift's is the seed's)
    double2* ps;         // [S][npad] shift directions (unused for the base)
    int64_t n, npad;
};

// init: r = b, p = b, x_s = 0, p_s = b; |b|^2 reduced into rho and bnorm2
cudaError_t launch_bcg_init(const Engine& e, BcgSys* sys, BcgSlot* slots, const BcgVec& v, int S,
                            cudaStream_t st);
// one iteration: five kernels (par = iteration parity)
cudaError_t launch_bcg_iter(const OpDev& A, const Engine& e, BcgSys* sys, BcgSlot* slots,
                            const BcgVec& v, int S, int par, cudaStream_t st);

}  // namespace msc
