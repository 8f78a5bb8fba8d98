/*
 * msc.h - multi-shift conjugate gradient on NVIDIA GB300 (sm_103a).
 *
 * Solves the shifted family of eq. (linprob), Sec. 2 of Galvez & van Anders,
 * "Accelerating the solution of families of shifted linear systems with
 * CUDA" (arXiv:1102.2143):
 *
 *     (A + sigma_s I) x_s = b,   s = 0 .. S-1,
 *
 * for every shift from one Krylov sequence (CG-M, Algorithm 1, Sec. 2; the
 * Krylov space is shift invariant, eq. krylov). A is Hermitian positive
 * definite and is given either as the staggered lattice operator
 * A = M^dagger M = m^2 - D^2 over SU(N) links, or as a generic block-CSR
 * matrix with complex bd x bd blocks (the generic matrix the paper's solver
 * takes, Sec. 3 and Fig. 1). The calls follow the paper's statement of the
 * problem: operator, source, list of shifts, tolerance and iteration cap in;
 * all x_s out in one array (Fig. 1: x holds N * N_s values).
 *
 * Conventions for every call:
 *   - complex numbers are interleaved (re, im) doubles; a vector of n complex
 *     unknowns is 2n doubles; a block is row-major;
 *   - a data pointer may point to host memory (pageable or pinned) or to
 *     device memory of the context's device; the library asks the CUDA
 *     runtime which one it is and copies as needed;
 *   - the caller owns every buffer it passes; the library copies operator
 *     data into its own device memory at creation, so the caller may free
 *     its arrays as soon as the call returns;
 *   - every call returns an int status: MSC_OK (0) or one of MSC_ERR_*;
 *     msc_strerror() names it. A context is not thread safe: calls on one
 *     context must not overlap.
 *   - work runs on the context's own CUDA stream, ordered after the work
 *     already queued on the stream given at creation; calls return after
 *     their results are in the caller's buffers.
 */
#ifndef MSC_H
#define MSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MSC_OK                0
#define MSC_ERR_ARG           1  /* invalid argument (null, size, negative shift...) */
#define MSC_ERR_CUDA          2  /* a CUDA runtime call failed */
#define MSC_ERR_OOM           3  /* device allocation failed */
#define MSC_ERR_NOT_HPD       4  /* p^dagger A p <= 0 met: A is not positive definite */
#define MSC_ERR_NONFINITE     5  /* NaN or Inf met in the source or the iteration */
#define MSC_ERR_NOT_CONVERGED 6  /* iteration cap reached; x is written, see info */
#define MSC_ERR_TIMEOUT       7  /* a kernel's bounded wait on its own asynchronous
                                    copies ran out (the solve's results are void;
                                    the context stays usable) */
#define MSC_ERR_UNSUPPORTED   8  /* valid request the library does not handle */
#define MSC_ERR_BREAKDOWN     9  /* msc_solve_nonherm: a BiCGStab denominator vanished */

/* precision of the iteration */
#define MSC_FP64  0  /* every vector, link, block and scalar in FP64 */
#define MSC_MIXED 1  /* FP32 operator and vector updates; FP64 zeta/alpha/beta
                        recurrences, FP64 dot-product accumulation, FP64
                        reliable updates of the base residual and FP64
                        solution accumulation; each shift is then refined to
                        the tolerance with a single-shift mixed solve */
#define MSC_FP32  2  /* msc_op_apply only: the FP32 operator kernel */

/* operator flags */
#define MSC_LINKS_FULL  1u  /* msc_op_staggered: keep all Nc*Nc FP32 link entries
                               (no SU(N) row reconstruction), e.g. for
                               non-unitary links */
#define MSC_CHECK_HERMITIAN 2u /* msc_op_bsr: check on the device at creation
                               that A is Hermitian (CG-M needs A = A^dagger,
                               eq. linprob, Sec. 2); see msc_op_bsr */

typedef struct msc_ctx msc_ctx;
typedef struct msc_op msc_op;

/* Create a context on CUDA device `device`. `cuda_stream` (a cudaStream_t,
 * may be NULL for the legacy default stream) is the stream the caller's own
 * work runs on; the library orders its work after it. */
int msc_create(msc_ctx** ctx, int device, void* cuda_stream);
int msc_destroy(msc_ctx* ctx);
/* Change the caller stream the context orders against. */
int msc_set_stream(msc_ctx* ctx, void* cuda_stream);

/* Staggered operator A = M^dagger M = m^2 - D^2 with
 *   D_xy = 1/2 sum_mu eta_mu(x) [U_mu(x) d_{y,x+mu} - U_mu(x-mu)^dagger d_{y,x-mu}],
 *   eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}), periodic boundaries.
 * nc: 2 or 3. dims[4]: extents, each even and >= 2; site index
 * x0 + L0*(x1 + L1*(x2 + L2*x3)). links: [4][V][nc][nc] complex (FP64),
 * U[mu][site][a][b]. A vector is [V][nc] complex. Unless MSC_LINKS_FULL is
 * given, FP32 links keep nc-1 rows and rebuild the last one from unitarity
 * when every link is in SU(nc) to 1e-9 (checked on the device); otherwise
 * all entries are kept. */
int msc_op_staggered(msc_ctx* ctx, msc_op** op, int nc, const int dims[4],
                     const double* links, double mass, unsigned flags);

/* Generic block-CSR operator: nbr block rows of complex bd x bd blocks
 * (bd = 1, 2 or 3), row_ptr[nbr+1] (int64, non-decreasing, row_ptr[0] = 0),
 * col_idx[nnzb] (int32 in [0, nbr)), vals[nnzb][bd][bd] complex FP64.
 * Repeated block columns in a row add. msc_solve needs A Hermitian
 * positive definite (CG-M, Sec. 2); msc_solve_nonherm takes any A.
 * flags: 0 or MSC_CHECK_HERMITIAN (other bits give MSC_ERR_ARG). With
 * MSC_CHECK_HERMITIAN a device kernel forms every entry A_ij (repeated
 * columns summed) and its partner A_ji and the call fails with
 * MSC_ERR_NOT_HPD, creating nothing, unless
 *     max |A_ij - conj(A_ji)| <= 1e-12 * max |A_ij|
 * over all entries (a block whose transposed partner is not stored counts
 * against a zero partner); its cost is, per stored block, the length of
 * its row and of its column's row. Without the flag Hermiticity is not
 * checked; positivity is never checked here (the solve reports
 * MSC_ERR_NOT_HPD when it meets p^dagger A p <= 0). n = nbr * bd. A block
 * row may hold at most 2^26 / (bd * bd) blocks (about 7.4 million 3 x 3
 * blocks); longer rows, like any other malformed input, give MSC_ERR_ARG. */
int msc_op_bsr(msc_ctx* ctx, msc_op** op, int64_t nbr, int bd, const int64_t* row_ptr,
               const int32_t* col_idx, const double* vals, unsigned flags);

/* Export the staggered operator's A = m^2 - D^2 as block-CSR on the device:
 * nbr = V block rows of nc x nc blocks, 33 blocks per row (the diagonal,
 * the 8 sites two hops along one axis, the 24 sites one hop along each of
 * two axes), row_ptr[i] = 33 i. Columns within a row are ordered by path
 * and repeat on extents <= 4 (repeated columns add). Sizes come from
 * msc_op_bsr_size(). Output buffers may be host or device. */
int msc_op_bsr_size(const msc_op* staggered, int64_t* nbr, int64_t* nnzb, int* bd);
int msc_staggered_export_bsr(msc_ctx* ctx, const msc_op* staggered, int64_t* row_ptr,
                             int32_t* col_idx, double* vals);

/* Number of complex unknowns n of an operator. */
int msc_op_size(const msc_op* op, int64_t* n);

/* recon = 1 when a staggered operator's FP32 links keep nc-1 rows and
 * rebuild the last from unitarity, 0 otherwise (block-CSR: 0). */
int msc_op_recon(const msc_op* op, int* recon);

/* out = (A + sigma) in, with `precision` MSC_FP64 or MSC_FP32 (FP32
 * operator kernel, FP64 in/out). in, out: [n] complex, host or device. */
int msc_op_apply(msc_ctx* ctx, const msc_op* op, double sigma, const double* in,
                 double* out, int precision);

/* out = D in for a staggered operator (FP64). */
int msc_op_dslash(msc_ctx* ctx, const msc_op* op, const double* in, double* out);

/* Free an operator and the solve graphs its context cached for it. Waits for
 * the context's queued work; the context must still exist. */
int msc_op_destroy(msc_op* op);

/* out = (A + sigma) in for a staggered operator, in FP64, without allocating
 * anything. The paper has no counterpart: this serves callers that may not
 * let a library call cudaMalloc at that point, such as code that runs under
 * another framework's memory pool or allocator, or a loop with latency
 * limits where an allocation could block or fail. The intermediate D in and
 * two small pass descriptors live in one fixed device array inside the
 * library (256 bytes + 16 MiB, held on every device that loads the library
 * until the process exits), so n may be at most 2^20 complex unknowns;
 * larger operators get MSC_ERR_ARG, block-CSR operators MSC_ERR_UNSUPPORTED.
 * in and out are device pointers on the operator's device, or managed
 * memory ([n] complex, out may equal in); device memory of another GPU or
 * host memory gives MSC_ERR_ARG before anything is launched. The work is queued on `stream` (a cudaStream_t, NULL
 * for the legacy default stream) and the call returns without waiting;
 * out is ready when the stream reaches that point. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Every call shares the one array and leaves its contents behind (nothing
 * in it needs to start at zero: each call overwrites what it reads), so
 * calls whose work overlaps on the GPU, on any streams, race with each other
 * and must be serialised by the caller. */
int msc_op_apply_noalloc(const msc_op* op, double sigma, const double* in, double* out,
                         void* stream);

typedef struct {
    double tol;          /* relative residual target per shift: |b-(A+s)x_s| <= tol |b| */
    int max_iter;        /* cap on multi-shift iterations (and per refinement round) */
    int precision;       /* MSC_FP64 or MSC_MIXED */
    int reliable_every;  /* MSC_MIXED: FP64 reliable update at the latest after this
                            many iterations since the last one (4x this many in
                            the refinement of a shift) */
    int freeze_converged;/* 1: stop updating a shift once it meets tol (default);
                            0: update every shift until all meet tol */
    int refine;          /* max refinement rounds after the multi-shift solve
                            (0 = none); a round re-solves each shift whose FP64
                            true residual is above tol, warm-started from x_s */
    double reliable_delta;/* MSC_MIXED: FP64 reliable update as soon as the iterated
                            residual norm falls below reliable_delta times its
                            largest value since the last update (0 <= delta < 1;
                            0: only the iteration count triggers it; a tenth of
                            it in the refinement of a shift). Keeps the FP32
                            drift small next to the residual it corrupts. */
} msc_params;

/* Fill defaults: tol 1e-10, max_iter 100000, MSC_MIXED, reliable_every 50,
 * freeze 1, refine 4, reliable_delta 0.01. */
void msc_params_default(msc_params* p);

typedef struct {
    int status;             /* same as the return value of the solve */
    int iters;              /* multi-shift iterations (max over right-hand sides) */
    int refine_rounds;      /* refinement rounds run */
    int refine_iters;       /* refinement iterations (sum over rounds of the
                               max over the systems refined in that round) */
    int reliable_updates;   /* FP64 reliable updates done (all systems, all stages) */
    int refine_reliable_updates; /* of which in the refinement stage */
    int kernel_launches;    /* kernels launched by this solve */
    double seconds;         /* host wall time of the call */
    /* optional caller arrays of nrhs*S entries (index rhs*S + s), or NULL */
    int* shift_iters;       /* iteration at which shift s met tol in the
                               multi-shift stage (-1: never) */
    int* shift_refine_iters;/* refinement iterations spent on shift s */
    double* true_rel_resid; /* final |b - (A+sigma_s) x_s| / |b| in FP64 */
    /* device time per launch, sampled with CUDA events on the solve's
       stream at the first iteration of each launch chunk of the
       multi-shift stage in which every system was still running:
       op_ms      the operator kernel (block-CSR SpMV with the fused P
                  reduction; staggered: first D pass with the fused P terms),
       rupdate_ms the residual kernel (block-CSR: r -= alpha Ap with the
                  fused |r|^2; staggered: second D pass with r -= alpha Ap
                  and |r|^2 fused),
       update_ms  the fused multi-shift update kernel;
       prof_samples the number of samples (0: not measured);
       prof_active  the mean, over the samples, of the number of non-base
                  shifts (summed over right-hand sides) still iterating at
                  the sampled iteration: the sampled update kernel moved
                  r, p (read) and p (write) and the base shift's x (read
                  and write) per right-hand side, and x_s and p_s (read
                  and write) per such shift */
    double op_ms, rupdate_ms, update_ms;
    int prof_samples;
    double prof_active;
} msc_info;

/* Solve (A + sigma_s) x_{r,s} = b_r for every shift s and right-hand side r.
 * b: [nrhs][n] complex; sigma: [S] host array, each >= 0; x: [nrhs][S][n]
 * complex, written for every shift (also on MSC_ERR_NOT_CONVERGED).
 * b and x may be host or device (independently). info may be NULL.
 * A zero b gives x = 0. */
int msc_solve(msc_ctx* ctx, const msc_op* op, const double* b, int nrhs,
              const double* sigma, int S, const msc_params* params, double* x,
              msc_info* info);

/* The shifted family for a source on the sites of one parity (staggered
 * operators): A = m^2 - D^2 couples no even site to an odd one (D hops one
 * site, so D^2 keeps the parity), so for b zero on the sites of parity
 * 1 - p the solution is zero there too and its parity-p part solves
 *     (m^2 - D_{p,1-p} D_{1-p,p} + sigma_s) x_s = b
 * on half the unknowns: every vector pass of the iteration moves half the
 * bytes of msc_solve on the embedded source (the links are still read
 * once per D pass). parity: 0 for even sites ((x0+x1+x2+x3) mod 2 = 0), 1
 * for odd. b: [nrhs][V/2][nc] and x: [nrhs][S][V/2][nc] complex, the
 * parity-p sites in increasing site order (site x at index x / 2). A
 * standard optimisation of staggered solvers, not in the paper. Other
 * arguments, the refinement and errors as in msc_solve; info->true_rel_resid
 * is |b - (A + sigma_s) x_s| / |b| over the parity-p sites (the whole
 * lattice's, since both vanish on the other parity). */
int msc_solve_parity(msc_ctx* ctx, const msc_op* op, int parity, const double* b, int nrhs,
                     const double* sigma, int S, const msc_params* params, double* x,
                     msc_info* info);

/* Different right-hand side per shift (Sec. 5, eq. linprobgen), for
 * right-hand sides of polynomial form in A:
 *     (A + sigma_s) x_s = b_s,   b_s = q_s(A) b,
 *     q_s(t) = sum_{k=0}^{deg} coef[s * (deg + 1) + k] t^k   (real coefficients).
 * The paper points to initial guesses x_s0 that make the shifted residuals
 * collinear, so that one CG-M sequence serves every shift; for this form
 * they follow from dividing q_s(t) by (t + sigma_s):
 *     q_s(t) = q_s(-sigma_s) + (t + sigma_s) s_s(t),   x_s0 = s_s(A) b,
 *     b_s - (A + sigma_s) x_s0 = q_s(-sigma_s) b,
 * so x_s = x_s0 + q_s(-sigma_s) (A + sigma_s)^{-1} b: one CG-M solve on b
 * (each shift stopping at |b - (A+sigma_s) z_s| <= tol |b_s| / |q_s(-sigma_s)|)
 * plus deg - 1 FP64 operator applications per shift for x_s0 and deg for
 * b_s. The FP64 true residual |b_s - (A + sigma_s) x_s| / |b_s| of every
 * shift is then checked and refined to tol exactly as in msc_solve.
 * b: [n] complex (one source); sigma: [S] host, each >= 0; coef: [S][deg+1]
 * host, finite; 0 <= deg <= MSC_MAX_POLY_DEGREE; x: [S][n] complex out. A
 * shift whose b_s is zero gets x_s = 0. info arrays hold S entries;
 * info->true_rel_resid is relative to |b_s|. Other arguments and errors as
 * in msc_solve. */
#define MSC_MAX_POLY_DEGREE 32
int msc_solve_poly_rhs(msc_ctx* ctx, const msc_op* op, const double* b, const double* sigma, int S,
                       const double* coef, int deg, const msc_params* params, double* x,
                       msc_info* info);

/* Non-Hermitian shifted families: (A + sigma_s I) x_{r,s} = b_r for every
 * shift by multi-shift BiCGStab (BiCGStab-M), the solver the paper names for
 * non-Hermitian operators (Sec. 1, Sec. 3; the recurrences are not printed
 * there). One BiCGStab sequence on A + sigma_0 (sigma_0 = the smallest shift,
 * shadow residual b) serves every shift: the BiCG part of each shifted
 * residual follows CG-M's zeta recurrence and the stabilising step becomes
 * omega_s = omega / (1 + (sigma_s - sigma_0) omega), so no shifted system
 * applies A (two operator applications per iteration in all).
 * op: a block-CSR operator from msc_op_bsr (any matrix; Hermiticity is not
 * required); a staggered operator gives MSC_ERR_UNSUPPORTED (the staggered
 * Dirac matrix m + D enters as block-CSR). params: tol, max_iter and
 * freeze_converged are used; precision must be MSC_FP64 (else
 * MSC_ERR_UNSUPPORTED). sigma: [S] host array, any finite values. b, x, info
 * as in msc_solve; info->true_rel_resid holds the FP64 true residual of
 * every x_s, computed after the iteration, and a shift above tol gives
 * MSC_ERR_NOT_CONVERGED. A vanishing denominator gives MSC_ERR_BREAKDOWN (x
 * is then left as it was at the breakdown). */
int msc_solve_nonherm(msc_ctx* ctx, const msc_op* op, const double* b, int nrhs,
                      const double* sigma, int S, const msc_params* params, double* x,
                      msc_info* info);

/* Rational pseudofermion action and its adjoint (the quadratic form that the
 * shifted family diagonalises, Sec. 1-2; sigma_s and c_s come from a rational
 * approximation):  S = sum_s c_s Re(phi^dagger x_s),  x_s = (A + sigma_s)^{-1} phi.
 * msc_quad_form: *value = S for solved x_s. phi: [n] complex; coef: [S]
 * host array of c_s; x: [S][n] complex (e.g. msc_solve's output for one
 * right-hand side). FP64 on the device. */
int msc_quad_form(msc_ctx* ctx, const msc_op* op, const double* phi, int S, const double* coef,
                  const double* x, double* value);

/* Gradients of S, in the convention grad = dS/dRe + i dS/dIm of each complex
 * entry (the one torch.autograd uses for a real loss of complex inputs):
 *   dphi = 2 sum_s c_s x_s                                     ([n] complex)
 *   dU_mu(x) = sum_s c_s eta_mu(x) [x_s(x) y_s(x+mu)^dagger - y_s(x) x_s(x+mu)^dagger],
 *   y_s = D x_s   ([4][V][nc][nc] complex, staggered operators only),
 * treating the link entries as free complex variables (no projection onto
 * SU(N)). Derived from dS = -sum_s c_s x_s^dagger dA x_s with dA = -(dD D + D dD).
 * Either output may be NULL; outputs may be host or device. FP64. */
int msc_quad_form_grad(msc_ctx* ctx, const msc_op* op, int S, const double* coef, const double* x,
                       double* dphi, double* dU);

/* Batched uneven systems: many independent staggered problems, each with
 * its own operator (any lattice, SU(2) or SU(3)), shift list and number of
 * right-hand sides, solved together: every pass of the iteration is one
 * kernel launch for the whole batch (blocks are divided among the systems in
 * proportion to their size), chunks of iterations are CUDA graphs, and each
 * system keeps its own recurrences, convergence and refinement. */
typedef struct {
    const msc_op* op;      /* staggered operator created on the same context */
    const double* b;       /* [nrhs][n] complex, host or device */
    int nrhs;
    const double* sigma;   /* [S] host array, each >= 0 */
    int S;
    double* x;             /* [nrhs][S][n] complex out, host or device */
    msc_info* info;        /* optional report for this problem (arrays nrhs*S) */
} msc_problem;

/* Launch shapes picked by the autotuner for a batch: it times candidate
 * block sizes of the operator pass and block sizes x units per thread of the
 * multi-shift update on the batch itself before the solve, and reuses the
 * winner for later batches of the same shape (same process). */
typedef struct {
    int site_threads;      /* threads per block of the operator passes */
    int vec_threads;       /* threads per block of the vector kernels */
    int vec_units;         /* 16-byte units per thread of the update */
    int tuned;             /* 1: measured for this call, 0: from the cache */
    double best_ms;        /* operator pass + update time of the winner */
} msc_tuning;

/* Solve every problem of the batch. Returns the worst status over the
 * problems (MSC_ERR_NOT_CONVERGED if any shift missed tol); each problem's
 * info holds its own status. `tuning` may be NULL. */
int msc_solve_batched(msc_ctx* ctx, int nprob, const msc_problem* probs, const msc_params* params,
                      msc_tuning* tuning);

const char* msc_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* MSC_H */
