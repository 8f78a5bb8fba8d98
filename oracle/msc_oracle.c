/*
 * FP64 CPU oracle for the shifted-family solve (A + sigma_i I) x_i = b.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA library is checked against. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it. It shares no code, header
 * or constant with the CUDA library.
 *
 * What it follows:
 *   - the problem, eq. (linprob), Sec. 2: (A + sigma_i I) x_i = b;
 *   - CG-M, Algorithm 1 (Sec. 2), with the Jegerlehner recurrences restated in
 *     the algorithm's own notation (beta0 = step length with the sign that
 *     makes r <- r + beta0*A p a residual update, alpha = direction
 *     coefficient, zeta_{-1}, zeta_0, zeta_1 per shift). The printed listing
 *     is garbled; the readings applied here are:
 *       (1) beta0 = -R0/P (so that r <- r + beta0*Ap and x <- x - beta0*p);
 *       (2) zeta_1 = zeta_0 zeta_{-1} beta_{-1} /
 *                   (beta0 alpha (zeta_{-1} - zeta_0)
 *                    + zeta_{-1} beta_{-1} (1 - sigma beta0)),
 *           with alpha the previous iteration's direction coefficient;
 *       (3) beta_sigma = beta0 zeta_1 / zeta_0;
 *       (4) alpha_sigma = alpha (zeta_1 / zeta_0)^2 with the new alpha;
 *       (5) p_sigma <- zeta_1 r + alpha_sigma p_sigma (the new zeta);
 *       (6) stopping is relative: shift sigma is converged once
 *           |zeta_1| sqrt(R1) <= tol * |b|;
 *       (7) optional freezing of converged shifts (off reproduces the
 *           listing, which keeps updating every shift to the end);
 *       (8) P = Re(p^dagger A p).
 *   - the operator of the synthetic workload: the staggered operator
 *       D_xy = 1/2 sum_mu eta_mu(x) [U_mu(x) delta_{y,x+mu}
 *                                    - U_mu(x-mu)^dagger delta_{y,x-mu}],
 *     eta_mu(x) = (-1)^(x_0+...+x_{mu-1}), periodic boundaries,
 *     M = m + D, A = M^dagger M = m^2 - D^2 (D is anti-Hermitian);
 *   - a generic block-CSR operator (complex bd x bd blocks), the generic
 *     matrix the paper's solver accepts (Sec. 3, Fig. 1).
 *
 *   - BiCGStab-M, the multi-shift BiCGStab the paper names for
 *     non-Hermitian families (Sec. 1, Sec. 3, Sec. 5) but does not print.
 *     Written here in textbook BiCGStab notation (van der Vorst): seed
 *     system A x = b with r~ = b; per iteration v = A p, alpha = rho /
 *     (r~, v), s = r - alpha v, t = A s, omega = (t, s)/(t, t),
 *     x += alpha p + omega s, r = s - omega t, rho' = (r~, r),
 *     beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v).
 *     The BiCG part of the residual polynomial obeys the same three-term
 *     recurrence as CG's, so shifted BiCG residuals are zeta_sigma times the
 *     seed's with the CG-M zeta recurrence; each stabilising factor is
 *     matched by (1 - omega t) = (1 + sigma omega)(1 - omega_sigma (t + sigma)),
 *     omega_sigma = omega / (1 + sigma omega). Then every shifted residual is
 *     (zeta_sigma / T_sigma) r with T_sigma = prod (1 + sigma omega), and
 *     s_sigma = (zeta'_sigma / T_sigma) s; the shifted direction update needs
 *     (A + sigma) p_sigma = (r_sigma - s_sigma) / alpha_sigma, so no shifted
 *     system ever applies A:
 *       zeta'_sigma as in CG-M with the seed's alpha, beta,
 *       alpha_sigma = alpha zeta' / zeta, beta_sigma = beta (zeta'/zeta)^2,
 *       x_sigma += alpha_sigma p_sigma + omega_sigma s_sigma,
 *       p_sigma = r'_sigma + beta_sigma (p_sigma
 *                 - (omega_sigma / alpha_sigma)(r_sigma - s_sigma)).
 *     Shift sigma is converged once |zeta_sigma / T_sigma| |r| <= tol |b|.
 *   - the staggered Dirac operator M = m + D itself, the non-Hermitian
 *     operator of the multi-mass family (M + sigma) x = b.
 *
 * Parity status: every function here is pinned by tests against closed
 * forms, dense solves, textbook CG and finite differences; none is
 * "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Lattice geometry                                                    */
/* ------------------------------------------------------------------ */

static void coords_of(long site, const int L[4], int x[4]) {
    for (int mu = 0; mu < 4; ++mu) {
        x[mu] = (int)(site % L[mu]);
        site /= L[mu];
    }
}

static long site_of(const int x[4], const int L[4]) {
    return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

/* site reached from `site` by one step of `step` (+1 or -1) along mu */
static long hop(long site, int mu, int step, const int L[4]) {
    int x[4];
    coords_of(site, L, x);
    x[mu] = (x[mu] + step + L[mu]) % L[mu];
    return site_of(x, L);
}

/* eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) */
static double eta(long site, int mu, const int L[4]) {
    int x[4];
    coords_of(site, L, x);
    int s = 0;
    for (int nu = 0; nu < mu; ++nu) s += x[nu];
    return (s & 1) ? -1.0 : 1.0;
}

static long vol(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* Staggered operator                                                  */
/* ------------------------------------------------------------------ */

/* U is [4][V][nc][nc]; U_mu(x)_{ab} = U[((mu*V + x)*nc + a)*nc + b] */
static const cplx* link(const cplx* U, int mu, long site, long V, int nc) {
    return U + ((long)mu * V + site) * nc * nc;
}

/* out = D in */
void orc_dslash(int nc, const int L[4], const cplx* U, const cplx* in, cplx* out) {
    long V = vol(L);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        cplx acc[4] = {0, 0, 0, 0};
        for (int mu = 0; mu < 4; ++mu) {
            double e = eta(x, mu, L);
            long xf = hop(x, mu, +1, L);
            long xb = hop(x, mu, -1, L);
            const cplx* Uf = link(U, mu, x, V, nc);   /* U_mu(x)     */
            const cplx* Ub = link(U, mu, xb, V, nc);  /* U_mu(x-mu)  */
            for (int a = 0; a < nc; ++a) {
                cplx fwd = 0, bwd = 0;
                for (int b = 0; b < nc; ++b) {
                    fwd += Uf[a * nc + b] * in[xf * nc + b];
                    bwd += conj(Ub[b * nc + a]) * in[xb * nc + b];
                }
                acc[a] += 0.5 * e * (fwd - bwd);
            }
        }
        for (int a = 0; a < nc; ++a) out[x * nc + a] = acc[a];
    }
}

/* out = (m^2 + sigma) in - D (D in) = (A + sigma) in */
void orc_staggered_apply(int nc, const int L[4], const cplx* U, double mass, double sigma,
                         const cplx* in, cplx* out) {
    long n = vol(L) * nc;
    cplx* t = malloc(sizeof(cplx) * n);
    orc_dslash(nc, L, U, in, t);
    orc_dslash(nc, L, U, t, out);
    double d = mass * mass + sigma;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) out[i] = d * in[i] - out[i];
    free(t);
}

/* ------------------------------------------------------------------ */
/* Generic block-CSR operator                                          */
/* ------------------------------------------------------------------ */

/* out = (A + sigma) in, A given by row_ptr[nbr+1], col_idx[nnzb],
 * vals[nnzb][bd][bd] (row-major blocks). */
void orc_bsr_apply(long nbr, int bd, const int64_t* row_ptr, const int32_t* col_idx,
                   const cplx* vals, double sigma, const cplx* in, cplx* out) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < nbr; ++i) {
        for (int a = 0; a < bd; ++a) {
            cplx acc = sigma * in[i * bd + a];
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                const cplx* blk = vals + k * bd * bd;
                long j = col_idx[k];
                for (int b = 0; b < bd; ++b) acc += blk[a * bd + b] * in[j * bd + b];
            }
            out[i * bd + a] = acc;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Operator handle used by the solvers                                 */
/* ------------------------------------------------------------------ */

typedef struct {
    int kind;               /* 0 staggered, 1 block-CSR */
    int nc;
    int L[4];
    const cplx* U;
    double mass;
    long nbr;
    int bd;
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const cplx* vals;
} orc_op;

static long op_n(const orc_op* op) {
    return op->kind != 1 ? vol(op->L) * op->nc : op->nbr * op->bd;
}

/* out = (m + sigma + D) in: the staggered Dirac operator M = m + D. */
void orc_dirac_apply(int nc, const int L[4], const cplx* U, double mass, double sigma,
                     const cplx* in, cplx* out) {
    long n = vol(L) * nc;
    orc_dslash(nc, L, U, in, out);
    for (long i = 0; i < n; ++i) out[i] += (mass + sigma) * in[i];
}

static void op_apply(const orc_op* op, double sigma, const cplx* in, cplx* out) {
    if (op->kind == 0)
        orc_staggered_apply(op->nc, op->L, op->U, op->mass, sigma, in, out);
    else if (op->kind == 2)
        orc_dirac_apply(op->nc, op->L, op->U, op->mass, sigma, in, out);
    else
        orc_bsr_apply(op->nbr, op->bd, op->row_ptr, op->col_idx, op->vals, sigma, in, out);
}

static cplx dot(long n, const cplx* a, const cplx* b) { /* a^dagger b */
    cplx s = 0;
    for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

static double norm2(long n, const cplx* a) {
    double s = 0;
    for (long i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* ------------------------------------------------------------------ */
/* CG-M (Algorithm 1 with readings (1)-(8))                             */
/* ------------------------------------------------------------------ */

enum { ORC_OK = 0, ORC_NOT_CONVERGED = 6, ORC_NOT_HPD = 4, ORC_NONFINITE = 5, ORC_ARG = 1,
       ORC_BREAKDOWN = 7 };

/*
 * x: [S][n] output. conv_iter[S] (optional): iteration at which each shift
 * met the tolerance (-1 if never). iters: iterations run. zeta_out[S] and
 * r_out[n] (optional): final zeta_0 per shift and final unshifted residual,
 * so that collinearity r_sigma = zeta_sigma r can be checked.
 * tol <= 0 runs exactly max_iter iterations.
 */
static int cgm(const orc_op* op, const cplx* b, int S, const double* sigma, double tol,
               int max_iter, int freeze, cplx* x, int* conv_iter, int* iters,
               double* zeta_out, cplx* r_out) {
    long n = op_n(op);
    if (S <= 0 || max_iter < 0) return ORC_ARG;
    cplx* r = malloc(sizeof(cplx) * n);
    cplx* p = malloc(sizeof(cplx) * n);
    cplx* pbar = malloc(sizeof(cplx) * n);
    cplx* ps = malloc(sizeof(cplx) * n * S);
    double* zm1 = malloc(sizeof(double) * S);   /* zeta_{-1 sigma} */
    double* z0 = malloc(sizeof(double) * S);    /* zeta_{0 sigma}  */
    double* z1 = malloc(sizeof(double) * S);    /* zeta_{1 sigma}  */
    double* bs = malloc(sizeof(double) * S);    /* beta_sigma      */
    double* as = malloc(sizeof(double) * S);    /* alpha_sigma     */
    int* done = calloc(S, sizeof(int));
    int status = ORC_OK;

    /* initialisation, lines 2-14 */
    double alpha = 0.0;
    double beta0 = 1.0, betam1;
    for (int s = 0; s < S; ++s) {
        zm1[s] = 1.0;
        z0[s] = 1.0;
        if (conv_iter) conv_iter[s] = -1;
    }
    memcpy(r, b, sizeof(cplx) * n);
    memcpy(p, b, sizeof(cplx) * n);
    for (int s = 0; s < S; ++s) memcpy(ps + (long)s * n, b, sizeof(cplx) * n);
    memset(x, 0, sizeof(cplx) * n * S);
    double R1 = norm2(n, r);
    double bnorm = sqrt(R1);
    int i = 0;

    if (bnorm == 0.0) { /* b = 0: x = 0 for every shift */
        for (int s = 0; s < S; ++s) if (conv_iter) conv_iter[s] = 0;
        goto out;
    }
    if (tol > 0) {
        int all = 1;
        for (int s = 0; s < S; ++s) {
            if (sqrt(R1) <= tol * bnorm) { done[s] = 1; if (conv_iter) conv_iter[s] = 0; }
            all &= done[s];
        }
        if (all) goto out;
    }

    /* loop, lines 15-32 */
    while (i < max_iter) {
        double R0 = R1;
        betam1 = beta0;
        op_apply(op, 0.0, p, pbar);                     /* pbar = A p      */
        double P = creal(dot(n, p, pbar));              /* P = p^dag A p   */
        if (!(P > 0.0)) { status = isfinite(P) ? ORC_NOT_HPD : ORC_NONFINITE; break; }
        beta0 = -R0 / P;                                /* reading (1)     */
        for (long k = 0; k < n; ++k) r[k] += beta0 * pbar[k];
        for (int s = 0; s < S; ++s) {                   /* reading (2),(3) */
            if (freeze && done[s]) continue;
            double den = beta0 * alpha * (zm1[s] - z0[s])
                       + zm1[s] * betam1 * (1.0 - sigma[s] * beta0);
            z1[s] = z0[s] * zm1[s] * betam1 / den;
            bs[s] = beta0 * z1[s] / z0[s];
        }
        R1 = norm2(n, r);
        alpha = R1 / R0;
        for (int s = 0; s < S; ++s) {                   /* reading (4)     */
            if (freeze && done[s]) continue;
            double q = z1[s] / z0[s];
            as[s] = alpha * q * q;
        }
        for (long k = 0; k < n; ++k) p[k] = r[k] + alpha * p[k];
        for (int s = 0; s < S; ++s) {                   /* lines 28-29     */
            if (freeze && done[s]) continue;
            cplx* xs = x + (long)s * n;
            cplx* pss = ps + (long)s * n;
            for (long k = 0; k < n; ++k) {
                xs[k] -= bs[s] * pss[k];
                pss[k] = z1[s] * r[k] + as[s] * pss[k];  /* reading (5)     */
            }
            zm1[s] = z0[s];
            z0[s] = z1[s];
        }
        ++i;
        if (!isfinite(R1)) { status = ORC_NONFINITE; break; }
        int all = 1;
        for (int s = 0; s < S; ++s) {                   /* reading (6),(7) */
            if (!done[s] && tol > 0 && fabs(z0[s]) * sqrt(R1) <= tol * bnorm) {
                done[s] = 1;
                if (conv_iter) conv_iter[s] = i;
            }
            all &= done[s];
        }
        if (tol > 0 && all) break;
    }
    if (status == ORC_OK && tol > 0) {
        for (int s = 0; s < S; ++s) if (!done[s]) status = ORC_NOT_CONVERGED;
    }
out:
    if (iters) *iters = i;
    if (zeta_out) for (int s = 0; s < S; ++s) zeta_out[s] = z0[s];
    if (r_out) memcpy(r_out, r, sizeof(cplx) * n);
    free(r); free(p); free(pbar); free(ps); free(zm1); free(z0); free(z1);
    free(bs); free(as); free(done);
    return status;
}

/* Textbook CG on (A + sigma) x = b from x = 0 (the unshifted solver the paper
 * times against, Sec. 4, applied to one shifted system). */
static int cg(const orc_op* op, const cplx* b, double sigma, double tol, int max_iter,
              cplx* x, int* iters) {
    long n = op_n(op);
    cplx* r = malloc(sizeof(cplx) * n);
    cplx* p = malloc(sizeof(cplx) * n);
    cplx* q = malloc(sizeof(cplx) * n);
    int status = ORC_OK;
    memset(x, 0, sizeof(cplx) * n);
    memcpy(r, b, sizeof(cplx) * n);
    memcpy(p, b, sizeof(cplx) * n);
    double rr = norm2(n, r), bn = sqrt(rr);
    int i = 0;
    while (i < max_iter && !(tol > 0 && sqrt(rr) <= tol * bn) && bn > 0) {
        op_apply(op, sigma, p, q);
        double pq = creal(dot(n, p, q));
        if (!(pq > 0.0)) { status = isfinite(pq) ? ORC_NOT_HPD : ORC_NONFINITE; break; }
        double a = rr / pq;
        for (long k = 0; k < n; ++k) { x[k] += a * p[k]; r[k] -= a * q[k]; }
        double rr2 = norm2(n, r);
        double be = rr2 / rr;
        for (long k = 0; k < n; ++k) p[k] = r[k] + be * p[k];
        rr = rr2;
        ++i;
    }
    if (status == ORC_OK && tol > 0 && bn > 0 && sqrt(rr) > tol * bn) status = ORC_NOT_CONVERGED;
    if (iters) *iters = i;
    free(r); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------ */
/* BiCGStab-M (see the header for the recurrences)                     */
/* ------------------------------------------------------------------ */

/*
 * Seed: the unshifted A (sigma = 0). x: [S][n] output. conv_iter[S]
 * (optional). c_out[S] (optional, complex): zeta_sigma / T_sigma at exit, and
 * r_out[n] the seed residual, so that b - (A + sigma) x_sigma =
 * c_sigma r can be checked. tol <= 0 runs exactly max_iter iterations.
 */
static int bicgstabm(const orc_op* op, const cplx* b, int S, const double* sigma, double tol,
                     int max_iter, int freeze, cplx* x, int* conv_iter, int* iters,
                     cplx* c_out, cplx* r_out) {
    long n = op_n(op);
    if (S <= 0 || max_iter < 0) return ORC_ARG;
    cplx* r = malloc(sizeof(cplx) * n);
    cplx* rt = malloc(sizeof(cplx) * n);
    cplx* p = malloc(sizeof(cplx) * n);
    cplx* v = malloc(sizeof(cplx) * n);
    cplx* sv = malloc(sizeof(cplx) * n);
    cplx* t = malloc(sizeof(cplx) * n);
    cplx* r_old = malloc(sizeof(cplx) * n);
    cplx* ps = malloc(sizeof(cplx) * n * S);
    cplx* zp = malloc(sizeof(cplx) * S);   /* zeta_{k-1} */
    cplx* z = malloc(sizeof(cplx) * S);    /* zeta_k     */
    cplx* T = malloc(sizeof(cplx) * S);    /* T_k = prod_{j<k} (1 + sigma omega_j) */
    int* done = calloc(S, sizeof(int));
    int status = ORC_OK;
    memcpy(r, b, sizeof(cplx) * n);
    memcpy(rt, b, sizeof(cplx) * n);
    memcpy(p, b, sizeof(cplx) * n);
    for (int s = 0; s < S; ++s) {
        memcpy(ps + (long)s * n, b, sizeof(cplx) * n);
        zp[s] = z[s] = T[s] = 1.0;
        if (conv_iter) conv_iter[s] = -1;
    }
    memset(x, 0, sizeof(cplx) * n * S);
    cplx rho = dot(n, rt, r);
    double bnorm = sqrt(norm2(n, b)), rnorm = bnorm;
    cplx alpha_prev = 1.0, beta_prev = 0.0;
    int i = 0;
    if (bnorm == 0.0) {
        for (int s = 0; s < S; ++s) if (conv_iter) conv_iter[s] = 0;
        goto out;
    }
    while (i < max_iter) {
        op_apply(op, 0.0, p, v);                              /* v = A p          */
        cplx rtv = dot(n, rt, v);
        if (rtv == 0.0 || rho == 0.0) { status = ORC_BREAKDOWN; break; }
        cplx alpha = rho / rtv;
        for (long k = 0; k < n; ++k) sv[k] = r[k] - alpha * v[k];
        op_apply(op, 0.0, sv, t);                             /* t = A s          */
        double tt = norm2(n, t);
        if (tt == 0.0) { status = ORC_BREAKDOWN; break; }
        cplx omega = dot(n, t, sv) / tt;
        if (omega == 0.0) { status = ORC_BREAKDOWN; break; }
        /* shifted updates of x and the coefficients (before r changes) */
        cplx rho_new;
        memcpy(r_old, r, sizeof(cplx) * n);                        /* r_k     */
        for (long k = 0; k < n; ++k) r[k] = sv[k] - omega * t[k];   /* r_{k+1} */
        rho_new = dot(n, rt, r);
        cplx beta = (rho_new / rho) * (alpha / omega);
        for (int s = 0; s < S; ++s) {
            if (freeze && done[s]) continue;
            cplx zn = z[s] * zp[s] * alpha_prev /
                      (alpha * beta_prev * (zp[s] - z[s]) + zp[s] * alpha_prev * (1.0 + sigma[s] * alpha));
            cplx as = alpha * zn / z[s];
            cplx os = omega / (1.0 + sigma[s] * omega);
            cplx Tn = T[s] * (1.0 + sigma[s] * omega);
            cplx cr = z[s] / T[s];      /* r_sigma = cr r_k         */
            cplx cs = zn / T[s];        /* s_sigma = cs s_k         */
            cplx crn = zn / Tn;         /* r'_sigma = crn r_{k+1}   */
            cplx bs = beta * (zn / z[s]) * (zn / z[s]);
            if (!isfinite(creal(zn)) || !isfinite(cimag(zn)) || Tn == 0.0 || as == 0.0) {
                status = ORC_BREAKDOWN;
                break;
            }
            cplx* xs = x + (long)s * n;
            cplx* pss = ps + (long)s * n;
            for (long k = 0; k < n; ++k) {
                cplx s_sig = cs * sv[k];
                cplx r_old_sig = cr * r_old[k];
                xs[k] += as * pss[k] + os * s_sig;
                pss[k] = crn * r[k] + bs * (pss[k] - (os / as) * (r_old_sig - s_sig));
            }
            zp[s] = z[s];
            z[s] = zn;
            T[s] = Tn;
        }
        if (status != ORC_OK) break;
        for (long k = 0; k < n; ++k) p[k] = r[k] + beta * (p[k] - omega * v[k]);
        rho = rho_new;
        alpha_prev = alpha;
        beta_prev = beta;
        ++i;
        rnorm = sqrt(norm2(n, r));
        if (!isfinite(rnorm)) { status = ORC_NONFINITE; break; }
        int all = 1;
        for (int s = 0; s < S; ++s) {
            if (!done[s] && tol > 0 && cabs(z[s] / T[s]) * rnorm <= tol * bnorm) {
                done[s] = 1;
                if (conv_iter) conv_iter[s] = i;
            }
            all &= done[s];
        }
        if (tol > 0 && all) break;
    }
    if (status == ORC_OK && tol > 0) {
        for (int s = 0; s < S; ++s) if (!done[s]) status = ORC_NOT_CONVERGED;
    }
out:
    if (iters) *iters = i;
    if (c_out) for (int s = 0; s < S; ++s) c_out[s] = z[s] / T[s];
    if (r_out) memcpy(r_out, r, sizeof(cplx) * n);
    free(r); free(rt); free(p); free(v); free(sv); free(t); free(r_old); free(ps);
    free(zp); free(z); free(T); free(done);
    return status;
}

/* ------------------------------------------------------------------ */
/* Exported entry points (plain pointers, complex as interleaved pairs) */
/* ------------------------------------------------------------------ */

static orc_op stag_op(int nc, const int L[4], const double* U, double mass) {
    orc_op op;
    memset(&op, 0, sizeof op);
    op.kind = 0;
    op.nc = nc;
    memcpy(op.L, L, sizeof op.L);
    op.U = (const cplx*)U;
    op.mass = mass;
    return op;
}

static orc_op bsr_op(long nbr, int bd, const int64_t* rp, const int32_t* ci, const double* v) {
    orc_op op;
    memset(&op, 0, sizeof op);
    op.kind = 1;
    op.nbr = nbr;
    op.bd = bd;
    op.row_ptr = rp;
    op.col_idx = ci;
    op.vals = (const cplx*)v;
    return op;
}

int orc_cgm_staggered(int nc, const int L[4], const double* U, double mass, const double* b,
                      int S, const double* sigma, double tol, int max_iter, int freeze,
                      double* x, int* conv_iter, int* iters, double* zeta_out, double* r_out) {
    orc_op op = stag_op(nc, L, U, mass);
    return cgm(&op, (const cplx*)b, S, sigma, tol, max_iter, freeze, (cplx*)x, conv_iter, iters,
               zeta_out, (cplx*)r_out);
}

int orc_cgm_bsr(long nbr, int bd, const int64_t* rp, const int32_t* ci, const double* v,
                const double* b, int S, const double* sigma, double tol, int max_iter,
                int freeze, double* x, int* conv_iter, int* iters, double* zeta_out,
                double* r_out) {
    orc_op op = bsr_op(nbr, bd, rp, ci, v);
    return cgm(&op, (const cplx*)b, S, sigma, tol, max_iter, freeze, (cplx*)x, conv_iter, iters,
               zeta_out, (cplx*)r_out);
}

int orc_cg_staggered(int nc, const int L[4], const double* U, double mass, const double* b,
                     double sigma, double tol, int max_iter, double* x, int* iters) {
    orc_op op = stag_op(nc, L, U, mass);
    return cg(&op, (const cplx*)b, sigma, tol, max_iter, (cplx*)x, iters);
}

int orc_cg_bsr(long nbr, int bd, const int64_t* rp, const int32_t* ci, const double* v,
               const double* b, double sigma, double tol, int max_iter, double* x, int* iters) {
    orc_op op = bsr_op(nbr, bd, rp, ci, v);
    return cg(&op, (const cplx*)b, sigma, tol, max_iter, (cplx*)x, iters);
}

int orc_bicgstabm_bsr(long nbr, int bd, const int64_t* rp, const int32_t* ci, const double* v,
                      const double* b, int S, const double* sigma, double tol, int max_iter,
                      int freeze, double* x, int* conv_iter, int* iters, double* c_out,
                      double* r_out) {
    orc_op op = bsr_op(nbr, bd, rp, ci, v);
    return bicgstabm(&op, (const cplx*)b, S, sigma, tol, max_iter, freeze, (cplx*)x, conv_iter,
                     iters, (cplx*)c_out, (cplx*)r_out);
}

int orc_bicgstabm_dirac(int nc, const int L[4], const double* U, double mass, const double* b,
                        int S, const double* sigma, double tol, int max_iter, int freeze,
                        double* x, int* conv_iter, int* iters, double* c_out, double* r_out) {
    orc_op op = stag_op(nc, L, U, mass);
    op.kind = 2;
    return bicgstabm(&op, (const cplx*)b, S, sigma, tol, max_iter, freeze, (cplx*)x, conv_iter,
                     iters, (cplx*)c_out, (cplx*)r_out);
}

void orc_dirac_apply_c(int nc, const int L[4], const double* U, double mass, double sigma,
                       const double* in, double* out) {
    orc_dirac_apply(nc, L, (const cplx*)U, mass, sigma, (const cplx*)in, (cplx*)out);
}

void orc_dslash_c(int nc, const int L[4], const double* U, const double* in, double* out) {
    orc_dslash(nc, L, (const cplx*)U, (const cplx*)in, (cplx*)out);
}

void orc_staggered_apply_c(int nc, const int L[4], const double* U, double mass, double sigma,
                           const double* in, double* out) {
    orc_staggered_apply(nc, L, (const cplx*)U, mass, sigma, (const cplx*)in, (cplx*)out);
}

void orc_bsr_apply_c(long nbr, int bd, const int64_t* rp, const int32_t* ci, const double* v,
                     double sigma, const double* in, double* out) {
    orc_bsr_apply(nbr, bd, rp, ci, (const cplx*)v, sigma, (const cplx*)in, (cplx*)out);
}

/* rho_s = |b - (A + sigma_s) x_s| / |b| for every shift (FP64). */
void orc_true_residual_staggered(int nc, const int L[4], const double* U, double mass,
                                 const double* b, int S, const double* sigma, const double* x,
                                 double* rho) {
    long n = vol(L) * nc;
    cplx* t = malloc(sizeof(cplx) * n);
    const cplx* bb = (const cplx*)b;
    double bn = sqrt(norm2(n, bb));
    for (int s = 0; s < S; ++s) {
        orc_staggered_apply(nc, L, (const cplx*)U, mass, sigma[s], (const cplx*)x + (long)s * n, t);
        double e = 0;
        for (long k = 0; k < n; ++k) {
            cplx d = bb[k] - t[k];
            e += creal(d) * creal(d) + cimag(d) * cimag(d);
        }
        rho[s] = bn > 0 ? sqrt(e) / bn : sqrt(e);
    }
    free(t);
}

/*
 * Link gradient of S = sum_s c_s Re(phi^dagger x_s), x_s = (A + sigma_s)^{-1} phi,
 * with respect to U_mu(x) taken as free complex entries, in the convention
 * grad = dS/dRe U + i dS/dIm U:
 *   G_mu(x) = sum_s c_s eta_mu(x) [ x_s(x) y_s(x+mu)^dagger - y_s(x) x_s(x+mu)^dagger ],
 *   y_s = D x_s.
 * Derivation: dS = -sum_s c_s x_s^dagger dA x_s with dA = -(dD D + D dD);
 * D and dD are anti-Hermitian, so dS = 2 sum_s c_s Re(x_s^dagger dD y_s), and
 * dU_mu(x) enters dD at (x, x+mu) as eta/2 dU and at (x+mu, x) as -eta/2 dU^dagger.
 * x: [S][n]; G: [4][V][nc][nc] complex (overwritten).
 */
void orc_link_force(int nc, const int L[4], const double* U, int S, const double* c,
                    const double* x, double* G) {
    long V = vol(L), n = V * nc;
    cplx* y = malloc(sizeof(cplx) * n);
    cplx* g = (cplx*)G;
    memset(g, 0, sizeof(cplx) * 4 * V * nc * nc);
    for (int s = 0; s < S; ++s) {
        const cplx* xs = (const cplx*)x + (long)s * n;
        orc_dslash(nc, L, (const cplx*)U, xs, y);
        for (int mu = 0; mu < 4; ++mu) {
#pragma omp parallel for schedule(static)
            for (long site = 0; site < V; ++site) {
                long fwd = hop(site, mu, +1, L);
                double w = c[s] * eta(site, mu, L);
                cplx* gm = g + ((long)mu * V + site) * nc * nc;
                for (int a = 0; a < nc; ++a)
                    for (int b2 = 0; b2 < nc; ++b2)
                        gm[a * nc + b2] += w * (xs[site * nc + a] * conj(y[fwd * nc + b2])
                                                - y[site * nc + a] * conj(xs[fwd * nc + b2]));
            }
        }
    }
    free(y);
}
