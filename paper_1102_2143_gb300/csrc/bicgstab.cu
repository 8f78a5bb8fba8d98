// BiCGStab-M kernels (see bicgstab.cuh for the recurrences): FP64, generic
// block-CSR operator. One iteration is five kernels: the two operator
// applications with their fused reductions, s = r - alpha v, the seed's
// x and r update with its reductions, and one fused update of every shift's
// x_s and p_s together with the seed's p. The scalar recurrences are run by
// the last block of each reducing kernel, so the host never waits inside an
// iteration.
#include "bicgstab.cuh"
#include "bsr.cuh"

namespace msc {

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ __forceinline__ bool czero(double2 a) { return a.x == 0.0 && a.y == 0.0; }
__device__ __forceinline__ double2 cfrom(double a) { return {a, 0.0}; }
__device__ __forceinline__ double2 caxpy(double2 a, double2 x, double2 y) {  // a x + y
    return {fma(a.x, x.x, fma(-a.y, x.y, y.x)), fma(a.x, x.y, fma(a.y, x.x, y.y))};
}

// Three block sums published to rows row0..row0+2; true in every thread of
// the last block to arrive, with the fixed-order totals.
__device__ bool reduce3_last(const Engine& e, int row0, double a, double b, double c, double (&tot)[3]) {
    __shared__ double sh[32];
    __shared__ int is_last;
    __shared__ double t3[3];
    const double s0 = block_sum(a, sh), s1 = block_sum(b, sh), s2 = block_sum(c, sh);
    if (threadIdx.x == 0) {
        e.partial[(size_t)row0 * kMaxBlocks + blockIdx.x] = s0;
        e.partial[(size_t)(row0 + 1) * kMaxBlocks + blockIdx.x] = s1;
        e.partial[(size_t)(row0 + 2) * kMaxBlocks + blockIdx.x] = s2;
        __threadfence();
        const unsigned k = atomicAdd(&e.counter[row0], 1u);
        is_last = (k == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[q] += __ldcg(&e.partial[(size_t)(row0 + q) * kMaxBlocks + i]);
    const double u0 = block_sum(acc[0], sh), u1 = block_sum(acc[1], sh), u2 = block_sum(acc[2], sh);
    if (threadIdx.x == 0) {
        t3[0] = u0;
        t3[1] = u1;
        t3[2] = u2;
        e.counter[row0] = 0u;
    }
    __syncthreads();
    tot[0] = t3[0];
    tot[1] = t3[1];
    tot[2] = t3[2];
    return true;
}

__device__ __forceinline__ bool running(const BcgSys* s) { return __ldcg(&s->status) == ST_RUNNING; }

// ---------------------------------------------------------------------------
// init: r = b, p = b, x_s = 0, p_s = b; rho = (b, b), bnorm2 = |b|^2
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_bcg_init(Engine e, BcgSys* sys, BcgSlot* slots, BcgVec v, int S) {
    const int base = sys->base;
    double local = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 b = v.rt[i];
        v.r[0][i] = b;
        v.p[i] = b;
        for (int k = 0; k < S; ++k) {
            v.x[(size_t)k * v.npad + i] = {0.0, 0.0};
            if (k != base) v.ps[(size_t)k * v.npad + i] = b;
        }
        local += b.x * b.x + b.y * b.y;
    }
    double tot[3];
    if (!reduce3_last(e, 0, local, 0.0, 0.0, tot)) return;
    const double b2 = tot[0];
    if (threadIdx.x == 0) {
        sys->bnorm2 = b2;
        sys->rnorm2 = b2;
        sys->rho = cfrom(b2);
        if (!isfinite(b2)) sys->status = ST_ERR_NONFINITE;
        else if (b2 == 0.0) sys->status = ST_DONE;
    }
    if (b2 == 0.0)
        for (int k = threadIdx.x; k < S; k += blockDim.x) {
            slots[k].active = 0;
            slots[k].conv_iter = 0;
        }
}

// ---------------------------------------------------------------------------
// K1: v = (A + sigma0) p, (r~, v); alpha = rho / (r~, v)
// K3: t = (A + sigma0) s, (t, s) and (t, t); omega and the shifted scalars
// ---------------------------------------------------------------------------
template <int BD, int STEP>
__global__ void __launch_bounds__(kThreads, 3) k_bcg_op(OpDev A, Engine e, BcgSys* sys, BcgSlot* slots, BcgVec v, int S) {
    if (!running(sys)) return;
    const double2* __restrict__ src = STEP == 1 ? v.p : v.s;
    double2* __restrict__ out = STEP == 1 ? v.v : v.t;
    const double s0 = sys->sigma0;
    double l0 = 0.0, l1 = 0.0, l2 = 0.0;
    const int nbr = (int)A.nbr;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < nbr; row += gridDim.x * blockDim.x) {
        double2 y[BD];
        bsr_row<double, BD>(A, A.vals64, src, row, y);
#pragma unroll
        for (int a = 0; a < BD; ++a) {
            const size_t i = (size_t)row * BD + a;
            const double2 x = src[i];
            const double2 o = {fma(s0, x.x, y[a].x), fma(s0, x.y, y[a].y)};
            out[i] = o;
            if (STEP == 1) {            // conj(r~) v
                const double2 w = v.rt[i];
                l0 += w.x * o.x + w.y * o.y;
                l1 += w.x * o.y - w.y * o.x;
            } else {                    // conj(t) s, |t|^2
                l0 += o.x * x.x + o.y * x.y;
                l1 += o.x * x.y - o.y * x.x;
                l2 += o.x * o.x + o.y * o.y;
            }
        }
    }
    double tot[3];
    if (!reduce3_last(e, 0, l0, l1, l2, tot)) return;
    if (STEP == 1) {
        if (threadIdx.x == 0) {
            const double2 c = {tot[0], tot[1]};
            if (!cfinite(c)) sys->status = ST_ERR_NONFINITE;
            else if (czero(c)) sys->status = ST_ERR_BREAKDOWN;
            else sys->alpha = cdiv(sys->rho, c);
        }
        return;
    }
    // STEP 3: omega and the shifted coefficients of this iteration
    const double2 ts = {tot[0], tot[1]};
    const double tt = tot[2];
    const bool ok = isfinite(tt) && cfinite(ts);
    const double2 omega = ok && tt > 0.0 ? double2{ts.x / tt, ts.y / tt} : double2{0.0, 0.0};
    const double2 alpha = sys->alpha, ap = sys->alpha_prev, bp = sys->beta_prev;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    if (ok && tt > 0.0 && !czero(omega)) {
        for (int k = threadIdx.x; k < S; k += blockDim.x) {
            BcgSlot* q = &slots[k];
            if (!q->active) { q->flag = 0; continue; }
            const double sr = q->sigma_rel;
            const double2 z = q->zeta, zp = q->zeta_prev;
            // den = alpha bp (zp - z) + zp ap (1 + sr alpha)
            const double2 d1 = cmul(cmul(alpha, bp), csub(zp, z));
            const double2 d2 = cmul(cmul(zp, ap), double2{1.0 + sr * alpha.x, sr * alpha.y});
            const double2 den = cadd(d1, d2);
            const double2 opw = {1.0 + sr * omega.x, sr * omega.y};
            if (czero(den) || czero(opw) || czero(z)) { bad = 1; continue; }
            const double2 zn = cdiv(cmul(cmul(z, zp), ap), den);
            const double2 Tn = cmul(q->T, opw);
            q->zeta_new = zn;
            q->T_new = Tn;
            q->a_s = cdiv(cmul(alpha, zn), z);
            q->o_s = cdiv(omega, opw);
            q->cr = cdiv(z, q->T);
            q->cs = cdiv(zn, q->T);
            q->crn = cdiv(zn, Tn);
            if (!cfinite(zn) || !cfinite(Tn) || czero(q->a_s)) bad = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!ok) sys->status = ST_ERR_NONFINITE;
        else if (!(tt > 0.0) || czero(omega) || bad) sys->status = ST_ERR_BREAKDOWN;
        else sys->omega = omega;
    }
}

// K2: s = r - alpha v
__global__ void __launch_bounds__(kThreads) k_bcg_s(BcgSys* sys, BcgVec v, int par) {
    if (!running(sys)) return;
    const double2 na = {-sys->alpha.x, -sys->alpha.y};
    const double2* __restrict__ r = v.r[par];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.n; i += (int64_t)gridDim.x * blockDim.x)
        v.s[i] = caxpy(na, v.v[i], r[i]);
}

// K4: seed x += alpha p + omega s, r' = s - omega t, (r~, r') and |r'|^2;
// beta, the shifted beta_s, convergence, rotation of the recurrences
__global__ void __launch_bounds__(kThreads) k_bcg_r(Engine e, BcgSys* sys, BcgSlot* slots, BcgVec v, int S, int par) {
    if (!running(sys)) return;
    const double2 alpha = sys->alpha, omega = sys->omega;
    const double2 no = {-omega.x, -omega.y};
    double2* __restrict__ xb = v.x + (size_t)sys->base * v.npad;
    double2* __restrict__ rn = v.r[1 - par];
    double l0 = 0.0, l1 = 0.0, l2 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 s = v.s[i];
        xb[i] = caxpy(omega, s, caxpy(alpha, v.p[i], xb[i]));
        const double2 r = caxpy(no, v.t[i], s);
        rn[i] = r;
        const double2 w = v.rt[i];
        l0 += w.x * r.x + w.y * r.y;
        l1 += w.x * r.y - w.y * r.x;
        l2 += r.x * r.x + r.y * r.y;
    }
    double tot[3];
    if (!reduce3_last(e, 0, l0, l1, l2, tot)) return;
    const double2 rho_n = {tot[0], tot[1]};
    const double R = tot[2];
    const double2 beta = cmul(cdiv(rho_n, sys->rho), cdiv(alpha, omega));
    const double thr = sys->tol2 * sys->bnorm2;
    const int it = sys->it, freeze = sys->freeze;
    int all = 1;
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        BcgSlot* q = &slots[k];
        if (!q->active) continue;
        const double2 ratio = cdiv(q->zeta_new, q->zeta);
        q->b_s = cmul(beta, cmul(ratio, ratio));
        const double2 c = q->crn;
        const bool conv = (c.x * c.x + c.y * c.y) * R <= thr;
        if (conv && q->conv_iter < 0) q->conv_iter = it + 1;
        if (conv && freeze) { q->active = 0; q->flag = 1; }
        else q->flag = 2;
        q->zeta_prev = q->zeta;
        q->zeta = q->zeta_new;
        q->T = q->T_new;
        if (q->conv_iter < 0) all = 0;
    }
    all = __syncthreads_and(all);
    if (threadIdx.x == 0) {
        sys->rnorm2 = R;
        sys->beta = beta;
        sys->rho = rho_n;
        sys->alpha_prev = alpha;
        sys->beta_prev = beta;
        sys->it = it + 1;
        if (!isfinite(R) || !cfinite(rho_n)) sys->status = ST_ERR_NONFINITE;
        else if (all) sys->status = ST_FINISHING;
        else if (czero(rho_n)) sys->status = ST_ERR_BREAKDOWN;
        else if (it + 1 >= sys->max_iter) { sys->status = ST_FINISHING; sys->capped = 1; }
    }
}

// K5: every non-base shift still moving: x_s += a_s p_s + o_s cs s and
//   p_s = crn r' + b_s p_s - b_s (o_s/a_s)(cr r - cs s); then p = r' + beta (p - omega v).
__global__ void __launch_bounds__(kThreads) k_bcg_update(Engine e, BcgSys* sys, BcgSlot* slots, BcgVec v, int S,
                                                         int par, unsigned* done_counter) {
    const int st = __ldcg(&sys->status);
    if (st != ST_RUNNING && st != ST_FINISHING) return;
    __shared__ double2 c1[kMaxShifts], c2[kMaxShifts], c3[kMaxShifts], c4[kMaxShifts], c5[kMaxShifts],
        c6[kMaxShifts];
    __shared__ int fl[kMaxShifts];
    const int base = sys->base;
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        const BcgSlot* q = &slots[k];
        fl[k] = k == base ? 0 : q->flag;
        if (fl[k] == 0) continue;
        const double2 g = cdiv(q->o_s, q->a_s);
        const double2 bg = cmul(q->b_s, g);
        c1[k] = q->a_s;
        c2[k] = cmul(q->o_s, q->cs);
        c3[k] = q->crn;
        c4[k] = q->b_s;
        c5[k] = cmul(double2{-bg.x, -bg.y}, q->cr);
        c6[k] = cmul(bg, q->cs);
    }
    __syncthreads();
    const double2 beta = sys->beta, omega = sys->omega;
    const double2 nbo = cmul(double2{-beta.x, -beta.y}, omega);
    const double2* __restrict__ ro = v.r[par];
    const double2* __restrict__ rn = v.r[1 - par];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 r0 = ro[i], r1 = rn[i], s = v.s[i];
        for (int k = 0; k < S; ++k) {
            const int f = fl[k];
            if (f == 0) continue;
            double2* xk = v.x + (size_t)k * v.npad + i;
            double2* pk = v.ps + (size_t)k * v.npad + i;
            const double2 pv = *pk;
            *xk = caxpy(c2[k], s, caxpy(c1[k], pv, *xk));
            if (f == 2) *pk = caxpy(c6[k], s, caxpy(c5[k], r0, caxpy(c4[k], pv, cmul(c3[k], r1))));
        }
        // p = r' + beta p - beta omega v
        v.p[i] = caxpy(nbo, v.v[i], caxpy(beta, v.p[i], r1));
    }
    // the last block retires a finishing system
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done_counter, 1u) == gridDim.x - 1;
        if (last) {
            *done_counter = 0u;
            if (sys->status == ST_FINISHING) sys->status = ST_DONE;
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_bcg_init(const Engine& e, BcgSys* sys, BcgSlot* slots, const BcgVec& v, int S,
                            cudaStream_t st) {
    k_bcg_init<<<resident_grid((const void*)k_bcg_init, v.n), kThreads, 0, st>>>(e, sys, slots, v, S);
    return cudaGetLastError();
}

template <int BD>
static void launch_iter_bd(const OpDev& A, const Engine& e, BcgSys* sys, BcgSlot* slots, const BcgVec& v,
                           int S, int par, cudaStream_t st) {
    auto k1 = k_bcg_op<BD, 1>;
    auto k3 = k_bcg_op<BD, 3>;
    const int g_op = resident_grid((const void*)k1, A.nbr);
    k1<<<g_op, kThreads, 0, st>>>(A, e, sys, slots, v, S);
    k_bcg_s<<<resident_grid((const void*)k_bcg_s, v.n), kThreads, 0, st>>>(sys, v, par);
    k3<<<resident_grid((const void*)k3, A.nbr), kThreads, 0, st>>>(A, e, sys, slots, v, S);
    k_bcg_r<<<resident_grid((const void*)k_bcg_r, v.n), kThreads, 0, st>>>(e, sys, slots, v, S, par);
    // the update's arrival counter sits in the engine's counter row 3
    k_bcg_update<<<resident_grid((const void*)k_bcg_update, v.n), kThreads, 0, st>>>(e, sys, slots, v, S, par,
                                                                                     e.counter + 3);
}

cudaError_t launch_bcg_iter(const OpDev& A, const Engine& e, BcgSys* sys, BcgSlot* slots, const BcgVec& v,
                            int S, int par, cudaStream_t st) {
    switch (A.bd) {
        case 1: launch_iter_bd<1>(A, e, sys, slots, v, S, par, st); break;
        case 2: launch_iter_bd<2>(A, e, sys, slots, v, S, par, st); break;
        default: launch_iter_bd<3>(A, e, sys, slots, v, S, par, st); break;
    }
    return cudaGetLastError();
}

}  // namespace msc
