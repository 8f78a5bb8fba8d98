// Shared device-side definitions of the multi-shift CG engine.
//
// The engine runs CG-M (Algorithm 1, Sec. 2) for `nsys` independent systems
// that share one operator. A system has S shifts; its base shift (the
// smallest) is the one the Krylov sequence is built on, so its direction
// vector p_s is p itself and its zeta is exactly 1. Per-shift vectors live in
// global "slots" g = slot0 + s.
//
// Recurrences, textbook convention (alpha = step, beta = direction weight;
// the paper writes beta0 = -alpha and alpha for our beta):
//   alpha = R / P,          P = p^dag (A + sigma0) p
//   zeta_s' = zeta_s zeta_s^- alpha^- /
//             (alpha beta^- (zeta_s^- - zeta_s) + zeta_s^- alpha^- (1 + (sigma_s - sigma0) alpha))
//   alpha_s = alpha zeta_s' / zeta_s,     x_s += alpha_s p_s
//   r -= alpha (A + sigma0) p,  R' = r^dag r,  beta = R'/R
//   beta_s = beta (zeta_s'/zeta_s)^2,     p_s = zeta_s' r + beta_s p_s
//   p = r + beta p
// Shift s has met the tolerance when |zeta_s'| sqrt(R') <= tol |b|.
//
// The per-iteration scalar work (a few flops per shift) is done on the
// device by the last block of the kernel that completes the reduction it
// needs, so the host never waits inside an iteration (Sec. 3: the shift
// constants are computed on the GPU to avoid host round trips).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace msc {

constexpr int kThreads = 256;        // threads per block of every engine kernel
constexpr int kMaxBlocks = 2048;     // partial-sum slots per reduction row
constexpr int kMaxShifts = 128;      // shifts per system

enum : int {
    ST_RUNNING = 0,    // iterate
    ST_FINISHING = 1,  // the current iteration is the last one
    ST_DONE = 2,       // converged or capped
    ST_ERR_NOT_HPD = 4,
    ST_ERR_NONFINITE = 5,
};

// finalize actions of the last block of a reducing kernel
enum : int {
    FIN_NONE = 0,
    FIN_P = 1,        // P known: alpha, zeta', alpha_s
    FIN_R = 2,        // R' known: beta, beta_s, convergence, iteration++
    FIN_SETR = 3,     // R := reduction (reliable update)
    FIN_SETR_INIT = 4,// R := reduction at the start of a solve from a residual
    FIN_INIT = 5,     // R = |b|^2 at the start of a solve from x = 0
    FIN_STORE = 6,    // store the reduction in out_red[row]
};

struct SysScalars {
    double R, P, alpha, alpha_prev, beta, beta_prev;
    double bnorm2;    // |b|^2
    double tol2;      // tol^2
    double d;         // diagonal shift of the operator pass (m^2+sigma0 or sigma0)
    double tol2_acc;  // start-of-solve acceptance: done at once if R <= tol2_acc |b|^2
    double Rmax;      // largest iterated R since the last reliable update
    double delta2;    // reliable update once R <= delta2 * Rmax
    int status, it, max_iter, capped;
    int S, base, slot0, rhs;
    int freeze;
    int ru_every;     // reliable update at the latest after this many iterations (0: never)
    int since_ru;     // iterations since the last reliable update
    int ru;           // 1: the reliable-update kernels of this iteration run
    int nru;          // reliable updates done
    int last_fold;    // iteration count at the last reliable update's fold
};

struct SlotScalars {
    double sigma_rel;                   // sigma_s - sigma0
    double zeta, zeta_prev, zeta_new;
    double alpha_s, beta_s;
    int active;                         // still iterating
    int flag;                           // this iteration: 0 skip, 1 x only, 2 x and p_s
    int conv_iter;                      // iteration at which tol was met (-1)
    int pad;
    double tol2;                        // > 0: this shift's own tol^2 (relative to |b|^2)
                                        //      in place of the system's
};

// One pass of an operator kernel: which vectors, which scalars, which
// reduction. An array of these is indexed by blockIdx.y.
struct PassDesc {
    const void* src;    // vector the operator acts on
    const void* aux;    // vector multiplied by d (p or x); may equal src
    const double2* b;   // right-hand side (residual passes)
    void* out;          // output vector (may be null for residual norms)
    double d;           // diagonal shift
    int sys;            // gating system (-1: always run)
    int row;            // reduction row (-1: no reduction)
    int fin;            // FIN_*
    int gate;           // 0: run while the system iterates; 1: also only when its
                        //    reliable update is due
};

struct Engine {
    SysScalars* sys;
    SlotScalars* slot;
    double* partial;     // [rows][kMaxBlocks]
    unsigned* counter;   // [rows]
    double* out_red;     // [rows]
    // CUDA-graph conditional of this iteration's reliable-update body (0: none)
    // and the flag that lets exactly one system set it
    unsigned long long cond;
    int* cond_flag;
    // error word (bit 0: a bounded wait of a kernel ran out), read by the host
    // after each launch chunk; may be null
    unsigned* err;
};

// ---------------------------------------------------------------------------
// complex helpers (T2 = float2 or double2)
// ---------------------------------------------------------------------------
template <class T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <class T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// conj(a) * b
template <class T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b) {
    return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <class T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return {a.x + b.x, a.y + b.y}; }
template <class T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return {a.x - b.x, a.y - b.y}; }
template <class T2, class T> __device__ __forceinline__ T2 cscale(T s, T2 a) { return {s * a.x, s * a.y}; }
template <class T2> __device__ __forceinline__ T2 cconj(T2 a) { return {a.x, -a.y}; }

// acc += a b, as four fused multiply-adds
template <class T2> __device__ __forceinline__ void cfma(T2& acc, T2 a, T2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc -= conj(a) b, as four fused multiply-adds
template <class T2> __device__ __forceinline__ void cfms_conj(T2& acc, T2 a, T2 b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

__device__ __forceinline__ int load_status(const SysScalars* s) {
    return __ldcg(&s->status);
}

// ---------------------------------------------------------------------------
// block reduction + "last block finalizes" (deterministic: fixed-order sums)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block, valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// Publishes this block's sum of v to row `row`; returns true in every thread
// of the last of the `nblocks` blocks that reduce into that row to arrive
// (`bidx` = this block's index among them), with the fixed-order total.
__device__ __forceinline__ bool reduce_last_n(const Engine& e, int row, double v, double& total,
                                              int nblocks, int bidx) {
    __shared__ double sh[32];
    __shared__ int is_last;
    __shared__ double tot;
    double bs = block_sum(v, sh);
    if (threadIdx.x == 0) {
        e.partial[(size_t)row * kMaxBlocks + bidx] = bs;
        __threadfence();
        unsigned t = atomicAdd(&e.counter[row], 1u);
        is_last = (t == (unsigned)nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x)
        acc += __ldcg(&e.partial[(size_t)row * kMaxBlocks + i]);
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        tot = s;
        e.counter[row] = 0u;
    }
    __syncthreads();
    total = tot;
    return true;
}

__device__ __forceinline__ bool reduce_last(const Engine& e, int row, double v, double& total) {
    return reduce_last_n(e, row, v, total, (int)gridDim.x, (int)blockIdx.x);
}

// Last block only: signals that every block of a non-reducing kernel is done.
__device__ __forceinline__ bool arrive_last_n(const Engine& e, int row, int nblocks) {
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(&e.counter[row], 1u);
        is_last = (t == (unsigned)nblocks - 1);
        if (is_last) e.counter[row] = 0u;
    }
    __syncthreads();
    return is_last != 0;
}

__device__ __forceinline__ bool arrive_last(const Engine& e, int row) {
    return arrive_last_n(e, row, (int)gridDim.x);
}

// ---------------------------------------------------------------------------
// real-scalar vector helpers on 16-byte units
// ---------------------------------------------------------------------------
template <class T> struct U16;
template <> struct U16<float> { using t = float4; static constexpr int cpu = 2; };
template <> struct U16<double> { using t = double2; static constexpr int cpu = 1; };

__device__ __forceinline__ float4 axpy(float a, float4 x, float4 y) {
    return {fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w)};
}
__device__ __forceinline__ double2 axpy(double a, double2 x, double2 y) {
    return {fma(a, x.x, y.x), fma(a, x.y, y.y)};
}
// a*x + b*y
__device__ __forceinline__ float4 axpby(float a, float4 x, float b, float4 y) {
    return {fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y), fmaf(a, x.z, b * y.z), fmaf(a, x.w, b * y.w)};
}
__device__ __forceinline__ double2 axpby(double a, double2 x, double b, double2 y) {
    return {fma(a, x.x, b * y.x), fma(a, x.y, b * y.y)};
}
__device__ __forceinline__ float sq(float4 v) { return v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w; }
__device__ __forceinline__ double sq(double2 v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ float4 to_unit(double2 a, double2 b) {
    return {(float)a.x, (float)a.y, (float)b.x, (float)b.y};
}

// ---------------------------------------------------------------------------
// scalar recurrences, run by the last block (all its threads)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fin_P(const Engine& e, int j, double P) {
    SysScalars* s = &e.sys[j];
    const double R = s->R, ap = s->alpha_prev, bp = s->beta_prev;
    const int S = s->S, slot0 = s->slot0;
    const bool ok = (P > 0.0) && isfinite(P) && isfinite(R);
    const double alpha = R / P;
    __syncthreads();
    if (!ok) {
        if (threadIdx.x == 0) s->status = isfinite(P) && isfinite(R) ? ST_ERR_NOT_HPD : ST_ERR_NONFINITE;
        return;
    }
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        SlotScalars* q = &e.slot[slot0 + k];
        if (!q->active) { q->flag = 0; continue; }
        const double z = q->zeta, zp = q->zeta_prev;
        const double den = alpha * bp * (zp - z) + zp * ap * (1.0 + q->sigma_rel * alpha);
        const double zn = z * zp * ap / den;
        q->zeta_new = zn;
        q->alpha_s = alpha * zn / z;
    }
    if (threadIdx.x == 0) { s->P = P; s->alpha = alpha; }
}

// COND: this kernel runs inside a chunk graph with conditional update nodes
// and sets the iteration's condition (a separate instance, so that kernels
// launched elsewhere contain no graph call and stay profilable).
template <bool COND>
__device__ __forceinline__ void fin_R(const Engine& e, int j, double Rn) {
    SysScalars* s = &e.sys[j];
    const double R = s->R, alpha = s->alpha;
    const double thr = s->tol2 * s->bnorm2;
    const int S = s->S, slot0 = s->slot0, it = s->it, freeze = s->freeze, maxit = s->max_iter;
    const double beta = Rn / R;
    const bool finite = isfinite(Rn);
    int all = 1;
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        SlotScalars* q = &e.slot[slot0 + k];
        if (!q->active) continue;
        const double z = q->zeta, zn = q->zeta_new;
        const double ratio = zn / z;
        q->beta_s = beta * ratio * ratio;
        const double tk = q->tol2 > 0.0 ? q->tol2 * s->bnorm2 : thr;
        const bool conv = (zn * zn * Rn <= tk) || !(fabs(zn) > 1e-290);
        if (conv && q->conv_iter < 0) q->conv_iter = it + 1;
        if (conv && freeze) { q->active = 0; q->flag = 1; }
        else q->flag = 2;
        q->zeta_prev = z;
        q->zeta = zn;
        if (q->conv_iter < 0) all = 0;
    }
    all = __syncthreads_and(all);
    if (threadIdx.x == 0) {
        s->alpha_prev = alpha;
        s->beta_prev = beta;
        s->beta = beta;
        s->R = Rn;
        s->it = it + 1;
        if (!finite) s->status = ST_ERR_NONFINITE;
        else if (all) s->status = ST_FINISHING;
        else if (it + 1 >= maxit) { s->status = ST_FINISHING; s->capped = 1; }
        // reliable update (mixed precision): once the iterated residual has
        // fallen by delta below its largest value since the last update, or
        // after ru_every iterations, so the FP32 drift stays small relative
        // to the residual being iterated
        const double Rmax = fmax(s->Rmax, Rn);
        s->Rmax = Rmax;
        const int since = s->since_ru + 1;
        s->since_ru = since;
        const int ru = (s->ru_every > 0 && s->status == ST_RUNNING &&
                        (Rn <= s->delta2 * Rmax || since >= s->ru_every)) ? 1 : 0;
        s->ru = ru;
        if constexpr (COND) {
            if (ru && e.cond_flag && atomicExch(e.cond_flag, 1) == 0)
                cudaGraphSetConditional((cudaGraphConditionalHandle)e.cond, 1u);
        }
    }
}

// R := reduction. At the start of a solve from a residual, a system that
// already meets the tolerance is done with nothing to iterate.
__device__ __forceinline__ void fin_setR(const Engine& e, int j, double Rv, bool init) {
    SysScalars* s = &e.sys[j];
    const double thr = s->tol2_acc * s->bnorm2;
    const int S = s->S, slot0 = s->slot0;
    __syncthreads();
    if (!isfinite(Rv)) {
        if (threadIdx.x == 0) s->status = ST_ERR_NONFINITE;
        return;
    }
    if (init && Rv <= thr) {
        for (int k = threadIdx.x; k < S; k += blockDim.x) {
            e.slot[slot0 + k].active = 0;
            e.slot[slot0 + k].flag = 0;
            e.slot[slot0 + k].conv_iter = 0;
        }
        if (threadIdx.x == 0) { s->R = Rv; s->status = ST_DONE; }
        return;
    }
    if (threadIdx.x == 0) {
        s->R = Rv;
        s->Rmax = Rv;
        s->since_ru = 0;
        s->ru = 0;
        if (!init) {
            s->nru += 1;
            s->last_fold = s->it;  // the update's fold ran before this residual
        }
    }
}

// A fold of the system's FP32 x accumulators skips slot k when nothing has
// been added to it since the last fold: it stopped iterating (frozen at
// conv_iter, its last x update) no later than that fold.
__device__ __forceinline__ bool fold_skips(const SlotScalars* q, int last_fold) {
    return !q->active && q->conv_iter >= 0 && q->conv_iter <= last_fold;
}

__device__ __forceinline__ void fin_init(const Engine& e, int j, double b2) {
    SysScalars* s = &e.sys[j];
    const int S = s->S, slot0 = s->slot0;
    __syncthreads();
    if (threadIdx.x == 0) {
        s->R = b2;
        s->Rmax = b2;
        s->since_ru = 0;
        s->ru = 0;
        s->bnorm2 = b2;
        if (!isfinite(b2)) s->status = ST_ERR_NONFINITE;
        else if (b2 == 0.0) s->status = ST_DONE;
    }
    if (b2 == 0.0) {
        for (int k = threadIdx.x; k < S; k += blockDim.x) {
            e.slot[slot0 + k].active = 0;
            e.slot[slot0 + k].conv_iter = 0;
        }
    }
}

template <bool COND = false>
__device__ __forceinline__ void finalize(const Engine& e, const PassDesc& d, double total) {
    switch (d.fin) {
        case FIN_P: fin_P(e, d.sys, total); break;
        case FIN_R: fin_R<COND>(e, d.sys, total); break;
        case FIN_SETR: fin_setR(e, d.sys, total, false); break;
        case FIN_SETR_INIT: fin_setR(e, d.sys, total, true); break;
        case FIN_INIT: fin_init(e, d.sys, total); break;
        case FIN_STORE: if (threadIdx.x == 0) e.out_red[d.row] = total; break;
        default: break;
    }
}

// Which system a block serves. Kernels over several systems use a 1-D grid
// whose blocks are dealt round-robin to the systems of the list `act`
// ({count, indices}, in device memory, rewritten by the host between graph
// launches) or to all `nsys` systems when act is null: block b serves system
// act[1 + b % count] as its block b / count of gridDim.x / count. Systems of
// one operator thus run side by side (shared matrix and link tiles are read
// from DRAM once), and as systems finish the same grid spreads over fewer.
struct SysBlock {
    int j;     // system
    int bx;    // block within the system
    int gx;    // blocks of the system
    bool ok;   // false: this block has no work
};

//
// A 2-D grid instead gives every system a whole grid row (blockIdx.y = system):
// used by passes that only some listed systems need (reliable updates, FP64
// checks), where the others' blocks exit at once and the busy ones keep the
// full device.
__device__ __forceinline__ SysBlock sys_block(int nsys, const int* act) {
    SysBlock s;
    if (gridDim.y > 1 || !act) {
        if (gridDim.y > 1) {
            s.j = blockIdx.y;
            s.bx = blockIdx.x;
            s.gx = gridDim.x;
            s.ok = s.j < nsys;
            return s;
        }
    }
    const int na = act ? __ldg(act) : nsys;
    s.ok = na > 0;
    if (!s.ok) { s.j = s.bx = s.gx = 0; return s; }
    const int k = blockIdx.x % na;
    s.bx = blockIdx.x / na;
    s.gx = gridDim.x / na;
    s.ok = s.bx < s.gx;
    s.j = act ? __ldg(act + 1 + k) : k;
    return s;
}

// Gate at kernel entry: true if this pass has nothing to do.
__device__ __forceinline__ bool gated_off(const Engine& e, const PassDesc& d) {
    if (d.sys < 0) return false;
    if (load_status(&e.sys[d.sys]) != ST_RUNNING) return true;
    return d.gate == 1 && __ldcg(&e.sys[d.sys].ru) == 0;
}

}  // namespace msc
