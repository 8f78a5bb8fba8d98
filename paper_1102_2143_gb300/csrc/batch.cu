// Batched uneven systems: many independent staggered problems (different
// lattices, SU(2) or SU(3), different shift counts, several right-hand sides)
// advanced together, one kernel launch per pass for the whole batch.
//
// Each system keeps its own FP64 scalars and runs CG-M (Algorithm 1, Sec. 2)
// exactly as in the single-operator engine; only the work distribution
// differs. Blocks are flattened over systems with a prefix-sum map, so a
// 4^4 lattice gets a few blocks and a 12^4 lattice many, and no block idles
// waiting for the largest system: block b serves system j with
// map[j] <= b < map[j+1] and is block b - map[j] of that system's
// map[j+1] - map[j] blocks (which also close its reductions).
#include "stencil.cuh"

namespace msc {

__device__ __forceinline__ int find_system(const int* __restrict__ map, int J, int b) {
    int lo = 0, hi = J;  // map[lo] <= b < map[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(map + mid) <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <class T, int KIND, class TO>
__global__ void __launch_bounds__(kThreads) kb_stag(Engine e, const PassDesc* descs, const BSys* sys,
                                                    const BOp* ops, const int* map, int J) {
    const int j = find_system(map, J, blockIdx.x);
    const int b0 = __ldg(map + j);
    const int nb = __ldg(map + j + 1) - b0, lb = blockIdx.x - b0;
    const PassDesc d = descs[j];
    if (gated_off(e, d)) return;
    const BOp op = ops[sys[j].op];
    const T alpha = KIND == PASS_B ? (T)e.sys[d.sys].alpha : T(0);
    double local = 0.0;
    const int x = lb * blockDim.x + threadIdx.x;
    if (x < op.g.V) {
        if constexpr (sizeof(T) == 4) {
            if (op.nc == 3) {
                if (op.recon) local = stag_site<T, 3, 1, KIND, TO>(d, op.g, op.l32, alpha, x);
                else local = stag_site<T, 3, 0, KIND, TO>(d, op.g, op.l32, alpha, x);
            } else {
                if (op.recon) local = stag_site<T, 2, 1, KIND, TO>(d, op.g, op.l32, alpha, x);
                else local = stag_site<T, 2, 0, KIND, TO>(d, op.g, op.l32, alpha, x);
            }
        } else {
            if (op.nc == 3) local = stag_site<T, 3, 0, KIND, TO>(d, op.g, op.l64, alpha, x);
            else local = stag_site<T, 2, 0, KIND, TO>(d, op.g, op.l64, alpha, x);
        }
    }
    if (d.row >= 0) {
        double tot;
        if (reduce_last_n(e, d.row, local, tot, nb, lb)) finalize(e, d, tot);
    }
}

// r = b, p = r, p_s = r, x = 0 (FP64 x and the iteration-precision accumulator)
template <class T>
__global__ void __launch_bounds__(kThreads) kb_init(Engine e, BVec v, const BSys* sys, const int* map, int J) {
    using V = typename U16<T>::t;
    constexpr int cpu = U16<T>::cpu;
    const int j = find_system(map, J, blockIdx.x);
    const int b0 = __ldg(map + j);
    const int nb = __ldg(map + j + 1) - b0, lb = blockIdx.x - b0;
    const BSys q = sys[j];
    const SysScalars* s = &e.sys[j];
    const int S = s->S, base = s->base;
    const int64_t upv = q.npad / cpu;
    V* r = (V*)v.r + q.voff / cpu;
    V* p = (V*)v.p + q.voff / cpu;
    V* ps = (V*)v.ps + q.soff / cpu;
    V* xit = (V*)v.xit + q.soff / cpu;
    double2* x64 = v.x64 + q.soff;
    const double2* b = v.b64 + q.boff;
    double local = 0.0;
    const int64_t i = (int64_t)lb * blockDim.x + threadIdx.x;
    if (i < upv) {
        V rv;
        if constexpr (cpu == 2) {
            const double2 b0v = b[2 * i], b1v = b[2 * i + 1];
            local = sq(b0v) + sq(b1v);
            rv = to_unit(b0v, b1v);
        } else {
            rv = b[i];
            local = sq(rv);
        }
        r[i] = rv;
        p[i] = rv;
        const V zero = {};
        for (int k = 0; k < S; ++k) {
            if (k != base) ps[(size_t)k * upv + i] = rv;
            xit[(size_t)k * upv + i] = zero;
            if constexpr (cpu == 2) {
                x64[(size_t)k * q.npad + 2 * i] = {0.0, 0.0};
                x64[(size_t)k * q.npad + 2 * i + 1] = {0.0, 0.0};
            }
        }
    }
    PassDesc d{};
    d.sys = j;
    d.row = j;
    d.fin = FIN_INIT;
    double tot;
    if (reduce_last_n(e, j, local, tot, nb, lb)) finalize(e, d, tot);
}

template <class T>
__global__ void __launch_bounds__(kThreads) kb_init_from_r(Engine e, BVec v, const BSys* sys, const int* map,
                                                           int J) {
    using V = typename U16<T>::t;
    constexpr int cpu = U16<T>::cpu;
    const int j = find_system(map, J, blockIdx.x);
    const int lb = blockIdx.x - __ldg(map + j);
    const SysScalars* s = &e.sys[j];
    if (load_status(s) != ST_RUNNING) return;
    const BSys q = sys[j];
    const int S = s->S, base = s->base;
    const int64_t upv = q.npad / cpu;
    const V* r = (const V*)v.r + q.voff / cpu;
    V* p = (V*)v.p + q.voff / cpu;
    V* ps = (V*)v.ps + q.soff / cpu;
    V* xit = (V*)v.xit + q.soff / cpu;
    const bool mixed = (void*)v.xit != (void*)v.x64;
    const int64_t i = (int64_t)lb * blockDim.x + threadIdx.x;
    if (i < upv) {
        const V rv = r[i];
        p[i] = rv;
        const V zero = {};
        for (int k = 0; k < S; ++k) {
            if (k != base) ps[(size_t)k * upv + i] = rv;
            if (mixed) xit[(size_t)k * upv + i] = zero;
        }
    }
}

// the fused multi-shift update (Algorithm 1, lines 28-29), U units per thread
template <class T, int U>
__global__ void __launch_bounds__(kThreads) kb_update(Engine e, BVec v, const BSys* sys, const int* map, int J) {
    using V = typename U16<T>::t;
    constexpr int cpu = U16<T>::cpu;
    const int j = find_system(map, J, blockIdx.x);
    const int b0 = __ldg(map + j);
    const int nb = __ldg(map + j + 1) - b0, lb = blockIdx.x - b0;
    SysScalars* s = &e.sys[j];
    const int st = load_status(s);
    if (st != ST_RUNNING && st != ST_FINISHING) return;
    __shared__ T sa[kMaxShifts], sz[kMaxShifts], sb[kMaxShifts];
    __shared__ int sf[kMaxShifts];
    const int S = s->S, base = s->base, slot0 = s->slot0;
    const T beta = (T)s->beta;
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        const SlotScalars* q = &e.slot[slot0 + k];
        sf[k] = q->flag;
        sa[k] = (T)q->alpha_s;
        sz[k] = (T)q->zeta_new;
        sb[k] = (T)q->beta_s;
    }
    __syncthreads();
    const BSys q = sys[j];
    const int64_t upv = q.npad / cpu;
    const V* __restrict__ r = (const V*)v.r + q.voff / cpu;
    V* __restrict__ p = (V*)v.p + q.voff / cpu;
    V* __restrict__ ps = (V*)v.ps + q.soff / cpu;
    V* __restrict__ xs = (V*)v.xit + q.soff / cpu;
    const int64_t i0 = (int64_t)lb * blockDim.x * U + threadIdx.x;
    V rv[U], pv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        if (i < upv) {
            rv[u] = r[i];
            pv[u] = p[i];
        }
    }
    for (int k = 0; k < S; ++k) {
        const int f = sf[k];
        if (f == 0) continue;
        V* __restrict__ xk = xs + (size_t)k * upv;
        V xv[U], pk[U];
        if (k == base) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + (int64_t)u * blockDim.x;
                if (i < upv) xv[u] = xk[i];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + (int64_t)u * blockDim.x;
                if (i < upv) xk[i] = axpy(sa[k], pv[u], xv[u]);
            }
            continue;
        }
        V* __restrict__ pks = ps + (size_t)k * upv;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            if (i < upv) {
                pk[u] = pks[i];
                xv[u] = xk[i];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            if (i < upv) {
                xk[i] = axpy(sa[k], pk[u], xv[u]);
                if (f == 2) pks[i] = axpby(sz[k], rv[u], sb[k], pk[u]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        if (i < upv) p[i] = axpy(beta, pv[u], rv[u]);
    }
    if (arrive_last_n(e, j, nb)) {
        if (threadIdx.x == 0 && s->status == ST_FINISHING) s->status = ST_DONE;
    }
}

// x_s(FP64) += x_s(FP32 accumulator); accumulator = 0
__global__ void __launch_bounds__(kThreads) kb_fold(Engine e, BVec v, const BSys* sys, const int* map, int J,
                                                    int only_ru) {
    const int j = find_system(map, J, blockIdx.x);
    const int lb = blockIdx.x - __ldg(map + j);
    const SysScalars* s = &e.sys[j];
    const int st = load_status(s);
    if (st == ST_ERR_NOT_HPD || st == ST_ERR_NONFINITE) return;
    if (only_ru && (st != ST_RUNNING || __ldcg(&s->ru) == 0)) return;
    const BSys q = sys[j];
    const int S = s->S;
    const int64_t upv = q.npad / 2;
    float4* xa = (float4*)v.xit + q.soff / 2;
    double2* x64 = v.x64 + q.soff;
    const int64_t i = (int64_t)lb * blockDim.x + threadIdx.x;
    if (i < upv) {
        for (int k = 0; k < S; ++k) {
            const float4 dx = xa[(size_t)k * upv + i];
            double2* x = x64 + (size_t)k * q.npad + 2 * i;
            double2 x0 = x[0], x1 = x[1];
            x0.x += dx.x; x0.y += dx.y; x1.x += dx.z; x1.y += dx.w;
            x[0] = x0;
            x[1] = x1;
            xa[(size_t)k * upv + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

template <class T, int KIND, class TO>
static void launch_bs(const Engine& e, const PassDesc* descs, const BSys* sys, const BOp* ops, const int* map,
                      int J, int nblk, int threads, cudaStream_t st) {
    kb_stag<T, KIND, TO><<<nblk, threads, 0, st>>>(e, descs, sys, ops, map, J);
}

cudaError_t launch_b_stag(int prec, int kind, int out_f32, const Engine& e, const PassDesc* descs,
                          const BSys* sys, const BOp* ops, const int* map, int J, int nblk, int threads,
                          cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (prec == PREC_F64) {
        switch (kind) {
            case PASS_A: launch_bs<double, PASS_A, double>(e, descs, sys, ops, map, J, nblk, threads, st); break;
            case PASS_B: launch_bs<double, PASS_B, double>(e, descs, sys, ops, map, J, nblk, threads, st); break;
            case PASS_C:
                if (out_f32) launch_bs<double, PASS_C, float>(e, descs, sys, ops, map, J, nblk, threads, st);
                else launch_bs<double, PASS_C, double>(e, descs, sys, ops, map, J, nblk, threads, st);
                break;
            default: launch_bs<double, PASS_D, double>(e, descs, sys, ops, map, J, nblk, threads, st); break;
        }
    } else {
        switch (kind) {
            case PASS_A: launch_bs<float, PASS_A, float>(e, descs, sys, ops, map, J, nblk, threads, st); break;
            case PASS_B: launch_bs<float, PASS_B, float>(e, descs, sys, ops, map, J, nblk, threads, st); break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_b_init(int prec, const Engine& e, const BVec& v, const BSys* sys, const int* map,
                          int J, int nblk, int threads, cudaStream_t st) {
    if (prec == PREC_F32) kb_init<float><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
    else kb_init<double><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
    return cudaGetLastError();
}

cudaError_t launch_b_init_from_r(int prec, const Engine& e, const BVec& v, const BSys* sys,
                                 const int* map, int J, int nblk, int threads, cudaStream_t st) {
    if (prec == PREC_F32) kb_init_from_r<float><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
    else kb_init_from_r<double><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
    return cudaGetLastError();
}

cudaError_t launch_b_update(int prec, int units, const Engine& e, const BVec& v, const BSys* sys,
                            const int* map, int J, int nblk, int threads, cudaStream_t st) {
    if (prec == PREC_F32) {
        if (units == 1) kb_update<float, 1><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
        else if (units == 2) kb_update<float, 2><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
        else kb_update<float, 4><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
    } else {
        if (units == 1) kb_update<double, 1><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
        else if (units == 2) kb_update<double, 2><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
        else kb_update<double, 4><<<nblk, threads, 0, st>>>(e, v, sys, map, J);
    }
    return cudaGetLastError();
}

cudaError_t launch_b_fold(const Engine& e, const BVec& v, const BSys* sys, const int* map, int J,
                          int nblk, int threads, int only_ru, cudaStream_t st) {
    kb_fold<<<nblk, threads, 0, st>>>(e, v, sys, map, J, only_ru);
    return cudaGetLastError();
}

}  // namespace msc
