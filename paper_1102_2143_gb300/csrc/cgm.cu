// Vector kernels of the multi-shift CG iteration (CG-M, Algorithm 1, Sec. 2).
//
// Every update in the iteration is a real scalar times a complex vector, so
// the kernels treat a vector as a flat array of reals and move it in 16-byte
// units (float4 = two complex FP32 values, double2 = one complex FP64 value).
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "engine.h"

namespace msc {

// r = b (in iteration precision), p = r, p_s = r (non-base shifts), x = 0;
// reduction |b|^2 in FP64 from the FP64 source.
template <class T>
__global__ void __launch_bounds__(kThreads) k_init(Engine e, VecSet v, const PassDesc* descs, int nsys) {
    using V = typename U16<T>::t;
    const SysBlock q = sys_block(nsys, nullptr);
    if (!q.ok) return;
    const PassDesc d = descs[q.j];
    const int j = d.sys;
    const SysScalars* s = &e.sys[j];
    const int S = s->S, base = s->base, slot0 = s->slot0, rhs = s->rhs;
    const int64_t upv = v.npad / U16<T>::cpu;
    V* r = (V*)v.r + (size_t)j * upv;
    V* p = (V*)v.p + (size_t)j * upv;
    V* ps = (V*)v.ps;
    V* xit = (V*)v.xit;
    const double2* b = v.b64 + (size_t)rhs * v.npad;
    double local = 0.0;
    const V zero = {};
    for (int64_t i = q.bx * (int64_t)blockDim.x + threadIdx.x; i < upv; i += (int64_t)q.gx * blockDim.x) {
        V rv;
        if constexpr (U16<T>::cpu == 2) {
            double2 b0 = b[2 * i], b1 = b[2 * i + 1];
            local += sq(b0) + sq(b1);
            rv = to_unit(b0, b1);
        } else {
            rv = b[i];
            local += sq(rv);
        }
        r[i] = rv;
        p[i] = rv;
        for (int k = 0; k < S; ++k) {
            const size_t g = (size_t)(slot0 + k) * upv + i;
            if (k != base) ps[g] = rv;
            xit[g] = zero;
        }
        if constexpr (U16<T>::cpu == 2) {
            for (int k = 0; k < S; ++k) {
                const size_t g = (size_t)(slot0 + k) * v.npad + 2 * i;
                v.x64[g] = {0.0, 0.0};
                v.x64[g + 1] = {0.0, 0.0};
            }
        }
    }
    double tot;
    if (reduce_last_n(e, d.row, local, tot, q.gx, q.bx)) finalize(e, d, tot);
}

// p = r, p_s = r, x accumulator of the system's shifts = 0 (start of a solve
// whose residual r was just computed from a warm start).
template <class T>
__global__ void __launch_bounds__(kThreads) k_init_from_r(Engine e, VecSet v, int nsys) {
    using V = typename U16<T>::t;
    const SysBlock q = sys_block(nsys, nullptr);
    if (!q.ok) return;
    const int j = q.j;
    const SysScalars* s = &e.sys[j];
    if (load_status(s) != ST_RUNNING) return;
    const int S = s->S, base = s->base, slot0 = s->slot0;
    const int64_t upv = v.npad / U16<T>::cpu;
    const V* r = (const V*)v.r + (size_t)j * upv;
    V* p = (V*)v.p + (size_t)j * upv;
    V* ps = (V*)v.ps;
    V* xit = (V*)v.xit;
    const V zero = {};
    const bool mixed = (void*)v.xit != (void*)v.x64;
    for (int64_t i = q.bx * (int64_t)blockDim.x + threadIdx.x; i < upv; i += (int64_t)q.gx * blockDim.x) {
        const V rv = r[i];
        p[i] = rv;
        for (int k = 0; k < S; ++k) {
            const size_t g = (size_t)(slot0 + k) * upv + i;
            if (k != base) ps[g] = rv;
            if (mixed) xit[g] = zero;
        }
    }
}

// The fused multi-shift update (Algorithm 1, lines 28-29, plus p): for every
// shift still iterating, x_s += alpha_s p_s and p_s = zeta_s' r + beta_s p_s;
// the base shift's direction is p itself, so only its x moves; then
// p = r + beta p. One read of r and p serves every shift. Each thread keeps
// U units of r and p in registers and issues the loads of one shift for all
// U units before using them, so enough bytes are in flight per SM.
constexpr int kUnits = 4;

template <class T>
__global__ void __launch_bounds__(kThreads, 2) k_update(Engine e, VecSet v, int nsys, const int* act) {
    using V = typename U16<T>::t;
    constexpr int U = kUnits;
    const SysBlock qb = sys_block(nsys, act);
    if (!qb.ok) return;
    const int j = qb.j;
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
    const int64_t upv = v.npad / U16<T>::cpu;
    const V* __restrict__ r = (const V*)v.r + (size_t)j * upv;
    V* __restrict__ p = (V*)v.p + (size_t)j * upv;
    V* __restrict__ ps = (V*)v.ps + (size_t)slot0 * upv;
    V* __restrict__ xs = (V*)v.xit + (size_t)slot0 * upv;
    const int64_t step = (int64_t)qb.gx * blockDim.x;
    for (int64_t i0 = qb.bx * (int64_t)blockDim.x + threadIdx.x; i0 < upv; i0 += step * U) {
        V rv[U], pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * step;
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
                for (int u = 0; u < U; ++u)
                    if (i0 + u * step < upv) xv[u] = xk[i0 + u * step];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (i0 + u * step < upv) xk[i0 + u * step] = axpy(sa[k], pv[u], xv[u]);
                continue;
            }
            V* __restrict__ pks = ps + (size_t)k * upv;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + u * step;
                if (i < upv) {
                    pk[u] = pks[i];
                    xv[u] = xk[i];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + u * step;
                if (i < upv) {
                    xk[i] = axpy(sa[k], pk[u], xv[u]);
                    if (f == 2) pks[i] = axpby(sz[k], rv[u], sb[k], pk[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * step;
            if (i < upv) p[i] = axpy(beta, pv[u], rv[u]);
        }
    }
    if (arrive_last_n(e, j, qb.gx)) {
        if (threadIdx.x == 0 && s->status == ST_FINISHING) s->status = ST_DONE;
    }
}

// Block-CSR path: r -= alpha Ap and R' = |r|^2 (Algorithm 1, lines 20 and 24).
template <class T, bool COND>
__global__ void __launch_bounds__(kThreads) k_axpy_norm(Engine e, VecSet v, const PassDesc* descs, int nsys,
                                                        const int* act) {
    using V = typename U16<T>::t;
    constexpr int U = kUnits;
    const SysBlock sb = sys_block(nsys, act);
    if (!sb.ok) return;
    const PassDesc d = descs[sb.j];
    if (gated_off(e, d)) return;
    const int j = d.sys;
    const T na = -(T)e.sys[j].alpha;
    const int64_t upv = v.npad / U16<T>::cpu;
    V* __restrict__ r = (V*)v.r + (size_t)j * upv;
    const V* __restrict__ ap = (const V*)v.t + (size_t)j * upv;
    double local = 0.0;
    const int64_t step = (int64_t)sb.gx * blockDim.x;
    for (int64_t i0 = sb.bx * (int64_t)blockDim.x + threadIdx.x; i0 < upv; i0 += step * U) {
        V rv[U], av[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * step;
            if (i < upv) {
                rv[u] = r[i];
                av[u] = ap[i];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * step;
            if (i < upv) {
                const V nv = axpy(na, av[u], rv[u]);
                r[i] = nv;
                local += (double)sq(nv);
            }
        }
    }
    double tot;
    if (reduce_last_n(e, d.row, local, tot, sb.gx, sb.bx)) finalize<COND>(e, d, tot);
}

// x_s(FP64) += x_s(FP32 accumulator); accumulator = 0, for every shift of
// the system (mixed precision; runs whatever the system's status).
__global__ void __launch_bounds__(kThreads) k_fold(Engine e, VecSet v, int only_ru, int nsys, const int* act) {
    const SysBlock sb = sys_block(nsys, act);
    if (!sb.ok) return;
    const int j = sb.j;
    const SysScalars* s = &e.sys[j];
    const int st = load_status(s);
    if (st == ST_ERR_NOT_HPD || st == ST_ERR_NONFINITE) return;
    if (only_ru && (st != ST_RUNNING || __ldcg(&s->ru) == 0)) return;
    const int S = s->S, slot0 = s->slot0;
    const int64_t upv = v.npad / 2;
    float4* xa = (float4*)v.xit;
    for (int64_t i = sb.bx * (int64_t)blockDim.x + threadIdx.x; i < upv; i += (int64_t)sb.gx * blockDim.x) {
        for (int k = 0; k < S; ++k) {
            const size_t g = (size_t)(slot0 + k);
            const float4 dx = xa[g * upv + i];
            double2* x = v.x64 + g * v.npad + 2 * i;
            double2 x0 = x[0], x1 = x[1];
            x0.x += dx.x; x0.y += dx.y; x1.x += dx.z; x1.y += dx.w;
            x[0] = x0;
            x[1] = x1;
            xa[g * upv + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

__global__ void k_convert(const void* src, int src_f32, void* dst, int dst_f32, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2 v;
        if (src_f32) { float2 f = ((const float2*)src)[i]; v = {f.x, f.y}; }
        else v = ((const double2*)src)[i];
        if (dst_f32) ((float2*)dst)[i] = make_float2((float)v.x, (float)v.y);
        else ((double2*)dst)[i] = v;
    }
}

int grid_blocks(int64_t work, int num_sms) {
    int64_t b = (work + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms * 8;
    if (cap > kMaxBlocks) cap = kMaxBlocks;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

int resident_grid(const void* fn, int64_t work) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    int cap;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find({fn, dev});
        if (it == cache.end()) {
            int per_sm = 0, sms = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess) {
                cudaGetLastError();
                per_sm = 1;
            }
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cap = std::max(1, per_sm) * std::max(1, sms);
            if (cap > kMaxBlocks) cap = kMaxBlocks;
            cache[{fn, dev}] = cap;
        } else {
            cap = it->second;
        }
    }
    int64_t b = (work + kThreads - 1) / kThreads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

dim3 multi_grid(const void* fn, int64_t work, int nsys, bool per_system) {
    if (per_system && nsys > 1) return dim3(resident_grid(fn, work), nsys);
    // enough blocks for all systems' work, capped at the resident blocks,
    // never fewer than one block per system
    const int64_t total = work * std::max(nsys, 1);
    return dim3(std::max(resident_grid(fn, total), std::max(nsys, 1)));
}

static int64_t upv_of(int prec, const VecSet& v) { return prec == PREC_F32 ? v.npad / 2 : v.npad; }

template <class K>
static dim3 vgrid(K kernel, int64_t upv, int units_per_thread, int nsys, bool per_system = false) {
    return multi_grid((const void*)kernel, (upv + units_per_thread - 1) / units_per_thread, nsys, per_system);
}

cudaError_t launch_init(int prec, const Engine& e, const VecSet& v, const PassDesc* d_descs,
                        int nsys, cudaStream_t st) {
    if (prec == PREC_F32) k_init<float><<<vgrid(k_init<float>, upv_of(prec, v), 1, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys);
    else k_init<double><<<vgrid(k_init<double>, upv_of(prec, v), 1, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys);
    return cudaGetLastError();
}

cudaError_t launch_init_from_r(int prec, const Engine& e, const VecSet& v, int nsys, cudaStream_t st) {
    if (prec == PREC_F32) k_init_from_r<float><<<vgrid(k_init_from_r<float>, upv_of(prec, v), 1, nsys), kThreads, 0, st>>>(e, v, nsys);
    else k_init_from_r<double><<<vgrid(k_init_from_r<double>, upv_of(prec, v), 1, nsys), kThreads, 0, st>>>(e, v, nsys);
    return cudaGetLastError();
}

cudaError_t launch_update(int prec, const Engine& e, const VecSet& v, int nsys, cudaStream_t st, const int* act) {
    if (prec == PREC_F32) k_update<float><<<vgrid(k_update<float>, upv_of(prec, v), kUnits, nsys), kThreads, 0, st>>>(e, v, nsys, act);
    else k_update<double><<<vgrid(k_update<double>, upv_of(prec, v), kUnits, nsys), kThreads, 0, st>>>(e, v, nsys, act);
    return cudaGetLastError();
}

cudaError_t launch_axpy_norm(int prec, const Engine& e, const VecSet& v, const PassDesc* d_descs,
                             int nsys, cudaStream_t st, const int* act) {
    if (prec == PREC_F32) {
        if (e.cond_flag) k_axpy_norm<float, true><<<vgrid(k_axpy_norm<float, true>, upv_of(prec, v), kUnits, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys, act);
        else k_axpy_norm<float, false><<<vgrid(k_axpy_norm<float, false>, upv_of(prec, v), kUnits, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys, act);
    } else {
        if (e.cond_flag) k_axpy_norm<double, true><<<vgrid(k_axpy_norm<double, true>, upv_of(prec, v), kUnits, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys, act);
        else k_axpy_norm<double, false><<<vgrid(k_axpy_norm<double, false>, upv_of(prec, v), kUnits, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys, act);
    }
    return cudaGetLastError();
}

cudaError_t launch_fold(const Engine& e, const VecSet& v, int nsys, int only_ru, cudaStream_t st, const int* act,
                        bool per_system) {
    k_fold<<<vgrid(k_fold, v.npad / 2, 1, nsys, per_system), kThreads, 0, st>>>(e, v, only_ru, nsys, act);
    return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int src_f32, void* dst, int dst_f32, int64_t n,
                           cudaStream_t st) {
    k_convert<<<resident_grid((const void*)k_convert, n), kThreads, 0, st>>>(src, src_f32, dst, dst_f32, n);
    return cudaGetLastError();
}

}  // namespace msc
