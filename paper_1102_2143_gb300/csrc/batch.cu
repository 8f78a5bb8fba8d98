// Batched uneven systems: many independent staggered problems (different
// lattices, SU(2) or SU(3), different shift counts, several right-hand sides)
// advanced together, one kernel launch per pass for the whole batch.
//
// Each system keeps its own FP64 scalars and runs CG-M (Algorithm 1, Sec. 2)
// exactly as in the single-operator engine; only the work distribution
// differs. Work is cut into virtual blocks flattened over the systems still
// iterating, with prefix-sum maps in device memory: virtual block b serves
// system act[k] for map[k] <= b < map[k+1] and is block b - map[k] of that
// system's map[k+1] - map[k] blocks (which also close its reductions). A
// fixed grid of resident blocks walks the virtual blocks, so the host can
// shrink the maps between graph launches as systems finish without changing
// the graph. hdr = {active systems, virtual blocks of the site, vector and
// update maps}.
#include <algorithm>

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

struct VBlock {
    int j;   // system
    int lb;  // block within the system
    int nb;  // blocks of the system
};

__device__ __forceinline__ VBlock vblock(const BTab& t, const int* map, int vb) {
    const int J = __ldg(t.hdr);
    const int k = find_system(map, J, vb);
    const int b0 = __ldg(map + k);
    VBlock v;
    v.j = __ldg(t.act + k);
    v.lb = vb - b0;
    v.nb = __ldg(map + k + 1) - b0;
    return v;
}

template <class T, int KIND, class TO>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 1) kb_stag(Engine e, const PassDesc* descs, BTab t) {
    const int total = __ldg(t.hdr + 1);
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const VBlock q = vblock(t, t.msite, vb);
        const PassDesc d = descs[q.j];
        if (gated_off(e, d)) continue;
        const BOp op = t.ops[t.sys[q.j].op];
        const T alpha = (KIND == PASS_B || KIND == PASS_BC) ? (T)e.sys[d.sys].alpha : T(0);
        double local = 0.0;
        const int x = q.lb * blockDim.x + threadIdx.x;
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
            if (reduce_last_n(e, d.row, local, tot, q.nb, q.lb)) finalize<KIND == PASS_BC>(e, d, tot);
        }
    }
}

// r = b, p = r, p_s = r, x = 0 (FP64 x and the iteration-precision accumulator)
template <class T>
__global__ void __launch_bounds__(kThreads) kb_init(Engine e, BVec v, BTab t) {
    using V = typename U16<T>::t;
    constexpr int cpu = U16<T>::cpu;
    const int total = __ldg(t.hdr + 2);
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const VBlock w = vblock(t, t.mvec, vb);
        const int j = w.j;
        const BSys q = t.sys[j];
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
        const int64_t i = (int64_t)w.lb * blockDim.x + threadIdx.x;
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
        if (reduce_last_n(e, j, local, tot, w.nb, w.lb)) finalize(e, d, tot);
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads) kb_init_from_r(Engine e, BVec v, BTab t) {
    using V = typename U16<T>::t;
    constexpr int cpu = U16<T>::cpu;
    const int total = __ldg(t.hdr + 2);
    const bool mixed = (void*)v.xit != (void*)v.x64;
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const VBlock w = vblock(t, t.mvec, vb);
        const int j = w.j;
        const SysScalars* s = &e.sys[j];
        if (load_status(s) != ST_RUNNING) continue;
        const BSys q = t.sys[j];
        const int S = s->S, base = s->base;
        const int64_t upv = q.npad / cpu;
        const V* r = (const V*)v.r + q.voff / cpu;
        V* p = (V*)v.p + q.voff / cpu;
        V* ps = (V*)v.ps + q.soff / cpu;
        V* xit = (V*)v.xit + q.soff / cpu;
        const int64_t i = (int64_t)w.lb * blockDim.x + threadIdx.x;
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
}

// the fused multi-shift update (Algorithm 1, lines 28-29), U units per thread
template <class T, int U>
__global__ void __launch_bounds__(kThreads) kb_update(Engine e, BVec v, BTab t) {
    using V = typename U16<T>::t;
    constexpr int cpu = U16<T>::cpu;
    __shared__ T sa[kMaxShifts], sz[kMaxShifts], sb[kMaxShifts];
    __shared__ int sf[kMaxShifts];
    const int total = __ldg(t.hdr + 3);
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const VBlock w = vblock(t, t.mupd, vb);
        const int j = w.j;
        SysScalars* s = &e.sys[j];
        const int st = load_status(s);
        if (st != ST_RUNNING && st != ST_FINISHING) continue;
        const int S = s->S, base = s->base, slot0 = s->slot0;
        const T beta = (T)s->beta;
        __syncthreads();  // the previous virtual block is done with the coefficients
        for (int k = threadIdx.x; k < S; k += blockDim.x) {
            const SlotScalars* q = &e.slot[slot0 + k];
            sf[k] = q->flag;
            sa[k] = (T)q->alpha_s;
            sz[k] = (T)q->zeta_new;
            sb[k] = (T)q->beta_s;
        }
        __syncthreads();
        const BSys q = t.sys[j];
        const int64_t upv = q.npad / cpu;
        const V* __restrict__ r = (const V*)v.r + q.voff / cpu;
        V* __restrict__ p = (V*)v.p + q.voff / cpu;
        V* __restrict__ ps = (V*)v.ps + q.soff / cpu;
        V* __restrict__ xs = (V*)v.xit + q.soff / cpu;
        const int64_t i0 = (int64_t)w.lb * blockDim.x * U + threadIdx.x;
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
        if (arrive_last_n(e, j, w.nb)) {
            if (threadIdx.x == 0 && s->status == ST_FINISHING) s->status = ST_DONE;
        }
    }
}

// x_s(FP64) += x_s(FP32 accumulator); accumulator = 0
__global__ void __launch_bounds__(kThreads) kb_fold(Engine e, BVec v, BTab t, int only_ru) {
    const int total = __ldg(t.hdr + 2);
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        const VBlock w = vblock(t, t.mvec, vb);
        const int j = w.j;
        const SysScalars* s = &e.sys[j];
        const int st = load_status(s);
        if (st == ST_ERR_NOT_HPD || st == ST_ERR_NONFINITE) continue;
        if (only_ru && (st != ST_RUNNING || __ldcg(&s->ru) == 0)) continue;
        const BSys q = t.sys[j];
        const int S = s->S;
        const int64_t upv = q.npad / 2;
        float4* xa = (float4*)v.xit + q.soff / 2;
        double2* x64 = v.x64 + q.soff;
        const int64_t i = (int64_t)w.lb * blockDim.x + threadIdx.x;
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
}

template <class K> static int fixed_grid(K kernel, int threads) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return std::max(1, per_sm) * std::max(1, sms);
}

template <class T, int KIND, class TO>
static void launch_bs(const Engine& e, const PassDesc* descs, const BTab& t, int threads, cudaStream_t st) {
    auto k = kb_stag<T, KIND, TO>;
    k<<<fixed_grid(k, threads), threads, 0, st>>>(e, descs, t);
}

cudaError_t launch_b_stag(int prec, int kind, int out_f32, const Engine& e, const PassDesc* descs,
                          const BTab& t, int threads, cudaStream_t st) {
    if (prec == PREC_F64) {
        switch (kind) {
            case PASS_A: launch_bs<double, PASS_A, double>(e, descs, t, threads, st); break;
            case PASS_B:
                if (e.cond_flag) launch_bs<double, PASS_BC, double>(e, descs, t, threads, st);
                else launch_bs<double, PASS_B, double>(e, descs, t, threads, st);
                break;
            case PASS_C:
                if (out_f32) launch_bs<double, PASS_C, float>(e, descs, t, threads, st);
                else launch_bs<double, PASS_C, double>(e, descs, t, threads, st);
                break;
            default: launch_bs<double, PASS_D, double>(e, descs, t, threads, st); break;
        }
    } else {
        switch (kind) {
            case PASS_A: launch_bs<float, PASS_A, float>(e, descs, t, threads, st); break;
            case PASS_B:
                if (e.cond_flag) launch_bs<float, PASS_BC, float>(e, descs, t, threads, st);
                else launch_bs<float, PASS_B, float>(e, descs, t, threads, st);
                break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_b_init(int prec, const Engine& e, const BVec& v, const BTab& t, int threads,
                          cudaStream_t st) {
    if (prec == PREC_F32) kb_init<float><<<fixed_grid(kb_init<float>, threads), threads, 0, st>>>(e, v, t);
    else kb_init<double><<<fixed_grid(kb_init<double>, threads), threads, 0, st>>>(e, v, t);
    return cudaGetLastError();
}

cudaError_t launch_b_init_from_r(int prec, const Engine& e, const BVec& v, const BTab& t, int threads,
                                 cudaStream_t st) {
    if (prec == PREC_F32)
        kb_init_from_r<float><<<fixed_grid(kb_init_from_r<float>, threads), threads, 0, st>>>(e, v, t);
    else
        kb_init_from_r<double><<<fixed_grid(kb_init_from_r<double>, threads), threads, 0, st>>>(e, v, t);
    return cudaGetLastError();
}

template <class T, int U>
static void launch_bu(const Engine& e, const BVec& v, const BTab& t, int threads, cudaStream_t st) {
    auto k = kb_update<T, U>;
    k<<<fixed_grid(k, threads), threads, 0, st>>>(e, v, t);
}

cudaError_t launch_b_update(int prec, int units, const Engine& e, const BVec& v, const BTab& t, int threads,
                            cudaStream_t st) {
    if (prec == PREC_F32) {
        if (units == 1) launch_bu<float, 1>(e, v, t, threads, st);
        else if (units == 2) launch_bu<float, 2>(e, v, t, threads, st);
        else launch_bu<float, 4>(e, v, t, threads, st);
    } else {
        if (units == 1) launch_bu<double, 1>(e, v, t, threads, st);
        else if (units == 2) launch_bu<double, 2>(e, v, t, threads, st);
        else launch_bu<double, 4>(e, v, t, threads, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_b_fold(const Engine& e, const BVec& v, const BTab& t, int threads, int only_ru,
                          cudaStream_t st) {
    kb_fold<<<fixed_grid(kb_fold, threads), threads, 0, st>>>(e, v, t, only_ru);
    return cudaGetLastError();
}

}  // namespace msc
