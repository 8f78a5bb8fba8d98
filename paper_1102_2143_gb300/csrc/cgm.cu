// Vector kernels of the multi-shift CG iteration (CG-M, Algorithm 1, Sec. 2).
//
// Every update in the iteration is a real scalar times a complex vector, so
// the kernels treat a vector as a flat array of reals and move it in 16-byte
// units (float4 = two complex FP32 values, double2 = one complex FP64 value).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
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

// k_init for colour-planar FP32 vectors (staggered operators, see VecSet):
// one thread per site and colour plane index, reading the site's FP64 source
// contiguously and writing each FP32 vector's planes coalesced; the pad
// entries [n, npad) of the FP32 vectors are zeroed.
template <int NC>
__global__ void __launch_bounds__(kThreads) k_init_pl(Engine e, VecSet v, const PassDesc* descs, int nsys) {
    const SysBlock q = sys_block(nsys, nullptr);
    if (!q.ok) return;
    const PassDesc d = descs[q.j];
    const int j = d.sys;
    const SysScalars* s = &e.sys[j];
    const int S = s->S, base = s->base, slot0 = s->slot0, rhs = s->rhs;
    const int V = v.pl_V;
    const int64_t npad = v.npad, n = (int64_t)V * NC;
    float2* r = (float2*)v.r + (size_t)j * npad;
    float2* p = (float2*)v.p + (size_t)j * npad;
    float2* ps = (float2*)v.ps;
    float2* xit = (float2*)v.xit;
    const double2* b = v.b64 + (size_t)rhs * npad;
    double local = 0.0;
    const int64_t step = (int64_t)q.gx * blockDim.x;
    for (int64_t x = q.bx * (int64_t)blockDim.x + threadIdx.x; x < V; x += step) {
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const double2 bv = b[x * NC + a];
            local += sq(bv);
            const float2 f = make_float2((float)bv.x, (float)bv.y);
            const size_t i = (size_t)a * V + x;
            r[i] = f;
            p[i] = f;
            for (int k = 0; k < S; ++k) {
                const size_t g = (size_t)(slot0 + k) * npad + i;
                if (k != base) ps[g] = f;
                xit[g] = make_float2(0.f, 0.f);
                v.x64[(size_t)(slot0 + k) * npad + x * NC + a] = {0.0, 0.0};
            }
        }
    }
    for (int64_t i = n + q.bx * (int64_t)blockDim.x + threadIdx.x; i < npad; i += step) {
        r[i] = p[i] = make_float2(0.f, 0.f);
        for (int k = 0; k < S; ++k) {
            const size_t g = (size_t)(slot0 + k) * npad + i;
            ps[g] = xit[g] = make_float2(0.f, 0.f);
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
// the system with something to fold (mixed precision; runs whatever the
// system's status).
__global__ void __launch_bounds__(kThreads) k_fold(Engine e, VecSet v, int only_ru, int nsys, const int* act) {
    const SysBlock sb = sys_block(nsys, act);
    if (!sb.ok) return;
    const int j = sb.j;
    const SysScalars* s = &e.sys[j];
    const int st = load_status(s);
    if (st == ST_ERR_NOT_HPD || st == ST_ERR_NONFINITE) return;
    if (only_ru && (st != ST_RUNNING || __ldcg(&s->ru) == 0)) return;
    const int S = s->S, slot0 = s->slot0, lf = s->last_fold;
    const int64_t upv = v.npad / 2;
    float4* xa = (float4*)v.xit;
    for (int64_t i = sb.bx * (int64_t)blockDim.x + threadIdx.x; i < upv; i += (int64_t)sb.gx * blockDim.x) {
        for (int k = 0; k < S; ++k) {
            if (fold_skips(&e.slot[slot0 + k], lf)) continue;
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

// k_fold for colour-planar FP32 accumulators: one thread per site, the
// site's FP64 entries of each shift read and written contiguously.
template <int NC>
__global__ void __launch_bounds__(kThreads) k_fold_pl(Engine e, VecSet v, int only_ru, int nsys, const int* act) {
    const SysBlock sb = sys_block(nsys, act);
    if (!sb.ok) return;
    const int j = sb.j;
    const SysScalars* s = &e.sys[j];
    const int st = load_status(s);
    if (st == ST_ERR_NOT_HPD || st == ST_ERR_NONFINITE) return;
    if (only_ru && (st != ST_RUNNING || __ldcg(&s->ru) == 0)) return;
    const int S = s->S, slot0 = s->slot0, lf = s->last_fold;
    const int V = v.pl_V;
    float2* xa = (float2*)v.xit;
    for (int64_t x = sb.bx * (int64_t)blockDim.x + threadIdx.x; x < V; x += (int64_t)sb.gx * blockDim.x) {
        for (int k = 0; k < S; ++k) {
            if (fold_skips(&e.slot[slot0 + k], lf)) continue;
            const size_t g = (size_t)(slot0 + k) * v.npad;
            double2* xs = v.x64 + g + x * NC;
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                float2* dp = xa + g + (size_t)a * V + x;
                const float2 dx = *dp;
                double2 xv = xs[a];
                xv.x += dx.x;
                xv.y += dx.y;
                xs[a] = xv;
                *dp = make_float2(0.f, 0.f);
            }
        }
    }
}

__global__ void k_convert_pl(const void* src, void* dst, int nc, int V, int to_planar) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < V; x += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < nc; ++a) {
            const size_t sm = (size_t)x * nc + a, pl = (size_t)a * V + x;
            if (to_planar) {
                const double2 u = ((const double2*)src)[sm];
                ((float2*)dst)[pl] = make_float2((float)u.x, (float)u.y);
            } else {
                const float2 u = ((const float2*)src)[pl];
                ((double2*)dst)[sm] = make_double2(u.x, u.y);
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

// ---------------------------------------------------------------------------
// right-hand sides of polynomial form (FP64, one launch for all shifts):
// blockIdx.y = shift s, vectors [s][npad] site-major
// ---------------------------------------------------------------------------

// v_s = Av_s + a_s b (Av = null: v_s = a_s b), one Horner step of every shift
__global__ void k_poly_step(double2* __restrict__ v, const double2* __restrict__ Av, ShiftCoef a,
                            const double2* __restrict__ b, int64_t n, int64_t npad) {
    const int s = blockIdx.y;
    const double as = a.v[s];
    double2* vs = v + (size_t)s * npad;
    const double2* As = Av ? Av + (size_t)s * npad : nullptr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 bi = b[i];
        double2 o = As ? As[i] : make_double2(0.0, 0.0);
        o.x = fma(as, bi.x, o.x);
        o.y = fma(as, bi.y, o.y);
        vs[i] = o;
    }
}

// x_s = c_s x_s + x0_s (x0 = null: x_s = c_s x_s)
__global__ void k_poly_combine(double2* __restrict__ x, const double2* __restrict__ x0, ShiftCoef c, int64_t n,
                               int64_t npad) {
    const int s = blockIdx.y;
    const double cs = c.v[s];
    double2* xs = x + (size_t)s * npad;
    const double2* x0s = x0 ? x0 + (size_t)s * npad : nullptr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 o = x0s ? x0s[i] : make_double2(0.0, 0.0);
        const double2 xi = xs[i];
        o.x = fma(cs, xi.x, o.x);
        o.y = fma(cs, xi.y, o.y);
        xs[i] = o;
    }
}

// out_red[s] = |v_s|^2 for s < count (reduction rows 0 .. count-1)
__global__ void __launch_bounds__(kThreads) k_norms(Engine e, const double2* __restrict__ v, int64_t n,
                                                     int64_t npad) {
    const int s = blockIdx.y;
    const double2* vs = v + (size_t)s * npad;
    double local = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        local += sq(vs[i]);
    double tot;
    if (reduce_last_n(e, s, local, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0) e.out_red[s] = tot;
}

static dim3 poly_grid(const void* fn, int64_t n, int count) {
    return dim3(std::max(1, resident_grid(fn, n) / std::max(1, count)), count);
}

cudaError_t launch_poly_step(double2* v, const double2* Av, const ShiftCoef& a, const double2* b, int S,
                             int64_t n, int64_t npad, cudaStream_t st) {
    k_poly_step<<<poly_grid((const void*)k_poly_step, n, S), kThreads, 0, st>>>(v, Av, a, b, n, npad);
    return cudaGetLastError();
}

cudaError_t launch_poly_combine(double2* x, const double2* x0, const ShiftCoef& c, int S, int64_t n, int64_t npad,
                                cudaStream_t st) {
    k_poly_combine<<<poly_grid((const void*)k_poly_combine, n, S), kThreads, 0, st>>>(x, x0, c, n, npad);
    return cudaGetLastError();
}

cudaError_t launch_norms(const Engine& e, const double2* v, int count, int64_t n, int64_t npad, cudaStream_t st) {
    k_norms<<<poly_grid((const void*)k_norms, n, count), kThreads, 0, st>>>(e, v, n, npad);
    return cudaGetLastError();
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

int resident_blocks(const void* fn, int threads) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({fn, dev, threads});
    if (it != cache.end()) return it->second;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int cap = std::min(std::max(1, per_sm) * std::max(1, sms), kMaxBlocks);
    cache[{fn, dev, threads}] = cap;
    return cap;
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
    if (prec == PREC_F32 && v.pl_nc == 3) k_init_pl<3><<<multi_grid((const void*)k_init_pl<3>, v.pl_V, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys);
    else if (prec == PREC_F32 && v.pl_nc == 2) k_init_pl<2><<<multi_grid((const void*)k_init_pl<2>, v.pl_V, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys);
    else if (prec == PREC_F32) k_init<float><<<vgrid(k_init<float>, upv_of(prec, v), 1, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys);
    else k_init<double><<<vgrid(k_init<double>, upv_of(prec, v), 1, nsys), kThreads, 0, st>>>(e, v, d_descs, nsys);
    return cudaGetLastError();
}

cudaError_t launch_init_from_r(int prec, const Engine& e, const VecSet& v, int nsys, cudaStream_t st) {
    if (prec == PREC_F32) k_init_from_r<float><<<vgrid(k_init_from_r<float>, upv_of(prec, v), 1, nsys), kThreads, 0, st>>>(e, v, nsys);
    else k_init_from_r<double><<<vgrid(k_init_from_r<double>, upv_of(prec, v), 1, nsys), kThreads, 0, st>>>(e, v, nsys);
    return cudaGetLastError();
}

static int device_sms() {
    static const int n = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return std::max(1, sms);
    }();
    return n;
}

cudaError_t launch_update(int prec, const Engine& e, const VecSet& v, int nsys, cudaStream_t st, const int* act) {
    if (prec == PREC_F32) {
        k_update<float><<<vgrid(k_update<float>, upv_of(prec, v), kUnits, nsys), kThreads, 0, st>>>(e, v, nsys, act);
        return cudaGetLastError();
    }
    // FP64 update of a small system: blocks of fewer threads, so that its
    // FP64 arithmetic spreads over more SMs (as for the FP64 stencil passes)
    const int64_t work = (upv_of(prec, v) + kUnits - 1) / kUnits;
    const int np = std::max(nsys, 1);
    int nt = kThreads;
    while (nt > 32 && ((work + nt - 1) / nt) * np < 2 * device_sms()) nt >>= 1;
    if (nt < kThreads)
        k_update<double><<<(unsigned)(((work + nt - 1) / nt) * np), nt, 0, st>>>(e, v, nsys, act);
    else
        k_update<double><<<vgrid(k_update<double>, upv_of(prec, v), kUnits, nsys), kThreads, 0, st>>>(e, v, nsys, act);
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
    if (v.pl_nc == 3) {
        k_fold_pl<3><<<multi_grid((const void*)k_fold_pl<3>, v.pl_V, nsys, per_system), kThreads, 0, st>>>(e, v, only_ru, nsys, act);
        return cudaGetLastError();
    }
    if (v.pl_nc == 2) {
        k_fold_pl<2><<<multi_grid((const void*)k_fold_pl<2>, v.pl_V, nsys, per_system), kThreads, 0, st>>>(e, v, only_ru, nsys, act);
        return cudaGetLastError();
    }
    k_fold<<<vgrid(k_fold, v.npad / 2, 1, nsys, per_system), kThreads, 0, st>>>(e, v, only_ru, nsys, act);
    return cudaGetLastError();
}

cudaError_t launch_convert_planar(const void* src, void* dst, int nc, int V, bool to_planar, cudaStream_t st) {
    k_convert_pl<<<resident_grid((const void*)k_convert_pl, V), kThreads, 0, st>>>(src, dst, nc, V, to_planar ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int src_f32, void* dst, int dst_f32, int64_t n,
                           cudaStream_t st) {
    k_convert<<<resident_grid((const void*)k_convert, n), kThreads, 0, st>>>(src, src_f32, dst, dst_f32, n);
    return cudaGetLastError();
}

}  // namespace msc
