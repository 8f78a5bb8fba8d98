// Generic block-CSR operator (the generic sparse matrix the paper's solver
// takes, Sec. 3 and Fig. 1; A p is Algorithm 1, line 18).
//
// The caller's block-CSR is repacked once into sliced ELL with 32 block rows
// per slice: inside a slice, block k of every row is stored lane-interleaved
// ([slot][component][lane]), so that one thread per row reads its blocks and
// a warp's loads of values and column indices are contiguous 256/128-byte
// runs. Rows shorter than the slice's longest row are padded with zero
// blocks pointing at column 0.
#include <algorithm>

#include "bsr.cuh"

namespace msc {

__global__ void k_bsr_pack(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const double2* __restrict__ vals, int64_t nbr, int bd,
                           const int32_t* __restrict__ slice_len,
                           const int64_t* __restrict__ slice_start, int32_t* __restrict__ pcol,
                           double2* __restrict__ v64, float2* __restrict__ v32, int* bad) {
    const int e2 = bd * bd;
    const int64_t nrow_pad = ((nbr + 31) / 32) * 32;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < nrow_pad;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slice = row >> 5;
        const int lane = (int)(row & 31);
        const int len = slice_len[slice];
        const int64_t st = slice_start[slice];
        const int64_t b0 = row < nbr ? row_ptr[row] : 0;
        const int64_t rl = row < nbr ? row_ptr[row + 1] - b0 : 0;
        for (int k = 0; k < len; ++k) {
            const int64_t slot = st + k;
            int c = 0;
            if (k < rl) {
                c = col[b0 + k];
                if (c < 0 || (int64_t)c >= nbr) { atomicExch(bad, 1); c = 0; }
            }
            pcol[slot * 32 + lane] = c;
            for (int q = 0; q < e2; ++q) {
                double2 v = {0.0, 0.0};
                if (k < rl) v = vals[(b0 + k) * e2 + q];
                v64[(slot * e2 + q) * 32 + lane] = v;
                v32[(slot * e2 + q) * 32 + lane] = make_float2((float)v.x, (float)v.y);
            }
        }
    }
}

// Hermiticity of a block-CSR matrix (repeated columns add): one thread per
// stored block k = (i, j); for the first block of column j in row i it forms
// S_ij = sum of row i's blocks in column j and S_ji from row j, and records
// max |S_ij[a][b] - conj(S_ji[b][a])| in out[0] and max |S_ij[a][b]| in
// out[1] (non-negative doubles, compared as their bit patterns; a NaN or
// Inf entry records the largest finite double as the difference). Work per
// block is the length of its two rows.
__global__ void k_bsr_herm(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const double2* __restrict__ vals, int64_t nbr, int bd,
                           unsigned long long* __restrict__ out) {
    const int64_t nnzb = row_ptr[nbr];
    double dmax = 0.0, amax = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnzb;
         k += (int64_t)gridDim.x * blockDim.x) {
        // row i of block k: the last row whose start is <= k
        int64_t lo = 0, hi = nbr - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (row_ptr[mid] <= k) lo = mid; else hi = mid - 1;
        }
        const int64_t i = lo;
        const int j = col[k];
        bool first = true;
        for (int64_t q = row_ptr[i]; q < k; ++q)
            if (col[q] == j) { first = false; break; }
        if (!first) continue;
        double2 sij[9], sji[9];
        for (int e = 0; e < bd * bd; ++e) sij[e] = sji[e] = {0.0, 0.0};
        for (int64_t q = k; q < row_ptr[i + 1]; ++q)
            if (col[q] == j)
                for (int e = 0; e < bd * bd; ++e) sij[e] = cadd(sij[e], vals[q * bd * bd + e]);
        for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q)
            if (col[q] == (int)i)
                for (int e = 0; e < bd * bd; ++e) sji[e] = cadd(sji[e], vals[q * bd * bd + e]);
        for (int a = 0; a < bd; ++a)
            for (int b = 0; b < bd; ++b) {
                const double2 u = sij[a * bd + b], v = sji[b * bd + a];
                const double d = fmax(fabs(u.x - v.x), fabs(u.y + v.y));
                const double m = fmax(fabs(u.x), fabs(u.y));
                dmax = (d == d && d <= 1.7e308) ? fmax(dmax, d) : 1.7e308;
                amax = (m == m && m <= 1.7e308) ? fmax(amax, m) : amax;
            }
    }
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(dmax));
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(amax));
}

cudaError_t bsr_check_hermitian(const int64_t* d_row_ptr, const int32_t* d_col, const double2* d_vals,
                                int64_t nbr, int bd, unsigned long long* d_out, cudaStream_t st) {
    k_bsr_herm<<<resident_grid((const void*)k_bsr_herm, std::max<int64_t>(nbr * 8, 1)), kThreads, 0, st>>>(
        d_row_ptr, d_col, d_vals, nbr, bd, d_out);
    return cudaGetLastError();
}

cudaError_t bsr_pack(OpDev& op, const int64_t* d_row_ptr, const int32_t* d_col,
                     const double2* d_vals, int* d_bad, cudaStream_t st) {
    int64_t rows = op.nslices * 32;
    int64_t b = (rows + 255) / 256;
    if (b > 65535) b = 65535;
    if (b < 1) b = 1;
    k_bsr_pack<<<(int)b, 256, 0, st>>>(d_row_ptr, d_col, d_vals, op.nbr, op.bd, op.slice_len,
                                        op.slice_start, op.cols, op.vals64, op.vals32, d_bad);
    return cudaGetLastError();
}

// FP32: four 256-thread blocks per SM at up to 64 registers (at five blocks
// the 48-register cap spills and the 24^4 SpMV takes 160 us instead of
// 150 us); FP64: three blocks at most 80 registers each: no spills, enough
// warps for the FP64 pipe.
template <class T, int BD, int KIND, class TO>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 4 : 3)
k_bsr(Engine e, const PassDesc* descs, int npass, const int* act, OpDev A, const T2<T>* __restrict__ vals) {
    const SysBlock q = sys_block(npass, act);
    if (!q.ok) return;
    const PassDesc d = descs[q.j];
    if (gated_off(e, d)) return;
    const T2<T>* __restrict__ src = (const T2<T>*)d.src;
    const T2<T>* __restrict__ aux = (const T2<T>*)d.aux;
    const T dd = (T)d.d;
    double local = 0.0;
    const int nbr = (int)A.nbr;
    for (int row = q.bx * blockDim.x + threadIdx.x; row < nbr; row += q.gx * blockDim.x) {
        T2<T> y[BD];
        bsr_row<T, BD>(A, vals, src, row, y);
        if (KIND == PASS_A) {  // out = (A + d) src, P term = Re src^dag out
            T2<T>* out = (T2<T>*)d.out;
            T loc = T(0);
#pragma unroll
            for (int a = 0; a < BD; ++a) {
                const T2<T> s = src[(size_t)row * BD + a];
                const T2<T> v = {y[a].x + dd * s.x, y[a].y + dd * s.y};
                out[(size_t)row * BD + a] = v;
                loc += s.x * v.x + s.y * v.y;
            }
            local += (double)loc;
        } else if (KIND == PASS_C) {  // out = b - (A + d) aux, |out|^2
            TO* out = (TO*)d.out;
#pragma unroll
            for (int a = 0; a < BD; ++a) {
                const T2<T> xa = aux[(size_t)row * BD + a];
                const double2 ba = d.b[(size_t)row * BD + a];
                const double vx = ba.x - ((double)y[a].x + (double)dd * xa.x);
                const double vy = ba.y - ((double)y[a].y + (double)dd * xa.y);
                if (out) {
                    out[2 * ((size_t)row * BD + a)] = (TO)vx;
                    out[2 * ((size_t)row * BD + a) + 1] = (TO)vy;
                }
                local += vx * vx + vy * vy;
            }
        } else {  // PASS_D: out = (A + d) aux
            T2<T>* out = (T2<T>*)d.out;
#pragma unroll
            for (int a = 0; a < BD; ++a) {
                const T2<T> xa = aux[(size_t)row * BD + a];
                out[(size_t)row * BD + a] = {y[a].x + dd * xa.x, y[a].y + dd * xa.y};
            }
        }
    }
    if (d.row >= 0) {
        double tot;
        if (reduce_last_n(e, d.row, local, tot, q.gx, q.bx)) finalize(e, d, tot);
    }
}

// Block shape of the FP32 SpMVs k_bsr_a1 and k_bsr_multi: 288 threads, four
// blocks per SM (36 warps, at most 56 registers). A thread takes rows
// blockDim.x * gridDim.x (per group of systems) apart, so the rows per
// thread are nbr / (36 x 32 x SMs) per group: 1.9 on the 24^4 matrix for
// one group, 3.8 for two, where 256 x 5 (40 warps) gives 1.7 and 3.4 and the
// last rows run on a part of the warps (24^4 solve: one-system SpMV 146.7 us
// against 152.4 us live, 224 x 5 and 192 x 6: 146.8 / 147.2 us, 256 x 4:
// 159.3 us; with the shared-matrix SpMV at this shape as well, the solve
// takes 242.6 against 244.7 ms, and that kernel no longer spills).
constexpr int kSpmvThreads = 288, kSpmvBlocks = 4;

// y_j = (A + d_j) src_j for up to G systems j sharing the matrix: each block
// value and column index is read once per thread and applied to every system
// of its group (the refinement stage and several right-hand sides). Epilogue
// as PASS_A, with one P reduction per system.
// Groups are interleaved in blockIdx.x, so the blocks of every group for the
// same rows run together: each matrix tile comes from DRAM once and from L2
// for the other groups. Two systems per thread is the measured optimum on
// the 24^4 staggered pattern (14 systems: 0.45 ms at G = 2, 1.0 ms at G = 8,
// where the 8 accumulators cost occupancy while the L2 source gathers, not
// the matrix stream, bound the kernel).
// `act` (optional): the passes still to run, act[0] = their count and
// act[1..] their indices, so that groups stay full as systems finish.
template <class T, int BD, int G>
__global__ void __launch_bounds__(kSpmvThreads, kSpmvBlocks)
k_bsr_multi(Engine e, const PassDesc* descs, int npass, const int* act, int groups, OpDev A,
            const T2<T>* __restrict__ vals) {
    __shared__ PassDesc sd[G];
    __shared__ unsigned s_mask;
    if (threadIdx.x == 0) s_mask = 0u;
    __syncthreads();
    const int grp = blockIdx.x % groups, bx = blockIdx.x / groups, gx = gridDim.x / groups;
    if (threadIdx.x < G) {
        const int na = act ? __ldg(act) : npass;
        const int j = grp * G + threadIdx.x;
        if (j < na) {
            sd[threadIdx.x] = descs[act ? __ldg(act + 1 + j) : j];
            if (!gated_off(e, sd[threadIdx.x])) atomicOr(&s_mask, 1u << threadIdx.x);
        }
    }
    __syncthreads();
    const unsigned mask = s_mask;
    if (!mask) return;
    const T2<T>* srcs[G];
#pragma unroll
    for (int g = 0; g < G; ++g) srcs[g] = ((mask >> g) & 1u) ? (const T2<T>*)sd[g].src : nullptr;
    double local[G];
#pragma unroll
    for (int g = 0; g < G; ++g) local[g] = 0.0;
    const int nbr = (int)A.nbr;
    for (int row = bx * blockDim.x + threadIdx.x; row < nbr; row += gx * blockDim.x) {
        const int slice = row >> 5;
        const int lane = row & 31;
        const int len = __ldg(&A.slice_len[slice]);
        const int64_t st = __ldg(&A.slice_start[slice]);
        T2<T> acc[G][BD];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int a = 0; a < BD; ++a) acc[g][a] = {T(0), T(0)};
        const int32_t* __restrict__ cp = A.cols + st * 32 + lane;
        const T2<T>* __restrict__ vp = vals + st * BD * BD * 32 + lane;
#pragma unroll 3
        for (int k = 0; k < len; ++k) {
            const int c = __ldg(cp + k * 32);
            const T2<T>* vk = vp + k * (BD * BD * 32);
            T2<T> v[BD][BD];
#pragma unroll
            for (int a = 0; a < BD; ++a)
#pragma unroll
                for (int b = 0; b < BD; ++b) v[a][b] = __ldg(vk + (a * BD + b) * 32);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (!srcs[g]) continue;
                T2<T> xv[BD];
#pragma unroll
                for (int b = 0; b < BD; ++b) xv[b] = __ldg(srcs[g] + (size_t)c * BD + b);
#pragma unroll
                for (int a = 0; a < BD; ++a)
#pragma unroll
                    for (int b = 0; b < BD; ++b) cfma(acc[g][a], v[a][b], xv[b]);
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (!srcs[g]) continue;
            T2<T>* out = (T2<T>*)sd[g].out;
            const T dd = (T)sd[g].d;
            T loc = T(0);
#pragma unroll
            for (int a = 0; a < BD; ++a) {
                const T2<T> s = __ldg(srcs[g] + (size_t)row * BD + a);
                const T2<T> y = {acc[g][a].x + dd * s.x, acc[g][a].y + dd * s.y};
                out[(size_t)row * BD + a] = y;
                loc += s.x * y.x + s.y * y.y;
            }
            local[g] += (double)loc;
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (!srcs[g] || sd[g].row < 0) continue;
        double tot;
        if (reduce_last_n(e, sd[g].row, local[g], tot, gx, bx)) finalize(e, sd[g], tot);
    }
}

// The FP32 PASS_A of a single system with its source and output passed as
// kernel parameters (the descriptor still gives the shift, gating and
// reduction): the addresses come from the constant bank instead of
// registers, which leaves the row loop the registers for its loads in
// flight (24^4, at 256 x 5: 142 us against 150 us with the pointers read
// from the descriptor).
template <int BD>
__global__ void __launch_bounds__(kSpmvThreads, kSpmvBlocks)
k_bsr_a1(Engine e, const PassDesc* descs, OpDev A, const float2* __restrict__ vals,
         const float2* __restrict__ src, float2* __restrict__ out) {
    const PassDesc d = descs[0];
    if (gated_off(e, d)) return;
    const float dd = (float)d.d;
    const int nbr = (int)A.nbr;
    double local = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < nbr; row += gridDim.x * blockDim.x) {
        const int slice = row >> 5, lane = row & 31;
        const int len = __ldg(&A.slice_len[slice]);
        const int64_t st = __ldg(&A.slice_start[slice]);
        float2 y[BD];
#pragma unroll
        for (int a = 0; a < BD; ++a) y[a] = {0.f, 0.f};
        const int32_t* __restrict__ cp = A.cols + st * 32 + lane;
        const float2* __restrict__ vp = vals + st * BD * BD * 32 + lane;
#pragma unroll 3
        for (int k = 0; k < len; ++k) {
            const int c = __ldg(cp + k * 32);
            float2 xv[BD];
#pragma unroll
            for (int b = 0; b < BD; ++b) xv[b] = src[(size_t)c * BD + b];
            const float2* vk = vp + k * (BD * BD * 32);
#pragma unroll
            for (int a = 0; a < BD; ++a)
#pragma unroll
                for (int b = 0; b < BD; ++b) cfma(y[a], __ldg(vk + (a * BD + b) * 32), xv[b]);
        }
        float loc = 0.f;
#pragma unroll
        for (int a = 0; a < BD; ++a) {
            const float2 s = src[(size_t)row * BD + a];
            const float2 v = {y[a].x + dd * s.x, y[a].y + dd * s.y};
            out[(size_t)row * BD + a] = v;
            loc += s.x * v.x + s.y * v.y;
        }
        local += (double)loc;
    }
    if (d.row >= 0) {
        double tot;
        if (reduce_last_n(e, d.row, local, tot, gridDim.x, blockIdx.x)) finalize(e, d, tot);
    }
}

template <int BD>
static void launch_a1(const Engine& e, const PassDesc* descs, const OpDev& A, const PassDesc& h,
                      cudaStream_t st) {
    auto k = k_bsr_a1<BD>;
    const int64_t need = (A.nbr + kSpmvThreads - 1) / kSpmvThreads;
    const int grid =
        (int)std::max<int64_t>(1, std::min<int64_t>(resident_blocks((const void*)k, kSpmvThreads), need));
    k<<<grid, kSpmvThreads, 0, st>>>(e, descs, A, A.vals32, (const float2*)h.src, (float2*)h.out);
}

template <class T, int BD, int KIND, class TO>
static void launch_one(const Engine& e, const PassDesc* descs, const OpDev& A, const T2<T>* vals,
                       int npass, const int* act, bool per, cudaStream_t st) {
    auto k = k_bsr<T, BD, KIND, TO>;
    k<<<multi_grid((const void*)k, A.nbr, npass, per), kThreads, 0, st>>>(e, descs, npass, act, A, vals);
}

template <class T, int BD>
static cudaError_t launch_bd(int kind, int out_f32, const Engine& e, const PassDesc* descs,
                             const OpDev& A, const T2<T>* vals, int npass, const int* act, bool per,
                             cudaStream_t st) {
    switch (kind) {
        case PASS_A: launch_one<T, BD, PASS_A, T>(e, descs, A, vals, npass, act, per, st); break;
        case PASS_C:
            if (out_f32) launch_one<T, BD, PASS_C, float>(e, descs, A, vals, npass, act, per, st);
            else launch_one<T, BD, PASS_C, double>(e, descs, A, vals, npass, act, per, st);
            break;
        case PASS_D: launch_one<T, BD, PASS_D, T>(e, descs, A, vals, npass, act, per, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int BD, int G>
static void launch_multi_g(const Engine& e, const PassDesc* descs, int npass, const int* act, int groups,
                           const OpDev& A, cudaStream_t st) {
    auto k = k_bsr_multi<float, BD, G>;
    // row blocks interleaved with groups in x
    const int64_t need = (A.nbr + kSpmvThreads - 1) / kSpmvThreads;
    const int nb = (int)std::max<int64_t>(
        1, std::min<int64_t>(resident_blocks((const void*)k, kSpmvThreads) / groups, need));
    k<<<nb * groups, kSpmvThreads, 0, st>>>(e, descs, npass, act, groups, A, A.vals32);
}

template <int BD>
static void launch_multi(const Engine& e, const PassDesc* descs, int npass, const int* act, int group,
                         int groups, const OpDev& A, cudaStream_t st) {
    if (group == 1) launch_multi_g<BD, 1>(e, descs, npass, act, groups, A, st);
    else launch_multi_g<BD, 2>(e, descs, npass, act, groups, A, st);
}

cudaError_t launch_bsr_multi(const OpDev& op, const Engine& e, const PassDesc* d_descs, int npass,
                             const int* act, int group, int groups, cudaStream_t st) {
    switch (op.bd) {
        case 1: launch_multi<1>(e, d_descs, npass, act, group, groups, op, st); break;
        case 2: launch_multi<2>(e, d_descs, npass, act, group, groups, op, st); break;
        default: launch_multi<3>(e, d_descs, npass, act, group, groups, op, st); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_bsr_pass(const OpDev& op, int prec, int kind, int out_f32, const Engine& e,
                            const PassDesc* d_descs, int npass, cudaStream_t st, const int* act, bool per,
                            const PassDesc* h_desc) {
    // one system: the active list (if any) holds at most that system, and the
    // kernel's gate stops it as the list would
    if (kind == PASS_A && npass == 1 && prec == PREC_F32 && !per && h_desc) {
        switch (op.bd) {
            case 1: launch_a1<1>(e, d_descs, op, *h_desc, st); break;
            case 2: launch_a1<2>(e, d_descs, op, *h_desc, st); break;
            default: launch_a1<3>(e, d_descs, op, *h_desc, st); break;
        }
        return cudaGetLastError();
    }
    if (kind == PASS_A && npass > 1 && prec == PREC_F32 && !per)
        return launch_bsr_multi(op, e, d_descs, npass, act, kMultiGroup,
                                (npass + kMultiGroup - 1) / kMultiGroup, st);
    if (prec == PREC_F64) {
        switch (op.bd) {
            case 1: return launch_bd<double, 1>(kind, out_f32, e, d_descs, op, op.vals64, npass, act, per, st);
            case 2: return launch_bd<double, 2>(kind, out_f32, e, d_descs, op, op.vals64, npass, act, per, st);
            default: return launch_bd<double, 3>(kind, out_f32, e, d_descs, op, op.vals64, npass, act, per, st);
        }
    }
    if (kind == PASS_C) return cudaErrorInvalidValue;
    switch (op.bd) {
        case 1: return launch_bd<float, 1>(kind, out_f32, e, d_descs, op, op.vals32, npass, act, per, st);
        case 2: return launch_bd<float, 2>(kind, out_f32, e, d_descs, op, op.vals32, npass, act, per, st);
        default: return launch_bd<float, 3>(kind, out_f32, e, d_descs, op, op.vals32, npass, act, per, st);
    }
}

}  // namespace msc
