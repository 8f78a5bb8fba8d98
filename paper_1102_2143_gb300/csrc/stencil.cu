// Staggered operator kernels: A = M^dagger M = m^2 - D^2 with
//   D_xy = 1/2 sum_mu eta_mu(x) [U_mu(x) d_{y,x+mu} - U_mu(x-mu)^dagger d_{y,x-mu}],
// the lattice operator of the synthetic workload (the paper's solver is
// operator-generic, Sec. 3; A = m^2 - D^2 follows from D^dagger = -D).
//
// A p is applied as two passes of D (t = D p, then Ap = (m^2+sigma0) p - D t)
// with the CG bookkeeping fused into the passes' epilogues:
//   pass 1 also reduces P = p^dag (A+sigma0) p = (m^2+sigma0)|p|^2 + |t|^2,
//   pass 2 also applies r -= alpha Ap and reduces R' = |r|^2,
// so Ap is never written to memory (Algorithm 1, lines 18-20 and 24).
//
// One thread handles one site. Links are stored structure-of-arrays
// ([mu][component][site]) so that a warp's link loads are contiguous. In
// FP32, SU(3) links keep two rows (third = conj(row0 x row1)) and SU(2)
// links keep one row (second = (-conj u01, conj u00)).
#include <algorithm>
#include <cstdlib>

#include "async.cuh"
#include "stencil.cuh"

namespace msc {

StagGeom stag_geom(const int dims[4]) {
    StagGeom g;
    int64_t V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        g.L[mu] = dims[mu];
        V *= dims[mu];
    }
    g.V = (int)V;
    const int div[4] = {dims[0], dims[1], dims[2], std::max(1, dims[0] / 2)};
    for (int k = 0; k < 4; ++k) {
        const uint64_t d = (uint64_t)div[k];
        int l = 0;
        while (((uint64_t)1 << l) < d) ++l;
        // M = floor(2^(32+l) / d) + 1 lies in (2^32, 2^33]; dm = M - 2^32
        const uint64_t M = ((uint64_t)1 << (32 + l)) / d + 1;
        g.dm[k] = (unsigned)(M - ((uint64_t)1 << 32));
        g.ds[k] = l;
    }
    return g;
}

// One D pass over every site with the epilogue `KIND` (see PASS_* in engine.h),
// for the systems of the pass list (see sys_block in common.cuh).
// FP32 passes: at most 80 registers (three 256-thread blocks per SM); the
// site loop is bound by the latency of its link and neighbour loads, and
// more resident warps beat the loads the compiler would otherwise hoist
// (32^4 solve: 1.81 s uncapped, 1.51 s at three blocks, 1.55 s at four).
#ifndef MSC_STAG_MINB
#define MSC_STAG_MINB 3
#endif
template <class T, int NC, int RECON, int KIND, class TO>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? MSC_STAG_MINB : 1)
k_stag(Engine e, const PassDesc* descs, int npass, const int* act, StagGeom g, const void* links) {
    const SysBlock q = sys_block(npass, act);
    if (!q.ok) return;
    const PassDesc d = descs[q.j];
    if (gated_off(e, d)) return;
    const T alpha = (KIND == PASS_B || KIND == PASS_BC) ? (T)e.sys[d.sys].alpha : T(0);
    SiteAcc<T, KIND> local = 0;
    const int nh = vlen(g);
    for (int h = q.bx * blockDim.x + threadIdx.x; h < nh; h += q.gx * blockDim.x)
        local += stag_site<T, NC, RECON, KIND, TO, true>(d, g, links, alpha, pass_site<KIND == PASS_A>(h, g));
    if (d.row >= 0) {
        double tot;
        if (reduce_last_n(e, d.row, (double)local, tot, q.gx, q.bx)) finalize<KIND == PASS_BC>(e, d, tot);
    }
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

template <class T, int NC, int RECON, int KIND, class TO>
static void launch_one(const Engine& e, const PassDesc* descs, StagGeom g, const void* links, int npass,
                       const int* act, bool per, cudaStream_t st) {
    auto k = k_stag<T, NC, RECON, KIND, TO>;
    if constexpr (sizeof(T) == 8) {
        // FP64 passes over few sites: smaller blocks, so that the FP64
        // arithmetic (about 1/64 of the FP32 rate on GB300) spreads over more
        // SMs; a 4^4 lattice's 256 sites in one 256-thread block would run on
        // one SM (a one-thread-per-site pass keeps one site per thread).
        const int64_t V = vlen(g);
        const int np = std::max(npass, 1);
        int nt = kThreads;
        while (nt > 32 && ((V + nt - 1) / nt) * np < 2 * device_sms()) nt >>= 1;
        if (nt < kThreads) {
            const int per_sys = (int)((V + nt - 1) / nt);
            const dim3 grid = (per && npass > 1) ? dim3(per_sys, npass) : dim3(per_sys * np);
            k<<<grid, nt, 0, st>>>(e, descs, npass, act, g, links);
            return;
        }
    }
    k<<<multi_grid((const void*)k, vlen(g), npass, per), kThreads, 0, st>>>(e, descs, npass, act, g, links);
}

template <class T, int NC, int RECON>
static cudaError_t launch_kind(int kind, int out_f32, const Engine& e, const PassDesc* descs,
                               StagGeom g, const void* links, int npass, const int* act, bool per,
                               cudaStream_t st) {
    switch (kind) {
        case PASS_A: launch_one<T, NC, RECON, PASS_A, T>(e, descs, g, links, npass, act, per, st); break;
        case PASS_B:
            if (e.cond_flag) launch_one<T, NC, RECON, PASS_BC, T>(e, descs, g, links, npass, act, per, st);
            else launch_one<T, NC, RECON, PASS_B, T>(e, descs, g, links, npass, act, per, st);
            break;
        case PASS_C:
            if (out_f32) launch_one<T, NC, RECON, PASS_C, float>(e, descs, g, links, npass, act, per, st);
            else launch_one<T, NC, RECON, PASS_C, double>(e, descs, g, links, npass, act, per, st);
            break;
        default: launch_one<T, NC, RECON, PASS_D, T>(e, descs, g, links, npass, act, per, st); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_stag_pass(const OpDev& op, int prec, int kind, int out_f32, const Engine& e,
                             const PassDesc* d_descs, int npass, cudaStream_t st, const int* act, bool per) {
    if (prec == PREC_F64) {
        if (op.nc == 3) return launch_kind<double, 3, 0>(kind, out_f32, e, d_descs, op.g, op.links64, npass, act, per, st);
        return launch_kind<double, 2, 0>(kind, out_f32, e, d_descs, op.g, op.links64, npass, act, per, st);
    }
    if (kind == PASS_C) return cudaErrorInvalidValue;  // residual passes run in FP64
    if (op.nc == 3) {
        if (op.recon) return launch_kind<float, 3, 1>(kind, out_f32, e, d_descs, op.g, op.links32, npass, act, per, st);
        return launch_kind<float, 3, 0>(kind, out_f32, e, d_descs, op.g, op.links32, npass, act, per, st);
    }
    if (op.recon) return launch_kind<float, 2, 1>(kind, out_f32, e, d_descs, op.g, op.links32, npass, act, per, st);
    return launch_kind<float, 2, 0>(kind, out_f32, e, d_descs, op.g, op.links32, npass, act, per, st);
}

// ---------------------------------------------------------------------------
// One FP32 system with the links staged in shared memory. The lattice is cut
// into tiles of kTile consecutive sites (one per thread) lying inside one
// x0-x1 plane (kTile divides L0 L1, L0 divides kTile). For a tile, one thread
// issues bulk asynchronous copies of every link the tile's sites use: the
// tile's own links in the four directions (the forward hops, and the
// backward hops along x0, whose neighbour sits in the same row), the links
// of the tile one plane below along x2 and along x3 (backward hops there),
// and one row of x1 links below the tile (the backward x1 hop of its first
// row). The copies complete on an mbarrier; the threads then apply D from
// shared memory, reading the neighbour spinors (colour-planar) from global
// memory. The link stream, 80% of a pass's bytes, is thus in flight in
// 75 KB per tile without holding registers. A wait that runs out (bounded by
// the global timer) marks the Engine's error word; the block skips its
// remaining tiles but still takes part in the reduction, so the context's
// counters stay consistent.
// Opt-in (MSC_STAG_TILE=1): on the 32^4 solve it takes 66 / 76 us per pass
// against 61 / 74 us for k_stag reading its links directly (and 92 / 114 us
// double-buffered at one block per SM): the passes are bound by the latency
// of the neighbour-spinor gathers at the resident warps, not by link bytes in
// flight. It sums in k_stag's order, so its results are the same bit for bit.
// ---------------------------------------------------------------------------
constexpr int kTile = kThreads;

template <int NC> struct TileE { static constexpr int E = NC == 3 ? 3 : 1; };  // float4 per stored link

// dynamic shared memory of a block: one tile's links
size_t stag_tile_smem(int nc, int L0) {
    const int E = nc == 3 ? 3 : 1;
    return (size_t)(6 * E * kTile + E * L0) * 16;
}

bool stag_tile_fits(const StagGeom& g, int nc) {
    const int P01 = g.L[0] * g.L[1];
    return g.eo == 0 && kTile % g.L[0] == 0 && P01 % kTile == 0 && g.V >= kTile &&
           stag_tile_smem(nc, g.L[0]) <= 76 * 1024;
}

// the link at shared-memory float4 index i (stride `st` between components)
template <int NC>
__device__ __forceinline__ void tile_link(const float4* __restrict__ p, int st, float2 (&u)[NC][NC]) {
    if constexpr (NC == 3) {
        const float4 q0 = p[0], q1 = p[st], q2 = p[2 * st];
        u[0][0] = {q0.x, q0.y}; u[0][1] = {q0.z, q0.w};
        u[0][2] = {q1.x, q1.y}; u[1][0] = {q1.z, q1.w};
        u[1][1] = {q2.x, q2.y}; u[1][2] = {q2.z, q2.w};
        u[2][0] = cconj(csub(cmul(u[0][1], u[1][2]), cmul(u[0][2], u[1][1])));
        u[2][1] = cconj(csub(cmul(u[0][2], u[1][0]), cmul(u[0][0], u[1][2])));
        u[2][2] = cconj(csub(cmul(u[0][0], u[1][1]), cmul(u[0][1], u[1][0])));
    } else {
        const float4 q = p[0];
        u[0][0] = {q.x, q.y};
        u[0][1] = {q.z, q.w};
        u[1][0] = {-q.z, q.w};
        u[1][1] = {q.x, -q.y};
    }
}

template <int NC, int KIND>
__global__ void __launch_bounds__(kThreads, 3)
k_stag_tile(Engine e, const PassDesc* descs, StagGeom g, const float4* __restrict__ links, uint64_t wait_ns,
            int no_copy) {
    constexpr int E = TileE<NC>::E;
    extern __shared__ float4 sl[];  // [4][E][T] forward, [E][T] back x2, [E][T] back x3, [E][L0] back x1 halo
    __shared__ uint64_t bar;
    __shared__ int s_bad;
    const PassDesc d = descs[0];
    if (gated_off(e, d)) return;
    const int V = g.V, L0 = g.L[0], L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
    const int P01 = L0 * L1, P012 = P01 * L2;
    const int ntiles = V / kTile;
    float4* fw = sl;
    float4* b2 = sl + 4 * E * kTile;
    float4* b3 = b2 + E * kTile;
    float4* b1 = b3 + E * kTile;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
        s_bad = 0;
    }
    __syncthreads();
    const float2* __restrict__ src = (const float2*)d.src;
    const float2* __restrict__ aux = (const float2*)d.aux;
    float2* out = (float2*)d.out;
    const float dd = (float)d.d;
    const float alpha = (KIND == PASS_B || KIND == PASS_BC) ? (float)e.sys[d.sys].alpha : 0.f;
    double local = 0.0;
    uint32_t parity = 0;
    bool inflight = false;  // thread 0: copies issued and not waited for
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int s0 = tile * kTile;
        if (threadIdx.x == 0) {
            async_proxy_fence();  // the previous tile's reads before the copies overwrite
            const uint32_t tb = kTile * 16, hb = (uint32_t)L0 * 16;
            mbar_arrive_expect_tx(&bar, 6u * E * tb + E * hb);
            if (!no_copy) {
                const int c1 = (s0 / L0) % L1, c2 = (s0 / P01) % L2, c3 = s0 / P012;
                const int h1 = c1 > 0 ? s0 - L0 : s0 + (L1 - 1) * L0;
                const int t2 = c2 > 0 ? s0 - P01 : s0 + (L2 - 1) * P01;
                const int t3 = c3 > 0 ? s0 - P012 : s0 + (L3 - 1) * P012;
                for (int mu = 0; mu < 4; ++mu)
                    for (int c = 0; c < E; ++c)
                        bulk_copy_g2s(fw + (mu * E + c) * kTile, links + ((size_t)mu * E + c) * V + s0, tb, &bar);
                for (int c = 0; c < E; ++c) {
                    bulk_copy_g2s(b2 + c * kTile, links + ((size_t)2 * E + c) * V + t2, tb, &bar);
                    bulk_copy_g2s(b3 + c * kTile, links + ((size_t)3 * E + c) * V + t3, tb, &bar);
                    bulk_copy_g2s(b1 + c * L0, links + ((size_t)E + c) * V + h1, hb, &bar);
                }
                inflight = true;
            }
        }
        if (mbar_wait_bounded(&bar, parity, wait_ns)) inflight = false;
        else s_bad = 1;
        parity ^= 1;
        __syncthreads();
        if (s_bad) break;
        const int l = threadIdx.x;
        const int x = s0 + l;
        const SiteNbrs nb = neighbours(x, g);
        float2 y[NC];
#pragma unroll
        for (int a = 0; a < NC; ++a) y[a] = {0.f, 0.f};
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            float2 u[NC][NC], w[NC][NC], v[NC], z[NC];
#pragma unroll
            for (int b = 0; b < NC; ++b) {
                v[b] = src[(size_t)b * V + nb.fwd[mu]];
                z[b] = src[(size_t)b * V + nb.bwd[mu]];
            }
            tile_link<NC>(fw + mu * E * kTile + l, kTile, u);
            if (mu == 0) tile_link<NC>(fw + (nb.bwd[0] - s0), kTile, w);
            else if (mu == 1) {
                if (l >= L0) tile_link<NC>(fw + E * kTile + (l - L0), kTile, w);
                else tile_link<NC>(b1 + l, L0, w);
            } else if (mu == 2) tile_link<NC>(b2 + l, kTile, w);
            else tile_link<NC>(b3 + l, kTile, w);
            const float eta = nb.par[mu] ? -0.5f : 0.5f;
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                float2 f = {0.f, 0.f};
#pragma unroll
                for (int b = 0; b < NC; ++b) {
                    cfma(f, u[a][b], v[b]);       // + U_mu(x) src(x+mu)
                    cfms_conj(f, w[b][a], z[b]);  // - U_mu(x-mu)^dag src(x-mu)
                }
                y[a].x = fmaf(eta, f.x, y[a].x);
                y[a].y = fmaf(eta, f.y, y[a].y);
            }
        }
        float loc = 0.f;
        if (KIND == PASS_A) {
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                out[(size_t)a * V + x] = y[a];
                if (d.row >= 0) {
                    const float2 pa = aux[(size_t)a * V + x];
                    loc += dd * (pa.x * pa.x + pa.y * pa.y) + y[a].x * y[a].x + y[a].y * y[a].y;
                }
            }
        } else {
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                const float2 pa = aux[(size_t)a * V + x];
                float2 ra = out[(size_t)a * V + x];
                ra.x -= alpha * (dd * pa.x - y[a].x);
                ra.y -= alpha * (dd * pa.y - y[a].y);
                out[(size_t)a * V + x] = ra;
                loc += ra.x * ra.x + ra.y * ra.y;
            }
        }
        local += (double)loc;
        __syncthreads();  // every thread is done with this tile's links
    }
    if (s_bad && threadIdx.x == 0) {
        if (e.err) atomicOr(e.err, 1u);
        // copies still in flight complete on the barrier's open phase
        if (inflight) mbar_wait_bounded(&bar, parity ^ 1, wait_ns);
    }
    if (d.row >= 0) {
        double tot;
        if (reduce_last_n(e, d.row, local, tot, gridDim.x, blockIdx.x)) finalize<KIND == PASS_BC>(e, d, tot);
    }
}

template <int NC, int KIND>
static cudaError_t launch_tile(const Engine& e, const PassDesc* descs, const StagGeom& g, const void* links,
                               uint64_t wait_ns, int no_copy, cudaStream_t st) {
    auto k = k_stag_tile<NC, KIND>;
    const size_t sm = stag_tile_smem(NC, g.L[0]);
    cudaError_t err = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessorWithFlags(&per_sm, (const void*)k, kThreads, sm, 0) != cudaSuccess)
        per_sm = 1;
    const int ntiles = g.V / kTile;
    const int grid = std::max(1, std::min(ntiles, std::max(1, per_sm) * std::max(1, sms)));
    k<<<grid, kThreads, sm, st>>>(e, descs, g, (const float4*)links, wait_ns, no_copy);
    return cudaGetLastError();
}

cudaError_t launch_stag_tile(const OpDev& op, int kind, const Engine& e, const PassDesc* d_descs, uint64_t wait_ns,
                             int no_copy, cudaStream_t st) {
    const int k = (kind == PASS_B && e.cond_flag) ? PASS_BC : kind;
    if (op.nc == 3) {
        if (k == PASS_A) return launch_tile<3, PASS_A>(e, d_descs, op.g, op.links32, wait_ns, no_copy, st);
        if (k == PASS_B) return launch_tile<3, PASS_B>(e, d_descs, op.g, op.links32, wait_ns, no_copy, st);
        return launch_tile<3, PASS_BC>(e, d_descs, op.g, op.links32, wait_ns, no_copy, st);
    }
    if (k == PASS_A) return launch_tile<2, PASS_A>(e, d_descs, op.g, op.links32, wait_ns, no_copy, st);
    if (k == PASS_B) return launch_tile<2, PASS_B>(e, d_descs, op.g, op.links32, wait_ns, no_copy, st);
    return launch_tile<2, PASS_BC>(e, d_descs, op.g, op.links32, wait_ns, no_copy, st);
}

// ---------------------------------------------------------------------------
// Several systems of one operator in one FP32 pass (right-hand sides of a
// multi-shift stage, or the shifts of a refinement round): each thread takes
// one site for up to NR systems: per hop it loads the NR neighbour spinors
// (colour-planar vectors, so each load of a warp is one contiguous run),
// then loads and rebuilds the link once and applies it to all of them, so a
// pass reads the links once per group of NR systems instead of once per
// system. The staggered phase eta_mu(x)/2 is folded into the link.
//
// The systems still iterating ({count, indices} in `act`, or all npass) are
// cut into ceil(count / NR) groups of near-equal size; block b serves group
// b % groups as its block b / groups (the groups of one site range run side
// by side, so the second group's link loads hit L2). Per system the epilogue
// is that of stag_site (PASS_A: out = D src, P terms; PASS_B/BC: r -= alpha
// (d aux - D src), |r|^2), and the reductions of a group complete together:
// its blocks publish one partial per system, then count themselves on the
// counter of the group's first system; the last block finalizes every
// system of the group in turn.
// ---------------------------------------------------------------------------
template <int NC, int RECON, int KIND, int NR, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
k_stag_group(Engine e, const PassDesc* descs, int npass, const int* act, StagGeom g, const void* links) {
    static_assert(NR <= kThreads / 32, "one warp per system of a group reduces its partial");
    using F2 = float2;
    __shared__ PassDesc sd[NR];
    __shared__ float sal[NR];
    __shared__ int son[NR];
    __shared__ double sred[NR][kThreads / 32];
    __shared__ int s_last;
    const int count = act ? __ldg(act) : npass;
    if (count <= 0) return;
    const int ng = (count + NR - 1) / NR;
    const int gi = (int)(blockIdx.x % ng);
    const int bx = (int)(blockIdx.x / ng);
    const int gx = (int)(gridDim.x / ng);
    if (bx >= gx) return;
    const int lo = (int)((int64_t)gi * count / ng);
    const int nr = (int)((int64_t)(gi + 1) * count / ng) - lo;
    if (threadIdx.x < NR) {
        const int r = threadIdx.x;
        int on = 0;
        float al = 0.f;
        if (r < nr) {
            const int j = act ? __ldg(act + 1 + lo + r) : lo + r;
            const PassDesc d = descs[j];
            sd[r] = d;
            on = gated_off(e, d) ? 0 : 1;
            if (on && (KIND == PASS_B || KIND == PASS_BC)) al = (float)e.sys[d.sys].alpha;
        }
        son[r] = on;
        sal[r] = al;
    }
    __syncthreads();
    unsigned mask = 0;
#pragma unroll
    for (int r = 0; r < NR; ++r) mask |= son[r] ? (1u << r) : 0u;
    if (mask == 0) return;
    const int V = vlen(g);  // sites (and colour-plane stride) of the vectors
    float local[NR];  // per-thread partial sums in FP32 (see SiteAcc)
#pragma unroll
    for (int r = 0; r < NR; ++r) local[r] = 0.f;
    for (int h = bx * blockDim.x + threadIdx.x; h < V; h += gx * blockDim.x) {
        const int x = pass_site<KIND == PASS_A>(h, g);
        const SiteNbrs nb = neighbours(x, g);
        F2 y[NR][NC];
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int a = 0; a < NC; ++a) y[r][a] = {0.f, 0.f};
#pragma unroll
        for (int hop = 0; hop < 8; ++hop) {
            // direction mu = hop / 2, forward (even hop) or backward
            const int mu = hop >> 1;
            const bool fwd = (hop & 1) == 0;
            const int xn = fwd ? nb.fwd[mu] : nb.bwd[mu];
            const int hn = vsite(xn, g);
            // the neighbour spinors of every system first (colour-planar:
            // each load of the warp is one contiguous run), then the link
            F2 v[NR][NC];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (!((mask >> r) & 1u)) continue;
                const F2* __restrict__ src = (const F2*)sd[r].src;
#pragma unroll
                for (int b = 0; b < NC; ++b) v[r][b] = src[(size_t)b * V + hn];
            }
            F2 u[NC][NC];
            Links<float, NC, RECON>::load(links, mu, fwd ? x : xn, g.V, u);
            const float eta = nb.par[mu] ? -0.5f : 0.5f;
#pragma unroll
            for (int a = 0; a < NC; ++a)
#pragma unroll
                for (int b = 0; b < NC; ++b) u[a][b] = {eta * u[a][b].x, eta * u[a][b].y};
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (!((mask >> r) & 1u)) continue;
#pragma unroll
                for (int a = 0; a < NC; ++a)
#pragma unroll
                    for (int b = 0; b < NC; ++b) {
                        if (fwd) cfma(y[r][a], u[a][b], v[r][b]);       // + eta U_mu(x) src(x+mu)
                        else cfms_conj(y[r][a], u[b][a], v[r][b]);      // - eta U_mu(x-mu)^dag src(x-mu)
                    }
            }
        }
    // epilogues
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (!((mask >> r) & 1u)) continue;
            const PassDesc& d = sd[r];
            const float dd = (float)d.d;
            const F2* __restrict__ aux = (const F2*)d.aux + h;
            F2* __restrict__ out = (F2*)d.out + h;
            float loc = 0.f;
            if (KIND == PASS_A) {
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    out[(size_t)a * V] = y[r][a];
                    const F2 pa = aux[(size_t)a * V];
                    loc += dd * (pa.x * pa.x + pa.y * pa.y) + y[r][a].x * y[r][a].x + y[r][a].y * y[r][a].y;
                }
            } else {
                const float al = sal[r];
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const F2 pa = aux[(size_t)a * V];
                    F2 ra = out[(size_t)a * V];
                    ra.x -= al * (dd * pa.x - y[r][a].x);
                    ra.y -= al * (dd * pa.y - y[r][a].y);
                    out[(size_t)a * V] = ra;
                    loc += ra.x * ra.x + ra.y * ra.y;
                }
            }
            local[r] += loc;
        }
    }
    if (sd[0].row < 0) return;  // apply-only passes reduce nothing
    // one partial per system of the group, then the group's arrival count
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const double v = warp_sum((double)local[r]);
        if (lane == 0) sred[r][w] = v;
    }
    __syncthreads();
    if (w < nr && ((mask >> w) & 1u)) {
        double t = lane < (int)(blockDim.x >> 5) ? sred[w][lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) e.partial[(size_t)sd[w].row * kMaxBlocks + bx] = t;
    }
    __syncthreads();
    unsigned* ctr = &e.counter[sd[0].row];
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(ctr, 1u);
        s_last = (t == (unsigned)gx - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int r = 0; r < nr; ++r) {
        if (!((mask >> r) & 1u)) continue;
        const PassDesc d = sd[r];
        double acc = 0.0;
        for (int i = threadIdx.x; i < gx; i += blockDim.x) acc += __ldcg(&e.partial[(size_t)d.row * kMaxBlocks + i]);
        const double tot = block_sum(acc, &sred[0][0]);
        __shared__ double s_tot;
        if (threadIdx.x == 0) s_tot = tot;
        __syncthreads();
        finalize<KIND == PASS_BC>(e, d, s_tot);
        __syncthreads();
    }
    if (threadIdx.x == 0) *ctr = 0u;
}

template <int NC, int RECON, int NR, int MINB>
static cudaError_t launch_group_kind(int kind, const Engine& e, const PassDesc* descs, StagGeom g,
                                     const void* links, int npass, const int* act, cudaStream_t st) {
    const int groups = (npass + NR - 1) / NR;
    switch (kind) {
        case PASS_A: {
            auto k = k_stag_group<NC, RECON, PASS_A, NR, MINB>;
            k<<<multi_grid((const void*)k, vlen(g), groups), kThreads, 0, st>>>(e, descs, npass, act, g, links);
            break;
        }
        case PASS_B:
            if (e.cond_flag) {
                auto k = k_stag_group<NC, RECON, PASS_BC, NR, MINB>;
                k<<<multi_grid((const void*)k, vlen(g), groups), kThreads, 0, st>>>(e, descs, npass, act, g, links);
            } else {
                auto k = k_stag_group<NC, RECON, PASS_B, NR, MINB>;
                k<<<multi_grid((const void*)k, vlen(g), groups), kThreads, 0, st>>>(e, descs, npass, act, g, links);
            }
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Launch shape of the grouped passes, 10 * systems per thread + blocks per
// SM: 21, 22, 42, 43 or 82; 0 runs every system through k_stag instead.
int stag_group_shape() {
    static int shape = [] {
        const char* v = getenv("MSC_STAG_GROUP");
        const int k = v ? atoi(v) : 43;
        return (k == 0 || k == 21 || k == 22 || k == 42 || k == 43 || k == 82) ? k : 43;
    }();
    return shape;
}

bool stag_group_applies(const OpDev& op, int prec, int kind, int npass) {
    return op.kind == OP_STAGGERED && prec == PREC_F32 && op.recon && npass >= 2 &&
           (kind == PASS_A || kind == PASS_B) && stag_group_shape() != 0;
}

// Group shapes: NR systems per thread, MINB blocks per SM.
template <int NC>
static cudaError_t launch_group_nc(int shape, int kind, const Engine& e, const PassDesc* d, const OpDev& op,
                                   int npass, const int* act, cudaStream_t st) {
    switch (shape) {
        case 21: return launch_group_kind<NC, 1, 2, 3>(kind, e, d, op.g, op.links32, npass, act, st);
        case 22: return launch_group_kind<NC, 1, 2, 2>(kind, e, d, op.g, op.links32, npass, act, st);
        case 42: return launch_group_kind<NC, 1, 4, 2>(kind, e, d, op.g, op.links32, npass, act, st);
        case 43: return launch_group_kind<NC, 1, 4, 3>(kind, e, d, op.g, op.links32, npass, act, st);
        default: return launch_group_kind<NC, 1, 8, 2>(kind, e, d, op.g, op.links32, npass, act, st);
    }
}

cudaError_t launch_stag_group(const OpDev& op, int kind, const Engine& e, const PassDesc* d_descs, int npass,
                              cudaStream_t st, const int* act) {
    int shape = stag_group_shape();
    if (npass <= 2 && shape > 22) shape = 21;
    if (npass <= 4 && shape > 43) shape = 43;
    if (op.nc == 3) return launch_group_nc<3>(shape, kind, e, d_descs, op, npass, act, st);
    return launch_group_nc<2>(shape, kind, e, d_descs, op, npass, act, st);
}

// ---------------------------------------------------------------------------
// set-up: link packing, unitarity check, block-CSR export
// ---------------------------------------------------------------------------

// AoS [4][V][nc][nc] double2 -> SoA [4][nc*nc][V] double2
__global__ void k_pack64(const double2* __restrict__ in, double2* __restrict__ out, int nc, int V) {
    const int e2 = nc * nc;
    const int64_t total = (int64_t)4 * V * e2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)(i % e2);
        const int64_t ml = i / e2;
        const int x = (int)(ml % V);
        const int mu = (int)(ml / V);
        out[((size_t)mu * e2 + comp) * V + x] = in[i];
    }
}

// max over links of max(|U U^dag - 1|_max, |det U - 1|)
__global__ void k_unitarity(const double2* __restrict__ in, int nc, int64_t nlinks,
                            unsigned long long* maxdev) {
    double m = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nlinks;
         l += (int64_t)gridDim.x * blockDim.x) {
        const double2* u = in + l * nc * nc;
        for (int a = 0; a < nc; ++a)
            for (int b = 0; b < nc; ++b) {
                double2 s = {0.0, 0.0};
                for (int c = 0; c < nc; ++c) s = cadd(s, cmul(u[a * nc + c], cconj(u[b * nc + c])));
                if (a == b) s.x -= 1.0;
                m = fmax(m, fmax(fabs(s.x), fabs(s.y)));
            }
        double2 det;
        if (nc == 2) {
            det = csub(cmul(u[0], u[3]), cmul(u[1], u[2]));
        } else {
            det = cmul(u[0], csub(cmul(u[4], u[8]), cmul(u[5], u[7])));
            det = csub(det, cmul(u[1], csub(cmul(u[3], u[8]), cmul(u[5], u[6]))));
            det = cadd(det, cmul(u[2], csub(cmul(u[3], u[7]), cmul(u[4], u[6]))));
        }
        det.x -= 1.0;
        m = fmax(m, fmax(fabs(det.x), fabs(det.y)));
        if (!(m == m)) m = 1e300;
    }
    // non-negative doubles order like their bit patterns
    atomicMax(maxdev, (unsigned long long)__double_as_longlong(m));
}

// FP32 links: full [4][nc*nc][V] float2, or rows [4][k][V] float4 (recon)
__global__ void k_pack32(const double2* __restrict__ in, void* out, int nc, int V, int recon) {
    const int e2 = nc * nc;
    const int64_t nl = (int64_t)4 * V;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nl;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(l % V);
        const int mu = (int)(l / V);
        const double2* u = in + l * e2;
        if (!recon) {
            float2* o = (float2*)out;
            for (int c = 0; c < e2; ++c)
                o[((size_t)mu * e2 + c) * V + x] = make_float2((float)u[c].x, (float)u[c].y);
        } else {
            float4* o = (float4*)out;
            const int k = nc == 3 ? 3 : 1;  // float4 per link: 6 or 2 complex
            for (int q = 0; q < k; ++q)
                o[((size_t)mu * k + q) * V + x] =
                    make_float4((float)u[2 * q].x, (float)u[2 * q].y, (float)u[2 * q + 1].x,
                                (float)u[2 * q + 1].y);
        }
    }
}

// hop matrix H(x, mu, s) of D: s=+1 -> 1/2 eta U_mu(x) (to x+mu);
// s=-1 -> -1/2 eta U_mu(x-mu)^dag (to x-mu).
template <int NC>
__device__ void hop_matrix(const double2* __restrict__ U, const StagGeom& g, int x, int mu, int s,
                           double2 (&h)[NC][NC], int& to) {
    const SiteNbrs nb = neighbours(x, g);
    const double eta = nb.par[mu] ? -0.5 : 0.5;
    if (s > 0) {
        to = nb.fwd[mu];
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) {
                const double2 u = U[((size_t)mu * NC * NC + a * NC + b) * g.V + x];
                h[a][b] = {eta * u.x, eta * u.y};
            }
    } else {
        to = nb.bwd[mu];
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) {
                const double2 u = U[((size_t)mu * NC * NC + b * NC + a) * g.V + to];
                h[a][b] = {-eta * u.x, eta * u.y};  // -eta * conj(u)
            }
    }
}

template <int NC>
__device__ void mat_acc(double2 (&acc)[NC][NC], const double2 (&a)[NC][NC], const double2 (&b)[NC][NC],
                        double sgn) {
    for (int i = 0; i < NC; ++i)
        for (int j = 0; j < NC; ++j) {
            double2 s = {0.0, 0.0};
            for (int k = 0; k < NC; ++k) s = cadd(s, cmul(a[i][k], b[k][j]));
            acc[i][j].x += sgn * s.x;
            acc[i][j].y += sgn * s.y;
        }
}

// A = m^2 - D^2 as 33 blocks per site row: slot 0 the diagonal, slots 1..8
// two hops along one axis (1 + 2 mu + (s<0)), slots 9..32 one hop along
// each of two axes mu < nu (9 + 4 pair + 2 (a<0) + (b<0)).
template <int NC>
__global__ void k_export_bsr(const double2* __restrict__ U, StagGeom g, double m2,
                             int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                             double2* __restrict__ vals) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.V; x += gridDim.x * blockDim.x) {
        const int64_t r0 = (int64_t)33 * x;
        row_ptr[x] = r0;
        if (x == g.V - 1) row_ptr[g.V] = r0 + 33;
        double2 blk[NC][NC];
        double2 h1[NC][NC], h2[NC][NC];
        int y, z;
        // diagonal: m^2 I - sum_{mu,s} H(x,mu,s) H(x+s mu, mu, -s)
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) blk[a][b] = {a == b ? m2 : 0.0, 0.0};
        for (int mu = 0; mu < 4; ++mu)
            for (int s = -1; s <= 1; s += 2) {
                hop_matrix<NC>(U, g, x, mu, s, h1, y);
                hop_matrix<NC>(U, g, y, mu, -s, h2, z);
                mat_acc<NC>(blk, h1, h2, -1.0);
            }
        col[r0] = x;
        for (int a = 0; a < NC; ++a)
            for (int b = 0; b < NC; ++b) vals[(size_t)r0 * NC * NC + a * NC + b] = blk[a][b];
        // two hops along one axis
        for (int mu = 0; mu < 4; ++mu)
            for (int s = -1; s <= 1; s += 2) {
                for (int a = 0; a < NC; ++a)
                    for (int b = 0; b < NC; ++b) blk[a][b] = {0.0, 0.0};
                hop_matrix<NC>(U, g, x, mu, s, h1, y);
                hop_matrix<NC>(U, g, y, mu, s, h2, z);
                mat_acc<NC>(blk, h1, h2, -1.0);
                const int64_t k = r0 + 1 + 2 * mu + (s < 0);
                col[k] = z;
                for (int a = 0; a < NC; ++a)
                    for (int b = 0; b < NC; ++b) vals[(size_t)k * NC * NC + a * NC + b] = blk[a][b];
            }
        // one hop along each of two axes, both orders of the hops
        int pair = 0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu, ++pair)
                for (int sa = -1; sa <= 1; sa += 2)
                    for (int sb = -1; sb <= 1; sb += 2) {
                        for (int a = 0; a < NC; ++a)
                            for (int b = 0; b < NC; ++b) blk[a][b] = {0.0, 0.0};
                        hop_matrix<NC>(U, g, x, mu, sa, h1, y);
                        hop_matrix<NC>(U, g, y, nu, sb, h2, z);
                        mat_acc<NC>(blk, h1, h2, -1.0);
                        hop_matrix<NC>(U, g, x, nu, sb, h1, y);
                        hop_matrix<NC>(U, g, y, mu, sa, h2, z);
                        mat_acc<NC>(blk, h1, h2, -1.0);
                        const int64_t k = r0 + 9 + 4 * pair + 2 * (sa < 0) + (sb < 0);
                        col[k] = z;
                        for (int a = 0; a < NC; ++a)
                            for (int b = 0; b < NC; ++b)
                                vals[(size_t)k * NC * NC + a * NC + b] = blk[a][b];
                    }
    }
}

static int setup_blocks(int64_t work) {
    int64_t b = (work + 255) / 256;
    if (b > 65535) b = 65535;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t stag_pack_links(OpDev& op, const double2* links_aos, double* d_maxdev, cudaStream_t st) {
    (void)d_maxdev;
    const int64_t total = (int64_t)4 * op.g.V * op.nc * op.nc;
    k_pack64<<<setup_blocks(total), 256, 0, st>>>(links_aos, op.links64, op.nc, op.g.V);
    return cudaGetLastError();
}

cudaError_t stag_unitarity(const OpDev& op, const double2* links_aos, double* d_maxdev,
                           cudaStream_t st) {
    const int64_t nl = (int64_t)4 * op.g.V;
    k_unitarity<<<setup_blocks(nl), 256, 0, st>>>(links_aos, op.nc, nl,
                                                  (unsigned long long*)d_maxdev);
    return cudaGetLastError();
}

cudaError_t stag_pack_links32(OpDev& op, const double2* links_aos, cudaStream_t st) {
    const int64_t nl = (int64_t)4 * op.g.V;
    k_pack32<<<setup_blocks(nl), 256, 0, st>>>(links_aos, op.links32, op.nc, op.g.V, op.recon);
    return cudaGetLastError();
}

cudaError_t stag_export_bsr(const OpDev& op, int64_t* row_ptr, int32_t* col, double2* vals,
                            cudaStream_t st) {
    const double m2 = op.mass * op.mass;
    if (op.nc == 3) k_export_bsr<3><<<setup_blocks(op.g.V), 128, 0, st>>>(op.links64, op.g, m2, row_ptr, col, vals);
    else k_export_bsr<2><<<setup_blocks(op.g.V), 128, 0, st>>>(op.links64, op.g, m2, row_ptr, col, vals);
    return cudaGetLastError();
}

}  // namespace msc
