// Device functions of the staggered operator shared by the single-operator
// and the batched kernels:
//   D_xy = 1/2 sum_mu eta_mu(x) [U_mu(x) d_{y,x+mu} - U_mu(x-mu)^dagger d_{y,x-mu}],
//   eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}), periodic boundaries.
#pragma once
#include <type_traits>

#include "engine.h"

namespace msc {

template <class T> using T2 = typename C2<T>::t;

struct SiteNbrs {
    int fwd[4], bwd[4];
    int par[4];  // parity of x_0 + ... + x_{mu-1}
};

__device__ __forceinline__ SiteNbrs neighbours(int x, const StagGeom& g) {
    SiteNbrs nb;
    int c[4];
    const int q0 = gdiv(x, g, 0), q1 = gdiv(q0, g, 1), q2 = gdiv(q1, g, 2);
    c[0] = x - q0 * g.L[0];
    c[1] = q0 - q1 * g.L[1];
    c[2] = q1 - q2 * g.L[2];
    c[3] = q2;
    int stride = 1, psum = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const int L = g.L[mu];
        nb.fwd[mu] = (c[mu] == L - 1) ? x - (L - 1) * stride : x + stride;
        nb.bwd[mu] = (c[mu] == 0) ? x + (L - 1) * stride : x - stride;
        nb.par[mu] = psum & 1;
        psum += c[mu];
        stride *= L;
    }
    return nb;
}

// Parity-reduced operator (g.eo = 1 + p): site x sits at compressed index
// x / 2 of a parity vector (each pair of sites (2k, 2k+1) along x0 holds one
// site of each parity), and the h-th site of parity par is eo_site(h, par).
__device__ __forceinline__ int vsite(int x, const StagGeom& g) { return g.eo ? (x >> 1) : x; }

__device__ __forceinline__ int eo_site(int h, int par, const StagGeom& g) {
    const int hl = g.L[0] >> 1;
    const int row = gdiv(h, g, 3);
    const int k = h - row * hl;
    const int r1 = gdiv(row, g, 1), r2 = gdiv(r1, g, 2);
    const int c1 = row - r1 * g.L[1];
    const int c2 = r1 - r2 * g.L[2];
    const int c3 = r2;
    return 2 * k + ((par + c1 + c2 + c3) & 1) + g.L[0] * row;
}

// The site a thread of a pass handles at loop index h: on the
// parity-reduced operator, t = D p (PASS_A, OTHER) lives on the other parity
// and every other pass's output on the source's.
template <bool OTHER>
__device__ __forceinline__ int pass_site(int h, const StagGeom& g) {
    if (!g.eo) return h;
    const int src_par = g.eo - 1;
    return eo_site(h, OTHER ? 1 - src_par : src_par, g);
}

// ---------------------------------------------------------------------------
// link loads
// ---------------------------------------------------------------------------
template <class T, int NC, int RECON> struct Links;

// full storage: T2 [4][NC*NC][V]
template <class T, int NC> struct Links<T, NC, 0> {
    __device__ static __forceinline__ void load(const void* base, int mu, int x, int V,
                                                T2<T> (&u)[NC][NC]) {
        const T2<T>* U = (const T2<T>*)base + (size_t)mu * NC * NC * V + x;
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int b = 0; b < NC; ++b) u[a][b] = U[(size_t)(a * NC + b) * V];
    }
};

// SU(3), two rows in three float4: (u00,u01) (u02,u10) (u11,u12)
template <> struct Links<float, 3, 1> {
    __device__ static __forceinline__ void load(const void* base, int mu, int x, int V,
                                                float2 (&u)[3][3]) {
        const float4* U = (const float4*)base + (size_t)mu * 3 * V + x;
        const float4 q0 = U[0], q1 = U[(size_t)V], q2 = U[(size_t)2 * V];
        u[0][0] = {q0.x, q0.y}; u[0][1] = {q0.z, q0.w};
        u[0][2] = {q1.x, q1.y}; u[1][0] = {q1.z, q1.w};
        u[1][1] = {q2.x, q2.y}; u[1][2] = {q2.z, q2.w};
        // row 2 = conj(row0 x row1)
        u[2][0] = cconj(csub(cmul(u[0][1], u[1][2]), cmul(u[0][2], u[1][1])));
        u[2][1] = cconj(csub(cmul(u[0][2], u[1][0]), cmul(u[0][0], u[1][2])));
        u[2][2] = cconj(csub(cmul(u[0][0], u[1][1]), cmul(u[0][1], u[1][0])));
    }
};

// SU(2), one row in one float4: (u00,u01); row 1 = (-conj u01, conj u00)
template <> struct Links<float, 2, 1> {
    __device__ static __forceinline__ void load(const void* base, int mu, int x, int V,
                                                float2 (&u)[2][2]) {
        const float4 q = ((const float4*)base)[(size_t)mu * V + x];
        u[0][0] = {q.x, q.y};
        u[0][1] = {q.z, q.w};
        u[1][0] = {-q.z, q.w};
        u[1][1] = {q.x, -q.y};
    }
};

// Index of the complex entry (site x, colour a) of a vector of element type
// T. Vectors are site-major (x * NC + a), except FP32 vectors of the
// single-operator stencil path (PL), which are colour-planar (a * V + x): the
// loads of one colour of a warp's 32 consecutive sites are then one
// contiguous 256-byte run instead of three 8-byte loads at a 24-byte stride.
template <class T, bool PL, int NC>
__device__ __forceinline__ size_t vix(int x, int a, int V) {
    return (PL && sizeof(T) == 4) ? (size_t)a * V + x : (size_t)x * NC + a;
}

// y = D src at site x
template <class T, int NC, int RECON, bool PL = false>
__device__ __forceinline__ void dslash_site(const void* links, const T2<T>* __restrict__ src, int x,
                                            const StagGeom& g, T2<T> (&y)[NC]) {
    const SiteNbrs nb = neighbours(x, g);
#pragma unroll
    for (int a = 0; a < NC; ++a) y[a] = {T(0), T(0)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        T2<T> u[NC][NC], v[NC];
        Links<T, NC, RECON>::load(links, mu, x, g.V, u);
#pragma unroll
        for (int b = 0; b < NC; ++b) v[b] = src[vix<T, PL, NC>(vsite(nb.fwd[mu], g), b, vlen(g))];
        T2<T> w[NC][NC], z[NC];
        Links<T, NC, RECON>::load(links, mu, nb.bwd[mu], g.V, w);
#pragma unroll
        for (int b = 0; b < NC; ++b) z[b] = src[vix<T, PL, NC>(vsite(nb.bwd[mu], g), b, vlen(g))];
        const T eta = nb.par[mu] ? T(-0.5) : T(0.5);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            T2<T> f = {T(0), T(0)};
#pragma unroll
            for (int b = 0; b < NC; ++b) {
                cfma(f, u[a][b], v[b]);        // + U_mu(x) src(x+mu)
                cfms_conj(f, w[b][a], z[b]);   // - U_mu(x-mu)^dag src(x-mu)
            }
            y[a].x = fma(eta, f.x, y[a].x);
            y[a].y = fma(eta, f.y, y[a].y);
        }
    }
}

// One site of a D pass: y = D src at x, then the epilogue KIND; returns this
// site's contribution to the pass's reduction (0 when d.row < 0).
//   PASS_A: out = y;                       P terms d|aux|^2 + |y|^2
//   PASS_B: r -= alpha (d aux - y);        |r|^2
//   PASS_C: out = b - (d aux - y) (FP64);  |out|^2
//   PASS_D: out = d aux - y
// PL: FP32 vectors (of type T or TO) are colour-planar (see vix).
// A site's share of a pass's reduction: FP32 for the FP32 passes (summed
// over a thread's sites in FP32, then reduced in FP64 across threads), FP64
// for the residual pass and FP64 operators.
template <class T, int KIND>
using SiteAcc = typename std::conditional<(sizeof(T) == 4 && KIND != PASS_C), float, double>::type;

template <class T, int NC, int RECON, int KIND, class TO, bool PL = false>
__device__ __forceinline__ SiteAcc<T, KIND> stag_site(const PassDesc& d, const StagGeom& g, const void* links,
                                            T alpha, int x) {
    const T2<T>* __restrict__ src = (const T2<T>*)d.src;
    const T2<T>* __restrict__ aux = (const T2<T>*)d.aux;
    const T dd = (T)d.d;
    const int V = vlen(g);
    T2<T> y[NC];
    dslash_site<T, NC, RECON, PL>(links, src, x, g, y);
    x = vsite(x, g);  // the site's index in the vectors
    if (KIND == PASS_A) {
        T2<T>* out = (T2<T>*)d.out;
        T loc = T(0);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            out[vix<T, PL, NC>(x, a, V)] = y[a];
            if (d.row >= 0) {
                const T2<T> pa = aux[vix<T, PL, NC>(x, a, V)];
                loc += dd * (pa.x * pa.x + pa.y * pa.y) + y[a].x * y[a].x + y[a].y * y[a].y;
            }
        }
        return (SiteAcc<T, KIND>)loc;
    } else if (KIND == PASS_B || KIND == PASS_BC) {
        T2<T>* r = (T2<T>*)d.out;
        T loc = T(0);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const T2<T> pa = aux[vix<T, PL, NC>(x, a, V)];
            const T2<T> ap = {dd * pa.x - y[a].x, dd * pa.y - y[a].y};
            T2<T> ra = r[vix<T, PL, NC>(x, a, V)];
            ra.x -= alpha * ap.x;
            ra.y -= alpha * ap.y;
            r[vix<T, PL, NC>(x, a, V)] = ra;
            loc += ra.x * ra.x + ra.y * ra.y;
        }
        return (SiteAcc<T, KIND>)loc;
    } else if (KIND == PASS_C) {
        TO* out = (TO*)d.out;
        double loc = 0.0;
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const T2<T> xa = aux[vix<T, PL, NC>(x, a, V)];
            const double2 ba = d.b[(size_t)x * NC + a];
            const double vx = ba.x - ((double)dd * xa.x - y[a].x);
            const double vy = ba.y - ((double)dd * xa.y - y[a].y);
            if (out) {
                const size_t o = vix<TO, PL, NC>(x, a, V);
                out[2 * o] = (TO)vx;
                out[2 * o + 1] = (TO)vy;
            }
            loc += vx * vx + vy * vy;
        }
        return loc;
    } else {
        T2<T>* out = (T2<T>*)d.out;
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const T2<T> xa = aux[vix<T, PL, NC>(x, a, V)];
            out[vix<T, PL, NC>(x, a, V)] = {dd * xa.x - y[a].x, dd * xa.y - y[a].y};
        }
        return SiteAcc<T, KIND>(0);
    }
}

}  // namespace msc
