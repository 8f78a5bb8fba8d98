// Adjoint of the rational pseudofermion action built on the shifted solves.
//
// S = sum_s c_s Re(phi^dag x_s), x_s = (A + sigma_s)^{-1} phi: the quadratic
// form the shifted family diagonalises in RHMC (Sec. 1-2: the shifts and
// weights come from a rational approximation). Its gradients, in the
// convention grad = dS/dRe + i dS/dIm:
//   dS/dphi   = 2 sum_s c_s x_s;
//   dS/dU_mu(x) = sum_s c_s eta_mu(x) [x_s(x) y_s(x+mu)^dag - y_s(x) x_s(x+mu)^dag],
//   y_s = D x_s,
// from dS = -sum_s c_s x_s^dag dA x_s, dA = -(dD D + D dD), D and dD
// anti-Hermitian, and dU_mu(x) entering D at (x, x+mu) as eta/2 dU and at
// (x+mu, x) as -eta/2 dU^dag. Everything here is FP64.
#include "engine.h"

namespace msc {

// out_red[row] = sum_s c_s Re(phi^dag x_s) (x: [S][npad])
__global__ void __launch_bounds__(kThreads) k_quad(Engine e, const double2* __restrict__ phi,
                                                   const double2* __restrict__ x, const double* c,
                                                   int S, int64_t n, int64_t npad, PassDesc d) {
    double local = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 f = phi[i];
        double acc = 0.0;
        for (int s = 0; s < S; ++s) {
            const double2 xv = x[(size_t)s * npad + i];
            acc = fma(c[s], f.x * xv.x + f.y * xv.y, acc);
        }
        local += acc;
    }
    double tot;
    if (reduce_last(e, d.row, local, tot)) finalize(e, d, tot);
}

// dphi = 2 sum_s c_s x_s
__global__ void __launch_bounds__(kThreads) k_dphi(const double2* __restrict__ x, const double* c, int S,
                                                   int64_t n, int64_t npad, double2* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = {0.0, 0.0};
        for (int s = 0; s < S; ++s) {
            const double2 xv = x[(size_t)s * npad + i];
            acc.x = fma(2.0 * c[s], xv.x, acc.x);
            acc.y = fma(2.0 * c[s], xv.y, acc.y);
        }
        out[i] = acc;
    }
}

// G_mu(x) for every site and direction; one thread per (site, mu).
// x, y: [S][npad] with site-major colour-inner vectors; G: [4][V][NC][NC].
template <int NC>
__global__ void __launch_bounds__(kThreads) k_force(const double2* __restrict__ x,
                                                    const double2* __restrict__ y, const double* c,
                                                    int S, int64_t npad, StagGeom g,
                                                    double2* __restrict__ G) {
    const int64_t total = (int64_t)4 * g.V;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int mu = (int)(t / g.V);
        const int site = (int)(t % g.V);
        int cc[4];
        int rem = site;
        cc[0] = rem % g.L[0]; rem /= g.L[0];
        cc[1] = rem % g.L[1]; rem /= g.L[1];
        cc[2] = rem % g.L[2]; rem /= g.L[2];
        cc[3] = rem;
        int stride = 1, par = 0;
        for (int nu = 0; nu < mu; ++nu) {
            par += cc[nu];
            stride *= g.L[nu];
        }
        const int fwd = (cc[mu] == g.L[mu] - 1) ? site - (g.L[mu] - 1) * stride : site + stride;
        const double eta = (par & 1) ? -1.0 : 1.0;
        double2 acc[NC][NC];
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int b = 0; b < NC; ++b) acc[a][b] = {0.0, 0.0};
        for (int s = 0; s < S; ++s) {
            const double w = eta * c[s];
            const double2* xs = x + (size_t)s * npad;
            const double2* ys = y + (size_t)s * npad;
            double2 xa[NC], ya[NC], xb[NC], yb[NC];
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                xa[a] = xs[(size_t)site * NC + a];
                ya[a] = ys[(size_t)site * NC + a];
                xb[a] = xs[(size_t)fwd * NC + a];
                yb[a] = ys[(size_t)fwd * NC + a];
            }
#pragma unroll
            for (int a = 0; a < NC; ++a)
#pragma unroll
                for (int b = 0; b < NC; ++b) {
                    // x(x)_a conj(y(x+mu)_b) - y(x)_a conj(x(x+mu)_b)
                    double2 t1 = {xa[a].x * yb[b].x + xa[a].y * yb[b].y, xa[a].y * yb[b].x - xa[a].x * yb[b].y};
                    double2 t2 = {ya[a].x * xb[b].x + ya[a].y * xb[b].y, ya[a].y * xb[b].x - ya[a].x * xb[b].y};
                    acc[a][b].x = fma(w, t1.x - t2.x, acc[a][b].x);
                    acc[a][b].y = fma(w, t1.y - t2.y, acc[a][b].y);
                }
        }
        double2* out = G + ((size_t)mu * g.V + site) * NC * NC;
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int b = 0; b < NC; ++b) out[a * NC + b] = acc[a][b];
    }
}

cudaError_t launch_quad(const Engine& e, const double2* phi, const double2* x, const double* c, int S,
                        int64_t n, int64_t npad, int row, cudaStream_t st) {
    PassDesc d{};
    d.sys = -1;
    d.row = row;
    d.fin = FIN_STORE;
    k_quad<<<resident_grid((const void*)k_quad, n), kThreads, 0, st>>>(e, phi, x, c, S, n, npad, d);
    return cudaGetLastError();
}

cudaError_t launch_dphi(const double2* x, const double* c, int S, int64_t n, int64_t npad,
                        double2* out, cudaStream_t st) {
    k_dphi<<<resident_grid((const void*)k_dphi, n), kThreads, 0, st>>>(x, c, S, n, npad, out);
    return cudaGetLastError();
}

cudaError_t launch_force(const OpDev& op, const double2* x, const double2* y, const double* c, int S,
                         int64_t npad, double2* G, cudaStream_t st) {
    const int64_t work = (int64_t)4 * op.g.V;
    if (op.nc == 3)
        k_force<3><<<resident_grid((const void*)k_force<3>, work), kThreads, 0, st>>>(x, y, c, S, npad, op.g, G);
    else
        k_force<2><<<resident_grid((const void*)k_force<2>, work), kThreads, 0, st>>>(x, y, c, S, npad, op.g, G);
    return cudaGetLastError();
}

}  // namespace msc
