// Direct solve of a 1D level's backward-Euler system (the 3-point operator of k_mg.cu,
//   -w_{i-1} x_{i-1} + (1 + w_{i-1} + w_i + Dirichlet) x_i - w_i x_{i+1} = b_i,
//   w_i the arithmetic or harmonic mean of K_i and K_{i+1}, a Dirichlet wall adding 2 K_i
//   to the diagonal)
// by parallel cyclic reduction: at stride s every row eliminates its neighbours i - s and
// i + s with their own rows, coupling it to i - 2s and i + 2s; after ceil(log2 n) steps each
// row holds one unknown. One launch per step over all cells (a 1D grid of a few thousand
// cells needs a dozen launches in place of the V-cycles' hundreds). The system is
// diagonally dominant, so no pivoting is needed. A periodic grid is made tridiagonal by
// the Sherman-Morrison formula: A = T + u v^T with the corner entries moved into u v^T
// (gamma = -diag_0; T's first and last diagonals take -gamma and -a_0 c_{n-1}/gamma), T is
// reduced with the two right-hand sides b and u, and x = y - (v.y)/(1 + v.z) z.
// FP64 throughout.
#include <algorithm>

#include "fld_internal.cuh"

namespace fld {

namespace {

constexpr int TRI_T = 256;

// rows of T and the right-hand sides b (d) and u (e, periodic only); sc[0] = a_0 / gamma
__global__ void k_tri_setup(int n, int lo_bc, int hi_bc, int fm, const double* __restrict__ K,
                            const double* __restrict__ rhs, double* __restrict__ a,
                            double* __restrict__ b, double* __restrict__ c, double* __restrict__ d,
                            double* __restrict__ e, double* __restrict__ sc) {
    const bool per = lo_bc == FLD_BC_PERIODIC;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double Ki = K[i];
        double wl = 0.0, wr = 0.0, dg = 1.0;
        if (i > 0) wl = fmean(Ki, K[i - 1], fm);
        else if (per) wl = fmean(Ki, K[n - 1], fm);
        else if (lo_bc == FLD_BC_DIRICHLET) dg += 2.0 * Ki;
        if (i < n - 1) wr = fmean(Ki, K[i + 1], fm);
        else if (per) wr = fmean(Ki, K[0], fm);
        else if (hi_bc == FLD_BC_DIRICHLET) dg += 2.0 * Ki;
        dg += wl + wr;
        double ai = -wl, ci = -wr;
        d[i] = rhs[i];
        if (per) {
            // corners a_0 (couples x_{n-1}) and c_{n-1} (couples x_0) into u v^T
            const double K0 = K[0], Kn = K[n - 1];
            const double wc = fmean(K0, Kn, fm);
            double dg0 = 1.0 + wc + (n > 1 ? fmean(K0, K[1], fm) : 0.0);
            const double gamma = -dg0;
            const double a0 = -wc, cn = -wc;
            e[i] = 0.0;
            if (i == 0) {
                ai = 0.0;
                dg -= gamma;
                e[i] = gamma;
                sc[0] = a0 / gamma;
            }
            if (i == n - 1) {
                ci = 0.0;
                dg -= a0 * cn / gamma;
                e[i] = cn;
            }
        }
        a[i] = ai;
        b[i] = dg;
        c[i] = ci;
    }
}

// one reduction step at stride s; rows outside [0, n) are identity rows
__global__ void k_pcr_step(int n, int s, int two, const double* __restrict__ a,
                           const double* __restrict__ b, const double* __restrict__ c,
                           const double* __restrict__ d, const double* __restrict__ e,
                           double* __restrict__ a2, double* __restrict__ b2,
                           double* __restrict__ c2, double* __restrict__ d2,
                           double* __restrict__ e2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int im = i - s, ip = i + s;
        const bool hm = im >= 0, hp = ip < n;
        const double k1 = hm ? a[i] / b[im] : 0.0;
        const double k2 = hp ? c[i] / b[ip] : 0.0;
        a2[i] = hm ? -a[im] * k1 : 0.0;
        c2[i] = hp ? -c[ip] * k2 : 0.0;
        b2[i] = b[i] - (hm ? c[im] * k1 : 0.0) - (hp ? a[ip] * k2 : 0.0);
        d2[i] = d[i] - (hm ? d[im] * k1 : 0.0) - (hp ? d[ip] * k2 : 0.0);
        if (two) e2[i] = e[i] - (hm ? e[im] * k1 : 0.0) - (hp ? e[ip] * k2 : 0.0);
    }
}

// x = d/b (and with two right-hand sides the Sherman-Morrison combination)
__global__ void k_tri_finish(int n, int two, const double* __restrict__ b,
                             const double* __restrict__ d, const double* __restrict__ e,
                             const double* __restrict__ sc, double* __restrict__ x) {
    double f = 0.0;
    if (two) {
        const double r = sc[0];
        const double y0 = d[0] / b[0], yn = d[n - 1] / b[n - 1];
        const double z0 = e[0] / b[0], zn = e[n - 1] / b[n - 1];
        f = (y0 + r * yn) / (1.0 + z0 + r * zn);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double y = d[i] / b[i];
        x[i] = two ? y - f * (e[i] / b[i]) : y;
    }
}

// r = b - A x in FP64 (the 3-point operator of k_tri_setup, periodic wrap or walls)
__global__ void k_tri_resid(int n, int lo_bc, int hi_bc, int fm, const double* __restrict__ K,
                            const double* __restrict__ b, const double* __restrict__ x,
                            double* __restrict__ r) {
    const bool per = lo_bc == FLD_BC_PERIODIC;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double Ki = K[i], xi = x[i];
        double ax = xi;
        const int il = i > 0 ? i - 1 : (per ? n - 1 : -1);
        const int ir = i < n - 1 ? i + 1 : (per ? 0 : -1);
        if (il >= 0) ax = fma(fmean(Ki, K[il], fm), xi - x[il], ax);
        else if (lo_bc == FLD_BC_DIRICHLET) ax = fma(2.0 * Ki, xi, ax);
        if (ir >= 0) ax = fma(fmean(Ki, K[ir], fm), xi - x[ir], ax);
        else if (hi_bc == FLD_BC_DIRICHLET) ax = fma(2.0 * Ki, xi, ax);
        r[i] = b[i] - ax;
    }
}

__global__ void k_tri_add(int n, double* __restrict__ x, const double* __restrict__ d) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] += d[i];
}

int tri_blocks(int n) { return std::max(1, std::min((n + TRI_T - 1) / TRI_T, num_sms() * 8)); }

}  // namespace

// Buffers: w holds 12 n + 1 doubles (two sets of a, b, c, d, e, one scalar, and the residual
// and correction of launch_tridiag_refine). Returns the number of kernels launched.
int launch_tridiag_solve(const Lvl& L, const double* K, const double* rhs, double* x, double* w,
                         cudaStream_t s) {
    const int n = L.n[0];
    double* A[2][5];
    for (int q = 0; q < 2; ++q)
        for (int f = 0; f < 5; ++f) A[q][f] = w + (long long)(5 * q + f) * n;
    double* sc = w + 10LL * n;
    const int two = L.bclo[0] == FLD_BC_PERIODIC ? 1 : 0;
    const int nb = tri_blocks(n);
    k_tri_setup<<<nb, TRI_T, 0, s>>>(n, L.bclo[0], L.bchi[0], L.fm, K, rhs, A[0][0], A[0][1], A[0][2],
                                     A[0][3], A[0][4], sc);
    int launches = 1, cur = 0;
    for (int st = 1; st < n; st *= 2) {
        k_pcr_step<<<nb, TRI_T, 0, s>>>(n, st, two, A[cur][0], A[cur][1], A[cur][2], A[cur][3],
                                        A[cur][4], A[cur ^ 1][0], A[cur ^ 1][1], A[cur ^ 1][2],
                                        A[cur ^ 1][3], A[cur ^ 1][4]);
        cur ^= 1;
        ++launches;
    }
    k_tri_finish<<<nb, TRI_T, 0, s>>>(n, two, A[cur][1], A[cur][3], A[cur][4], sc, x);
    return launches + 1;
}

// One step of iterative refinement of x: r = b - A x (FP64), A d = r by the same reduction,
// x += d. The reduction's rounding grows with the coupling (dt D / h^2 far above 1 on fine
// 1D grids) and with the Sherman-Morrison combination of a periodic grid; a step brings
// the residual back to the rounding of the operator. Returns the kernels launched.
int launch_tridiag_refine(const Lvl& L, const double* K, const double* rhs, double* x, double* w,
                          cudaStream_t s) {
    const int n = L.n[0];
    double* r = w + 10LL * n + 1;
    double* d = r + n;
    const int nb = tri_blocks(n);
    k_tri_resid<<<nb, TRI_T, 0, s>>>(n, L.bclo[0], L.bchi[0], L.fm, K, rhs, x, r);
    const int nl = launch_tridiag_solve(L, K, r, d, w, s);
    k_tri_add<<<nb, TRI_T, 0, s>>>(n, x, d);
    return nl + 2;
}

}  // namespace fld
