// Pointwise kernels of the FLD substep: the gas-radiation exchange quartic and the
// flux limiter (Levermore-Pomraning, 4th-order 5-point gradient).
#include <algorithm>

#include "fld_internal.cuh"

namespace fld {

// ----------------------------------------------------------------- exchange
// Backward Euler on de/dt = +qdot, dE/dt = -qdot with qdot = c kappa rho (E - a_r T^4)
// (Eqs. heating, qdot). Eliminating E' leaves, per cell,
//   f(T) = alpha T + beta T^4 - q = 0,  alpha = rho c_v, beta = a_r chi/(1+chi),
//   q = e + chi E/(1+chi),  chi = dt c kappa rho,
// increasing and convex for T > 0 with f(0) < 0: one positive root, bounded above by
// min(q/alpha, (q/beta)^(1/4)), from where Newton decreases monotonically to it.
//
// FP64 arithmetic is the scarce resource on this GPU, so the root is found in two
// stages: Newton in FP32 on a scaled form of the quartic (all quantities O(1)), then
// one FP64 Newton step, whose residual f(T) is evaluated in FP64 and whose derivative
// only needs FP32 accuracy (the step is ~1e-7 T, so a 1e-7 relative error in it leaves
// ~1e-14 T). Cells whose coefficients fall outside the FP32 range take a plain FP64
// Newton iteration instead.

__device__ __forceinline__ bool f32_ok(double v) { return v > 1e-30 && v < 1e30; }

__device__ double exchange_root(double alpha, double beta, double q) {
    const float af = (float)alpha, bf = (float)beta, qf = (float)q;
    const float T1 = qf / af;                       // root if beta were 0
    const float T1sq = T1 * T1;
    const float g = (bf * T1sq) * (T1sq / qf);      // beta T1^4 / q
    const bool fast = f32_ok(alpha) && f32_ok(q) && (beta == 0.0 || f32_ok(beta)) &&
                      T1 > 1e-9f && T1 < 1e9f && g < 1e30f;
    if (fast) {
        float x = 1.f, scale = T1;
        if (g <= 1.f) {
            // phi(x) = g x^4 + x - 1, root in (0.72, 1]
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const float x2 = x * x;
                x -= (fmaf(g * x2, x2, x) - 1.f) / fmaf(4.f * g * x2, x, 1.f);
            }
        } else {
            // psi(y) = y^4 + h y - 1 with h = g^(-1/4), T = y T1 h, root in (0.8, 1]
            const float hh = rsqrtf(sqrtf(g));
            scale = T1 * hh;
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const float x2 = x * x;
                x -= (fmaf(x2, x2, hh * x) - 1.f) / fmaf(4.f * x2, x, hh);
            }
        }
        const double T = (double)x * (double)scale;
        // one FP64 Newton step: FP64 residual, FP32 derivative
        const double T2 = T * T;
        const double f = fma(beta * T2, T2, fma(alpha, T, -q));
        const float fpf = fmaf(4.f * bf * (float)T2, (float)T, af);
        return fma(-f, (double)__frcp_rn(fpf), T);
    }
    // outside the FP32 range: plain FP64 Newton from the upper bound
    double x = q / alpha;
    if (beta > 0.0) x = fmin(x, sqrt(sqrt(q / beta)));
    for (int it = 0; it < 60; ++it) {
        const double x2 = x * x;
        const double f = fma(beta * x2, x2, fma(alpha, x, -q));
        const double dx = f / fma(4.0 * beta * x2, x, alpha);
        x -= dx;
        if (fabs(dx) <= 4e-16 * x) break;
    }
    return x;
}

__global__ void k_exchange(long long n, const double* __restrict__ rho, double* __restrict__ T,
                           double* __restrict__ E, Opacity op, double dtc, double a_r, double cv,
                           unsigned* err) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = rho[i], t = T[i], er = E[i];
        if (!(pos_finite(r) && pos_finite(t) && pos_finite(er))) {
            atomicOr(err, ERRBIT_DOMAIN);
            continue;
        }
        const double kap = opacity_eval(op, r, t);
        if (!pos_finite(kap)) {
            atomicOr(err, ERRBIT_DOMAIN);
            continue;
        }
        const double chi = dtc * kap * r;
        const double alpha = r * cv;
        const double d1 = 1.0 + chi;
        const double inv1 = (d1 < 1e30) ? rcp_nr(d1) : 1.0 / d1;
        const double w = chi * inv1;
        const double beta = w * a_r;
        const double q = fma(w, er, alpha * t);
        const double x = exchange_root(alpha, beta, q);
        const double x2 = x * x;
        T[i] = x;
        E[i] = fma(chi * a_r, x2 * x2, er) * inv1;
    }
}

void launch_exchange(long long n, const double* rho, double* T, double* E, Opacity op,
                     double dtc, double a_r, double cv, unsigned* err, cudaStream_t s) {
    if (n <= 0) return;
    const int block = 256;
    long long nb = (n + block - 1) / block;
    if (nb > 152 * 32) nb = 152 * 32;
    k_exchange<<<(int)nb, block, 0, s>>>(n, rho, T, E, op, dtc, a_r, cv, err);
}

// ----------------------------------------------------------------- limiter
struct BcOff {
    long long off[6];   // offset of each Dirichlet face block in E_bc (-1: not Dirichlet)
};

__device__ __forceinline__ long long face_index(const Lvl& L, int d, int i, int j, int k) {
    if (d == 0) return (long long)k * L.n[1] + j;
    if (d == 1) return (long long)k * L.n[0] + i;
    return (long long)j * L.n[0] + i;
}

__device__ __forceinline__ long long lin(const Lvl& L, int i, int j, int k) {
    return ((long long)k * L.n[1] + j) * L.n[0] + i;
}

// E at offset o (|o| <= 2) from cell (i,j,k) along axis d, with ghost values:
// periodic wrap, Neumann even mirror, Dirichlet odd reflection about the face value.
__device__ __forceinline__ double fetch_E(const Lvl& L, const double* __restrict__ E,
                                          const double* __restrict__ Ebc, const BcOff& bo,
                                          int i, int j, int k, int d, int o) {
    int c[3] = {i, j, k};
    const int n = L.n[d];
    int m = c[d] + o;
    if (m >= 0 && m < n) {
        c[d] = m;
        return E[lin(L, c[0], c[1], c[2])];
    }
    int kind, side, mirror;
    if (m < 0) {
        kind = L.bclo[d];
        side = 0;
        mirror = -m - 1;            // E_{-k} pairs with E_{k-1}
        if (kind == FLD_BC_PERIODIC) mirror = m + n;
    } else {
        kind = L.bchi[d];
        side = 1;
        mirror = 2 * n - 1 - m;     // E_{n-1+k} pairs with E_{n-k}
        if (kind == FLD_BC_PERIODIC) mirror = m - n;
    }
    const long long fi = face_index(L, d, i, j, k);
    c[d] = mirror;
    const double v = E[lin(L, c[0], c[1], c[2])];
    if (kind == FLD_BC_DIRICHLET) return 2.0 * Ebc[bo.off[2 * d + side] + fi] - v;
    return v;
}

__global__ void k_limiter(Lvl L, double3 inv12h, const double* __restrict__ E,
                          const double* __restrict__ rho, const double* __restrict__ T,
                          const double* __restrict__ Ebc, BcOff bo, Opacity op, double c,
                          int mode, double* __restrict__ D, double* __restrict__ lam,
                          unsigned* err) {
    const double ih[3] = {inv12h.x, inv12h.y, inv12h.z};
    const int nrows = L.n[1] * L.n[2];
    for (int rw = blockIdx.x; rw < nrows; rw += gridDim.x)
    for (int i = threadIdx.x; i < L.n[0]; i += blockDim.x) {
        const int j = rw % L.n[1], k = rw / L.n[1];
        const long long p = (long long)rw * L.n[0] + i;
        const double Ec = E[p], r = rho[p];
        const double t = (op.kind == FLD_OPACITY_CONST) ? 1.0 : T[p];
        const double kap = opacity_eval(op, r, t);
        if (!(pos_finite(Ec) && pos_finite(r) && pos_finite(t) && pos_finite(kap))) {
            atomicOr(err, ERRBIT_DOMAIN);
            continue;
        }
        const double kr = kap * r;
        double lm = 1.0 / 3.0;
        if (mode == FLD_LIMITER_LP) {
            double g2 = 0.0;
            for (int d = 0; d < L.ndim; ++d) {
                const double em2 = fetch_E(L, E, Ebc, bo, i, j, k, d, -2);
                const double em1 = fetch_E(L, E, Ebc, bo, i, j, k, d, -1);
                const double ep1 = fetch_E(L, E, Ebc, bo, i, j, k, d, 1);
                const double ep2 = fetch_E(L, E, Ebc, bo, i, j, k, d, 2);
                const double g = ((em2 - 8.0 * em1) + 8.0 * ep1 - ep2) * ih[d];
                g2 = fma(g, g, g2);
            }
            // R = |grad E| / (kappa rho E), lambda = (2 + R)/(6 + 3R + R^2) and
            // D = c lambda / (kappa rho) = c lambda E v with v = 1/(kappa rho E): two
            // reciprocals and one square root, by FP32-seeded Newton-Raphson where the
            // operands allow it (FP64 issues at a small fraction of the FP32 rate).
            const double m = kr * Ec;
            if (in_f32_range(m) && (g2 == 0.0 || in_f32_range(g2))) {
                const double v = rcp_nr(m);
                const double R = g2 > 0.0 ? g2 * rsqrt_nr(g2, 2) * v : 0.0;
                const double P = 2.0 + R, Q = fma(R, R + 3.0, 6.0);
                const double rQ = in_f32_range(Q) ? rcp_nr(Q) : 1.0 / Q;
                lm = P * rQ;
                D[p] = c * lm * (Ec * v);
                if (lam) lam[p] = lm;
                continue;
            }
            const double R = sqrt(g2) / m;
            lm = (2.0 + R) / (6.0 + 3.0 * R + R * R);
        }
        D[p] = in_f32_range(kr) ? c * lm * rcp_nr(kr) : c * lm / kr;
        if (lam) lam[p] = lm;
    }
}

void launch_limiter(const Lvl& L, const double* h, const double* E, const double* rho,
                    const double* T, const double* E_bc, const long long* bc_off, Opacity op,
                    double c, int mode, double* D, double* lam, unsigned* err, cudaStream_t s) {
    BcOff bo;
    for (int q = 0; q < 6; ++q) bo.off[q] = bc_off[q];
    double3 ih = make_double3(1.0 / (12.0 * h[0]), L.ndim > 1 ? 1.0 / (12.0 * h[1]) : 0.0,
                              L.ndim > 2 ? 1.0 / (12.0 * h[2]) : 0.0);
    const int block = 256;
    const int nb = (int)std::min<long long>((long long)L.n[1] * L.n[2], 152 * 64);
    k_limiter<<<nb, block, 0, s>>>(L, ih, E, rho, T, E_bc, bo, op, c, mode, D, lam, err);
}

}  // namespace fld
