// Pointwise kernels of the FLD substep: the gas-radiation exchange quartic and the
// flux limiter (Levermore-Pomraning, 4th-order 5-point gradient).
#include "fld_internal.cuh"

namespace fld {

// ----------------------------------------------------------------- exchange
// Backward Euler on de/dt = +qdot, dE/dt = -qdot with qdot = c kappa rho (E - a_r T^4)
// (Eqs. heating, qdot). Eliminating E' leaves, per cell,
//   f(T) = alpha T + beta T^4 - q = 0,  alpha = rho c_v, beta = a_r chi/(1+chi),
//   q = e + chi E/(1+chi),  chi = dt c kappa rho,
// increasing and convex for T > 0 with f(0) < 0: one positive root, bounded above by
// min(q/alpha, (q/beta)^(1/4)). Newton from that bound decreases monotonically to the
// root, so a fixed iteration cap with a relative-step stop is safe.
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
        const double e = alpha * t;
        const double w = chi / (1.0 + chi);
        const double beta = w * a_r;
        const double q = fma(w, er, e);
        double x = q / alpha;
        if (beta > 0.0) x = fmin(x, sqrt(sqrt(q / beta)));
        for (int it = 0; it < 100; ++it) {
            const double x2 = x * x;
            const double f = fma(beta * x2, x2, fma(alpha, x, -q));
            const double fp = fma(4.0 * beta * x2, x, alpha);
            const double dx = f / fp;
            x -= dx;
            if (fabs(dx) <= 1e-16 * x) break;
        }
        const double x2 = x * x;
        T[i] = x;
        E[i] = fma(chi * a_r, x2 * x2, er) / (1.0 + chi);
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
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L.ncell;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % L.n[0]);
        const long long q = p / L.n[0];
        const int j = (int)(q % L.n[1]);
        const int k = (int)(q / L.n[1]);
        const double Ec = E[p], r = rho[p];
        const double t = (op.kind == FLD_OPACITY_CONST) ? 1.0 : T[p];
        const double kap = opacity_eval(op, r, t);
        if (!(pos_finite(Ec) && pos_finite(r) && pos_finite(t) && pos_finite(kap))) {
            atomicOr(err, ERRBIT_DOMAIN);
            continue;
        }
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
            const double R = sqrt(g2) / (kap * r * Ec);
            lm = (2.0 + R) / (6.0 + 3.0 * R + R * R);
        }
        D[p] = c * lm / (kap * r);
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
    long long nb = (L.ncell + block - 1) / block;
    if (nb > 152 * 32) nb = 152 * 32;
    k_limiter<<<(int)nb, block, 0, s>>>(L, ih, E, rho, T, E_bc, bo, op, c, mode, D, lam, err);
}

}  // namespace fld
