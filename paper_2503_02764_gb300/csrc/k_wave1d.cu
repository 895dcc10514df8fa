// Kernels of the one-dimensional radiation-MHD wave step (Sect. 3 scheme, Sect. 4.3
// tests): primitive variables, WENO3 + HLL interface fluxes, the Runge-Kutta stage
// update with the explicit coupling sources, the exchange's energy feedback and the
// CFL signal speed. State arrays are variable-major [8][n]: rho, rho v_x, rho v_y,
// rho v_z, B_y, B_z, e (total gas energy), E; B_x is a constant.
#include <math_constants.h>

#include "fld_wave1d.cuh"

namespace fld {

namespace {

constexpr int W1_THREADS = 256;

// conservative <-> primitive (rho, v_x, v_y, v_z, B_y, B_z, p, E)
__device__ __forceinline__ void to_prim(const double* U, double Bx, double g, double* W) {
    const double rho = U[0];
    const double vx = U[1] / rho, vy = U[2] / rho, vz = U[3] / rho;
    W[0] = rho;
    W[1] = vx;
    W[2] = vy;
    W[3] = vz;
    W[4] = U[4];
    W[5] = U[5];
    W[6] = (g - 1.0) * (U[6] - 0.5 * rho * (vx * vx + vy * vy + vz * vz) -
                        0.5 * (Bx * Bx + U[4] * U[4] + U[5] * U[5]));
    W[7] = U[7];
}

__device__ __forceinline__ void to_cons(const double* W, double Bx, double g, double* U) {
    const double rho = W[0], vx = W[1], vy = W[2], vz = W[3];
    U[0] = rho;
    U[1] = rho * vx;
    U[2] = rho * vy;
    U[3] = rho * vz;
    U[4] = W[4];
    U[5] = W[5];
    U[6] = W[6] / (g - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) +
           0.5 * (Bx * Bx + W[4] * W[4] + W[5] * W[5]);
    U[7] = W[7];
}

// x-fluxes of the MHD equations and of E v_x (the advection term of the E equation)
__device__ __forceinline__ void phys_flux(const double* W, double Bx, double g, double* F) {
    const double rho = W[0], vx = W[1], vy = W[2], vz = W[3], By = W[4], Bz = W[5];
    const double p = W[6];
    const double B2 = Bx * Bx + By * By + Bz * Bz;
    const double pt = p + 0.5 * B2;
    const double e = p / (g - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * B2;
    const double Bv = Bx * vx + By * vy + Bz * vz;
    F[0] = rho * vx;
    F[1] = rho * vx * vx + pt - Bx * Bx;
    F[2] = rho * vx * vy - Bx * By;
    F[3] = rho * vx * vz - Bx * Bz;
    F[4] = vx * By - Bx * vy;
    F[5] = vx * Bz - Bx * vz;
    F[6] = (e + pt) * vx - Bv * Bx;
    F[7] = W[7] * vx;
}

// fast magnetosonic speed from the gas sound speed sqrt(gamma p / rho)
__device__ __forceinline__ double fast_speed(const double* W, double Bx, double g) {
    const double rho = W[0];
    const double cs2 = g * W[6] / rho;
    const double va2 = (Bx * Bx + W[4] * W[4] + W[5] * W[5]) / rho;
    const double vax2 = Bx * Bx / rho;
    const double s = cs2 + va2;
    return sqrt(0.5 * (s + sqrt(fmax(s * s - 4.0 * cs2 * vax2, 0.0))));
}

// WENO3 states on both sides of the face between q0 and qp: two two-cell stencils per
// side with linear weights 1/3 and 2/3 and Jiang-Shu nonlinear weights; the smoothness
// indicators are divided by the largest square of the four cells (unit-free).
__device__ __forceinline__ void weno3(double qm, double q0, double qp, double qpp, double& qL,
                                      double& qR) {
    const double eps = 1e-6;
    const double scale = fmax(fmax(qm * qm, q0 * q0), fmax(qp * qp, qpp * qpp)) + 1e-300;
    const double dm = q0 - qm, dc = qp - q0, dp = qpp - qp;
    const double bm = eps + dm * dm / scale, bc = eps + dc * dc / scale, bp = eps + dp * dp / scale;
    const double a0 = (1.0 / 3.0) / (bm * bm), a1 = (2.0 / 3.0) / (bc * bc);
    qL = (a0 * (1.5 * q0 - 0.5 * qm) + a1 * (0.5 * q0 + 0.5 * qp)) / (a0 + a1);
    const double b0 = (1.0 / 3.0) / (bp * bp), b1 = (2.0 / 3.0) / (bc * bc);
    qR = (b0 * (1.5 * qp - 0.5 * qpp) + b1 * (0.5 * q0 + 0.5 * qp)) / (b0 + b1);
}

// driving wave at cell centre x and time t, primitive variables
__device__ __forceinline__ void drive_prim(const Wave1dDev& P, double x, double t, double* W) {
    const double s = sin(P.k * x - P.omega * t);
#pragma unroll
    for (int v = 0; v < 8; ++v) W[v] = P.W0[v] + P.hat[v] * s;
}

// primitive state of cell c: the driving wave left of the grid, zero gradient right of it
__device__ __forceinline__ void cell_prim(const Wave1dDev& P, const double* __restrict__ U,
                                          int c, double t, double* W) {
    if (c < 0) {
        drive_prim(P, (c + 0.5) * P.dx, t, W);
        return;
    }
    if (c >= P.n) c = P.n - 1;
    double u[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) u[v] = U[(long long)v * P.n + c];
    to_prim(u, P.Bx, P.gamma, W);
}

__global__ void k_w1_prim(Wave1dDev P, const double* __restrict__ U, double* __restrict__ rho,
                          double* __restrict__ vx, double* __restrict__ T,
                          double* __restrict__ T0, double* __restrict__ E) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    double W[8];
    cell_prim(P, U, i, 0.0, W);
    const double Tg = W[6] / (W[0] * P.R_gas);
    rho[i] = W[0];
    vx[i] = W[1];
    T[i] = Tg;
    if (T0) T0[i] = Tg;
    E[i] = W[7];
}

// one thread per face j = 0 .. n (between cells j-1 and j)
__global__ void k_w1_iface(Wave1dDev P, const double* __restrict__ U, double t,
                           double* __restrict__ Fi) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > P.n) return;
    double Wm[8], W0[8], Wp[8], Wpp[8];
    cell_prim(P, U, j - 2, t, Wm);
    cell_prim(P, U, j - 1, t, W0);
    cell_prim(P, U, j, t, Wp);
    cell_prim(P, U, j + 1, t, Wpp);
    double WL[8], WR[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) weno3(Wm[v], W0[v], Wp[v], Wpp[v], WL[v], WR[v]);
    double UL[8], UR[8], FL[8], FR[8];
    to_cons(WL, P.Bx, P.gamma, UL);
    to_cons(WR, P.Bx, P.gamma, UR);
    phys_flux(WL, P.Bx, P.gamma, FL);
    phys_flux(WR, P.Bx, P.gamma, FR);
    const double cL = fast_speed(WL, P.Bx, P.gamma), cR = fast_speed(WR, P.Bx, P.gamma);
    const double SL = fmin(fmin(WL[1] - cL, WR[1] - cR), 0.0);
    const double SR = fmax(fmax(WL[1] + cL, WR[1] + cR), 0.0);
    const long long m = P.n + 1;
#pragma unroll
    for (int v = 0; v < 8; ++v)
        Fi[v * m + j] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
}

// Uout = a U0 + b (Uin + dt L(Uin)), L = -dF/dx + (0, f_r, 0, 0, 0, 0, v.f_r, -P:grad v);
// the driven cells then take the driving wave at t_stage. Uout may alias U0.
__global__ void k_w1_stage(Wave1dDev P, const double* U0, const double* __restrict__ Uin,
                           double* Uout, const double* __restrict__ Fi,
                           const double* __restrict__ fr, const double* __restrict__ vfr,
                           const double* __restrict__ pt, double a, double b, double dt,
                           double t_stage) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const long long n = P.n, m = P.n + 1;
    if (i < P.nd) {
        double W[8], u[8];
        drive_prim(P, (i + 0.5) * P.dx, t_stage, W);
        to_cons(W, P.Bx, P.gamma, u);
#pragma unroll
        for (int v = 0; v < 8; ++v) Uout[v * n + i] = u[v];
        return;
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        double dU = -(Fi[v * m + i + 1] - Fi[v * m + i]) / P.dx;
        if (v == 1) dU += fr[i];
        if (v == 6) dU += vfr[i];
        if (v == 7) dU -= pt[i];
        Uout[v * n + i] = a * U0[v * n + i] + b * (Uin[v * n + i] + dt * dU);
    }
}

// L(Uin) = -dF/dx + (0, f_r, 0, 0, 0, 0, v.f_r, -P:grad v), every cell (the driven ones are
// reset by whatever combines it)
__global__ void k_w1_rhs(Wave1dDev P, const double* __restrict__ Fi, const double* __restrict__ fr,
                         const double* __restrict__ vfr, const double* __restrict__ pt,
                         double* __restrict__ Lout) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const long long n = P.n, m = P.n + 1;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        double dU = -(Fi[v * m + i + 1] - Fi[v * m + i]) / P.dx;
        if (v == 1) dU += fr[i];
        if (v == 6) dU += vfr[i];
        if (v == 7) dU -= pt[i];
        Lout[v * n + i] = dU;
    }
}

// Uout = U0 + dt (c1 L1 + c2 L2 + c3 L3) + dt (d2 G2 + d3 G3), the G's ([2][n]: gas energy,
// E) entering variables 6 and 7; null operands have zero weight. Driven cells take the
// driving wave at t_stage. Uout may alias U0.
__global__ void k_w1_comb(Wave1dDev P, const double* U0, const double* __restrict__ L1,
                          const double* __restrict__ L2, const double* __restrict__ L3,
                          double c1, double c2, double c3, const double* __restrict__ G2,
                          const double* __restrict__ G3, double d2, double d3, double dt,
                          double* Uout, double t_stage) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const long long n = P.n;
    if (i < P.nd) {
        double W[8], u[8];
        drive_prim(P, (i + 0.5) * P.dx, t_stage, W);
        to_cons(W, P.Bx, P.gamma, u);
#pragma unroll
        for (int v = 0; v < 8; ++v) Uout[v * n + i] = u[v];
        return;
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        double inc = 0.0;
        if (L1) inc += c1 * L1[v * n + i];
        if (L2) inc += c2 * L2[v * n + i];
        if (L3) inc += c3 * L3[v * n + i];
        if (v >= 6) {
            if (G2) inc += d2 * G2[(v - 6) * n + i];
            if (G3) inc += d3 * G3[(v - 6) * n + i];
        }
        Uout[v * n + i] = U0[v * n + i] + dt * inc;
    }
}

// the implicit increment of a stage: G = (Uafter - Ubefore) / tau for variables 6, 7
__global__ void k_w1_incr(Wave1dDev P, const double* __restrict__ Ua,
                          const double* __restrict__ Ub, double inv_tau, double* __restrict__ G) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const long long n = P.n;
    G[i] = (Ua[6 * n + i] - Ub[6 * n + i]) * inv_tau;
    G[n + i] = (Ua[7 * n + i] - Ub[7 * n + i]) * inv_tau;
}

// after the FLD substep: e += rho R_gas (T' - T) / (gamma - 1), E = E'; driven cells reset
__global__ void k_w1_post(Wave1dDev P, double* __restrict__ U, const double* __restrict__ rho,
                          const double* __restrict__ T0, const double* __restrict__ T,
                          const double* __restrict__ E, double t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const long long n = P.n;
    if (i < P.nd) {
        double W[8], u[8];
        drive_prim(P, (i + 0.5) * P.dx, t, W);
        to_cons(W, P.Bx, P.gamma, u);
#pragma unroll
        for (int v = 0; v < 8; ++v) U[v * n + i] = u[v];
        return;
    }
    U[6 * n + i] += rho[i] * P.R_gas * (T[i] - T0[i]) / (P.gamma - 1.0);
    U[7 * n + i] = E[i];
}

// max over cells of |v_x| + c_f, as the bits of a non-negative double (integer order)
__global__ void k_w1_speed(Wave1dDev P, const double* __restrict__ U,
                           unsigned long long* __restrict__ out) {
    __shared__ double sh[W1_THREADS / 32];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        double W[8];
        cell_prim(P, U, i, 0.0, W);
        const double c = fabs(W[1]) + fast_speed(W, P.Bx, P.gamma);
        // a cell with rho <= 0, p <= 0 or a non-finite speed makes the maximum +inf, which
        // the host reports as a domain error (fmax alone would drop a NaN)
        const bool ok = W[0] > 0.0 && W[6] > 0.0 && c < CUDART_INF;
        s = ok ? fmax(s, c) : CUDART_INF;
    }
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < W1_THREADS / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
    }
}

int blocks_for(long long n) { return (int)((n + W1_THREADS - 1) / W1_THREADS); }

}  // namespace

void launch_w1_prim(const Wave1dDev& P, const double* U, double* rho, double* vx, double* T,
                    double* T0, double* E, cudaStream_t s) {
    k_w1_prim<<<blocks_for(P.n), W1_THREADS, 0, s>>>(P, U, rho, vx, T, T0, E);
}

void launch_w1_iface(const Wave1dDev& P, const double* U, double t, double* Fi, cudaStream_t s) {
    k_w1_iface<<<blocks_for(P.n + 1), W1_THREADS, 0, s>>>(P, U, t, Fi);
}

void launch_w1_stage(const Wave1dDev& P, const double* U0, const double* Uin, double* Uout,
                     const double* Fi, const double* fr, const double* vfr, const double* pt,
                     double a, double b, double dt, double t_stage, cudaStream_t s) {
    k_w1_stage<<<blocks_for(P.n), W1_THREADS, 0, s>>>(P, U0, Uin, Uout, Fi, fr, vfr, pt, a, b,
                                                       dt, t_stage);
}

void launch_w1_post(const Wave1dDev& P, double* U, const double* rho, const double* T0,
                    const double* T, const double* E, double t, cudaStream_t s) {
    k_w1_post<<<blocks_for(P.n), W1_THREADS, 0, s>>>(P, U, rho, T0, T, E, t);
}

void launch_w1_rhs(const Wave1dDev& P, const double* Fi, const double* fr, const double* vfr,
                   const double* pt, double* Lout, cudaStream_t s) {
    k_w1_rhs<<<blocks_for(P.n), W1_THREADS, 0, s>>>(P, Fi, fr, vfr, pt, Lout);
}

void launch_w1_comb(const Wave1dDev& P, const double* U0, const double* L1, const double* L2,
                    const double* L3, double c1, double c2, double c3, const double* G2,
                    const double* G3, double d2, double d3, double dt, double* Uout,
                    double t_stage, cudaStream_t s) {
    k_w1_comb<<<blocks_for(P.n), W1_THREADS, 0, s>>>(P, U0, L1, L2, L3, c1, c2, c3, G2, G3, d2,
                                                      d3, dt, Uout, t_stage);
}

void launch_w1_incr(const Wave1dDev& P, const double* Ua, const double* Ub, double inv_tau,
                    double* G, cudaStream_t s) {
    k_w1_incr<<<blocks_for(P.n), W1_THREADS, 0, s>>>(P, Ua, Ub, inv_tau, G);
}

void launch_w1_speed(const Wave1dDev& P, const double* U, unsigned long long* out,
                     cudaStream_t s) {
    const int nb = std::min(blocks_for(P.n), num_sms() * 4);
    k_w1_speed<<<nb, W1_THREADS, 0, s>>>(P, U, out);
}

}  // namespace fld
