// Pointwise kernels of the FLD substep: the gas-radiation exchange quartic and the
// flux limiter (Levermore-Pomraning, 4th-order 5-point gradient).
#include <algorithm>

#include "fld_device.cuh"

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

// kr (nullable): kappa rho of every cell, frozen at the step's start by the limiter of the
// same substep; without it kappa is evaluated from (rho, T). DF as for k_limiter.
template <bool DF>
__global__ void __launch_bounds__(256, DF ? 5 : 6) k_exchange(long long n, const double* __restrict__ rho, double* __restrict__ T,
                           double* __restrict__ E, const double* __restrict__ kr, Opacity op,
                           double dtc, double a_r, double cv, int use_df, DfConst K,
                           unsigned* err, double one) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = rho[i];
        double t = T[i], er = E[i];
        const double kri = kr ? kr[i] : 0.0;
        if (kr && !pos_finite(kri)) {
            atomicOr(err, ERRBIT_DOMAIN);
            continue;
        }
        if (DF && use_df && exchange_cell_df(r, t, er, op, K, kri)) {
            T[i] = t;
            E[i] = er;
            continue;
        }
        t = T[i];
        er = E[i];
        if (kr) {
            if (!(pos_finite(r) && pos_finite(t) && pos_finite(er))) {
                atomicOr(err, ERRBIT_DOMAIN);
                continue;
            }
            exchange_cell_kr(r, kri, t, er, dtc, a_r, cv, one);
        } else if (!exchange_cell(r, t, er, op, dtc, a_r, cv)) {
            atomicOr(err, ERRBIT_DOMAIN);
            continue;
        }
        T[i] = t;
        E[i] = er;
    }
}

DfConst make_dfconst(double c, double kappa0, double dtc, double a_r, double cv) {
    DfConst K;
    split_host(c, K.c_h, K.c_l);
    split_host(kappa0, K.kap_h, K.kap_l);
    split_host(dtc, K.dtc_h, K.dtc_l);
    split_host(a_r, K.ar_h, K.ar_l);
    split_host(cv, K.cv_h, K.cv_l);
    return K;
}

void launch_exchange(long long n, const double* rho, double* T, double* E, Opacity op,
                     double dtc, double a_r, double cv, int use_df, unsigned* err, cudaStream_t s,
                     const double* kr) {
    if (n <= 0) return;
    const int block = 256;
    long long nb = (n + block - 1) / block;
    if (nb > num_sms() * 32) nb = num_sms() * 32;
    const DfConst K = make_dfconst(0.0, op.kappa0, dtc, a_r, cv);
    if (use_df)
        k_exchange<true><<<(int)nb, block, 0, s>>>(n, rho, T, E, kr, op, dtc, a_r, cv, use_df, K,
                                                   err, 1.0);
    else
        k_exchange<false><<<(int)nb, block, 0, s>>>(n, rho, T, E, kr, op, dtc, a_r, cv, use_df, K,
                                                    err, 1.0);
}

// ----------------------------------------------------------------- limiter
// E split into FP32 (hi, lo) pairs, once per cell, for the double-FP32 limiter's gradient
__global__ void k_split_df(long long n, const double* __restrict__ v, float* __restrict__ hi,
                           float* __restrict__ lo) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const df d = df_from_double_i(v[p]);
        hi[p] = d.hi;
        lo[p] = d.lo;
    }
}

// kr (nullable): receives kappa rho of every cell, for the exchange of the same substep.
// DF: the double-FP32 cell routine first (FP64 for the cells it declines); the FP64-only
// instantiation carries none of its registers.
template <bool DF>
__global__ void __launch_bounds__(256, DF ? 5 : 6) k_limiter(Lvl L, double3 inv12h, const double* __restrict__ E,
                          const double* __restrict__ rho, const double* __restrict__ T,
                          const double* __restrict__ Ebc, BcOff bo, Opacity op, double c,
                          int mode, int use_df, DfConst K, const float* __restrict__ Eh,
                          const float* __restrict__ El, double* __restrict__ D,
                          double* __restrict__ lam, double* __restrict__ kr, unsigned* err,
                          double one) {
    const double ih[3] = {inv12h.x, inv12h.y, inv12h.z};
    df ihd[3];
    if (DF)
        for (int d = 0; d < 3; ++d) ihd[d] = df_from_double(ih[d]);
    const int nrows = L.n[1] * L.n[2];
    for (int rw = blockIdx.x; rw < nrows; rw += gridDim.x)
        for (int i = threadIdx.x; i < L.n[0]; i += blockDim.x) {
            const int j = rw % L.n[1], k = rw / L.n[1];
            const long long p = (long long)rw * L.n[0] + i;
            double Dv, lm, kv;
            if (DF && use_df && limiter_cell_df(L, ih, E, rho, T, Ebc, bo, op, K, mode, i, j, k, p, Dv, lm,
                                          Eh, El, ihd, kr ? &kv : nullptr)) {
                D[p] = Dv;
                if (lam) lam[p] = lm;
                if (kr) kr[p] = kv;
                continue;
            }
            if (!limiter_cell(L, ih, E, rho, T, Ebc, bo, op, c, mode, i, j, k, p, Dv, lm,
                              kr ? &kv : nullptr, lam != nullptr, one)) {
                atomicOr(err, ERRBIT_DOMAIN);
                continue;
            }
            D[p] = Dv;
            if (lam) lam[p] = lm;
            if (kr) kr[p] = kv;
        }
}

// ----------------------------------------------------------------- coupling terms
// v_c at offset o (|o| <= 2) along axis d: periodic wrap, an even mirror at walls.
__device__ __forceinline__ double fetch_v(const Lvl& L, const double* __restrict__ v, int i,
                                          int j, int k, int d, int o) {
    int c[3] = {i, j, k};
    const int n = L.n[d];
    int m = c[d] + o;
    if (m < 0) m = L.bclo[d] == FLD_BC_PERIODIC ? m + n : -m - 1;
    else if (m >= n) m = L.bchi[d] == FLD_BC_PERIODIC ? m - n : 2 * n - 1 - m;
    c[d] = m;
    return v[lin(L, c[0], c[1], c[2])];
}

// Explicit coupling terms of one cell, in FP64 from the limiter's gradient: F = -D grad E,
// f_r = -lambda grad E, f = lambda + lambda^2 R^2, and with v: v . f_r and
// P : grad v, P = E ((1 - f) I + (3f - 1) n n) / 2, n = grad E / |grad E|.
__global__ void k_coupling(Lvl L, double3 inv12h, double3 inv12hv, const double* __restrict__ E,
                           const double* __restrict__ rho, const double* __restrict__ T,
                           const double* __restrict__ Ebc, BcOff bo, Opacity op, double c,
                           int mode, const double* __restrict__ v, double* __restrict__ F,
                           double* __restrict__ fr, double* __restrict__ fe,
                           double* __restrict__ vfr, double* __restrict__ pt, unsigned* err) {
    const double ih[3] = {inv12h.x, inv12h.y, inv12h.z};
    const double ihv[3] = {inv12hv.x, inv12hv.y, inv12hv.z};
    const int nd = L.ndim;
    const long long nc = L.ncell;
    const int nrows = L.n[1] * L.n[2];
    for (int rw = blockIdx.x; rw < nrows; rw += gridDim.x)
        for (int i = threadIdx.x; i < L.n[0]; i += blockDim.x) {
            const int j = rw % L.n[1], k = rw / L.n[1];
            const long long p = (long long)rw * L.n[0] + i;
            const double Ec = E[p], r = rho[p];
            const double t = op.kind == FLD_OPACITY_CONST ? 1.0 : T[p];
            if (!(pos_finite(Ec) && pos_finite(r) && pos_finite(t))) {
                atomicOr(err, ERRBIT_DOMAIN);
                continue;
            }
            const double kap = opacity_eval(op, r, t);
            if (!pos_finite(kap)) {
                atomicOr(err, ERRBIT_DOMAIN);
                continue;
            }
            double g[3] = {0.0, 0.0, 0.0};
            double g2 = 0.0;
            for (int d = 0; d < nd; ++d) {
                const double em2 = fetch_E(L, E, Ebc, bo, i, j, k, d, -2);
                const double em1 = fetch_E(L, E, Ebc, bo, i, j, k, d, -1);
                const double ep1 = fetch_E(L, E, Ebc, bo, i, j, k, d, 1);
                const double ep2 = fetch_E(L, E, Ebc, bo, i, j, k, d, 2);
                g[d] = ((em2 - 8.0 * em1) + 8.0 * ep1 - ep2) * ih[d];
                g2 = fma(g[d], g[d], g2);
            }
            const double gn = sqrt(g2);
            const double kr = kap * r;
            const double R = gn / (kr * Ec);
            const double lam = mode == FLD_LIMITER_LP        ? (2.0 + R) / (6.0 + 3.0 * R + R * R)
                               : mode == FLD_LIMITER_MINERBO ? minerbo_lambda(R)
                                                             : 1.0 / 3.0;
            const double D = c * lam / kr;
            const double f = lam + lam * lam * R * R;
            double vf = 0.0;
            for (int d = 0; d < nd; ++d) {
                const double frd = -lam * g[d];
                if (F) F[d * nc + p] = -D * g[d];
                if (fr) fr[d * nc + p] = frd;
                if (v) vf = fma(v[d * nc + p], frd, vf);
            }
            if (fe) fe[p] = f;
            if (v && vfr) vfr[p] = vf;
            if (v && pt) {
                double n[3] = {0.0, 0.0, 0.0};
                if (gn > 0.0)
                    for (int d = 0; d < nd; ++d) n[d] = g[d] / gn;
                const double a = 0.5 * (1.0 - f), bq = 0.5 * (3.0 * f - 1.0);
                double acc = 0.0;
                for (int a1 = 0; a1 < nd; ++a1) {            // velocity component
                    const double* vi = v + a1 * nc;
                    for (int a2 = 0; a2 < nd; ++a2) {        // derivative axis
                        const double gv = ((fetch_v(L, vi, i, j, k, a2, -2) -
                                            8.0 * fetch_v(L, vi, i, j, k, a2, -1)) +
                                           8.0 * fetch_v(L, vi, i, j, k, a2, 1) -
                                           fetch_v(L, vi, i, j, k, a2, 2)) * ihv[a2];
                        const double Pij = ((a1 == a2 ? a : 0.0) + bq * n[a1] * n[a2]) * Ec;
                        acc = fma(Pij, gv, acc);
                    }
                }
                pt[p] = acc;
            }
        }
}

void launch_coupling(const Lvl& L, const double* h, const double* E, const double* rho,
                     const double* T, const double* E_bc, const long long* bc_off, Opacity op,
                     double c, int mode, const double* v, double* F, double* fr, double* fe,
                     double* vfr, double* pt, unsigned* err, cudaStream_t s) {
    BcOff bo;
    for (int q = 0; q < 6; ++q) bo.off[q] = bc_off[q];
    const double3 ih = make_double3(1.0 / (12.0 * h[0]), L.ndim > 1 ? 1.0 / (12.0 * h[1]) : 0.0,
                                    L.ndim > 2 ? 1.0 / (12.0 * h[2]) : 0.0);
    const int nb = (int)std::min<long long>((long long)L.n[1] * L.n[2], num_sms() * 64);
    k_coupling<<<nb, 256, 0, s>>>(L, ih, ih, E, rho, T, E_bc, bo, op, c, mode, v, F, fr, fe, vfr,
                                  pt, err);
}

void launch_split_df(long long n, const double* v, float* hi, float* lo, cudaStream_t s) {
    const long long nb = std::min<long long>((n + 255) / 256, num_sms() * 32);
    k_split_df<<<(int)nb, 256, 0, s>>>(n, v, hi, lo);
}

void launch_limiter(const Lvl& L, const double* h, const double* E, const double* rho,
                    const double* T, const double* E_bc, const long long* bc_off, Opacity op,
                    double c, int mode, int use_df, double* D, double* lam, unsigned* err,
                    cudaStream_t s, float* Eh, float* El, double* kr) {
    BcOff bo;
    for (int q = 0; q < 6; ++q) bo.off[q] = bc_off[q];
    double3 ih = make_double3(1.0 / (12.0 * h[0]), L.ndim > 1 ? 1.0 / (12.0 * h[1]) : 0.0,
                              L.ndim > 2 ? 1.0 / (12.0 * h[2]) : 0.0);
    const int block = 256;
    const int nb = (int)std::min<long long>((long long)L.n[1] * L.n[2], num_sms() * 64);
    const DfConst K = make_dfconst(c, op.kappa0, 0.0, 0.0, 0.0);
    if (!(use_df && mode != FLD_LIMITER_DIFFUSION)) Eh = El = nullptr;
    if (use_df)
        k_limiter<true><<<nb, block, 0, s>>>(L, ih, E, rho, T, E_bc, bo, op, c, mode, use_df, K,
                                             Eh, El, D, lam, kr, err, 1.0);
    else
        k_limiter<false><<<nb, block, 0, s>>>(L, ih, E, rho, T, E_bc, bo, op, c, mode, use_df, K,
                                              Eh, El, D, lam, kr, err, 1.0);
}

}  // namespace fld
