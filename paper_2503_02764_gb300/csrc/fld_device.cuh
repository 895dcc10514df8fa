// Per-cell device routines shared by the grid kernels and the batched persistent
// kernel: index decoding, the level operator's stencil, linear prolongation weights,
// block reductions, limiter ghost values and the exchange root.
#pragma once
#include "df64.cuh"
#include "fld_internal.cuh"

namespace fld {

__device__ __forceinline__ void decode(const Lvl& L, long long p, int& i, int& j, int& k) {
    const int pp = (int)p;
    i = pp % L.n[0];
    const int q = pp / L.n[0];
    j = q % L.n[1];
    k = q / L.n[1];
}

// Off-diagonal sum and diagonal excess of the level operator at cell p:
//   sw  = sum of face weights (+ 2 K_p w_d per Dirichlet face),  acc = sum w_f x_q,
// so (A x)_p = (1 + sw) x_p - acc. FM >= 0 fixes the face mean at compile time (the
// level's fm otherwise).
template <typename T, int FM = -1>
__device__ __forceinline__ void stencil(const Lvl& L, const T* __restrict__ K,
                                        const T* __restrict__ x, int i, int j, int k, long long p64,
                                        T& sw, T& acc) {
    const int fm = FM < 0 ? L.fm : FM;
    // cell indices fit in 32 bits (the handle rejects grids of 2^31 cells or more)
    const int p = (int)p64;
    const T Kc = K[fld_at(p, L.ncell)];
    const int c[3] = {i, j, k};
    int stride = 1;
    sw = T(0);
    acc = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d < L.ndim) {
            const int n = L.n[d];
            const T wd = wgt<T>(L, d);
            // low face
            int q = -1;
            if (c[d] > 0) q = p - stride;
            else if (L.bclo[d] == FLD_BC_PERIODIC) q = p + (n - 1) * stride;
            if (q >= 0) {
                q = (int)fld_at(q, L.ncell);
                const T w = fmean(Kc, K[q], fm) * wd;
                sw += w;
                acc += w * x[q];
            } else if (L.bclo[d] == FLD_BC_DIRICHLET) {
                sw += T(2) * Kc * wd;
            }
            // high face
            q = -1;
            if (c[d] < n - 1) q = p + stride;
            else if (L.bchi[d] == FLD_BC_PERIODIC) q = p - (n - 1) * stride;
            if (q >= 0) {
                q = (int)fld_at(q, L.ncell);
                const T w = fmean(Kc, K[q], fm) * wd;
                sw += w;
                acc += w * x[q];
            } else if (L.bchi[d] == FLD_BC_DIRICHLET) {
                sw += T(2) * Kc * wd;
            }
            stride *= n;
        }
    }
}

template <typename T>
__device__ __forceinline__ T div_fast(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float div_fast<float>(float a, float b) { return __fdividef(a, b); }

// Cell-centred linear prolongation: along a coarsened axis a fine cell takes 3/4 of
// its parent I = i/2 and 1/4 of the coarse neighbour on its side (I-1 for an even i,
// I+1 for an odd one); tensor product over the axes. A missing neighbour at a wall is
// the mirror value: +e_I (Neumann, zero flux) or -e_I (Dirichlet, zero correction).
struct Interp {
    int idx[2];
    float wt[2];
};

__device__ __forceinline__ Interp interp1(int i, int nf, int nc, int lo_bc, int hi_bc,
                                          int constant = 0) {
    Interp r;
    if (constant && nc != nf) {   // piecewise constant: the parent's value
        r.idx[0] = r.idx[1] = i >> 1;
        r.wt[0] = 1.f;
        r.wt[1] = 0.f;
        return r;
    }
    if (nc == nf) {           // axis not coarsened
        r.idx[0] = r.idx[1] = i;
        r.wt[0] = 1.f;
        r.wt[1] = 0.f;
        return r;
    }
    const int I = i >> 1;
    int J = (i & 1) ? I + 1 : I - 1;
    float sgn = 1.f;
    if (J < 0 || J >= nc) {
        const int kind = (J < 0) ? lo_bc : hi_bc;
        if (kind == FLD_BC_PERIODIC) J = (J + nc) % nc;
        else {
            sgn = (kind == FLD_BC_DIRICHLET) ? -1.f : 1.f;
            J = I;
        }
    }
    r.idx[0] = I;
    r.idx[1] = J;
    r.wt[0] = 0.75f;
    r.wt[1] = 0.25f * sgn;
    return r;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}


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
        return E[fld_at(lin(L, c[0], c[1], c[2]), L.ncell)];
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
    const double v = E[fld_at(lin(L, c[0], c[1], c[2]), L.ncell)];
    if (kind == FLD_BC_DIRICHLET) return 2.0 * Ebc[bo.off[2 * d + side] + fi] - v;
    return v;
}

// Minerbo's limiter (the paper implements it but does not print it; the published closed
// form): 2 / (3 + sqrt(9 + 12 R^2)) for R <= 3/2, 1 / (1 + R + sqrt(1 + 2R)) above; both
// branches give 2/9 and the same slope at R = 3/2, and lambda R -> 1 as R -> infinity.
__device__ __forceinline__ double minerbo_lambda(double R) {
    return R <= 1.5 ? 2.0 / (3.0 + sqrt(fma(12.0 * R, R, 9.0)))
                    : 1.0 / ((1.0 + R) + sqrt(fma(2.0, R, 1.0)));
}

__device__ __forceinline__ df minerbo_lambda_df(df R) {
    if (R.hi <= 1.5f)
        return df_div({2.f, 0.f}, df_add_f(df_sqrt(df_add_f(df_mul_f(df_mul(R, R), 12.f), 9.f)), 3.f));
    return df_div({1.f, 0.f}, df_add(df_add_f(R, 1.f), df_sqrt(df_add_f(df_mul_f(R, 2.f), 1.f))));
}

// fetch_E from the double-FP32 split copy (Eh, El) of E: the same ghost rules, a Dirichlet
// ghost 2 E_b - E_mirror formed in FP64 and split.
__device__ __forceinline__ df fetch_Edf(const Lvl& L, const float* __restrict__ Eh,
                                        const float* __restrict__ El,
                                        const double* __restrict__ E,
                                        const double* __restrict__ Ebc, const BcOff& bo, int i,
                                        int j, int k, int d, int o) {
    int c[3] = {i, j, k};
    const int n = L.n[d];
    const int m = c[d] + o;
    if (m >= 0 && m < n) {
        c[d] = m;
        const long long q = lin(L, c[0], c[1], c[2]);
        return {Eh[q], El[q]};
    }
    int kind, side, mirror;
    if (m < 0) {
        kind = L.bclo[d];
        side = 0;
        mirror = kind == FLD_BC_PERIODIC ? m + n : -m - 1;
    } else {
        kind = L.bchi[d];
        side = 1;
        mirror = kind == FLD_BC_PERIODIC ? m - n : 2 * n - 1 - m;
    }
    c[d] = mirror;
    const long long q = lin(L, c[0], c[1], c[2]);
    if (kind == FLD_BC_DIRICHLET)
        return df_from_double(2.0 * Ebc[bo.off[2 * d + side] + face_index(L, d, i, j, k)] - E[q]);
    return {Eh[q], El[q]};
}

__device__ __forceinline__ bool f32_ok(double v) { return v > 1e-30 && v < 1e30; }

// Root of alpha T + beta T^4 = q (alpha, q > 0, beta >= 0): Newton in FP32 on a scaled
// form of the quartic (all quantities O(1)) from FP32 images of the coefficients, then
// one FP64 Newton step whose residual is FP64 and whose derivative is the FP32 one (the
// step is ~1e-7 T, so the derivative's 1e-7 relative error leaves ~1e-14 T). The FP32
// images and the seed's FP64 value are converted in integer arithmetic. Coefficients
// outside the FP32 range take a plain FP64 Newton iteration from the upper bound.
__device__ __forceinline__ double exchange_root(double alpha, double beta, double q) {
    const bool bzero = (__double_as_longlong(beta) << 1) == 0;
    if (in_f32_range(alpha) && in_f32_range(q) && (bzero || in_f32_range(beta))) {
        const float af = f32_near_pos(alpha), qf = f32_near_pos(q);
        const float bf = bzero ? 0.f : f32_near_pos(beta);
        const float T1 = qf / af;                       // root if beta were 0
        const float T1sq = T1 * T1;
        const float g = (bf * T1sq) * (T1sq / qf);      // beta T1^4 / q
        if (T1 > 1e-9f && T1 < 1e9f && g < 1e30f) {
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
            const float Tf = x * scale;
            const double T = f64_of_pos(Tf);
            // one FP64 Newton step: FP64 residual, FP32 derivative
            const double T2 = T * T;
            const double f = fma(beta * T2, T2, fma(alpha, T, -q));
            const float fpf = fmaf(4.f * bf * Tf * Tf, Tf, af);
            return fma(-f, f64_of_pos(__frcp_rn(fpf)), T);
        }
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

// ----------------------------------------------------------------- limiter, one cell
// R = |grad E| / (kappa rho E) (Eq. fld_R), lambda = (2 + R)/(6 + 3R + R^2)
// (Eq. fld_lambda), D = c lambda / (kappa rho) (Eq. fld_F), grad E by the 5-point
// 4th-order difference. With a = kappa rho E and g = |grad E| (R = g/a), multiplying the
// limiter's numerator and denominator by a^2 gives
//   D = c E (2a + g) / (6a^2 + 3ag + g^2),
// one square root and one division (FP32-seeded Newton-Raphson where the operands allow
// it): FP64 issues at a small fraction of the FP32 rate here. Minerbo's limiter and
// operands outside the FP32 range take R itself. kr_out receives kappa rho (the exchange
// of the same substep reuses it). Returns false on a domain error.
template <bool kTables = true>
__device__ __forceinline__ bool limiter_cell(const Lvl& L, const double* ih,
                                             const double* __restrict__ E,
                                             const double* __restrict__ rho,
                                             const double* __restrict__ T,
                                             const double* __restrict__ Ebc, const BcOff& bo,
                                             const Opacity& op, double c, int mode, int i, int j,
                                             int k, long long p, double& Dout, double& lmout,
                                             double* kr_out = nullptr, bool want_lm = true,
                                             double one = 1.0) {
    const double Ec = E[p], r = rho[p];
    const double t = (op.kind == FLD_OPACITY_CONST) ? 1.0 : T[p];
    const double kap = opacity_eval<kTables>(op, r, t);
    if (!(pos_finite(Ec) && pos_finite(r) && pos_finite(t) && pos_finite(kap))) return false;
    const double kr = kap * r;
    if (kr_out) *kr_out = kr;
    double lm = 1.0 / 3.0;
    if (mode != FLD_LIMITER_DIFFUSION) {
        double g2 = 0.0;
        // unrolled over the three axes, so that every index into the level and the
        // spacings is a constant (no local-memory copy of them)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= L.ndim) break;
            const double em2 = fetch_E(L, E, Ebc, bo, i, j, k, d, -2);
            const double em1 = fetch_E(L, E, Ebc, bo, i, j, k, d, -1);
            const double ep1 = fetch_E(L, E, Ebc, bo, i, j, k, d, 1);
            const double ep2 = fetch_E(L, E, Ebc, bo, i, j, k, d, 2);
            // (E_-2 - 8 E_-1) + 8 E_+1 - E_+2 as three FMAs (`one` = 1.0 from the kernel's
            // arguments: an FP64 add costs the FP64 pipe twice an FMA's time on this GPU)
            const double g = fma(ep2, -one, fma(8.0, ep1, fma(-8.0, em1, em2))) * ih[d];
            g2 = fma(g, g, g2);
        }
        const double a = kr * Ec;
        const bool gzero = __double_as_longlong(g2) == 0;
        if (mode == FLD_LIMITER_LP && in_f32_range(a) && (gzero || in_f32_range(g2))) {
            const double g = gzero ? 0.0 : sqrt_nr(g2);
            const double den = fma(a, fma(6.0, a, 3.0 * g), g2);
            const double n2 = fma(2.0, a, g);
            if (in_f32_range(den)) {
                Dout = div_nr((c * Ec) * n2, den);
                if (want_lm) lmout = div_nr(a * n2, den);
                return true;
            }
        }
        if (in_f32_range(a) && (gzero || in_f32_range(g2))) {
            const double v = rcp_nr(a);
            const double R = gzero ? 0.0 : sqrt_nr(g2) * v;
            if (mode == FLD_LIMITER_MINERBO) {
                lmout = minerbo_lambda(R);
            } else {
                const double P = 2.0 + R, Q = fma(R, R + 3.0, 6.0);
                const double rQ = in_f32_range(Q) ? rcp_nr(Q) : 1.0 / Q;
                lmout = P * rQ;
            }
            Dout = c * lmout * (Ec * v);
            return true;
        }
        const double R = sqrt(g2) / a;
        lm = mode == FLD_LIMITER_MINERBO ? minerbo_lambda(R) : (2.0 + R) / (6.0 + 3.0 * R + R * R);
    }
    lmout = lm;
    Dout = in_f32_range(kr) ? c * lm * rcp_nr(kr) : c * lm / kr;
    return true;
}

// ----------------------------------------------------------------- exchange, one cell
// Backward Euler on de/dt = +qdot, dE/dt = -qdot (Eqs. heating, qdot), given
// kr = kappa rho (frozen at the step's start): chi = dt c kr, solves
// alpha T' + beta T'^4 = q (exchange_root) with alpha = rho c_v, beta = a_r chi/(1+chi),
// q = alpha T + chi E/(1+chi), and sets E' = (E + chi a_r T'^4)/(1 + chi)
// = E/(1+chi) + beta T'^4. The caller checks r, t, er and kr.
__device__ __forceinline__ void exchange_cell_kr(double r, double kr, double& t, double& er,
                                                 double dtc, double a_r, double cv,
                                                 double one = 1.0) {
    const double chi = dtc * kr;
    const double alpha = r * cv;
    const double d1 = fma(chi, one, 1.0);      // 1 + chi as an FMA (see limiter_cell)
    const double inv1 = in_f32_range(d1) ? rcp_nr(d1) : 1.0 / d1;
    const double w = chi * inv1;
    const double beta = w * a_r;
    const double q = fma(w, er, alpha * t);
    const double x = exchange_root(alpha, beta, q);
    const double x2 = x * x;
    er = fma(beta, x2 * x2, er * inv1);
    t = x;
}

// The same with kappa from (rho, T on entry). Returns false (cell unchanged) on a domain
// error.
template <bool kTables = true>
__device__ __forceinline__ bool exchange_cell(double r, double& t, double& er, const Opacity& op,
                                              double dtc, double a_r, double cv) {
    if (!(pos_finite(r) && pos_finite(t) && pos_finite(er))) return false;
    const double kap = opacity_eval<kTables>(op, r, t);
    if (!pos_finite(kap)) return false;
    exchange_cell_kr(r, kap * r, t, er, dtc, a_r, cv);
    return true;
}

// ----------------------------------------------------------------- double-FP32 variants
// The same limiter and exchange with the FP64 work cut to the gradient and the format
// conversions: every other operation runs as FP32 double-word arithmetic (df64.cuh).
// They return false when a value leaves the window where that arithmetic keeps 48 bits
// (the caller then uses the FP64 routines above).

struct DfConst {        // per-launch constants as (hi, lo) pairs
    float c_h, c_l, kap_h, kap_l, dtc_h, dtc_l, ar_h, ar_l, cv_h, cv_l;
};

// kappa as df: constant, or the Kramers-like law kappa0 rho T^-3.5; false otherwise
__device__ __forceinline__ bool df_opacity(const Opacity& op, const DfConst& K, df rho, df T,
                                           df& kap) {
    const df k0 = {K.kap_h, K.kap_l};
    if (op.kind == FLD_OPACITY_CONST) {
        kap = k0;
        return true;
    }
    if (op.kind != FLD_OPACITY_POWER || op.a_rho != 1.0 || op.a_T != -3.5) return false;
    const df y = df_rsqrt(T);                 // T^-1/2
    const df y2 = df_mul(y, y);
    const df y7 = df_mul(df_mul(df_mul(y2, y2), y2), y);
    kap = df_mul(df_mul(k0, rho), y7);
    return df_safe(kap.hi);
}

// With Eh/El (the split copy of E, nullable) the gradient is formed in double-FP32 from the
// split values (FP64 work left: the cell's rho and T, the output, wall ghosts); without it
// the gradient is FP64. ihd holds 1/(12 h_d) as (hi, lo) pairs for the split form.
__device__ __forceinline__ bool limiter_cell_df(const Lvl& L, const double* ih,
                                                const double* __restrict__ E,
                                                const double* __restrict__ rho,
                                                const double* __restrict__ T,
                                                const double* __restrict__ Ebc, const BcOff& bo,
                                                const Opacity& op, const DfConst& K, int mode,
                                                int i, int j, int k, long long p, double& Dout,
                                                double& lmout, const float* __restrict__ Eh = nullptr,
                                                const float* __restrict__ El = nullptr,
                                                const df* ihd = nullptr,
                                                double* kr_out = nullptr) {
    const double r = rho[p];
    const double t = (op.kind == FLD_OPACITY_CONST) ? 1.0 : T[p];
    df Ed;
    if (Eh) {
        Ed = {Eh[p], El[p]};
        if (!(pos_finite(r) && pos_finite(t) && Ed.hi > 0.f)) return false;
    } else {
        const double Ec = E[p];
        if (!(pos_finite(Ec) && pos_finite(r) && pos_finite(t))) return false;
        Ed = df_from_double(Ec);
    }
    // FP64 conversions here: this kernel is bound by instruction issue, where the integer
    // forms would cost more than the FP64 pipe does
    const df rd = df_from_double(r), td = df_from_double(t);
    if (!(df_safe(Ed.hi) && df_safe(rd.hi) && df_safe(td.hi))) return false;
    df kap;
    if (!df_opacity(op, K, rd, td, kap)) return false;
    const df kr = df_mul(kap, rd);
    const df m = df_mul(kr, Ed);
    if (!df_safe(m.hi)) return false;
    if (kr_out) *kr_out = df_to_double_i(kr);
    df lm = {0.33333334f, -9.9341077e-09f};   // 1/3 as a double-FP32 pair
    if (mode != FLD_LIMITER_DIFFUSION) {
        df g2d = {0.f, 0.f};
        if (Eh) {
            // (E_-2 - 8 E_-1) + 8 E_+1 - E_+2 in double-word form (the factors 8 are exact)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d >= L.ndim) break;
                const df em2 = fetch_Edf(L, Eh, El, E, Ebc, bo, i, j, k, d, -2);
                const df em1 = fetch_Edf(L, Eh, El, E, Ebc, bo, i, j, k, d, -1);
                const df ep1 = fetch_Edf(L, Eh, El, E, Ebc, bo, i, j, k, d, 1);
                const df ep2 = fetch_Edf(L, Eh, El, E, Ebc, bo, i, j, k, d, 2);
                if (!(df_safe(em2.hi) && df_safe(em1.hi) && df_safe(ep1.hi) && df_safe(ep2.hi)))
                    return false;
                df t = dw_sub(em2, df{8.f * em1.hi, 8.f * em1.lo});
                t = dw_add(t, df{8.f * ep1.hi, 8.f * ep1.lo});
                t = dw_sub(t, ep2);
                t = two_sum(t.hi, t.lo);
                const df g = df_mul(t, ihd[d]);
                // g^2 must stay a normal FP32 number (else the FP64 form decides)
                const float ga = fabsf(g.hi);
                if (ga != 0.f && !(ga > 1e-18f && ga < 1e18f)) return false;
                g2d = dw_add(g2d, dw_mul(g, g));
            }
            g2d = two_sum(g2d.hi, g2d.lo);
        } else {
            double g2 = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d >= L.ndim) break;
                const double em2 = fetch_E(L, E, Ebc, bo, i, j, k, d, -2);
                const double em1 = fetch_E(L, E, Ebc, bo, i, j, k, d, -1);
                const double ep1 = fetch_E(L, E, Ebc, bo, i, j, k, d, 1);
                const double ep2 = fetch_E(L, E, Ebc, bo, i, j, k, d, 2);
                const double g = ((em2 - 8.0 * em1) + 8.0 * ep1 - ep2) * ih[d];
                g2 = fma(g, g, g2);
            }
            if (g2 > 0.0) {
                g2d = df_from_double(g2);
                if (!df_safe(g2d.hi)) return false;
            }
        }
        if (g2d.hi > 0.f) {
            const df R = df_div(df_sqrt(g2d), m);
            if (!(R.hi < 1e12f)) return false;
            if (mode == FLD_LIMITER_MINERBO) {
                lm = minerbo_lambda_df(R);
            } else {
                const df P = df_add_f(R, 2.f);
                const df Q = df_add_f(df_mul(R, df_add_f(R, 3.f)), 6.f);
                lm = df_div(P, Q);
            }
        }
    }
    const df D = df_div(df_mul({K.c_h, K.c_l}, lm), kr);
    if (!df_safe(D.hi)) return false;
    Dout = df_to_double(D);
    lmout = df_to_double(lm);
    return true;
}

// kr > 0: kappa rho given (frozen at the step's start); else kappa from (rho, T).
__device__ __forceinline__ bool exchange_cell_df(double r, double& t, double& er,
                                                 const Opacity& op, const DfConst& K,
                                                 double kr = 0.0) {
    if (!(pos_finite(r) && pos_finite(t) && pos_finite(er))) return false;
    const df rd = df_from_double_i(r), td = df_from_double_i(t), Ed = df_from_double_i(er);
    if (!(df_safe(rd.hi) && df_safe(td.hi) && df_safe(Ed.hi))) return false;
    df chi;
    if (kr > 0.0) {
        const df krd = df_from_double_i(kr);
        if (!df_safe(krd.hi)) return false;
        chi = df_mul({K.dtc_h, K.dtc_l}, krd);
    } else {
        df kap;
        if (!df_opacity(op, K, rd, td, kap)) return false;
        chi = df_mul(df_mul({K.dtc_h, K.dtc_l}, kap), rd);
    }
    if (!(chi.hi < 1e20f)) return false;
    const df d1 = df_add_f(chi, 1.f);
    const df w = df_div(chi, d1);                         // chi/(1+chi)
    const df onemw = df_div({1.f, 0.f}, d1);              // 1/(1+chi)
    const df alpha = df_mul(rd, {K.cv_h, K.cv_l});
    const df beta = df_mul(w, {K.ar_h, K.ar_l});
    const df q = df_add(df_mul(alpha, td), df_mul(w, Ed));
    if (!(df_safe(alpha.hi) && df_safe(q.hi) && (beta.hi == 0.f || df_safe(beta.hi)))) return false;
    // FP32 Newton on the scaled quartic (all quantities O(1)), as in exchange_root
    const float T1 = q.hi / alpha.hi;
    if (!(T1 > 1e-9f && T1 < 1e9f)) return false;
    const float T1sq = T1 * T1;
    const float g = (beta.hi * T1sq) * (T1sq / q.hi);
    if (!(g < 1e30f)) return false;
    float x = 1.f, scale = T1;
    if (g <= 1.f) {
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const float x2 = x * x;
            x -= (fmaf(g * x2, x2, x) - 1.f) / fmaf(4.f * g * x2, x, 1.f);
        }
    } else {
        const float hh = rsqrtf(sqrtf(g));
        scale = T1 * hh;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const float x2 = x * x;
            x -= (fmaf(x2, x2, hh * x) - 1.f) / fmaf(4.f * x2, x, hh);
        }
    }
    // one df Newton step on f(T) = beta T^4 + alpha T - q, derivative in FP32
    df Tn = two_prod(x, scale);
    const df T2 = df_mul(Tn, Tn);
    const df f = df_sub(df_add(df_mul(beta, df_mul(T2, T2)), df_mul(alpha, Tn)), q);
    const float fp = fmaf(4.f * beta.hi * T2.hi, Tn.hi, alpha.hi);
    Tn = df_add_f(Tn, -__fdiv_rn(f.hi, fp));
    // E' = E/(1+chi) + beta T'^4  (= (E + chi a_r T'^4)/(1+chi))
    const df T2n = df_mul(Tn, Tn);
    const df En = df_add(df_mul(Ed, onemw), df_mul(beta, df_mul(T2n, T2n)));
    if (!(df_safe(Tn.hi) && df_safe(En.hi))) return false;
    // inputs split in integer arithmetic, outputs joined on the FP64 pipe: the two pipes
    // share the conversion work
    t = df_to_double(Tn);
    er = df_to_double(En);
    return true;
}

}  // namespace fld
