// Residual and correction of the mixed-precision refinement carried in double-FP32
// (df64.cuh): the iterate x, the right-hand side b and the operator coefficient K are
// held as FP32 (hi, lo) pairs scaled by a power of two S (exact), so that the FP64-grade
// residual r = b - A x costs FP32 instructions only and the kernel stays memory-bound.
#include "df64.cuh"
#include "fld_device.cuh"

namespace fld {

__global__ void k_df_setup(long long n, double S, const double* __restrict__ E,
                           const double* __restrict__ b, const double* __restrict__ K,
                           float* __restrict__ xh, float* __restrict__ xl, float* __restrict__ bh,
                           float* __restrict__ bl, float* __restrict__ Kh, float* __restrict__ Kl) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        df v = df_from_double(S * E[p]);
        xh[p] = v.hi;
        xl[p] = v.lo;
        v = df_from_double(S * b[p]);
        bh[p] = v.hi;
        bl[p] = v.lo;
        v = df_from_double(K[p]);
        Kh[p] = v.hi;
        Kl[p] = v.lo;
    }
}

__global__ void k_df_finish(long long n, double invS, const float* __restrict__ xh,
                            const float* __restrict__ xl, double* __restrict__ E) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        E[p] = ((double)xh[p] + (double)xl[p]) * invS;
}

// x_new = x + e (when e is given), written out of place; r = b - A x_new in double-FP32;
// r32 = r rounded to FP32; per-block partial sums of r^2.
//
// A x_new = x_new + sum_d (w_d/2) sum_faces (K_p + K_q)(x_p - x_q): per face the sum
// K_p + K_q and the difference x_p - x_q in renormalised double-FP32, their product and
// the accumulation in the unnormalised double-word forms (no renormalisation between
// them); the error stays a few units of 2^-48 of |x| and |K x|, far below the refinement
// tolerance. x_new of the cell itself is renormalised (it is stored); the neighbours'
// x + e are formed as the exact sum of the hi words and e plus the lo word. The squares
// are summed in FP32 per thread (a norm needs no more) and in FP64 across the block.
__global__ void k_df_resid(Lvl L, DfW wd, const float* __restrict__ xh, const float* __restrict__ xl,
                           const float* __restrict__ e, const float* __restrict__ bh,
                           const float* __restrict__ bl, const float* __restrict__ Kh,
                           const float* __restrict__ Kl, float* __restrict__ oh,
                           float* __restrict__ ol, float* __restrict__ r32,
                           double* __restrict__ partials) {
    __shared__ double sh[32];
    float acc2 = 0.f;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int nrows = ny * nz;
    const int sy = nx, sz = nx * ny;
    auto Xn = [&](int q) -> df {   // neighbour value x + e, lo unnormalised
        if (!e) return df{xh[q], xl[q]};
        df s = two_sum(xh[q], e[q]);
        s.lo = __fadd_rn(s.lo, xl[q]);
        return s;
    };
    for (int rr = blockIdx.x; rr < nrows; rr += gridDim.x) {
        const int j = rr % ny, k = rr / ny;
        const int base = rr * nx;
        int oym = 0, oyp = 0, ozm = 0, ozp = 0;
        bool hym = false, hyp = false, hzm = false, hzp = false;
        if (L.ndim >= 2) {
            hym = j > 0 || L.bclo[1] == FLD_BC_PERIODIC;
            hyp = j < ny - 1 || L.bchi[1] == FLD_BC_PERIODIC;
            oym = j > 0 ? -sy : (ny - 1) * sy;
            oyp = j < ny - 1 ? sy : -(ny - 1) * sy;
        }
        if (L.ndim >= 3) {
            hzm = k > 0 || L.bclo[2] == FLD_BC_PERIODIC;
            hzp = k < nz - 1 || L.bchi[2] == FLD_BC_PERIODIC;
            ozm = k > 0 ? -sz : (nz - 1) * sz;
            ozp = k < nz - 1 ? sz : -(nz - 1) * sz;
        }
        // Dirichlet face count weights of this row (y, z walls)
        int ndy = 0, ndz = 0;
        if (L.ndim >= 2) ndy = (!hym && L.bclo[1] == FLD_BC_DIRICHLET) + (!hyp && L.bchi[1] == FLD_BC_DIRICHLET);
        if (L.ndim >= 3) ndz = (!hzm && L.bclo[2] == FLD_BC_DIRICHLET) + (!hzp && L.bchi[2] == FLD_BC_DIRICHLET);
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int p = base + i;
            const df x0 = {xh[p], xl[p]};
            const df xc = e ? df_add_f(x0, e[p]) : x0;
            const df kc = {Kh[p], Kl[p]};
            df res = dw_sub({bh[p], bl[p]}, xc);
            auto face = [&](int q, df acc, bool first) -> df {
                const df t = dw_mul(df_add(kc, df{Kh[q], Kl[q]}), df_sub(xc, Xn(q)));
                return first ? t : dw_add(acc, t);
            };
            const bool hxm = i > 0 || L.bclo[0] == FLD_BC_PERIODIC;
            const bool hxp = i < nx - 1 || L.bchi[0] == FLD_BC_PERIODIC;
            df ax = {0.f, 0.f};
            if (hxm) ax = face(i > 0 ? p - 1 : p + nx - 1, ax, true);
            if (hxp) ax = face(i < nx - 1 ? p + 1 : p - nx + 1, ax, !hxm);
            res = dw_sub(res, dw_mul({wd.hh[0], wd.hl[0]}, ax));
            if (L.ndim >= 2) {
                df ay = {0.f, 0.f};
                if (hym) ay = face(p + oym, ay, true);
                if (hyp) ay = face(p + oyp, ay, !hym);
                res = dw_sub(res, dw_mul({wd.hh[1], wd.hl[1]}, ay));
            }
            if (L.ndim >= 3) {
                df az = {0.f, 0.f};
                if (hzm) az = face(p + ozm, az, true);
                if (hzp) az = face(p + ozp, az, !hzm);
                res = dw_sub(res, dw_mul({wd.hh[2], wd.hl[2]}, az));
            }
            // Dirichlet walls: 2 w_d K_p x_p per wall face (= 4 (w_d/2) K_p x_p)
            const int ndx = (!hxm && L.bclo[0] == FLD_BC_DIRICHLET) + (!hxp && L.bchi[0] == FLD_BC_DIRICHLET);
            if (ndx + ndy + ndz) {
                df dw = {0.f, 0.f};
                if (ndx) dw = df_add(dw, df_mul({wd.hh[0], wd.hl[0]}, {4.f * ndx, 0.f}));
                if (ndy) dw = df_add(dw, df_mul({wd.hh[1], wd.hl[1]}, {4.f * ndy, 0.f}));
                if (ndz) dw = df_add(dw, df_mul({wd.hh[2], wd.hl[2]}, {4.f * ndz, 0.f}));
                res = dw_sub(res, df_mul(df_mul(dw, kc), xc));
            }
            if (oh) {
                oh[p] = xc.hi;
                ol[p] = xc.lo;
            }
            const float r = __fadd_rn(res.hi, res.lo);
            r32[p] = r;
            acc2 = fmaf(r, r, acc2);
        }
    }
    const double a2 = block_sum((double)acc2, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = a2;
}

void launch_df_setup(long long n, double S, const double* E, const double* b, const double* K,
                     float* xh, float* xl, float* bh, float* bl, float* Kh, float* Kl,
                     cudaStream_t s) {
    long long nb = (n + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    k_df_setup<<<(int)nb, 256, 0, s>>>(n, S, E, b, K, xh, xl, bh, bl, Kh, Kl);
}

void launch_df_finish(long long n, double invS, const float* xh, const float* xl, double* E,
                      cudaStream_t s) {
    long long nb = (n + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    k_df_finish<<<(int)nb, 256, 0, s>>>(n, invS, xh, xl, E);
}

void launch_df_resid(const Lvl& L, const DfW& wd, const float* xh, const float* xl, const float* e,
                     const float* bh, const float* bl, const float* Kh, const float* Kl, float* oh,
                     float* ol, float* r32, double* partials, int nblocks, int block,
                     cudaStream_t s) {
    k_df_resid<<<nblocks, block, 0, s>>>(L, wd, xh, xl, e, bh, bl, Kh, Kl, oh, ol, r32, partials);
}

}  // namespace fld
