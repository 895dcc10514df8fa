// Batched FLD substep: many independent problems of uneven sizes in ONE persistent
// launch. A group of CS blocks (a thread-block cluster when CS > 1, one block when
// CS == 1) takes the next problem from a queue ordered by decreasing size and runs the
// whole substep on it: limiter -> multigrid solve (FP32 V-cycles inside FP64 or
// double-FP32 iterative refinement, to the relative-residual tolerance) -> exchange, the
// limiter and the exchange in the refinement's arithmetic.
//
// The group's threads split every phase's cells; phases are separated by the hardware
// cluster barrier (or __syncthreads), reductions go through distributed shared memory
// in a fixed order, and no block ever spins on memory written by another: the launch
// cannot deadlock and its results do not depend on which group solves which problem.
#include <cooperative_groups.h>

#include <algorithm>

#include "df64.cuh"
#include "fld_batch.cuh"
#include "fld_device.cuh"

namespace cg = cooperative_groups;

namespace fld {

namespace {

constexpr int BMAX_DENSE = 64;

struct GroupShared {
    double red[32];
    double part;                                   // this block's partial sum
    double total;                                  // group total (rank 0 holds it)
    int qi;                                        // problem index (rank 0 holds it)
    double A[BMAX_DENSE][BMAX_DENSE + 1];          // dense coarsest system (rank 0)
};

template <int CS>
struct Grp {
    int tid;     // thread index within the group
    int nthr;    // threads in the group
    int rank;    // block rank within the group
    __device__ __forceinline__ void sync() const {
        if constexpr (CS == 1) __syncthreads();
        else cg::this_cluster().sync();
    }
    // a shared variable of block `r` of the group
    template <typename V>
    __device__ __forceinline__ V* at(V* p, int r) const {
        if constexpr (CS == 1) return p;
        else return cg::this_cluster().map_shared_rank(p, r);
    }
};

// Group-wide sum: block sums in fixed trees, then the blocks' partials in rank order.
template <int CS>
__device__ double grp_sum(double v, GroupShared& sh, const Grp<CS>& g) {
    v = block_sum(v, sh.red);
    if (threadIdx.x == 0) sh.part = v;
    g.sync();
    if (g.rank == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < CS; ++r) t += *g.at(&sh.part, r);
        sh.total = t;
    }
    g.sync();
    const double t = *g.at(&sh.total, 0);
    g.sync();
    return t;
}

// Half sweep of colour `color`; in place, or through t (ping-pong) when a periodic
// extent is odd (two same-colour neighbours meet across the wrap).
template <int CS>
__device__ void grp_half(const Grp<CS>& g, const Lvl& L, int color, float* x, float* t,
                         const float* b, const float* K, bool pingpong) {
    const int nx = L.n[0], ny = L.n[1];
    const int pairs = (nx + 1) >> 1;
    const int total = pairs * ny * L.n[2];
    for (int q = g.tid; q < total; q += g.nthr) {
        const int ip = q % pairs;
        const int row = q / pairs;
        const int j = row % ny, k = row / ny;
        const int par = (j + k + color) & 1;
        const int ia = 2 * ip + par;                 // the cell of `color` in this pair
        const int ib = 2 * ip + (par ^ 1);           // the other one
        const long long base = (long long)row * nx;
        if (pingpong) {
            if (ib < nx) t[base + ib] = x[base + ib];
            if (ia < nx) {
                float sw, acc;
                stencil<float>(L, K, x, ia, j, k, base + ia, sw, acc);
                t[base + ia] = div_fast<float>(b[base + ia] + acc, 1.f + sw);
            }
        } else if (ia < nx) {
            float sw, acc;
            stencil<float>(L, K, x, ia, j, k, base + ia, sw, acc);
            x[base + ia] = div_fast<float>(b[base + ia] + acc, 1.f + sw);
        }
    }
    g.sync();
}

template <int CS>
__device__ void grp_smooth(const Grp<CS>& g, const Lvl& L, int sweeps, float* x, float* t,
                           const float* b, const float* K) {
    bool odd = false;
    for (int d = 0; d < L.ndim; ++d) odd |= (L.bclo[d] == FLD_BC_PERIODIC) && (L.n[d] & 1);
    for (int s = 0; s < sweeps; ++s) {
        if (odd) {
            grp_half(g, L, 0, x, t, b, K, true);     // t = red(x) | black(x)
            grp_half(g, L, 1, t, x, b, K, true);     // x = black(t) | red(t)
        } else {
            grp_half(g, L, 0, x, (float*)nullptr, b, K, false);
            grp_half(g, L, 1, x, (float*)nullptr, b, K, false);
        }
    }
}

__device__ __forceinline__ void children(const Lvl& F, const Lvl& C, int I, int J, int Kc,
                                         int lo[3], int hi[3]) {
    const int c[3] = {I, J, Kc};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (C.n[d] < F.n[d]) {
            lo[d] = 2 * c[d];
            hi[d] = min(2 * c[d] + 1, F.n[d] - 1);
        } else {
            lo[d] = hi[d] = c[d];
        }
    }
}

template <int CS>
__device__ void grp_restrict_K(const Grp<CS>& g, const Lvl& F, const Lvl& C, float scale,
                               const float* Kf, float* Kc) {
    for (int P = g.tid; P < (int)C.ncell; P += g.nthr) {
        int c0, c1, c2;
        decode(C, P, c0, c1, c2);
        int lo[3], hi[3];
        children(F, C, c0, c1, c2, lo, hi);
        float s = 0.f;
        int cnt = 0;
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    s += Kf[((long long)k * F.n[1] + j) * F.n[0] + i];
                    ++cnt;
                }
        Kc[P] = scale * s / (float)cnt;
    }
    g.sync();
}

template <int CS>
__device__ void grp_resid_restrict(const Grp<CS>& g, const Lvl& F, const Lvl& C, const float* x,
                                   const float* b, const float* K, float* bc, float* xc) {
    for (int P = g.tid; P < (int)C.ncell; P += g.nthr) {
        int c0, c1, c2;
        decode(C, P, c0, c1, c2);
        int lo[3], hi[3];
        children(F, C, c0, c1, c2, lo, hi);
        float s = 0.f;
        int cnt = 0;
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    const long long p = ((long long)k * F.n[1] + j) * F.n[0] + i;
                    float sw, acc;
                    stencil<float>(F, K, x, i, j, k, p, sw, acc);
                    s += b[p] - (1.f + sw) * x[p] + acc;
                    ++cnt;
                }
        bc[P] = s / (float)cnt;
        xc[P] = 0.f;
    }
    g.sync();
}

template <int CS>
__device__ void grp_prolong(const Grp<CS>& g, const Lvl& F, const Lvl& C, float* xf,
                            const float* xc) {
    for (int p = g.tid; p < (int)F.ncell; p += g.nthr) {
        int i, j, k;
        decode(F, p, i, j, k);
        const Interp ix = interp1(i, F.n[0], C.n[0], F.bclo[0], F.bchi[0]);
        const Interp iy = interp1(j, F.n[1], C.n[1], F.bclo[1], F.bchi[1]);
        const Interp iz = interp1(k, F.n[2], C.n[2], F.bclo[2], F.bchi[2]);
        float acc = 0.f;
        for (int c = 0; c < 2; ++c)
            for (int bb = 0; bb < 2; ++bb) {
                const float wzy = iz.wt[c] * iy.wt[bb];
                if (wzy == 0.f) continue;
                const long long rowc = ((long long)iz.idx[c] * C.n[1] + iy.idx[bb]) * C.n[0];
                acc += wzy * (ix.wt[0] * xc[rowc + ix.idx[0]] + ix.wt[1] * xc[rowc + ix.idx[1]]);
            }
        xf[p] += acc;
    }
    g.sync();
}

// Coarsest level: exact dense FP64 solve by the group's first block when small, else
// red-black sweeps by the whole group.
template <int CS>
__device__ void grp_coarse(const Grp<CS>& g, const Lvl& L, float* x, float* t, const float* b,
                           const float* K, int sweeps, GroupShared& sh) {
    const int n = (int)L.ncell;
    if (n > BMAX_DENSE) {
        for (int p = g.tid; p < n; p += g.nthr) x[p] = 0.f;
        g.sync();
        grp_smooth(g, L, sweeps, x, t, b, K);
        return;
    }
    if (g.rank == 0) {
        const int r = threadIdx.x;
        if (r < n) {
            for (int c = 0; c <= n; ++c) sh.A[r][c] = 0.0;
            int i, j, k;
            decode(L, r, i, j, k);
            const int c3[3] = {i, j, k};
            const double kc = (double)K[r];
            double diag = 1.0;
            int stride = 1;
            for (int d = 0; d < L.ndim; ++d) {
                const int nd = L.n[d];
                for (int side = 0; side < 2; ++side) {
                    const int kind = side ? L.bchi[d] : L.bclo[d];
                    int q = -1;
                    if (side == 0) {
                        if (c3[d] > 0) q = r - stride;
                        else if (kind == FLD_BC_PERIODIC) q = r + (nd - 1) * stride;
                    } else {
                        if (c3[d] < nd - 1) q = r + stride;
                        else if (kind == FLD_BC_PERIODIC) q = r - (nd - 1) * stride;
                    }
                    if (q >= 0) {
                        const double w = 0.5 * (kc + (double)K[q]) * L.w[d];
                        diag += w;
                        sh.A[r][q] -= w;
                    } else if (kind == FLD_BC_DIRICHLET) {
                        diag += 2.0 * kc * L.w[d];
                    }
                }
                stride *= nd;
            }
            sh.A[r][r] += diag;
            sh.A[r][n] = (double)b[r];
        }
        for (int p = 0; p < n; ++p) {
            __syncthreads();
            double f = 0.0;
            if (r < n && r != p) f = sh.A[r][p] / sh.A[p][p];
            __syncthreads();
            if (r < n && r != p)
                for (int c = p; c <= n; ++c) sh.A[r][c] = fma(-f, sh.A[p][c], sh.A[r][c]);
        }
        __syncthreads();
        if (r < n) x[r] = (float)(sh.A[r][n] / sh.A[r][r]);
    }
    g.sync();
}

template <int CS>
__device__ void grp_vcycle(const Grp<CS>& g, const BProb& P, float* F, int nu1, int nu2,
                           int csweeps, GroupShared& sh) {
    const int L = P.nlev;
    for (int l = 0; l < L - 1; ++l) {
        float* x = F + P.o32[l];
        const long long n = P.lv[l].ncell;
        grp_smooth(g, P.lv[l], nu1, x, x + 3 * n, x + n, x + 2 * n);
        float* xc = F + P.o32[l + 1];
        const long long nc = P.lv[l + 1].ncell;
        grp_resid_restrict(g, P.lv[l], P.lv[l + 1], x, x + n, x + 2 * n, xc + nc, xc);
    }
    {
        float* x = F + P.o32[L - 1];
        const long long n = P.lv[L - 1].ncell;
        grp_coarse(g, P.lv[L - 1], x, x + 3 * n, x + n, x + 2 * n, csweeps, sh);
    }
    for (int l = L - 2; l >= 0; --l) {
        float* x = F + P.o32[l];
        const long long n = P.lv[l].ncell;
        grp_prolong(g, P.lv[l], P.lv[l + 1], x, F + P.o32[l + 1]);
        grp_smooth(g, P.lv[l], nu2, x, x + 3 * n, x + n, x + 2 * n);
    }
}

// Level-0 residual in double-FP32: r = b - A x (renormalised face factors, unnormalised
// double-word products and sums: a few units of 2^-48 of |x| and |K x|), r32 = r rounded
// to FP32; returns the group's sum of r^2.
template <int CS>
__device__ double grp_df_resid(const Grp<CS>& g, const Lvl& L, const DfW& wd, const float* xh,
                               const float* xl, const float* bh, const float* bl, const float* Kh,
                               const float* Kl, float* r32, GroupShared& sh) {
    double a2 = 0.0;
    for (int p = g.tid; p < (int)L.ncell; p += g.nthr) {
        int i, j, k;
        decode(L, p, i, j, k);
        const df xc = {xh[p], xl[p]};
        const df kc = {Kh[p], Kl[p]};
        df res = dw_sub({bh[p], bl[p]}, xc);
        const int c[3] = {i, j, k};
        int stride = 1;
        df dw = {0.f, 0.f};
        for (int d = 0; d < L.ndim; ++d) {
            const int nd = L.n[d];
            df ax = {0.f, 0.f};
            for (int side = 0; side < 2; ++side) {
                const int kind = side ? L.bchi[d] : L.bclo[d];
                int q = -1;
                if (side == 0) {
                    if (c[d] > 0) q = p - stride;
                    else if (kind == FLD_BC_PERIODIC) q = p + (nd - 1) * stride;
                } else {
                    if (c[d] < nd - 1) q = p + stride;
                    else if (kind == FLD_BC_PERIODIC) q = p - (nd - 1) * stride;
                }
                if (q >= 0) {
                    const df kq = {Kh[q], Kl[q]};
                    const df xq = {xh[q], xl[q]};
                    ax = dw_add(ax, dw_mul(df_add(kc, kq), df_sub(xc, xq)));
                } else if (kind == FLD_BC_DIRICHLET) {
                    dw = df_add(dw, df_mul({wd.hh[d], wd.hl[d]}, {4.f, 0.f}));
                }
            }
            res = dw_sub(res, dw_mul({wd.hh[d], wd.hl[d]}, ax));
            stride *= nd;
        }
        if (dw.hi != 0.f) res = dw_sub(res, df_mul(df_mul(dw, kc), xc));
        const float r = __fadd_rn(res.hi, res.lo);
        r32[p] = r;
        a2 = fma((double)r, (double)r, a2);
    }
    g.sync();
    return grp_sum(a2, sh, g);
}

// Level-0 residual in FP64: r = b - A x with the level operator's stencil, r32 = r rounded
// to FP32; returns the group's sum of r^2.
template <int CS>
__device__ double grp_resid64(const Grp<CS>& g, const Lvl& L, const double* x, const double* b,
                              const double* K, float* r32, GroupShared& sh) {
    double a2 = 0.0;
    for (int p = g.tid; p < (int)L.ncell; p += g.nthr) {
        int i, j, k;
        decode(L, p, i, j, k);
        double sw, acc;
        stencil<double>(L, K, x, i, j, k, p, sw, acc);
        const double r = b[p] - fma(1.0 + sw, x[p], -acc);
        r32[p] = (float)r;
        a2 = fma(r, r, a2);
    }
    g.sync();
    return grp_sum(a2, sh, g);
}

template <int NT, int CS>
__global__ void __launch_bounds__(NT)
k_batch_step(const BProb* __restrict__ probs, const BDyn* __restrict__ dyn,
             const int* __restrict__ order, int nprob, int* __restrict__ queue, BatchParams prm,
             const double* __restrict__ rho, double* __restrict__ T, double* __restrict__ E,
             const double* __restrict__ Ebc, double* __restrict__ wsd, float* __restrict__ wsf,
             BatchStat* __restrict__ stats, unsigned* __restrict__ err) {
    __shared__ GroupShared sh;
    Grp<CS> g;
    if constexpr (CS == 1) g.rank = 0;
    else g.rank = (int)cg::this_cluster().block_rank();
    g.tid = g.rank * NT + threadIdx.x;
    g.nthr = CS * NT;
    for (;;) {
        if (g.rank == 0 && threadIdx.x == 0) sh.qi = atomicAdd(queue, 1);
        g.sync();
        const int qi = *g.at(&sh.qi, 0);
        g.sync();
        if (qi >= nprob) break;
        const int pid = order[qi];
        const BProb& P = probs[pid];
        const double dt = dyn[pid].dt;
        const Opacity op = dyn[pid].op;
        const Lvl& L0 = P.lv[0];
        const int n0 = (int)L0.ncell;
        const double* r_ = rho + P.cell_off;
        double* T_ = T + P.cell_off;
        double* E_ = E + P.cell_off;
        const double* eb = P.ebc_off >= 0 ? Ebc + P.ebc_off : nullptr;
        double* D = wsd + P.ws_d;
        double* x64 = D + n0;              // FP64 refinement (prm.fp64): iterate, rhs, K
        double* b64 = D + 2 * n0;
        double* K64 = D + 3 * n0;
        float* F = wsf + P.ws_f;
        float* xh = F;
        float* xl = F + n0;
        float* bh = F + 2 * n0;
        float* bl = F + 3 * n0;
        float* Kh = F + 4 * n0;
        float* Kl = F + 5 * n0;
        float* x32 = F + P.o32[0];
        float* b32 = x32 + n0;
        float* K32 = x32 + 2 * n0;
        BcOff bo;
        for (int q = 0; q < 6; ++q) bo.off[q] = P.bc_off[q];
        const double ih[3] = {1.0 / (12.0 * P.h[0]), 1.0 / (12.0 * P.h[1]), 1.0 / (12.0 * P.h[2])};

        // per-problem constants as double-FP32 pairs
        DfConst KC;
        {
            const df c2 = df_from_double(prm.c), k2 = df_from_double(op.kappa0),
                     t2 = df_from_double(dt * prm.c), a2 = df_from_double(prm.a_r),
                     v2 = df_from_double(prm.cv);
            KC = {c2.hi, c2.lo, k2.hi, k2.lo, t2.hi, t2.lo, a2.hi, a2.lo, v2.hi, v2.lo};
        }
        // ---- limiter -> D; count domain errors
        double bad = 0.0;
        for (int p = g.tid; p < n0; p += g.nthr) {
            int i, j, k;
            decode(L0, p, i, j, k);
            double Dv = 0.0, lm;
            if (!(!prm.fp64 && limiter_cell_df(L0, ih, E_, r_, T_, eb, bo, op, KC, prm.limiter, i,
                                               j, k, p, Dv, lm)) &&
                !limiter_cell<false>(L0, ih, E_, r_, T_, eb, bo, op, prm.c, prm.limiter, i, j, k,
                                     p, Dv, lm))
                bad += 1.0;
            D[p] = Dv;
        }
        g.sync();
        const bool bad_any = grp_sum(bad, sh, g) > 0.0;

        // ---- set-up: K = dt D / h_x^2, b = E + Dirichlet terms, power-of-two scaling
        const double kscale = dt / (P.h[0] * P.h[0]);
        auto bval = [&](int p, double Kp) -> double {
            double bp = E_[p];
            if (eb) {
                int c[3];
                decode(L0, p, c[0], c[1], c[2]);
                for (int d = 0; d < L0.ndim; ++d) {
                    const long long fi = face_index(L0, d, c[0], c[1], c[2]);
                    if (c[d] == 0 && L0.bclo[d] == FLD_BC_DIRICHLET)
                        bp += 2.0 * Kp * L0.w[d] * eb[bo.off[2 * d] + fi];
                    if (c[d] == L0.n[d] - 1 && L0.bchi[d] == FLD_BC_DIRICHLET)
                        bp += 2.0 * Kp * L0.w[d] * eb[bo.off[2 * d + 1] + fi];
                }
            }
            return bp;
        };
        double rel = -1.0, rel0 = -1.0;
        int cyc = 0;
        if (!bad_any) {
            double b2 = 0.0;
            for (int p = g.tid; p < n0; p += g.nthr) {
                const double bp = bval(p, kscale * D[p]);
                b2 = fma(bp, bp, b2);
            }
            b2 = grp_sum(b2, sh, g);
            if (prm.fp64) {
                // ---- FP64 refinement: x = E^n, b and K in FP64, FP32 V-cycles on A e = r
                for (int p = g.tid; p < n0; p += g.nthr) {
                    const double Kp = kscale * D[p];
                    x64[p] = E_[p];
                    b64[p] = bval(p, Kp);
                    K64[p] = Kp;
                    K32[p] = (float)Kp;
                }
                g.sync();
                for (int l = 0; l + 1 < P.nlev; ++l) {
                    const long long nf = P.lv[l].ncell, nc = P.lv[l + 1].ncell;
                    grp_restrict_K(g, P.lv[l], P.lv[l + 1], (float)P.kdown[l],
                                   F + P.o32[l] + 2 * nf, F + P.o32[l + 1] + 2 * nc);
                }
                const double bnorm = sqrt(b2);
                rel = bnorm > 0.0 ? sqrt(grp_resid64(g, L0, x64, b64, K64, b32, sh)) / bnorm : 0.0;
                rel0 = rel;
                while (rel > prm.tol && cyc < prm.max_cycles && isfinite(rel)) {
                    for (int p = g.tid; p < n0; p += g.nthr) x32[p] = 0.f;
                    g.sync();
                    for (int ic = 0; ic < prm.inner; ++ic)
                        grp_vcycle(g, P, F, prm.nu1, prm.nu2, prm.coarse_sweeps, sh);
                    for (int p = g.tid; p < n0; p += g.nthr) x64[p] += (double)x32[p];
                    g.sync();
                    rel = sqrt(grp_resid64(g, L0, x64, b64, K64, b32, sh)) / bnorm;
                    ++cyc;
                }
                // ---- the exchange in FP64 with kappa(rho, T^n)
                const double dtc = dt * prm.c;
                for (int p = g.tid; p < n0; p += g.nthr) {
                    double t = T_[p], e_new = x64[p];
                    exchange_cell<false>(r_[p], t, e_new, op, dtc, prm.a_r, prm.cv);
                    T_[p] = t;
                    E_[p] = e_new;
                }
            } else {
            int ex = 0;
            frexp(b2 > 0.0 ? sqrt(b2 / n0) : 1.0, &ex);
            const double S = ldexp(1.0, -ex);
            for (int p = g.tid; p < n0; p += g.nthr) {
                const double Kp = kscale * D[p];
                df v = df_from_double(S * E_[p]);
                xh[p] = v.hi;
                xl[p] = v.lo;
                v = df_from_double(S * bval(p, Kp));
                bh[p] = v.hi;
                bl[p] = v.lo;
                v = df_from_double(Kp);
                Kh[p] = v.hi;
                Kl[p] = v.lo;
                K32[p] = (float)Kp;
            }
            g.sync();
            for (int l = 0; l + 1 < P.nlev; ++l) {
                const long long nf = P.lv[l].ncell, nc = P.lv[l + 1].ncell;
                grp_restrict_K(g, P.lv[l], P.lv[l + 1], (float)P.kdown[l], F + P.o32[l] + 2 * nf,
                               F + P.o32[l + 1] + 2 * nc);
            }
            DfW wd;
            for (int d = 0; d < 3; ++d) {
                const double wh = 0.5 * L0.w[d];
                wd.hh[d] = (float)wh;
                wd.hl[d] = (float)(wh - (double)wd.hh[d]);
            }
            // ---- refinement: FP32 V-cycle on A e = r, x += e in double-FP32
            const double bnorm = sqrt(b2) * S;
            rel = bnorm > 0.0
                      ? sqrt(grp_df_resid(g, L0, wd, xh, xl, bh, bl, Kh, Kl, b32, sh)) / bnorm
                      : 0.0;
            rel0 = rel;
            while (rel > prm.tol && cyc < prm.max_cycles && isfinite(rel)) {
                for (int p = g.tid; p < n0; p += g.nthr) x32[p] = 0.f;
                g.sync();
                for (int ic = 0; ic < prm.inner; ++ic)
                    grp_vcycle(g, P, F, prm.nu1, prm.nu2, prm.coarse_sweeps, sh);
                for (int p = g.tid; p < n0; p += g.nthr) {
                    const df v = df_add_f({xh[p], xl[p]}, x32[p]);
                    xh[p] = v.hi;
                    xl[p] = v.lo;
                }
                g.sync();
                rel = sqrt(grp_df_resid(g, L0, wd, xh, xl, bh, bl, Kh, Kl, b32, sh)) / bnorm;
                ++cyc;
            }
            // ---- E back from the scaled iterate, then the exchange with kappa(rho, T^n)
            const double invS = 1.0 / S;
            const double dtc = dt * prm.c;
            for (int p = g.tid; p < n0; p += g.nthr) {
                const double e_sol = ((double)xh[p] + (double)xl[p]) * invS;
                double t = T_[p], e_new = e_sol;
                if (!exchange_cell_df(r_[p], t, e_new, op, KC)) {
                    t = T_[p];
                    e_new = e_sol;
                    exchange_cell<false>(r_[p], t, e_new, op, dtc, prm.a_r, prm.cv);
                }
                T_[p] = t;
                E_[p] = e_new;
            }
            }
        }
        if (g.rank == 0 && threadIdx.x == 0) {
            stats[pid].cycles = cyc;
            stats[pid].rel_resid = rel;
            stats[pid].rel_resid0 = rel0;
            if (bad_any) atomicOr(err, ERRBIT_DOMAIN);
            else if (!(rel <= prm.tol)) atomicOr(err, ERRBIT_NOTCONV);
        }
        g.sync();
    }
}

template <int NT, int CS>
void launch_one(int nblocks, const BProb* probs, const BDyn* dyn, const int* order, int nprob,
                int* queue, const BatchParams& prm, const double* rho, double* T, double* E,
                const double* Ebc, double* wsd, float* wsf, BatchStat* stats, unsigned* err,
                cudaStream_t s) {
    if constexpr (CS == 1) {
        k_batch_step<NT, 1><<<nblocks, NT, 0, s>>>(probs, dyn, order, nprob, queue, prm, rho, T, E,
                                                   Ebc, wsd, wsf, stats, err);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nblocks);
        cfg.blockDim = dim3(NT);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_batch_step<NT, CS>, probs, dyn, order, nprob, queue, prm, rho,
                           T, E, Ebc, wsd, wsf, stats, err);
    }
}

template <int NT, int CS>
int max_groups() {
    if constexpr (CS == 1) {
        int nb = 0, dev = 0, nsm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<NT, 1>, NT, 0);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        return nb * nsm;
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CS * 64);
        cfg.blockDim = dim3(NT);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_batch_step<NT, CS>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return nc;
    }
}

}  // namespace

int batch_threads_supported(int nt) { return nt == 256 || nt == 512 || nt == 1024; }
int batch_cluster_supported(int cs) { return cs == 1 || cs == 2 || cs == 4 || cs == 8; }

#define FLD_BATCH_DISPATCH(NT_, CALL) \
    switch (cs) {                     \
        case 2: CALL(NT_, 2); break;  \
        case 4: CALL(NT_, 4); break;  \
        case 8: CALL(NT_, 8); break;  \
        default: CALL(NT_, 1);        \
    }

int batch_max_groups(int nt, int cs) {
    int r = 0;
#define MG(NT_, CS_) r = max_groups<NT_, CS_>()
    if (nt == 256) {
        FLD_BATCH_DISPATCH(256, MG)
    } else if (nt == 1024) {
        FLD_BATCH_DISPATCH(1024, MG)
    } else {
        FLD_BATCH_DISPATCH(512, MG)
    }
#undef MG
    return r;
}

void launch_batch_step(int nt, int cs, int ngroups, const BProb* probs, const BDyn* dyn,
                       const int* order, int nprob, int* queue, const BatchParams& prm,
                       const double* rho, double* T, double* E, const double* Ebc, double* wsd,
                       float* wsf, BatchStat* stats, unsigned* err, cudaStream_t s) {
#define LB(NT_, CS_)                                                                        \
    launch_one<NT_, CS_>(ngroups * CS_, probs, dyn, order, nprob, queue, prm, rho, T, E, Ebc, \
                         wsd, wsf, stats, err, s)
    if (nt == 256) {
        FLD_BATCH_DISPATCH(256, LB)
    } else if (nt == 1024) {
        FLD_BATCH_DISPATCH(1024, LB)
    } else {
        FLD_BATCH_DISPATCH(512, LB)
    }
#undef LB
}

}  // namespace fld
