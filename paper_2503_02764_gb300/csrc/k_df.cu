// Residual and correction of the mixed-precision refinement carried in double-FP32
// (df64.cuh): the iterate x, the right-hand side b and the operator coefficient K are
// held as FP32 (hi, lo) pairs scaled by a power of two S (exact), so that the FP64-grade
// residual r = b - A x costs FP32 instructions only and the kernel stays memory-bound.
#include <algorithm>
#include <cmath>

#include "df64.cuh"
#include "fld_device.cuh"

namespace fld {

// x = S E, b = S b, K split into double-FP32 pairs; S = 2^k2 (exact), applied in the
// exponent by the integer split.
__global__ void k_df_setup(long long n, int k2, const double* __restrict__ E,
                           const double* __restrict__ b, const double* __restrict__ K,
                           float* __restrict__ xh, float* __restrict__ xl, float* __restrict__ bh,
                           float* __restrict__ bl, float* __restrict__ Kh, float* __restrict__ Kl) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        df v = df_from_double_i(E[p], k2);
        xh[p] = v.hi;
        xl[p] = v.lo;
        v = df_from_double_i(b[p], k2);
        bh[p] = v.hi;
        bl[p] = v.lo;
        v = df_from_double_i(K[p]);
        Kh[p] = v.hi;
        Kl[p] = v.lo;
    }
}

// E = (hi + lo) / S, S = 2^-k2 applied in the exponent by the integer join
__global__ void k_df_finish(long long n, int k2, const float* __restrict__ xh,
                            const float* __restrict__ xl, double* __restrict__ E) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        E[p] = df_to_double_i(df{xh[p], xl[p]}, k2);
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

// 3D levels: the same residual with every face evaluated once. A block owns a DR_TX x DR_TY
// tile of the x-y plane and marches along z over [z0, z1); thread (lx, ly) owns one
// column. For each plane it forms x_new = x + e (renormalised) for its cell, and the
// threads of the tile's ring (the cells at distance 1 outside the tile in x and y; ghosts
// beyond a wall: x = 0, K = -K or 3 K of the wall cell) for theirs, into shared memory.
// Each thread then evaluates the flux G = (K_c + K_q)(x_c - x_q) of its cell's -x and
// -y faces (the last column and row also the +x, +y faces of the tile edge) and, from
// its registers, of the -z face against the plane below. A cell's residual is
//   b - x - h_x (G_x(-) - G_x(+)) - h_y (G_y(-) - G_y(+)) - h_z (G_z(-) - G_z(+)),
// its +z term arriving one plane later. Per face: renormalised K_c + K_q and x_c - x_q,
// an unnormalised product; every flux is used with both signs, exactly antisymmetric.
constexpr int DR_TX = 32, DR_TY = 8, DR_NT = DR_TX * DR_TY;
constexpr int DR_PW = DR_TX + 2;                   // shared row pitch (tile + ring)

__device__ __forceinline__ int dr_axis(int g, int n, bool per) {
    if (g >= 0 && g < n) return g;
    if (per) return g < 0 ? g + n : g - n;
    return -1;
}

__device__ __forceinline__ float dr_factor(int bc) { return bc == FLD_BC_DIRICHLET ? 3.f : -1.f; }

__global__ void __launch_bounds__(DR_NT)
k_df_resid3(Lvl L, DfW wd, const float* __restrict__ xh, const float* __restrict__ xl,
            const float* __restrict__ e, const float* __restrict__ bh,
            const float* __restrict__ bl, const float* __restrict__ Kh,
            const float* __restrict__ Kl, float* __restrict__ oh, float* __restrict__ ol,
            float* __restrict__ r32, double* __restrict__ partials, int cz) {
    __shared__ float XH[(DR_TY + 2) * DR_PW], XL[(DR_TY + 2) * DR_PW];
    __shared__ float KH[(DR_TY + 2) * DR_PW], KL[(DR_TY + 2) * DR_PW];
    __shared__ float FXH[DR_TY * (DR_TX + 1)], FXL[DR_TY * (DR_TX + 1)];
    __shared__ float FYH[(DR_TY + 1) * DR_TX], FYL[(DR_TY + 1) * DR_TX];
    __shared__ double sh[32];

    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int tilesx = (nx + DR_TX - 1) / DR_TX, tilesy = (ny + DR_TY - 1) / DR_TY;
    int bid = blockIdx.x;
    const int tx0 = (bid % tilesx) * DR_TX;
    bid /= tilesx;
    const int ty0 = (bid % tilesy) * DR_TY;
    bid /= tilesy;
    const int z0 = bid * cz, z1 = min(z0 + cz, nz);
    const bool xper = L.bclo[0] == FLD_BC_PERIODIC, yper = L.bclo[1] == FLD_BC_PERIODIC;
    const bool zper = L.bclo[2] == FLD_BC_PERIODIC;
    const long long plane = (long long)nx * ny;
    const df hx = {wd.hh[0], wd.hl[0]}, hy = {wd.hh[1], wd.hl[1]}, hz = {wd.hh[2], wd.hl[2]};

    const int tid = threadIdx.x;
    const int lx = tid % DR_TX, ly = tid / DR_TX;
    const int ax = min(DR_TX, nx - tx0), ay = min(DR_TY, ny - ty0);
    const bool act = lx < ax && ly < ay;
    const long long own = act ? (long long)(ty0 + ly) * nx + tx0 + lx : 0;
    const int so = (ly + 1) * DR_PW + lx + 1;

    // ring cell of this thread: left/right columns, then bottom/top rows
    int rso = -1;              // its shared offset (-1: none)
    long long rsrc = 0;        // plane offset of the value it copies (the wall cell for a ghost)
    bool rghost = false;
    float rfac = 0.f;
    {
        int qx = 0, qy = 0;
        bool has = true;
        if (tid < ay) { qx = -1; qy = tid; }
        else if (tid < 2 * ay) { qx = ax; qy = tid - ay; }
        else if (tid < 2 * ay + ax) { qx = tid - 2 * ay; qy = -1; }
        else if (tid < 2 * ay + 2 * ax) { qx = tid - 2 * ay - ax; qy = ay; }
        else has = false;
        if (has) {
            rso = (qy + 1) * DR_PW + qx + 1;
            const int gx = dr_axis(tx0 + qx, nx, xper), gy = dr_axis(ty0 + qy, ny, yper);
            if (gx >= 0 && gy >= 0) {
                rsrc = (long long)gy * nx + gx;
            } else {
                // the ghost next to a wall mirrors the adjacent tile cell
                rghost = true;
                const int wx = qx < 0 ? 0 : (qx >= ax ? ax - 1 : qx);
                const int wy = qy < 0 ? 0 : (qy >= ay ? ay - 1 : qy);
                rsrc = (long long)(ty0 + wy) * nx + tx0 + wx;
                const int bc = gx < 0 ? (qx < 0 ? L.bclo[0] : L.bchi[0])
                                      : (qy < 0 ? L.bclo[1] : L.bchi[1]);
                rfac = dr_factor(bc);
            }
        }
    }

    // Raw words of one plane for this thread's column and ring cell, loaded one plane ahead
    // of use so the loads are in flight during the previous plane's flux work.
    struct Raw {
        float xh, xl, e, kh, kl, bh, bl;      // own column
        float rxh, rxl, re, rkh, rkl;         // ring cell
    };
    auto load_raw = [&](int m, Raw& R) {
        const int gz = dr_axis(m, nz, zper);
        if (gz < 0) return;                   // a wall ghost plane: formed from K below
        const long long pk = gz * plane;
        if (act) {
            const long long q = pk + own;
            R.xh = xh[q];
            R.xl = xl[q];
            R.e = e ? e[q] : 0.f;
            R.kh = Kh[q];
            R.kl = Kl[q];
            if (m < z1) {
                R.bh = bh[q];
                R.bl = bl[q];
            }
        }
        if (rso >= 0 && m < z1) {
            const long long q = pk + rsrc;
            R.rkh = Kh[q];
            R.rkl = Kl[q];
            if (!rghost) {
                R.rxh = xh[q];
                R.rxl = xl[q];
                R.re = e ? e[q] : 0.f;
            }
        }
    };
    auto xform = [&](float h, float l, float ev) -> df {
        const df v = {h, l};
        return e ? df_add_f(v, ev) : v;
    };
    // own column's x_new and K at plane m from its raw words (wrap), or the wall ghost of Kwall
    auto column = [&](int m, const Raw& R, df Kwall, df& xv, df& kv) {
        if (dr_axis(m, nz, zper) >= 0) {
            xv = xform(R.xh, R.xl, R.e);
            kv = {R.kh, R.kl};
        } else {
            xv = {0.f, 0.f};
            kv = df_mul_f(Kwall, dr_factor(m < 0 ? L.bclo[2] : L.bchi[2]));
        }
    };

    float acc2 = 0.f;
    df xprev = {0.f, 0.f}, kprev = {0.f, 0.f}, gzprev = {0.f, 0.f}, part = {0.f, 0.f};
    Raw cur = {}, nxt = {};
    load_raw(z0, cur);
    if (act) {
        Raw below = {};
        load_raw(z0 - 1, below);
        column(z0 - 1, below, df{cur.kh, cur.kl}, xprev, kprev);
    }
    for (int k = z0; k <= z1; ++k) {
        const bool inplane = k < z1;
        // x_new and K of this plane's column (the plane z1 only for the z face)
        df xk = {0.f, 0.f}, kk = {0.f, 0.f};
        if (act) column(k, cur, kprev, xk, kk);
        if (inplane) {
            const long long pk = (long long)k * plane;
            if (act) {
                XH[so] = xk.hi; XL[so] = xk.lo; KH[so] = kk.hi; KL[so] = kk.lo;
                if (oh) {
                    oh[pk + own] = xk.hi;
                    ol[pk + own] = xk.lo;
                }
            }
            if (rso >= 0) {
                df xr, kr;
                if (rghost) {
                    xr = {0.f, 0.f};
                    kr = df_mul_f(df{cur.rkh, cur.rkl}, rfac);
                } else {
                    xr = xform(cur.rxh, cur.rxl, cur.re);
                    kr = {cur.rkh, cur.rkl};
                }
                XH[rso] = xr.hi; XL[rso] = xr.lo; KH[rso] = kr.hi; KL[rso] = kr.lo;
            }
        }
        if (k < z1) load_raw(k + 1, nxt);
        __syncthreads();
        // -z face against the plane below (registers); fluxes of the -x, -y faces (shared)
        df gz = {0.f, 0.f};
        if (act) gz = dw_mul(df_add(kk, kprev), df_sub(xk, xprev));
        auto flux = [&](int c, int q) -> df {    // (K_c + K_q)(x_c - x_q)
            return dw_mul(df_add(df{KH[c], KL[c]}, df{KH[q], KL[q]}),
                          df_sub(df{XH[c], XL[c]}, df{XH[q], XL[q]}));
        };
        if (inplane && act) {
            df f = flux(so, so - 1);
            FXH[ly * (DR_TX + 1) + lx] = f.hi; FXL[ly * (DR_TX + 1) + lx] = f.lo;
            if (lx == ax - 1) {
                f = flux(so + 1, so);
                FXH[ly * (DR_TX + 1) + lx + 1] = f.hi; FXL[ly * (DR_TX + 1) + lx + 1] = f.lo;
            }
            f = flux(so, so - DR_PW);
            FYH[ly * DR_TX + lx] = f.hi; FYL[ly * DR_TX + lx] = f.lo;
            if (ly == ay - 1) {
                f = flux(so + DR_PW, so);
                FYH[(ly + 1) * DR_TX + lx] = f.hi; FYL[(ly + 1) * DR_TX + lx] = f.lo;
            }
        }
        // the plane below is complete: its +z face is this plane's -z face
        if (act && k - 1 >= z0) {
            const df az = dw_sub(gzprev, gz);
            const df res = dw_sub(part, dw_mul(hz, az));
            const float r = __fadd_rn(res.hi, res.lo);
            r32[(long long)(k - 1) * plane + own] = r;
            acc2 = fmaf(r, r, acc2);
        }
        __syncthreads();
        if (inplane && act) {
            const int fx = ly * (DR_TX + 1) + lx, fy = ly * DR_TX + lx;
            const df axv = dw_sub(df{FXH[fx], FXL[fx]}, df{FXH[fx + 1], FXL[fx + 1]});
            const df ayv = dw_sub(df{FYH[fy], FYL[fy]}, df{FYH[fy + DR_TX], FYL[fy + DR_TX]});
            df res = dw_sub(df{cur.bh, cur.bl}, xk);
            res = dw_sub(res, dw_mul(hx, axv));
            part = dw_sub(res, dw_mul(hy, ayv));
        }
        xprev = xk;
        kprev = kk;
        gzprev = gz;
        cur = nxt;
    }
    const double a2 = block_sum((double)acc2, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = a2;
}

void launch_df_setup(long long n, double S, const double* E, const double* b, const double* K,
                     float* xh, float* xl, float* bh, float* bl, float* Kh, float* Kl,
                     cudaStream_t s) {
    long long nb = (n + 255) / 256;
    if (nb > num_sms() * 32) nb = num_sms() * 32;
    k_df_setup<<<(int)nb, 256, 0, s>>>(n, std::ilogb(S), E, b, K, xh, xl, bh, bl, Kh, Kl);
}

void launch_df_finish(long long n, double invS, const float* xh, const float* xl, double* E,
                      cudaStream_t s) {
    long long nb = (n + 255) / 256;
    if (nb > num_sms() * 32) nb = num_sms() * 32;
    k_df_finish<<<(int)nb, 256, 0, s>>>(n, std::ilogb(invS), xh, xl, E);
}

// Returns the number of partial sums written (the blocks of the launch, <= nblocks).
int launch_df_resid(const Lvl& L, const DfW& wd, const float* xh, const float* xl, const float* e,
                    const float* bh, const float* bl, const float* Kh, const float* Kl, float* oh,
                    float* ol, float* r32, double* partials, int nblocks, int block,
                    cudaStream_t s) {
    if (L.ndim == 3) {
        const int tiles = ((L.n[0] + DR_TX - 1) / DR_TX) * ((L.n[1] + DR_TY - 1) / DR_TY);
        if (tiles <= nblocks) {
            // z-chunks sized against the resident blocks of the whole GPU, within the
            // partial-sum slots, at least 8 planes each
            static int slots = 0;
            if (slots == 0) {
                int dev = 0, nsm = 0, occ = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_df_resid3, DR_NT, 0);
                slots = std::max(1, nsm * occ);
            }
            // the chunk count minimising waves x (planes per chunk + the 2 halo planes)
            int best = 1;
            long long bestc = -1;
            for (int c = 1; c <= std::max(1, nblocks / tiles); ++c) {
                const int czc = (L.n[2] + c - 1) / c;
                if (czc < 8 && c > 1) break;
                const long long waves = ((long long)tiles * c + slots - 1) / slots;
                const long long cost = waves * (czc + 2);
                if (bestc < 0 || cost < bestc) {
                    bestc = cost;
                    best = c;
                }
            }
            const int cz = (L.n[2] + best - 1) / best;
            const int nch = (L.n[2] + cz - 1) / cz;
            k_df_resid3<<<tiles * nch, DR_NT, 0, s>>>(L, wd, xh, xl, e, bh, bl, Kh, Kl, oh, ol,
                                                       r32, partials, cz);
            return tiles * nch;
        }
    }
    k_df_resid<<<nblocks, block, 0, s>>>(L, wd, xh, xl, e, bh, bl, Kh, Kl, oh, ol, r32, partials);
    return nblocks;
}

}  // namespace fld
