// FP64 refinement residual on 3D levels, each face flux evaluated once:
//   r = b - A x,  (A x)_p = x_p + sum_d (w_d/2) sum_faces (K_p + K_q)(x_p - x_q)
//                         + sum_Dirichlet 2 w_d K_p x_p,
// optionally on the corrected iterate x + e (e the FP32 correction of the refinement step,
// written out of place), with the residual's FP32 image for the next FP32 V-cycles and
// per-block partial sums of r^2.
//
// FP64 instructions issue at a small fraction of the FP32 rate on this GPU, so the kernel
// is built around their count: a block owns a RZ_TX x RZ_TY tile of the x-y plane and
// marches along z; thread (lx, ly) owns one column. For each plane the tile's x and K (and
// a one-cell ring around it: periodic neighbours, or at a wall a ghost with x = 0 and
// K = 3 K_wall for Dirichlet, -K_wall for Neumann, which gives the wall face's flux
// 4 K_p x_p and 0) go to shared memory; each thread forms the flux G = (K_c + K_q)(x_c -
// x_q) of its cell's -x and -y faces (the tile's last column and row also the +x, +y
// faces of the edge) and, in registers, of its -z face against the plane below, and uses
// every flux with both signs. Per cell: three fluxes of three operations, their
// differences and the three weighted sums, against six fluxes of three operations each
// when every cell evaluates all its faces.
#include <algorithm>

#include "fld_device.cuh"

namespace fld {

namespace {

constexpr int RZ_TX = 32, RZ_TY = 8, RZ_NT = RZ_TX * RZ_TY;
constexpr int RZ_PW = RZ_TX + 2;                   // shared row pitch (tile + ring)

__device__ __forceinline__ int rz_axis(int g, int n, bool per) {
    if (g >= 0 && g < n) return g;
    if (per) return g < 0 ? g + n : g - n;
    return -1;
}

__device__ __forceinline__ double rz_factor(int bc) { return bc == FLD_BC_DIRICHLET ? 3.0 : -1.0; }

// FP64 value of an FP32 number in integer arithmetic (normal numbers and zeros; the rest
// through the conversion instruction, a branch the FP64 residual takes only for such
// values).
__device__ __forceinline__ double f64_of(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned a = u & 0x7FFFFFFFu;
    const unsigned long long sg = (unsigned long long)(u >> 31) << 63;
    if (a >= 0x00800000u && a < 0x7F800000u)
        return __longlong_as_double((long long)(((((unsigned long long)a) + (896ull << 23)) << 29) | sg));
    if (a == 0) return __longlong_as_double((long long)sg);
    return (double)f;
}

// a + b and a - b as FMAs whose multiplier `one` (1.0) arrives at run time, so the compiler
// cannot turn them back into adds: the result is the same rounded sum, and on this GPU an
// FP64 add holds the FP64 pipe about twice as long as an FMA (measured: per-cell FP64 add,
// multiply and FMA counts against the pipe's busy time in three kernels).
__device__ __forceinline__ double addf(double a, double b, double one) { return fma(a, one, b); }
__device__ __forceinline__ double subf(double a, double b, double one) { return fma(b, -one, a); }

// FP32 number nearest to v (ties away from zero) in integer arithmetic where the result is
// a normal number or zero; the rest through the conversion instruction.
__device__ __forceinline__ float f32_of(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
    const unsigned e = (unsigned)(a >> 52);
    const unsigned sg = (unsigned)(b >> 63) << 31;
    if (e >= 897u && e <= 1149u)
        return __uint_as_float(((unsigned)((a + (1ull << 28)) >> 29) - (896u << 23)) | sg);
    if (a == 0) return __uint_as_float(sg);
    return (float)v;
}

// The same conversion in integer arithmetic only, for the FP32 residual (no branch to a
// conversion instruction): below the FP32 normal range zero (subnormals flush), above it
// infinity, NaN stays NaN.
__device__ __forceinline__ float f32_of_i(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
    const unsigned e = (unsigned)(a >> 52);
    const unsigned sg = (unsigned)(b >> 63) << 31;
    unsigned r = (unsigned)((a + (1ull << 28)) >> 29) - (896u << 23);        // normal
    if (e < 897u) r = 0;
    if (e > 1149u) r = (e == 2047u && (a << 12)) ? 0x7FC00000u : 0x7F800000u;
    return __uint_as_float(r | sg);
}

__global__ void __launch_bounds__(RZ_NT, 5)
k_resid64z(Lvl L, const double* __restrict__ x, const float* __restrict__ e,
           double* __restrict__ xo, const double* __restrict__ b, const double* __restrict__ K,
           float* __restrict__ r32, double* __restrict__ partials, int cz, double one) {
    __shared__ double XS[(RZ_TY + 2) * RZ_PW], KS[(RZ_TY + 2) * RZ_PW];
    __shared__ double FX[RZ_TY * (RZ_TX + 1)], FY[(RZ_TY + 1) * RZ_TX];
    __shared__ double sh[32];

    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int tilesx = (nx + RZ_TX - 1) / RZ_TX, tilesy = (ny + RZ_TY - 1) / RZ_TY;
    int bid = blockIdx.x;
    const int tx0 = (bid % tilesx) * RZ_TX;
    bid /= tilesx;
    const int ty0 = (bid % tilesy) * RZ_TY;
    bid /= tilesy;
    const int z0 = bid * cz, z1 = min(z0 + cz, nz);
    const bool xper = L.bclo[0] == FLD_BC_PERIODIC, yper = L.bclo[1] == FLD_BC_PERIODIC;
    const bool zper = L.bclo[2] == FLD_BC_PERIODIC;
    const long long plane = (long long)nx * ny;
    const double hx = 0.5 * L.w[0], hy = 0.5 * L.w[1], hz = 0.5 * L.w[2];

    const int tid = threadIdx.x;
    const int lx = tid % RZ_TX, ly = tid / RZ_TX;
    const int ax = min(RZ_TX, nx - tx0), ay = min(RZ_TY, ny - ty0);
    const bool act = lx < ax && ly < ay;
    const long long own = act ? (long long)(ty0 + ly) * nx + tx0 + lx : 0;
    const int so = (ly + 1) * RZ_PW + lx + 1;

    // ring cell of this thread: left/right columns, then bottom/top rows
    int rso = -1;              // its shared offset (-1: none)
    long long rsrc = 0;        // plane offset of the value it copies (the wall cell for a ghost)
    bool rghost = false;
    double rfac = 0.0;
    {
        int qx = 0, qy = 0;
        bool has = true;
        if (tid < ay) { qx = -1; qy = tid; }
        else if (tid < 2 * ay) { qx = ax; qy = tid - ay; }
        else if (tid < 2 * ay + ax) { qx = tid - 2 * ay; qy = -1; }
        else if (tid < 2 * ay + 2 * ax) { qx = tid - 2 * ay - ax; qy = ay; }
        else has = false;
        if (has) {
            rso = (qy + 1) * RZ_PW + qx + 1;
            const int gx = rz_axis(tx0 + qx, nx, xper), gy = rz_axis(ty0 + qy, ny, yper);
            if (gx >= 0 && gy >= 0) {
                rsrc = (long long)gy * nx + gx;
            } else {
                rghost = true;
                const int wx = qx < 0 ? 0 : (qx >= ax ? ax - 1 : qx);
                const int wy = qy < 0 ? 0 : (qy >= ay ? ay - 1 : qy);
                rsrc = (long long)(ty0 + wy) * nx + tx0 + wx;
                const int bc = gx < 0 ? (qx < 0 ? L.bclo[0] : L.bchi[0])
                                      : (qy < 0 ? L.bclo[1] : L.bchi[1]);
                rfac = rz_factor(bc);
            }
        }
    }

    // words of one plane for the own column and the ring cell, loaded a plane ahead
    struct Raw {
        double x, k, b, rx, rk;
        float e, re;
    };
    auto load_raw = [&](int m, Raw& R) {
        const int gz = rz_axis(m, nz, zper);
        if (gz < 0) return;                   // a wall ghost plane: formed from K below
        const long long pk = gz * plane;
        if (act) {
            const long long q = fld_at(pk + own, L.ncell);
            R.x = x[q];
            R.k = K[q];
            R.e = e ? e[q] : 0.f;
            if (m < z1) R.b = b[q];
        }
        if (rso >= 0 && m < z1) {
            const long long q = fld_at(pk + rsrc, L.ncell);
            R.rk = K[q];
            if (!rghost) {
                R.rx = x[q];
                R.re = e ? e[q] : 0.f;
            }
        }
    };
    auto xnew = [&](double v, float ev) -> double { return e ? addf(v, f64_of(ev), one) : v; };
    // own column's x_new and K at plane m (wrapped), or the wall ghost from Kwall
    auto column = [&](int m, const Raw& R, double Kwall, double& xv, double& kv) {
        if (rz_axis(m, nz, zper) >= 0) {
            xv = xnew(R.x, R.e);
            kv = R.k;
        } else {
            xv = 0.0;
            kv = Kwall * rz_factor(m < 0 ? L.bclo[2] : L.bchi[2]);
        }
    };

    double acc2 = 0.0;
    double xprev = 0.0, kprev = 0.0, gzprev = 0.0, part = 0.0;
    Raw cur = {}, nxt = {};
    load_raw(z0, cur);
    if (act) {
        Raw below = {};
        load_raw(z0 - 1, below);
        column(z0 - 1, below, cur.k, xprev, kprev);
    }
    for (int k = z0; k <= z1; ++k) {
        const bool inplane = k < z1;
        double xk = 0.0, kk = 0.0;
        if (act) column(k, cur, kprev, xk, kk);
        if (inplane) {
            if (act) {
                XS[so] = xk;
                KS[so] = kk;
                if (xo) xo[fld_at((long long)k * plane + own, L.ncell)] = xk;
            }
            if (rso >= 0) {
                XS[rso] = rghost ? 0.0 : xnew(cur.rx, cur.re);
                KS[rso] = rghost ? rfac * cur.rk : cur.rk;
            }
        }
        if (k < z1) load_raw(k + 1, nxt);
        __syncthreads();
        // -z face against the plane below (registers); fluxes of the -x, -y faces (shared)
        // the flux (K_c + K_q)(x_c - x_q) of a face
        auto flux = [&](double kc, double kq, double xc, double xq) {
            return addf(kc, kq, one) * subf(xc, xq, one);
        };
        double gz = 0.0;
        if (act) gz = flux(kk, kprev, xk, xprev);
        if (inplane && act) {
            FX[ly * (RZ_TX + 1) + lx] = flux(KS[so], KS[so - 1], XS[so], XS[so - 1]);
            if (lx == ax - 1)
                FX[ly * (RZ_TX + 1) + lx + 1] = flux(KS[so + 1], KS[so], XS[so + 1], XS[so]);
            FY[ly * RZ_TX + lx] = flux(KS[so], KS[so - RZ_PW], XS[so], XS[so - RZ_PW]);
            if (ly == ay - 1)
                FY[(ly + 1) * RZ_TX + lx] = flux(KS[so + RZ_PW], KS[so], XS[so + RZ_PW], XS[so]);
        }
        // the plane below is complete: its +z face is this plane's -z face
        if (act && k - 1 >= z0) {
            const double r = fma(-hz, subf(gzprev, gz, one), part);
            if (r32) r32[fld_at((long long)(k - 1) * plane + own, L.ncell)] = f32_of(r);
            acc2 = fma(r, r, acc2);
        }
        __syncthreads();
        if (inplane && act) {
            const int fx = ly * (RZ_TX + 1) + lx, fy = ly * RZ_TX + lx;
            const double r = fma(-hx, subf(FX[fx], FX[fx + 1], one), subf(cur.b, xk, one));
            part = fma(-hy, subf(FY[fy], FY[fy + RZ_TX], one), r);
        }
        xprev = xk;
        kprev = kk;
        gzprev = gz;
        cur = nxt;
    }
    const double a2 = block_sum(acc2, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = a2;
}

int g_rz_slots[64];        // resident blocks of the kernel on the whole GPU, per device

}  // namespace

bool resid64z_ok(const Lvl& L, int nblocks) {
    if (L.ndim != 3 || L.fm) return false;     // arithmetic face mean only
    const int tiles = ((L.n[0] + RZ_TX - 1) / RZ_TX) * ((L.n[1] + RZ_TY - 1) / RZ_TY);
    return tiles <= nblocks;
}

// Returns the number of partial sums written (the blocks of the launch, <= nblocks).
int launch_resid64z(const Lvl& L, const double* x, const float* e, double* xo, const double* b,
                    const double* K, float* r32, double* partials, int nblocks, cudaStream_t s) {
    const int tiles = ((L.n[0] + RZ_TX - 1) / RZ_TX) * ((L.n[1] + RZ_TY - 1) / RZ_TY);
    int dev = 0;
    cudaGetDevice(&dev);
    int slots = (dev >= 0 && dev < 64) ? g_rz_slots[dev] : 0;
    if (slots <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_resid64z, RZ_NT, 0);
        slots = std::max(1, num_sms() * occ);
        if (dev >= 0 && dev < 64) g_rz_slots[dev] = slots;
    }
    // the chunk count minimising waves x (planes per chunk + the 2 halo planes), within
    // the partial-sum slots, at least 8 planes a chunk
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
    k_resid64z<<<tiles * nch, RZ_NT, 0, s>>>(L, x, e, xo, b, K, r32, partials, cz, 1.0);
    return tiles * nch;
}


// ----------------------------------------------------------------- FP32 initial residual
// The right-hand side of the mixed refinement's first correction: r = b - A x in FP32
// arithmetic from the FP64 iterate x and right-hand side b (their FP32 images, formed in
// integer arithmetic) and the FP32 coefficients K, with per-block partial sums of r^2 (the
// first entry of the residual history). The first FP32 V-cycles then start the iterate from
// an FP32 solve, as mixed-precision iterative refinement does; every later residual, which
// decides convergence, is the FP64 one above.
namespace {

__global__ void k_resid32_init(Lvl L, const double* __restrict__ x, const double* __restrict__ b,
                               const float* __restrict__ K, float* __restrict__ r32,
                               double* __restrict__ partials) {
    __shared__ double sh[32];
    double acc2 = 0.0;
    const int nx = L.n[0], ny = L.n[1];
    const int nrows = ny * L.n[2];
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int j = r % ny, k = r / ny;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const long long p = (long long)r * nx + i;
            float sw, acc;
            // the level operator's stencil on the FP32 images of x
            const float Kc = K[p];
            const int c[3] = {i, j, k};
            long long stride = 1;
            sw = 0.f;
            acc = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d < L.ndim) {
                    const int n = L.n[d];
                    const float wd = L.wf[d];
                    long long q = -1;
                    if (c[d] > 0) q = p - stride;
                    else if (L.bclo[d] == FLD_BC_PERIODIC) q = p + (n - 1) * stride;
                    if (q >= 0) {
                        const float w = fmean(Kc, K[q], L.fm) * wd;
                        sw += w;
                        acc = fmaf(w, f32_of(x[q]), acc);
                    } else if (L.bclo[d] == FLD_BC_DIRICHLET) {
                        sw += 2.f * Kc * wd;
                    }
                    q = -1;
                    if (c[d] < n - 1) q = p + stride;
                    else if (L.bchi[d] == FLD_BC_PERIODIC) q = p - (n - 1) * stride;
                    if (q >= 0) {
                        const float w = fmean(Kc, K[q], L.fm) * wd;
                        sw += w;
                        acc = fmaf(w, f32_of(x[q]), acc);
                    } else if (L.bchi[d] == FLD_BC_DIRICHLET) {
                        sw += 2.f * Kc * wd;
                    }
                    stride *= n;
                }
            }
            const float rv = f32_of(b[p]) - fmaf(1.f + sw, f32_of(x[p]), -acc);
            r32[p] = rv;
            acc2 = fma((double)rv, (double)rv, acc2);
        }
    }
    acc2 = block_sum(acc2, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc2;
}

// The same residual on 3D levels, marching along z like k_resid64z: a block owns a
// RZ_TX x RZ_TY tile, the FP32 images of x and K of the current plane (and the one-cell
// ring: periodic neighbours, or the wall ghosts x = 0, K = 3 K_wall for Dirichlet and
// -K_wall for Neumann) sit in shared memory, the planes below and above in registers. Each
// cell evaluates its seven-point stencil in FP32; x and b are read once as FP64 and
// converted in integer arithmetic.
__global__ void __launch_bounds__(RZ_NT)
k_resid32z(Lvl L, const double* __restrict__ x, const double* __restrict__ b,
           const float* __restrict__ K, float* __restrict__ r32, double* __restrict__ partials,
           int cz) {
    __shared__ float XS[(RZ_TY + 2) * RZ_PW], KS[(RZ_TY + 2) * RZ_PW];
    __shared__ double sh[32];

    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int tilesx = (nx + RZ_TX - 1) / RZ_TX, tilesy = (ny + RZ_TY - 1) / RZ_TY;
    int bid = blockIdx.x;
    const int tx0 = (bid % tilesx) * RZ_TX;
    bid /= tilesx;
    const int ty0 = (bid % tilesy) * RZ_TY;
    bid /= tilesy;
    const int z0 = bid * cz, z1 = min(z0 + cz, nz);
    const bool xper = L.bclo[0] == FLD_BC_PERIODIC, yper = L.bclo[1] == FLD_BC_PERIODIC;
    const bool zper = L.bclo[2] == FLD_BC_PERIODIC;
    const long long plane = (long long)nx * ny;
    const float hx = 0.5f * L.wf[0], hy = 0.5f * L.wf[1], hz = 0.5f * L.wf[2];

    const int tid = threadIdx.x;
    const int lx = tid % RZ_TX, ly = tid / RZ_TX;
    const int ax = min(RZ_TX, nx - tx0), ay = min(RZ_TY, ny - ty0);
    const bool act = lx < ax && ly < ay;
    const long long own = act ? (long long)(ty0 + ly) * nx + tx0 + lx : 0;
    const int so = (ly + 1) * RZ_PW + lx + 1;

    int rso = -1;
    long long rsrc = 0;
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
            rso = (qy + 1) * RZ_PW + qx + 1;
            const int gx = rz_axis(tx0 + qx, nx, xper), gy = rz_axis(ty0 + qy, ny, yper);
            if (gx >= 0 && gy >= 0) {
                rsrc = (long long)gy * nx + gx;
            } else {
                rghost = true;
                const int wx = qx < 0 ? 0 : (qx >= ax ? ax - 1 : qx);
                const int wy = qy < 0 ? 0 : (qy >= ay ? ay - 1 : qy);
                rsrc = (long long)(ty0 + wy) * nx + tx0 + wx;
                const int bc = gx < 0 ? (qx < 0 ? L.bclo[0] : L.bchi[0])
                                      : (qy < 0 ? L.bclo[1] : L.bchi[1]);
                rfac = (float)rz_factor(bc);
            }
        }
    }
    // the own column at plane m: the FP32 images, or the z-wall ghost from the wall cell's K
    auto column = [&](int m, float kwall, float& xv, float& kv) {
        const int gz = rz_axis(m, nz, zper);
        if (gz >= 0) {
            const long long q = fld_at(gz * plane + own, L.ncell);
            xv = f32_of_i(x[q]);
            kv = K[q];
        } else {
            xv = 0.f;
            kv = kwall * (float)rz_factor(m < 0 ? L.bclo[2] : L.bchi[2]);
        }
    };
    // the words plane k needs besides the planes below: the own column at k + 1, b at k and
    // the ring at k, loaded one plane ahead (while plane k - 1 is computed)
    struct Raw {
        double x, b, rx;
        float k, rk;
    };
    auto fetch = [&](int k, Raw& R) {
        const int g1 = rz_axis(k + 1, nz, zper);
        if (act) {
            if (g1 >= 0) {
                const long long q = fld_at(g1 * plane + own, L.ncell);
                R.x = x[q];
                R.k = K[q];
            }
            R.b = b[fld_at((long long)k * plane + own, L.ncell)];
        }
        if (rso >= 0) {
            const long long q = fld_at((long long)k * plane + rsrc, L.ncell);
            R.rk = K[q];
            if (!rghost) R.rx = x[q];
        }
    };

    float acc2f = 0.f;
    float xm = 0.f, km = 0.f, xc = 0.f, kc = 0.f, xp = 0.f, kp = 0.f;
    if (act) {
        column(z0, 0.f, xc, kc);
        column(z0 - 1, kc, xm, km);
    }
    Raw cur = {}, nxt = {};
    fetch(z0, cur);
    for (int k = z0; k < z1; ++k) {
        const long long pk = (long long)k * plane;
        if (k + 1 < z1) fetch(k + 1, nxt);
        float bk = 0.f;
        if (act) {
            if (rz_axis(k + 1, nz, zper) >= 0) {
                xp = f32_of_i(cur.x);
                kp = cur.k;
            } else {
                xp = 0.f;
                kp = kc * (float)rz_factor(L.bchi[2]);
            }
            bk = f32_of_i(cur.b);
            XS[so] = xc;
            KS[so] = kc;
        }
        if (rso >= 0) {
            XS[rso] = rghost ? 0.f : f32_of_i(cur.rx);
            KS[rso] = rghost ? rfac * cur.rk : cur.rk;
        }
        __syncthreads();
        if (act) {
            float sx = (kc + KS[so - 1]) * (xc - XS[so - 1]);
            sx = fmaf(kc + KS[so + 1], xc - XS[so + 1], sx);
            float sy = (kc + KS[so - RZ_PW]) * (xc - XS[so - RZ_PW]);
            sy = fmaf(kc + KS[so + RZ_PW], xc - XS[so + RZ_PW], sy);
            float sz = (kc + km) * (xc - xm);
            sz = fmaf(kc + kp, xc - xp, sz);
            float rv = fmaf(-hx, sx, bk - xc);
            rv = fmaf(-hy, sy, rv);
            rv = fmaf(-hz, sz, rv);
            r32[fld_at(pk + own, L.ncell)] = rv;
            acc2f = fmaf(rv, rv, acc2f);
        }
        __syncthreads();
        xm = xc;
        km = kc;
        xc = xp;
        kc = kp;
        cur = nxt;
    }
    // the squares of this column summed in FP32 (a chunk's planes at most: the norm only
    // reports and screens the first residual), then in FP64 across the block
    const double acc2 = (double)acc2f;
    const double a2 = block_sum(acc2, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = a2;
}

}  // namespace

// Returns the number of partial sums written (<= nblocks).
int launch_resid32_init(const Lvl& L, const double* x, const double* b, const float* K,
                        float* r32, double* partials, int nblocks, cudaStream_t s) {
    if (resid64z_ok(L, nblocks)) {
        const int tiles = ((L.n[0] + RZ_TX - 1) / RZ_TX) * ((L.n[1] + RZ_TY - 1) / RZ_TY);
        // chunks of at least 16 planes, as many as the partial sums allow
        int nch = std::max(1, std::min(nblocks / tiles, (L.n[2] + 15) / 16));
        const int cz = (L.n[2] + nch - 1) / nch;
        nch = (L.n[2] + cz - 1) / cz;
        k_resid32z<<<tiles * nch, RZ_NT, 0, s>>>(L, x, b, K, r32, partials, cz);
        return tiles * nch;
    }
    const int nb = (int)std::max<long long>(1, std::min<long long>((long long)L.n[1] * L.n[2],
                                                                      nblocks));
    k_resid32_init<<<nb, 256, 0, s>>>(L, x, b, K, r32, partials);
    return nb;
}

}  // namespace fld
