// Recursive refinement residual on 3D levels. After a refinement residual r_k = b - A x_k
// has been formed in FP64 and the FP32 V-cycles have returned the correction e, the next
// iterate and its residual are
//   x_{k+1} = x_k + e (FP64),   r_{k+1} = r_k - A e,
// where A e is evaluated in FP32 from the level's FP32 coefficients: e is of the size of
// r_k, so the FP32 rounding of A e is a few units of 2^-24 of |r_k| and of the face fluxes of
// e, far below the FP64 residual's size once r_k is. The residual is updated rather than
// recomputed (the "recursive residual" of iterative solvers), so the kernel also returns a
// bound on what the update adds to the gap between it and the true residual b - A x_{k+1}:
// per cell
//   beta = 2^-20 (|r_k| + |e_c| + sum_d (w_d/2) sum_faces |(K_c + K_q)(e_c - e_q)|),
// which covers the rounding of the stored r_k (one unit of 2^-24), the FP32 coefficients
// K = fl(K64) and weights (a unit each on every face term, three for the Dirichlet ghost's
// 3K), and the seven roundings on the longest path of the stencil's evaluation, with
// margin (2^-20 = 16 units). The rounding of the FP64 update itself, delta = fl(x + e) -
// (x + e) with |delta| <= 2^-53 |x + e|, moves the true residual by A delta, at most
// 2^-53 ||A||_2 ||x + e||_2; the kernel returns the largest absolute row sum of A (which
// bounds ||A||_2, A being symmetric) and the host bounds ||x + e||_2 by ||b||_2 (A = I plus a
// positive semi-definite part, so ||A^-1||_2 <= 1). The host adds both bounds over the
// updates since the last FP64 residual and stops only when ||r|| plus that sum is below
// the tolerance, so the reported relative residual bounds the true one up to the rounding
// of the last FP64 residual, which every refinement scheme has.
//
// The kernel has the structure of the FP32 residual of E^n: a block owns a UZ_TX x UZ_TY
// tile of the x-y plane and marches along z; the tile's e and K (and the one-cell ring:
// periodic neighbours, or the wall ghosts e = 0 with K = 3 K_wall for Dirichlet and -K_wall
// for Neumann) sit in shared memory, the planes below and above in registers, the next
// plane's words are loaded while the current one is computed. Per cell it moves 32 bytes
// (x 8 + e 4 + K 4 + r 4 read, x 8 + r 4 written) and issues one FP64 instruction (x + e,
// an FMA with a unit multiplier).
#include <algorithm>

#include "fld_device.cuh"

namespace fld {

namespace {

constexpr int UZ_TX = 32, UZ_TY = 8, UZ_NT = UZ_TX * UZ_TY;
constexpr int UZ_PW = UZ_TX + 2;                   // shared row pitch (tile + ring)

__device__ __forceinline__ int uz_axis(int g, int n, bool per) {
    if (g >= 0 && g < n) return g;
    if (per) return g < 0 ? g + n : g - n;
    return -1;
}

__device__ __forceinline__ float uz_factor(int bc) { return bc == FLD_BC_DIRICHLET ? 3.f : -1.f; }

// FP64 value of an FP32 number: integer arithmetic for normal numbers and zeros, the
// conversion instruction for the rest.
__device__ __forceinline__ double uz_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned a = u & 0x7FFFFFFFu;
    const unsigned long long sg = (unsigned long long)(u >> 31) << 63;
    if (a >= 0x00800000u && a < 0x7F800000u)
        return __longlong_as_double((long long)(((((unsigned long long)a) + (896ull << 23)) << 29) | sg));
    if (a == 0) return __longlong_as_double((long long)sg);
    return (double)f;
}

// largest value over the block (thread 0 holds it; values >= 0)
__device__ __forceinline__ float uz_block_max(float v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = (double)v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? (float)sh[threadIdx.x] : 0.f;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// The kernel forms the bracket of beta, beta' = 2^20 beta; rs (a power of two chosen from
// ||b|| on the host, so that the FP32 squares neither underflow nor overflow) scales r, and
// bs = 2^-20 rs turns beta' into rs beta. The block writes sum (rs r)^2 to
// partials[blockIdx.x], sum (rs beta)^2 to partials[gridDim.x + blockIdx.x] and its largest
// row sum of |A| to partials[2 gridDim.x + blockIdx.x].
__global__ void __launch_bounds__(UZ_NT, 5)
k_resid_update(Lvl L, const double* __restrict__ x, const float* __restrict__ e,
               double* __restrict__ xo, const float* __restrict__ K, float* __restrict__ r32,
               double* __restrict__ partials, int cz, float rs, float bs, double one) {
    __shared__ float ES[(UZ_TY + 2) * UZ_PW], KS[(UZ_TY + 2) * UZ_PW];
    __shared__ double sh[32];

    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int tilesx = (nx + UZ_TX - 1) / UZ_TX, tilesy = (ny + UZ_TY - 1) / UZ_TY;
    int bid = blockIdx.x;
    const int tx0 = (bid % tilesx) * UZ_TX;
    bid /= tilesx;
    const int ty0 = (bid % tilesy) * UZ_TY;
    bid /= tilesy;
    const int z0 = bid * cz, z1 = min(z0 + cz, nz);
    const bool xper = L.bclo[0] == FLD_BC_PERIODIC, yper = L.bclo[1] == FLD_BC_PERIODIC;
    const bool zper = L.bclo[2] == FLD_BC_PERIODIC;
    const long long plane = (long long)nx * ny;
    const float hx = 0.5f * L.wf[0], hy = 0.5f * L.wf[1], hz = 0.5f * L.wf[2];

    const int tid = threadIdx.x;
    const int lx = tid % UZ_TX, ly = tid / UZ_TX;
    const int ax = min(UZ_TX, nx - tx0), ay = min(UZ_TY, ny - ty0);
    const bool act = lx < ax && ly < ay;
    const long long own = act ? (long long)(ty0 + ly) * nx + tx0 + lx : 0;
    const int so = (ly + 1) * UZ_PW + lx + 1;

    // ring cell of this thread: left/right columns, then bottom/top rows
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
            rso = (qy + 1) * UZ_PW + qx + 1;
            const int gx = uz_axis(tx0 + qx, nx, xper), gy = uz_axis(ty0 + qy, ny, yper);
            if (gx >= 0 && gy >= 0) {
                rsrc = (long long)gy * nx + gx;
            } else {
                rghost = true;
                const int wx = qx < 0 ? 0 : (qx >= ax ? ax - 1 : qx);
                const int wy = qy < 0 ? 0 : (qy >= ay ? ay - 1 : qy);
                rsrc = (long long)(ty0 + wy) * nx + tx0 + wx;
                const int bc = gx < 0 ? (qx < 0 ? L.bclo[0] : L.bchi[0])
                                      : (qy < 0 ? L.bclo[1] : L.bchi[1]);
                rfac = uz_factor(bc);
            }
        }
    }
    // the own column at plane m: e and K, or the z-wall ghost from the wall cell's K
    auto column = [&](int m, float kwall, float& ev, float& kv) {
        const int gz = uz_axis(m, nz, zper);
        if (gz >= 0) {
            const long long q = fld_at(gz * plane + own, L.ncell);
            ev = e[q];
            kv = K[q];
        } else {
            ev = 0.f;
            kv = kwall * uz_factor(m < 0 ? L.bclo[2] : L.bchi[2]);
        }
    };
    // the words plane k needs besides the planes below: the own column's e and K at k + 1,
    // x and r at k, the ring's e and K at k; loaded one plane ahead
    struct Raw {
        double x;
        float r, e, k, re, rk;
    };
    auto fetch = [&](int k, Raw& R) {
        const int g1 = uz_axis(k + 1, nz, zper);
        if (act) {
            if (g1 >= 0) {
                const long long q = fld_at(g1 * plane + own, L.ncell);
                R.e = e[q];
                R.k = K[q];
            }
            const long long p = fld_at((long long)k * plane + own, L.ncell);
            R.x = x[p];
            R.r = r32[p];
        }
        if (rso >= 0) {
            const long long q = fld_at((long long)k * plane + rsrc, L.ncell);
            R.rk = K[q];
            if (!rghost) R.re = e[q];
        }
    };

    float accr = 0.f, accb = 0.f, amax = 0.f;
    float em = 0.f, km = 0.f, ec = 0.f, kc = 0.f, ep = 0.f, kp = 0.f;
    if (act) {
        column(z0, 0.f, ec, kc);
        column(z0 - 1, kc, em, km);
    }
    Raw cur = {}, nxt = {};
    fetch(z0, cur);
    for (int k = z0; k < z1; ++k) {
        const long long pk = (long long)k * plane;
        if (k + 1 < z1) fetch(k + 1, nxt);
        if (act) {
            if (uz_axis(k + 1, nz, zper) >= 0) {
                ep = cur.e;
                kp = cur.k;
            } else {
                ep = 0.f;
                kp = kc * uz_factor(L.bchi[2]);
            }
            ES[so] = ec;
            KS[so] = kc;
        }
        if (rso >= 0) {
            ES[rso] = rghost ? 0.f : cur.re;
            KS[rso] = rghost ? rfac * cur.rk : cur.rk;
        }
        __syncthreads();
        if (act) {
            const float a1 = kc + KS[so - 1], a2 = kc + KS[so + 1];
            const float a3 = kc + KS[so - UZ_PW], a4 = kc + KS[so + UZ_PW];
            const float a5 = kc + km, a6 = kc + kp;
            const float p1 = a1 * (ec - ES[so - 1]);
            const float p2 = a2 * (ec - ES[so + 1]);
            const float p3 = a3 * (ec - ES[so - UZ_PW]);
            const float p4 = a4 * (ec - ES[so + UZ_PW]);
            const float p5 = a5 * (ec - em);
            const float p6 = a6 * (ec - ep);
            // the row's absolute sum: 1 + 2 sum_d (w_d/2) (|a_-| + |a_+|)
            float rsum = fmaf(hx, fabsf(a1) + fabsf(a2), 0.f);
            rsum = fmaf(hy, fabsf(a3) + fabsf(a4), rsum);
            rsum = fmaf(hz, fabsf(a5) + fabsf(a6), rsum);
            amax = fmaxf(amax, fmaf(2.f, rsum, 1.f));
            const float r1 = cur.r;
            float rv = fmaf(-hx, p1 + p2, r1 - ec);
            rv = fmaf(-hy, p3 + p4, rv);
            rv = fmaf(-hz, p5 + p6, rv);
            float bnd = fmaf(hx, fabsf(p1) + fabsf(p2), fabsf(r1) + fabsf(ec));
            bnd = fmaf(hy, fabsf(p3) + fabsf(p4), bnd);
            bnd = fmaf(hz, fabsf(p5) + fabsf(p6), bnd);
            const long long p = fld_at(pk + own, L.ncell);
            r32[p] = rv;
            xo[p] = fma(uz_f64(ec), one, cur.x);
            const float rvs = rv * rs, bns = bnd * bs;
            accr = fmaf(rvs, rvs, accr);
            accb = fmaf(bns, bns, accb);
        }
        __syncthreads();
        em = ec;
        km = kc;
        ec = ep;
        kc = kp;
        cur = nxt;
    }
    // a column's squares summed in FP32 (a chunk's planes), then in FP64 across the block
    const double sr = block_sum((double)accr, sh);
    __syncthreads();
    const double sb = block_sum((double)accb, sh);
    __syncthreads();
    const float bm = uz_block_max(amax, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = sr;
        partials[gridDim.x + blockIdx.x] = sb;
        partials[2 * gridDim.x + blockIdx.x] = (double)bm;
    }
}

// The three reductions of the blocks' partials in one launch: out[0], out[1] the sums of
// the first two groups, out[2] the largest of the third.
__global__ void k_finish_update(const double* __restrict__ partials, int nparts, double* out0,
                                double* out1, double* out2) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    float m = 0.f;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) {
        a += partials[q];
        b += partials[nparts + q];
        m = fmaxf(m, (float)partials[2 * nparts + q]);
    }
    a = block_sum(a, sh);
    __syncthreads();
    b = block_sum(b, sh);
    __syncthreads();
    m = uz_block_max(m, sh);
    if (threadIdx.x == 0) {
        *out0 = a;
        *out1 = b;
        *out2 = (double)m;
    }
}

}  // namespace

bool resid_update_ok(const Lvl& L, int nblocks) {
    if (L.ndim != 3 || L.fm) return false;     // arithmetic face mean only
    const int tiles = ((L.n[0] + UZ_TX - 1) / UZ_TX) * ((L.n[1] + UZ_TY - 1) / UZ_TY);
    return tiles <= nblocks;
}

// Returns the number of blocks (nparts <= nblocks): sums of squares of the scaled residual
// in partials[0, nparts), of the scaled bound in partials[nparts, 2 nparts), the blocks'
// largest row sums in partials[2 nparts, 3 nparts).
int launch_resid_update(const Lvl& L, const double* x, const float* e, double* xo,
                        const float* K, float* r32, double* partials, int nblocks, float rs,
                        float bs, cudaStream_t s) {
    const int tiles = ((L.n[0] + UZ_TX - 1) / UZ_TX) * ((L.n[1] + UZ_TY - 1) / UZ_TY);
    // chunks of at least 16 planes, as many as the partial sums allow
    int nch = std::max(1, std::min(nblocks / tiles, (L.n[2] + 15) / 16));
    const int cz = (L.n[2] + nch - 1) / nch;
    nch = (L.n[2] + cz - 1) / cz;
    k_resid_update<<<tiles * nch, UZ_NT, 0, s>>>(L, x, e, xo, K, r32, partials, cz, rs, bs,
                                                  1.0);
    return tiles * nch;
}

void launch_finish_update(const double* partials, int nparts, double* out0, double* out1,
                          double* out2, cudaStream_t s) {
    k_finish_update<<<1, 1024, 0, s>>>(partials, nparts, out0, out1, out2);
}

}  // namespace fld
