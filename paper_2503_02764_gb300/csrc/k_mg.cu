// Geometric multigrid kernels for the backward-Euler diffusion solve
//   A x = x - dt div(D grad x) = b
// on cell-centred finite volumes (face D = arithmetic or harmonic mean of the two cell
// values, the level's fm). Per level the operator is stored as K = dt D / H_x^2 per cell
// with axis weights w_d = (H_x/H_d)^2:
//   (A x)_p = x_p + sum_{faces p|q} mean(K_p, K_q) w_d (x_p - x_q) + sum_{Dirichlet} 2 K_p w_d x_p.
// Coarse levels average K over the (up to 2^d) children and rescale it to the coarse
// spacing; restriction averages residuals; prolongation is cell-centred linear (weights
// 3/4 and 1/4 per coarsened axis, tensor product over the axes) or, with the level's pk,
// piecewise constant.
// Every kernel here is templated on the storage/arithmetic type (double or float).
#include <algorithm>

#include "fld_device.cuh"

namespace fld {

static inline int grid_for(long long n, int block, int cap = 0) {
    if (cap <= 0) cap = num_sms() * 32;
    long long nb = (n + block - 1) / block;
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    return (int)nb;
}

// Row mapping: a block walks rows r = (j, k) (grid-stride over ny*nz rows) and its
// threads walk i along the row, so no per-cell integer division is needed.
static inline int rows_grid(const Lvl& L, int cap = 0) {
    if (cap <= 0) cap = num_sms() * 64;
    long long nr = (long long)L.n[1] * L.n[2];
    return (int)std::min<long long>(std::max<long long>(nr, 1), cap);
}

// ----------------------------------------------------------------- level-0 set-up
// K = kscale D (kscale = dt / h_x^2), its FP32 copy, and b = E + Dirichlet face terms
// 2 K w_d E_b. With kmax, the largest K (its FP32 value, K >= 0) is folded into *kmax by
// an integer atomicMax of its bits (non-negative FP32 numbers order as their bit patterns).
struct BcOffM {
    long long off[6];
};

__global__ void __launch_bounds__(256)
k_prep_level0(Lvl L, double kscale, const double* __restrict__ D,
              const double* __restrict__ E, const double* __restrict__ Ebc, BcOffM bo,
              double* __restrict__ K64, float* __restrict__ K32, double* __restrict__ b,
              unsigned* err, unsigned* kmax) {
    __shared__ float wmax[8];
    float km = 0.f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L.ncell;
         p += (long long)gridDim.x * blockDim.x) {
        const double Dp = D[p];
        if (!pos_finite(Dp)) atomicOr(err, ERRBIT_DOMAIN);
        const double Kp = kscale * Dp;
        km = fmaxf(km, (float)Kp);
        K64[p] = Kp;
        if (K32) K32[p] = (float)Kp;
        double bp = E[p];
        if (Ebc) {
            int c[3];
            decode(L, p, c[0], c[1], c[2]);
            for (int d = 0; d < L.ndim; ++d) {
                long long fi;
                if (d == 0) fi = (long long)c[2] * L.n[1] + c[1];
                else if (d == 1) fi = (long long)c[2] * L.n[0] + c[0];
                else fi = (long long)c[1] * L.n[0] + c[0];
                if (c[d] == 0 && L.bclo[d] == FLD_BC_DIRICHLET)
                    bp += 2.0 * Kp * L.w[d] * Ebc[bo.off[2 * d] + fi];
                if (c[d] == L.n[d] - 1 && L.bchi[d] == FLD_BC_DIRICHLET)
                    bp += 2.0 * Kp * L.w[d] * Ebc[bo.off[2 * d + 1] + fi];
            }
        }
        b[p] = bp;
    }
    if (!kmax) return;
    for (int o = 16; o > 0; o >>= 1) km = fmaxf(km, __shfl_down_sync(0xffffffffu, km, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = km;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) km = fmaxf(km, wmax[q]);
        if (km > 0.f) atomicMax(kmax, __float_as_uint(km));
    }
}

void launch_prep_level0(const Lvl& L, double kscale, const double* D, const double* E,
                        const double* E_bc, const long long* bc_off, double* K64, float* K32,
                        double* b, unsigned* err, unsigned* kmax, cudaStream_t s) {
    BcOffM bo;
    for (int q = 0; q < 6; ++q) bo.off[q] = bc_off[q];
    k_prep_level0<<<grid_for(L.ncell, 256), 256, 0, s>>>(L, kscale, D, E, E_bc, bo, K64, K32, b,
                                                         err, kmax);
}

// ----------------------------------------------------------------- transfers
// Children of coarse index I along axis d: {2I, 2I+1} (clipped) if the axis was
// coarsened, else {I}.
template <typename T>
__global__ void k_restrict_K(Lvl F, Lvl C, double scale, const T* __restrict__ Kf,
                             T* __restrict__ Kc) {
    const T sc = (T)scale;
    for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < C.ncell;
         P += (long long)gridDim.x * blockDim.x) {
        int c[3];
        decode(C, P, c[0], c[1], c[2]);
        int lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            if (C.n[d] < F.n[d]) {
                lo[d] = 2 * c[d];
                hi[d] = min(2 * c[d] + 1, F.n[d] - 1);
            } else {
                lo[d] = hi[d] = c[d];
            }
        }
        // the mean in the level's own type (the FP32 pyramid preconditions only; the FP64
        // one keeps FP64 sums); the child count is a power of two, so its reciprocal is exact
        T s = T(0);
        int cnt = 0;
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    s += Kf[((long long)k * F.n[1] + j) * F.n[0] + i];
                    ++cnt;
                }
        const T inv = cnt == 8 ? T(0.125) : cnt == 4 ? T(0.25) : cnt == 2 ? T(0.5) : T(1);
        Kc[P] = (sc * inv) * s;
    }
}

template <typename T>
void launch_restrict_K(const Lvl& F, const Lvl& C, double scale, const T* Kf, T* Kc,
                       cudaStream_t s) {
    k_restrict_K<T><<<grid_for(C.ncell, 256), 256, 0, s>>>(F, C, scale, Kf, Kc);
}

// Red-black Gauss-Seidel half sweep, out of place: cells of `color` ((i+j+k) mod 2)
// get (b + acc)/(1 + sw) from xin; the other colour is copied. Reading xin only makes
// the result independent of thread order; on an odd periodic extent two same-colour
// neighbours across the wrap then couple Jacobi-style.
template <typename T>
__global__ void k_smooth(Lvl L, int color, const T* __restrict__ xin, T* __restrict__ xout,
                         const T* __restrict__ b, const T* __restrict__ K) {
    const int nrows = L.n[1] * L.n[2];
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int j = r % L.n[1], k = r / L.n[1];
        const long long base = (long long)r * L.n[0];
        for (int i = threadIdx.x; i < L.n[0]; i += blockDim.x) {
            const long long p = base + i;
            if (((i + j + k) & 1) != color) {
                xout[p] = xin[p];
                continue;
            }
            T sw, acc;
            stencil<T>(L, K, xin, i, j, k, p, sw, acc);
            xout[p] = (b[p] + acc) / (T(1) + sw);
        }
    }
}

template <typename T>
void launch_smooth(const Lvl& L, int color, const T* xin, T* xout, const T* b, const T* K,
                   int block, cudaStream_t s) {
    k_smooth<T><<<rows_grid(L), block, 0, s>>>(L, color, xin, xout, b, K);
}

// In-place red-black half sweep: only cells of `color` are updated, from neighbours
// of the other colour. One thread per pair of cells along x (the one of `color`),
// a row (j, k) per block row, so the index arithmetic is a few integer operations.
// Valid when no periodic axis has an odd extent (otherwise two same-colour cells
// meet across the wrap and would race); the caller checks.
// One colour-`color` cell (i, j, k) of an in-place half sweep.
template <typename T>
__device__ __forceinline__ void rb_cell(const Lvl& L, int i, int j, int k, T* __restrict__ x,
                                        const T* __restrict__ b, const T* __restrict__ K) {
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int sy = nx, sz = nx * ny;
    const int p = (int)fld_at((k * ny + j) * nx + i, L.ncell);
    const T kc = K[p];
    T sw = T(0), acc = T(0);
    const T wx = wgt<T>(L, 0);
    int q = i > 0 ? p - 1 : (L.bclo[0] == FLD_BC_PERIODIC ? p + nx - 1 : -1);
    if (q >= 0) { q = (int)fld_at(q, L.ncell); const T w = fmean(kc, K[q], L.fm) * wx; sw += w; acc += w * x[q]; }
    else if (L.bclo[0] == FLD_BC_DIRICHLET) sw += T(2) * kc * wx;
    q = i < nx - 1 ? p + 1 : (L.bchi[0] == FLD_BC_PERIODIC ? p - nx + 1 : -1);
    if (q >= 0) { q = (int)fld_at(q, L.ncell); const T w = fmean(kc, K[q], L.fm) * wx; sw += w; acc += w * x[q]; }
    else if (L.bchi[0] == FLD_BC_DIRICHLET) sw += T(2) * kc * wx;
    if (L.ndim >= 2) {
        const T wy = wgt<T>(L, 1);
        q = j > 0 ? p - sy : (L.bclo[1] == FLD_BC_PERIODIC ? p + (ny - 1) * sy : -1);
        if (q >= 0) { q = (int)fld_at(q, L.ncell); const T w = fmean(kc, K[q], L.fm) * wy; sw += w; acc += w * x[q]; }
        else if (L.bclo[1] == FLD_BC_DIRICHLET) sw += T(2) * kc * wy;
        q = j < ny - 1 ? p + sy : (L.bchi[1] == FLD_BC_PERIODIC ? p - (ny - 1) * sy : -1);
        if (q >= 0) { q = (int)fld_at(q, L.ncell); const T w = fmean(kc, K[q], L.fm) * wy; sw += w; acc += w * x[q]; }
        else if (L.bchi[1] == FLD_BC_DIRICHLET) sw += T(2) * kc * wy;
    }
    if (L.ndim >= 3) {
        const T wz = wgt<T>(L, 2);
        q = k > 0 ? p - sz : (L.bclo[2] == FLD_BC_PERIODIC ? p + (nz - 1) * sz : -1);
        if (q >= 0) { q = (int)fld_at(q, L.ncell); const T w = fmean(kc, K[q], L.fm) * wz; sw += w; acc += w * x[q]; }
        else if (L.bclo[2] == FLD_BC_DIRICHLET) sw += T(2) * kc * wz;
        q = k < nz - 1 ? p + sz : (L.bchi[2] == FLD_BC_PERIODIC ? p - (nz - 1) * sz : -1);
        if (q >= 0) { q = (int)fld_at(q, L.ncell); const T w = fmean(kc, K[q], L.fm) * wz; sw += w; acc += w * x[q]; }
        else if (L.bchi[2] == FLD_BC_DIRICHLET) sw += T(2) * kc * wz;
    }
    x[p] = div_fast<T>(b[p] + acc, T(1) + sw);
}

// In-place red-black half sweep: only cells of `color` are updated, from neighbours
// of the other colour. One thread per pair of cells along x (the one of `color`) on
// ZU planes spaced nz/ZU apart (independent cells in flight per thread), a row (j, k)
// per block row, so the index arithmetic is a few integer operations. Valid when no
// periodic axis has an odd extent (two same-colour cells would meet across the wrap and
// race); the caller checks.
template <typename T>
__global__ void k_rb_half(Lvl L, int color, T* __restrict__ x, const T* __restrict__ b,
                          const T* __restrict__ K) {
    // block = (pairs along x) x (rows along y): neighbouring rows of a tile share L1
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (j >= L.n[1]) return;
    const int i = 2 * ip + ((j + k + color) & 1);
    if (i < L.n[0]) rb_cell<T>(L, i, j, k, x, b, K);
}

template <typename T>
bool rb_half_supported(const Lvl& L) {
    for (int d = 0; d < L.ndim; ++d)
        if (L.bclo[d] == FLD_BC_PERIODIC && (L.n[d] & 1)) return false;
    return L.n[1] <= 65535 && L.n[2] <= 65535;
}

template <typename T>
void launch_rb_half(const Lvl& L, int color, T* x, const T* b, const T* K, cudaStream_t s) {
    const int pairs = (L.n[0] + 1) / 2;
    // x-y tiles of 32 pairs x 8 rows on wide levels, one row of up to 128 pairs otherwise
    const int bx = pairs >= 32 ? 32 : ((pairs + 7) / 8) * 8;
    const int by = pairs >= 32 ? 8 : 1;
    dim3 block(pairs >= 32 ? bx : (pairs >= 128 ? 128 : ((pairs + 31) / 32) * 32), by);
    dim3 grid((pairs + block.x - 1) / block.x, (L.n[1] + by - 1) / by, L.n[2]);
    k_rb_half<T><<<grid, block, 0, s>>>(L, color, x, b, K);
}

// Coarse right-hand side = average of the fine residuals b - A x over the children.
template <typename T>
__global__ void k_resid_restrict(Lvl F, Lvl C, const T* __restrict__ x, const T* __restrict__ b,
                                 const T* __restrict__ K, T* __restrict__ bc) {
    for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < C.ncell;
         P += (long long)gridDim.x * blockDim.x) {
        int c[3];
        decode(C, P, c[0], c[1], c[2]);
        int lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            if (C.n[d] < F.n[d]) {
                lo[d] = 2 * c[d];
                hi[d] = min(2 * c[d] + 1, F.n[d] - 1);
            } else {
                lo[d] = hi[d] = c[d];
            }
        }
        T s = T(0);
        int cnt = 0;
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    const long long p = ((long long)k * F.n[1] + j) * F.n[0] + i;
                    T sw, acc;
                    stencil<T>(F, K, x, i, j, k, p, sw, acc);
                    s += b[p] - (T(1) + sw) * x[p] + acc;
                    ++cnt;
                }
        bc[P] = s / T(cnt);
    }
}

template <typename T>
void launch_resid_restrict(const Lvl& F, const Lvl& C, const T* x, const T* b, const T* K, T* bc,
                           int block, bool red_only, cudaStream_t s) {
    if (transfer3_ok(F, C) && !F.fm)
        return launch_resid_restrict3<T>(F, C, x, b, K, bc, red_only, s);
    k_resid_restrict<T><<<grid_for(C.ncell, block), block, 0, s>>>(F, C, x, b, K, bc);
}

template <typename T>
__global__ void k_prolong(Lvl F, Lvl C, T* __restrict__ xf, const T* __restrict__ xc) {
    const int nrows = F.n[1] * F.n[2];
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int j = r % F.n[1], k = r / F.n[1];
        const long long base = (long long)r * F.n[0];
        const Interp iy = interp1(j, F.n[1], C.n[1], F.bclo[1], F.bchi[1], F.pk);
        const Interp iz = interp1(k, F.n[2], C.n[2], F.bclo[2], F.bchi[2], F.pk);
        for (int i = threadIdx.x; i < F.n[0]; i += blockDim.x) {
            const Interp ix = interp1(i, F.n[0], C.n[0], F.bclo[0], F.bchi[0], F.pk);
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const T wzy = (T)(iz.wt[c] * iy.wt[b]);
                    if (wzy == T(0)) continue;
                    const long long rowc = ((long long)iz.idx[c] * C.n[1] + iy.idx[b]) * C.n[0];
                    acc += wzy * ((T)ix.wt[0] * xc[rowc + ix.idx[0]] +
                                  (T)ix.wt[1] * xc[rowc + ix.idx[1]]);
                }
            xf[base + i] += acc;
        }
    }
}

template <typename T>
void launch_prolong(const Lvl& F, const Lvl& C, T* xf, const T* xc, int block, cudaStream_t s) {
    if (transfer3_ok(F, C) && !F.pk) return launch_prolong3<T>(F, C, xf, xc, s);
    k_prolong<T><<<rows_grid(F), block, 0, s>>>(F, C, xf, xc);
}

// Coarsest level: `sweeps` red-black sweeps from x = 0 by one block, in FP64 whatever
// the storage type, the level held in shared memory (ncell <= MAX_COARSE, 32 KB).
constexpr int MAX_COARSE = 1024;

template <typename T>
__global__ void k_coarse_solve(Lvl L, T* __restrict__ x, const T* __restrict__ b,
                               const T* __restrict__ K, int sweeps) {
    __shared__ double xs[MAX_COARSE], bs[MAX_COARSE], Ks[MAX_COARSE], nx[MAX_COARSE];
    const int n = (int)L.ncell;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        xs[p] = 0.0;
        bs[p] = (double)b[p];
        Ks[p] = (double)K[p];
    }
    __syncthreads();
    for (int it = 0; it < sweeps; ++it) {
        for (int color = 0; color < 2; ++color) {
            for (int p = threadIdx.x; p < n; p += blockDim.x) {
                int i, j, k;
                decode(L, p, i, j, k);
                if (((i + j + k) & 1) != color) continue;
                double sw, acc;
                stencil<double>(L, Ks, xs, i, j, k, p, sw, acc);
                nx[p] = (bs[p] + acc) / (1.0 + sw);
            }
            __syncthreads();
            for (int p = threadIdx.x; p < n; p += blockDim.x) {
                int i, j, k;
                decode(L, p, i, j, k);
                if (((i + j + k) & 1) == color) xs[p] = nx[p];
            }
            __syncthreads();
        }
    }
    for (int p = threadIdx.x; p < n; p += blockDim.x) x[p] = (T)xs[p];
}

// Coarsest level with at most MAX_DENSE cells: the level matrix is assembled in shared
// memory and solved exactly by Gauss-Jordan elimination in FP64 (no pivoting: the
// matrix is symmetric, diagonally dominant with a unit-or-larger excess). One thread
// per row.
constexpr int MAX_DENSE = 64;

template <typename T>
__global__ void k_coarse_dense(Lvl L, T* __restrict__ x, const T* __restrict__ b,
                               const T* __restrict__ K) {
    __shared__ double A[MAX_DENSE][MAX_DENSE + 1];
    const int n = (int)L.ncell;
    const int r = threadIdx.x;
    if (r < n) {
        for (int c = 0; c <= n; ++c) A[r][c] = 0.0;
        int i, j, k;
        decode(L, r, i, j, k);
        const int c3[3] = {i, j, k};
        const double kc = (double)K[r];
        double diag = 1.0;
        int stride = 1;
        for (int d = 0; d < L.ndim; ++d) {
            const int nd = L.n[d];
            const double wd = L.w[d];
            for (int side = 0; side < 2; ++side) {
                int q = -1;
                const int kind = side ? L.bchi[d] : L.bclo[d];
                if (side == 0) {
                    if (c3[d] > 0) q = r - stride;
                    else if (kind == FLD_BC_PERIODIC) q = r + (nd - 1) * stride;
                } else {
                    if (c3[d] < nd - 1) q = r + stride;
                    else if (kind == FLD_BC_PERIODIC) q = r - (nd - 1) * stride;
                }
                if (q >= 0) {
                    const double w = fmean(kc, (double)K[q], L.fm) * wd;
                    diag += w;
                    A[r][q] -= w;
                } else if (kind == FLD_BC_DIRICHLET) {
                    diag += 2.0 * kc * wd;
                }
            }
            stride *= nd;
        }
        A[r][r] += diag;
        A[r][n] = (double)b[r];
    }
    for (int p = 0; p < n; ++p) {
        __syncthreads();
        double f = 0.0;
        if (r < n && r != p) f = A[r][p] / A[p][p];
        __syncthreads();
        if (r < n && r != p)
            for (int c = p; c <= n; ++c) A[r][c] = fma(-f, A[p][c], A[r][c]);
    }
    __syncthreads();
    if (r < n) x[r] = (T)(A[r][n] / A[r][r]);
}

template <typename T>
void launch_coarse_solve(const Lvl& L, T* x, const T* b, const T* K, int sweeps, cudaStream_t s) {
    if (L.ncell <= MAX_DENSE)
        k_coarse_dense<T><<<1, MAX_DENSE, 0, s>>>(L, x, b, K);
    else
        k_coarse_solve<T><<<1, 256, 0, s>>>(L, x, b, K, sweeps);
}

// ----------------------------------------------------------------- FP64 residual + norms
// FP64 residual with the fewest FP64 operations per cell (FP64 issues at 1/58 of the
// FP32 rate here): per face one sum of coefficients, one difference and one FMA,
//   r = b - x - sum_d (w_d/2) sum_faces (K_p + K_q)(x_p - x_q) - sum_Dirichlet 2 w_d K_p x_p.
__global__ void k_resid64(Lvl L, const double* __restrict__ x, const double* __restrict__ b,
                          const double* __restrict__ K, float* __restrict__ r32,
                          double* __restrict__ partials) {
    __shared__ double sh[32];
    double acc2 = 0.0;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int nrows = ny * nz;
    const int sy = nx, sz = nx * ny;
    const double hx = 0.5 * L.w[0], hy = 0.5 * L.w[1], hz = 0.5 * L.w[2];
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int j = r % ny, k = r / ny;
        const int base = r * nx;
        // neighbour row offsets (periodic wrap, or -1 for a wall)
        int oym = -1, oyp = -1, ozm = -1, ozp = -1;
        if (L.ndim >= 2) {
            oym = j > 0 ? -sy : (L.bclo[1] == FLD_BC_PERIODIC ? (ny - 1) * sy : -1);
            oyp = j < ny - 1 ? sy : (L.bchi[1] == FLD_BC_PERIODIC ? -(ny - 1) * sy : -1);
        }
        if (L.ndim >= 3) {
            ozm = k > 0 ? -sz : (L.bclo[2] == FLD_BC_PERIODIC ? (nz - 1) * sz : -1);
            ozp = k < nz - 1 ? sz : (L.bchi[2] == FLD_BC_PERIODIC ? -(nz - 1) * sz : -1);
        }
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int p = (int)fld_at(base + i, L.ncell);
            const double xc = x[p], kc = K[p];
            double ax = 0.0, ay = 0.0, az = 0.0, dir = 0.0;
            // x faces
            int q = i > 0 ? p - 1 : (L.bclo[0] == FLD_BC_PERIODIC ? p + nx - 1 : -1);
            if (q >= 0) { q = (int)fld_at(q, L.ncell); ax = fma(fsum2(kc, K[q], L.fm), xc - x[q], ax); }
            else if (L.bclo[0] == FLD_BC_DIRICHLET) dir += L.w[0];
            q = i < nx - 1 ? p + 1 : (L.bchi[0] == FLD_BC_PERIODIC ? p - nx + 1 : -1);
            if (q >= 0) { q = (int)fld_at(q, L.ncell); ax = fma(fsum2(kc, K[q], L.fm), xc - x[q], ax); }
            else if (L.bchi[0] == FLD_BC_DIRICHLET) dir += L.w[0];
            if (L.ndim >= 2) {
                if (oym != -1) { const int q2 = (int)fld_at(p + oym, L.ncell); ay = fma(fsum2(kc, K[q2], L.fm), xc - x[q2], ay); }
                else if (L.bclo[1] == FLD_BC_DIRICHLET) dir += L.w[1];
                if (oyp != -1) { const int q2 = (int)fld_at(p + oyp, L.ncell); ay = fma(fsum2(kc, K[q2], L.fm), xc - x[q2], ay); }
                else if (L.bchi[1] == FLD_BC_DIRICHLET) dir += L.w[1];
            }
            if (L.ndim >= 3) {
                if (ozm != -1) { const int q2 = (int)fld_at(p + ozm, L.ncell); az = fma(fsum2(kc, K[q2], L.fm), xc - x[q2], az); }
                else if (L.bclo[2] == FLD_BC_DIRICHLET) dir += L.w[2];
                if (ozp != -1) { const int q2 = (int)fld_at(p + ozp, L.ncell); az = fma(fsum2(kc, K[q2], L.fm), xc - x[q2], az); }
                else if (L.bchi[2] == FLD_BC_DIRICHLET) dir += L.w[2];
            }
            double res = fma(-hx, ax, b[p] - xc);
            res = fma(-hy, ay, res);
            res = fma(-hz, az, res);
            if (dir != 0.0) res = fma(-2.0 * dir * kc, xc, res);
            if (r32) r32[p] = (float)res;
            acc2 = fma(res, res, acc2);
        }
    }
    acc2 = block_sum(acc2, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc2;
}

void launch_resid64(const Lvl& L, const double* x, const double* b, const double* K, float* r32,
                    double* partials, int nblocks, int block, cudaStream_t s) {
    k_resid64<<<nblocks, block, 0, s>>>(L, x, b, K, r32, partials);
}

__global__ void k_add_correction(long long n, double* __restrict__ x, const float* __restrict__ e) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        x[p] += (double)e[p];
}

void launch_add_correction(long long n, double* x, const float* e, cudaStream_t s) {
    k_add_correction<<<grid_for(n, 256), 256, 0, s>>>(n, x, e);
}

__global__ void k_sumsq(long long n, const double* __restrict__ v, double* __restrict__ partials) {
    __shared__ double sh[32];
    double a = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        a = fma(v[p], v[p], a);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
}

void launch_sumsq(long long n, const double* v, double* partials, int nblocks, cudaStream_t s) {
    k_sumsq<<<nblocks, 256, 0, s>>>(n, v, partials);
}

__global__ void k_finish_sum(const double* __restrict__ partials, int nparts, double* out) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) a += partials[q];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) *out = a;
}

void launch_finish_sum(const double* partials, int nparts, double* out, cudaStream_t s) {
    k_finish_sum<<<1, 1024, 0, s>>>(partials, nparts, out);
}

// partial sums of the energy density per cell, c_v rho T + E (E alone when rho is null)
__global__ void k_energy_sum(long long n, const double* __restrict__ rho,
                             const double* __restrict__ T, const double* __restrict__ E,
                             double cv, double* __restrict__ partials) {
    __shared__ double sh[32];
    double a = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        a += E[p];
        if (rho) a = fma(cv * rho[p], T[p], a);
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
}

void launch_energy_sum(long long n, const double* rho, const double* T, const double* E, double cv,
                       double* partials, int nblocks, cudaStream_t s) {
    k_energy_sum<<<nblocks, 256, 0, s>>>(n, rho, T, E, cv, partials);
}

// explicit instantiations
#define FLD_INST(T)                                                                              \
    template void launch_restrict_K<T>(const Lvl&, const Lvl&, double, const T*, T*, cudaStream_t); \
    template void launch_smooth<T>(const Lvl&, int, const T*, T*, const T*, const T*, int,         \
                                   cudaStream_t);                                                \
    template void launch_resid_restrict<T>(const Lvl&, const Lvl&, const T*, const T*, const T*,  \
                                           T*, int, bool, cudaStream_t);                         \
    template void launch_prolong<T>(const Lvl&, const Lvl&, T*, const T*, int, cudaStream_t);     \
    template void launch_coarse_solve<T>(const Lvl&, T*, const T*, const T*, int, cudaStream_t); \
    template bool rb_half_supported<T>(const Lvl&);                                              \
    template void launch_rb_half<T>(const Lvl&, int, T*, const T*, const T*, cudaStream_t);
FLD_INST(double)
FLD_INST(float)

}  // namespace fld
