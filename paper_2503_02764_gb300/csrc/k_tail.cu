// The coarse end of a V-cycle in ONE single-block launch, its levels held in shared memory.
// From the first level with at most TAIL_MAX_CELLS cells down to the coarsest, every step
// of the V-cycle (the pre- and post-smoothing sweeps, residual restriction, zeroing of the
// coarse iterate, the exact coarsest solve, prolongation) runs as block-stride loops over
// shared memory separated by block barriers. Those levels are small (8^3 and below, the
// measured best start), so the steps cost microseconds of one SM, where separate launches
// would each cost their launch and tail latency (about two dozen launches per V-cycle).
//
// The arithmetic is that of the per-level kernels: red-black sweeps as two out-of-place
// colour phases (the half-sweep update; on even periodic extents identical to the
// in-place form), the average of the children's residuals b - A x, cell-centred
// trilinear prolongation with mirrored walls, and Gauss-Jordan elimination in FP64 on
// the coarsest level (at most TAIL_MAX_DENSE cells).
#include <atomic>
#include <mutex>

#include "fld_device.cuh"

namespace fld {

namespace {

constexpr int TAIL_THREADS = 1024;

template <typename T, int FM>
__device__ void tail_colour(const Lvl& L, int color, const T* __restrict__ xin,
                            T* __restrict__ xout, const T* __restrict__ b,
                            const T* __restrict__ K) {
    for (int p = threadIdx.x; p < (int)L.ncell; p += blockDim.x) {
        int i, j, k;
        decode(L, p, i, j, k);
        if (((i + j + k) & 1) != color) {
            xout[p] = xin[p];
            continue;
        }
        T sw, acc;
        stencil<T, FM>(L, K, xin, i, j, k, p, sw, acc);
        xout[p] = div_fast<T>(b[p] + acc, T(1) + sw);
    }
}

template <typename T, int FM>
__device__ void tail_smooth(const Lvl& L, int n, T* x, T* tmp, const T* b, const T* K) {
    for (int s = 0; s < n; ++s) {
        tail_colour<T, FM>(L, 0, x, tmp, b, K);
        __syncthreads();
        tail_colour<T, FM>(L, 1, tmp, x, b, K);
        __syncthreads();
    }
}

// coarse b = mean over the children of the fine residual b - A x
template <typename T, int FM>
__device__ void tail_restrict(const Lvl& F, const Lvl& C, const T* __restrict__ x,
                              const T* __restrict__ b, const T* __restrict__ K,
                              T* __restrict__ bc) {
    for (int P = threadIdx.x; P < (int)C.ncell; P += blockDim.x) {
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
                    stencil<T, FM>(F, K, x, i, j, k, p, sw, acc);
                    s += b[p] - (T(1) + sw) * x[p] + acc;
                    ++cnt;
                }
        bc[P] = s / T(cnt);
    }
}

// x_f += trilinear interpolant of the coarse correction
template <typename T>
__device__ void tail_prolong(const Lvl& F, const Lvl& C, T* __restrict__ xf,
                             const T* __restrict__ xc) {
    for (int p = threadIdx.x; p < (int)F.ncell; p += blockDim.x) {
        int i, j, k;
        decode(F, p, i, j, k);
        const Interp ix = interp1(i, F.n[0], C.n[0], F.bclo[0], F.bchi[0], F.pk);
        const Interp iy = interp1(j, F.n[1], C.n[1], F.bclo[1], F.bchi[1], F.pk);
        const Interp iz = interp1(k, F.n[2], C.n[2], F.bclo[2], F.bchi[2], F.pk);
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                const T wzy = (T)(iz.wt[c] * iy.wt[bb]);
                if (wzy == T(0)) continue;
                const long long rowc = ((long long)iz.idx[c] * C.n[1] + iy.idx[bb]) * C.n[0];
                acc += wzy * ((T)ix.wt[0] * xc[rowc + ix.idx[0]] + (T)ix.wt[1] * xc[rowc + ix.idx[1]]);
            }
        xf[p] += acc;
    }
}

// exact solve of the coarsest level (n <= TAIL_MAX_DENSE) by Gauss-Jordan in FP64
template <typename T, int FM>
__device__ void tail_dense(const Lvl& L, T* __restrict__ x, const T* __restrict__ b,
                           const T* __restrict__ K, double (*A)[TAIL_MAX_DENSE + 1]) {
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
                    const double w = fmean(kc, (double)K[q], FM) * wd;
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
    __syncthreads();
}

// All tail levels live in shared memory for the whole launch: the first level's x and b
// and every level's K are read once, the first level's x written back once; every phase
// in between touches shared memory only.
// FM: the levels' face mean (0 arithmetic, 1 harmonic), fixed per instantiation
template <typename T, int FM>
__global__ void __launch_bounds__(TAIL_THREADS) k_vcycle_tail(TailLevels<T> t) {
    __shared__ double A[TAIL_MAX_DENSE][TAIL_MAX_DENSE + 1];
    extern __shared__ __align__(16) unsigned char tail_smem[];
    T* xs[TAIL_MAX_LEVELS];
    T* bs[TAIL_MAX_LEVELS];
    T* Ks[TAIL_MAX_LEVELS];
    T* ts[TAIL_MAX_LEVELS];
    {
        T* p = reinterpret_cast<T*>(tail_smem);
        for (int q = 0; q < t.n; ++q) {
            const int n = (int)t.L[q].ncell;
            xs[q] = p; bs[q] = p + n; Ks[q] = p + 2 * n; ts[q] = p + 3 * n;
            p += 4 * n;
        }
    }
    for (int q = 0; q < t.n; ++q)
        for (int p = threadIdx.x; p < (int)t.L[q].ncell; p += blockDim.x) {
            Ks[q][p] = t.K[q][p];
            if (q == 0) {
                xs[0][p] = t.x[0][p];
                bs[0][p] = t.b[0][p];
            }
        }
    __syncthreads();
    const int last = t.n - 1;
    // down: pre-smooth, restrict the residual, clear the coarse iterate
    for (int l = 0; l < last; ++l) {
        tail_smooth<T, FM>(t.L[l], t.nu1, xs[l], ts[l], bs[l], Ks[l]);
        tail_restrict<T, FM>(t.L[l], t.L[l + 1], xs[l], bs[l], Ks[l], bs[l + 1]);
        for (int p = threadIdx.x; p < (int)t.L[l + 1].ncell; p += blockDim.x) xs[l + 1][p] = T(0);
        __syncthreads();
    }
    tail_dense<T, FM>(t.L[last], xs[last], bs[last], Ks[last], A);
    // up: prolong the correction, post-smooth
    for (int l = last - 1; l >= 0; --l) {
        tail_prolong<T>(t.L[l], t.L[l + 1], xs[l], xs[l + 1]);
        __syncthreads();
        tail_smooth<T, FM>(t.L[l], t.nu2, xs[l], ts[l], bs[l], Ks[l]);
    }
    for (int p = threadIdx.x; p < (int)t.L[0].ncell; p += blockDim.x) t.x[0][p] = xs[0][p];
}

}  // namespace

template <typename T>
size_t tail_smem_bytes(const Lvl* lv, int n) {
    size_t c = 0;
    for (int q = 0; q < n; ++q) c += (size_t)lv[q].ncell;
    return 4 * sizeof(T) * c;
}

template <typename T>
void launch_vcycle_tail(const TailLevels<T>& t, cudaStream_t s) {
    const size_t sm = tail_smem_bytes<T>(t.L, t.n);
    if (t.L[0].fm)
        k_vcycle_tail<T, 1><<<1, TAIL_THREADS, sm, s>>>(t);
    else
        k_vcycle_tail<T, 0><<<1, TAIL_THREADS, sm, s>>>(t);
}

// Opt the tail kernels into TAIL_SMEM_MAX bytes of dynamic shared memory, once per device
// (the attribute is a per-device setting), with that device current and outside any stream
// capture (called when a handle is created).
void prepare_vcycle_tail() {
    constexpr int MAXDEV = 64;
    static std::atomic<bool> done[MAXDEV];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev].load()) return;
    cudaFuncSetAttribute(k_vcycle_tail<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)TAIL_SMEM_MAX);
    cudaFuncSetAttribute(k_vcycle_tail<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)TAIL_SMEM_MAX);
    cudaFuncSetAttribute(k_vcycle_tail<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)TAIL_SMEM_MAX);
    cudaFuncSetAttribute(k_vcycle_tail<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)TAIL_SMEM_MAX);
    done[dev].store(true);
}

template size_t tail_smem_bytes<float>(const Lvl*, int);
template size_t tail_smem_bytes<double>(const Lvl*, int);

template void launch_vcycle_tail<float>(const TailLevels<float>&, cudaStream_t);
template void launch_vcycle_tail<double>(const TailLevels<double>&, cudaStream_t);

}  // namespace fld
