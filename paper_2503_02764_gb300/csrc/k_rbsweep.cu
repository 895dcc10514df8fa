// One full red-black Gauss-Seidel sweep (red half, then black half) in a single pass
// over memory, for 2D and 3D levels.
//
// Each block owns a TX x TY column of the x-y plane and marches along z over a chunk
// of planes. Shared memory holds rings of planes: the input iterate x and the operator
// coefficient K with a 2-cell halo, the right-hand side b and the red-updated iterate R
// with a 1-cell halo. For plane m the red half-sweep is evaluated on the tile plus its
// 1-cell ring (recomputing the neighbours' red values instead of exchanging them), so
// the black half-sweep of plane m-1 only needs shared memory. Per sweep each cell is
// read once (x, b, K) and written once (x_out) from/to global memory: 16 B in FP32,
// 32 B in FP64.
//
// Semantics (identical to two out-of-place half sweeps): red cells take
// (b + acc)/(1 + sw) of the input iterate; black cells take it of the red-updated one.
// Same-colour neighbours across an odd periodic extent therefore couple through their
// input values, independently of the tiling.
#include <algorithm>

#include "fld_internal.cuh"

namespace fld {

namespace {

// Global index of a (possibly out-of-range) tile coordinate: periodic axes wrap (any
// overhang: a tile may be wider than the level), other axes give -1 outside.
__device__ __forceinline__ int wrap_idx(int g, int n, bool periodic) {
    if (g >= 0 && g < n) return g;
    if (!periodic) return -1;
    g %= n;
    return g < 0 ? g + n : g;
}

}  // namespace

// Asynchronous 4- or 8-byte global -> shared copy (zero-filled when !valid).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int sz = valid ? BYTES : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES),
                 "r"(sz)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Ring depths: x needs planes m-1..m+1 for red(m) plus the prefetched m+2 (4);
// K needs m-2..m+1 (black(m-1) and red(m)) plus m+2 (5); b needs m-1, m plus m+1 (3);
// the red-updated iterate needs m-2..m (3).
constexpr int NXR = 4, NKR = 5, NBR = 3, NRR = 3;

template <typename T>
__device__ __forceinline__ T fast_div(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float fast_div<float>(float a, float b) { return __fdividef(a, b); }

// Shared-memory plane layout (all four arrays): TY + 4 rows of XWP = TX + 2 XL
// elements, row r holding global y = ty0 - 2 + r and column c global x = tx0 - XL + c.
// XL >= 2 is a whole 16-byte chunk, so interior rows are copied with 16-byte
// cp.async when the row length nx is a multiple of the chunk.
template <typename T, int TX, int TY>
struct RbLayout {
    static constexpr int V = 16 / (int)sizeof(T);
    static constexpr int XL = V > 2 ? V : 2;
    static constexpr int XWP = TX + 2 * XL;
    static constexpr int NROW = TY + 4;
    static constexpr int PL = XWP * NROW;
    static constexpr int CPR = XWP / V;
};

template <typename T, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB)
k_rb_sweep(Lvl L, const T* __restrict__ xin, T* __restrict__ xout, const T* __restrict__ b,
           const T* __restrict__ K, int cz, int vec_ok) {
    using LY = RbLayout<T, TX, TY>;
    constexpr int V = LY::V, XL = LY::XL, XWP = LY::XWP, NROW = LY::NROW, PL = LY::PL;
    constexpr int CPR = LY::CPR, NT = TX * TY;
    constexpr int NXK = NROW * CPR, NB = (NROW - 2) * CPR;   // x/K chunks, b chunks
    constexpr int RWID = TX + 2, NRED = (TY + 2) * RWID;     // red region (halo 1)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Xs = reinterpret_cast<T*>(smem_raw);
    T* Ks = Xs + NXR * PL;
    T* Bs = Ks + NKR * PL;
    T* Rs = Bs + NBR * PL;

    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int tiles_x = (nx + TX - 1) / TX, tiles_y = (ny + TY - 1) / TY;
    int bid = blockIdx.x;
    const int tx0 = (bid % tiles_x) * TX;
    bid /= tiles_x;
    const int ty0 = (bid % tiles_y) * TY;
    bid /= tiles_y;
    const int z0 = bid * cz;
    const int z1 = min(z0 + cz, nz);
    const bool xper = L.bclo[0] == FLD_BC_PERIODIC;
    const bool yper = L.bclo[1] == FLD_BC_PERIODIC;
    const bool three = L.ndim == 3;
    const bool zper = three && L.bclo[2] == FLD_BC_PERIODIC;
    const T wx = wgt<T>(L, 0), wy = wgt<T>(L, 1), wz = wgt<T>(L, 2);
    const bool xd_lo = L.bclo[0] == FLD_BC_DIRICHLET, xd_hi = L.bchi[0] == FLD_BC_DIRICHLET;
    const bool yd_lo = L.bclo[1] == FLD_BC_DIRICHLET, yd_hi = L.bchi[1] == FLD_BC_DIRICHLET;
    const bool zd_lo = L.bclo[2] == FLD_BC_DIRICHLET, zd_hi = L.bchi[2] == FLD_BC_DIRICHLET;
    const int plane = nx * ny;
    const int tid = threadIdx.x;

    auto zmap = [&](int m) { return three ? wrap_idx(m, nz, zper) : (m == 0 ? 0 : -1); };
    auto ring = [](int m, int n) { return ((m % n) + n) % n; };

    // copy plane m of x and K (all rows) and plane mb of b (halo-1 rows)
    auto issue = [&](int m, int mb) {
        const int gzx = zmap(m), gzb = zmap(mb);
        T* xd = Xs + ring(m, NXR) * PL;
        T* kd = Ks + ring(m, NKR) * PL;
        T* bd = Bs + ring(mb, NBR) * PL;
        for (int c = tid; c < NXK + NB; c += NT) {
            const bool isb = c >= NXK;
            const int cc = isb ? c - NXK + CPR : c;          // b skips the first row
            const int gz = isb ? gzb : gzx;
            if (gz < 0) continue;
            const int row = cc / CPR, ch = cc - row * CPR;
            const int gy = wrap_idx(ty0 - 2 + row, ny, yper);
            const int gx0 = tx0 - XL + V * ch;
            const int so = row * XWP + V * ch;
            if (isb) {
                T* dst = bd + so;
                const T* src = b + (long long)gz * plane;
                if (gy >= 0 && vec_ok && gx0 >= 0 && gx0 + V <= nx) {
                    cp_async<16>(dst, src + gy * nx + gx0, true);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int gx = wrap_idx(gx0 + v, nx, xper);
                        const bool ok = gy >= 0 && gx >= 0;
                        cp_async<sizeof(T)>(dst + v, src + (ok ? gy * nx + gx : 0), ok);
                    }
                }
            } else {
                const long long zo = (long long)gz * plane;
                if (gy >= 0 && vec_ok && gx0 >= 0 && gx0 + V <= nx) {
                    const int go = gy * nx + gx0;
                    cp_async<16>(xd + so, xin + zo + go, true);
                    cp_async<16>(kd + so, K + zo + go, true);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int gx = wrap_idx(gx0 + v, nx, xper);
                        const bool ok = gy >= 0 && gx >= 0;
                        const long long go = zo + (ok ? gy * nx + gx : 0);
                        cp_async<sizeof(T)>(xd + so + v, xin + go, ok);
                        cp_async<sizeof(T)>(kd + so + v, K + go, ok);
                    }
                }
            }
        }
        cp_async_commit();
    };

    // (b + acc)/(1 + sw) of the cell at index c of value planes V0 (Vm, Vq below and
    // above) and coefficient planes K0 (Km, Kq), all in the common layout.
    auto relax = [&](int gx, int gy, int gz, const T* V0, const T* Vm, const T* Vq,
                     const T* K0, const T* Km, const T* Kq, int c, T bval) -> T {
        const T kc = K0[c];
        T sw = T(0), acc = T(0);
        if (gx > 0 || xper) {
            const T w = T(0.5) * (kc + K0[c - 1]) * wx;
            sw += w;
            acc += w * V0[c - 1];
        } else if (xd_lo) sw += T(2) * kc * wx;
        if (gx < nx - 1 || xper) {
            const T w = T(0.5) * (kc + K0[c + 1]) * wx;
            sw += w;
            acc += w * V0[c + 1];
        } else if (xd_hi) sw += T(2) * kc * wx;
        if (gy > 0 || yper) {
            const T w = T(0.5) * (kc + K0[c - XWP]) * wy;
            sw += w;
            acc += w * V0[c - XWP];
        } else if (yd_lo) sw += T(2) * kc * wy;
        if (gy < ny - 1 || yper) {
            const T w = T(0.5) * (kc + K0[c + XWP]) * wy;
            sw += w;
            acc += w * V0[c + XWP];
        } else if (yd_hi) sw += T(2) * kc * wy;
        if (three) {
            if (gz > 0 || zper) {
                const T w = T(0.5) * (kc + Km[c]) * wz;
                sw += w;
                acc += w * Vm[c];
            } else if (zd_lo) sw += T(2) * kc * wz;
            if (gz < nz - 1 || zper) {
                const T w = T(0.5) * (kc + Kq[c]) * wz;
                sw += w;
                acc += w * Vq[c];
            } else if (zd_hi) sw += T(2) * kc * wz;
        }
        return fast_div<T>(bval + acc, T(1) + sw);
    };

    // red half of plane m on the tile and its 1-cell ring
    auto red_plane = [&](int m) {
        const int gz = zmap(m);
        if (gz < 0) return;
        const T* X0 = Xs + ring(m, NXR) * PL;
        const T* Xm = Xs + ring(m - 1, NXR) * PL;
        const T* Xq = Xs + ring(m + 1, NXR) * PL;
        const T* K0 = Ks + ring(m, NKR) * PL;
        const T* Km = Ks + ring(m - 1, NKR) * PL;
        const T* Kq = Ks + ring(m + 1, NKR) * PL;
        const T* B0 = Bs + ring(m, NBR) * PL;
        T* R0 = Rs + ring(m, NRR) * PL;
        for (int e = tid; e < NRED; e += NT) {
            const int ry = e / RWID, rx = e - ry * RWID;
            const int gx = wrap_idx(tx0 - 1 + rx, nx, xper);
            const int gy = wrap_idx(ty0 - 1 + ry, ny, yper);
            const int c = (ry + 1) * XWP + rx - 1 + XL;
            T v = X0[c];
            if (gx >= 0 && gy >= 0 && ((gx + gy + gz) & 1) == 0)
                v = relax(gx, gy, gz, X0, Xm, Xq, K0, Km, Kq, c, B0[c]);
            R0[c] = v;
        }
    };

    // black half of plane m on the tile, written to xout
    auto black_plane = [&](int m) {
        const int gz = zmap(m);
        const T* R0 = Rs + ring(m, NRR) * PL;
        const T* Rm = Rs + ring(m - 1, NRR) * PL;
        const T* Rq = Rs + ring(m + 1, NRR) * PL;
        const T* K0 = Ks + ring(m, NKR) * PL;
        const T* Km = Ks + ring(m - 1, NKR) * PL;
        const T* Kq = Ks + ring(m + 1, NKR) * PL;
        const T* B0 = Bs + ring(m, NBR) * PL;
        const long long zb = (long long)gz * plane;
        for (int e = tid; e < TX * TY; e += NT) {
            const int ly = e / TX, lx = e - ly * TX;
            const int gx = tx0 + lx, gy = ty0 + ly;
            if (gx >= nx || gy >= ny) continue;
            const int c = (ly + 2) * XWP + lx + XL;
            T v = R0[c];
            if (((gx + gy + gz) & 1) == 1) v = relax(gx, gy, gz, R0, Rm, Rq, K0, Km, Kq, c, B0[c]);
            xout[zb + gy * nx + gx] = v;
        }
    };

    // Pipeline. Iteration m computes red(m) and black(m-1); it needs x, K at m-1..m+1
    // (and K at m-2), b at m-1 and m. The copies for the next iteration (x, K at m+2,
    // b at m+1) are issued first so they overlap this iteration's arithmetic.
    issue(z0 - 2, z0 - 1);
    issue(z0 - 1, z0 - 1);     // (b plane reissued: harmless, same slot and data)
    issue(z0, z0);
    for (int m = z0 - 1; m <= z1; ++m) {
        issue(m + 2, m + 1);
        cp_async_wait<1>();    // all but the group just issued have landed
        __syncthreads();
        red_plane(m);
        __syncthreads();
        if (m - 1 >= z0) black_plane(m - 1);
        __syncthreads();
    }
    cp_async_wait<0>();
}

template <typename T, int TX, int TY>
static size_t rb_smem() {
    return sizeof(T) * (size_t)(NXR + NKR + NBR + NRR) * RbLayout<T, TX, TY>::PL;
}

template <typename T>
bool rb_sweep_supported(const Lvl& L) {
    return L.ndim >= 2 && L.n[0] >= 8;
}

template <typename T>
void launch_rb_sweep(const Lvl& L, const T* xin, T* xout, const T* b, const T* K, cudaStream_t s) {
    constexpr int TX = 32, TY = 8, MINB = sizeof(T) == 4 ? 5 : 3;
    const int tiles = ((L.n[0] + TX - 1) / TX) * ((L.n[1] + TY - 1) / TY);
    int cz = 1;
    if (L.ndim == 3) {
        // enough z-chunks for ~3 waves of blocks, each chunk >= 8 planes
        const int want = (152 * MINB * 3 + tiles - 1) / tiles;
        cz = std::max(8, (L.n[2] + want - 1) / std::max(want, 1));
        cz = std::min(cz, L.n[2]);
    }
    const int zch = (L.n[2] + cz - 1) / cz;
    const size_t sm = rb_smem<T, TX, TY>();
    const int vec_ok = (L.n[0] % RbLayout<T, TX, TY>::V) == 0;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_rb_sweep<T, TX, TY, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
        attr_set = true;
    }
    k_rb_sweep<T, TX, TY, MINB><<<tiles * zch, TX * TY, sm, s>>>(L, xin, xout, b, K, cz, vec_ok);
}

template bool rb_sweep_supported<float>(const Lvl&);
template bool rb_sweep_supported<double>(const Lvl&);
template void launch_rb_sweep<float>(const Lvl&, const float*, float*, const float*, const float*,
                                     cudaStream_t);
template void launch_rb_sweep<double>(const Lvl&, const double*, double*, const double*,
                                      const double*, cudaStream_t);

}  // namespace fld
