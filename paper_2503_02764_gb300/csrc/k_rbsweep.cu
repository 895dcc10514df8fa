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

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
k_rb_sweep(Lvl L, const T* __restrict__ xin, T* __restrict__ xout, const T* __restrict__ b,
           const T* __restrict__ K, int cz) {
    constexpr int XW = TX + 4, XH = TY + 4, XP = XW * XH;   // halo-2 plane
    constexpr int RW = TX + 2, RH = TY + 2, RP = RW * RH;   // halo-1 plane
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Xs = reinterpret_cast<T*>(smem_raw);   // 3 planes
    T* Ks = Xs + 3 * XP;                      // 4 planes
    T* Bs = Ks + 4 * XP;                      // 2 planes (halo 1)
    T* Rs = Bs + 2 * RP;                      // 3 planes (halo 1)

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
    const T wx = (T)L.w[0], wy = (T)L.w[1], wz = (T)L.w[2];
    const long long plane = (long long)nx * ny;
    const int tid = threadIdx.x;
    constexpr int NT = TX * TY;

    auto zmap = [&](int m) { return three ? wrap_idx(m, nz, zper) : (m == 0 ? 0 : -1); };

    // load plane m (if it exists) of x and K (halo 2), and of b (halo 1)
    auto load_xk = [&](int m) {
        const int gz = zmap(m);
        if (gz < 0) return;
        T* xd = Xs + ((m + 3) % 3) * XP;
        T* kd = Ks + ((m + 4) % 4) * XP;
        const long long zb = (long long)gz * plane;
        for (int e = tid; e < XP; e += NT) {
            const int ly = e / XW, lx = e - ly * XW;
            const int gx = wrap_idx(tx0 - 2 + lx, nx, xper);
            const int gy = wrap_idx(ty0 - 2 + ly, ny, yper);
            T xv = T(0), kv = T(0);
            if (gx >= 0 && gy >= 0) {
                const long long p = zb + (long long)gy * nx + gx;
                xv = xin[p];
                kv = K[p];
            }
            xd[e] = xv;
            kd[e] = kv;
        }
    };
    auto load_b = [&](int m) {
        const int gz = zmap(m);
        if (gz < 0) return;
        T* bd = Bs + ((m + 2) % 2) * RP;
        const long long zb = (long long)gz * plane;
        for (int e = tid; e < RP; e += NT) {
            const int ly = e / RW, lx = e - ly * RW;
            const int gx = wrap_idx(tx0 - 1 + lx, nx, xper);
            const int gy = wrap_idx(ty0 - 1 + ly, ny, yper);
            bd[e] = (gx >= 0 && gy >= 0) ? b[zb + (long long)gy * nx + gx] : T(0);
        }
    };

    // Stencil of cell with global (wrapped) coordinates (gx, gy, gz) whose centre sits at
    // index c of a plane of width W in the arrays V (values) and Kp (coefficients);
    // Vm/Vp, Km/Kp2 are the planes below/above.
    auto update = [&](int gx, int gy, int gz, const T* V, const T* Vm, const T* Vp, const T* Kc_,
                      const T* Km, const T* Kq, int c, int W, T bval) -> T {
        const T kc = Kc_[c];
        T sw = T(0), acc = T(0);
        // x faces
        if (gx > 0 || xper) {
            const T w = T(0.5) * (kc + Kc_[c - 1]) * wx;
            sw += w;
            acc += w * V[c - 1];
        } else if (L.bclo[0] == FLD_BC_DIRICHLET) sw += T(2) * kc * wx;
        if (gx < nx - 1 || xper) {
            const T w = T(0.5) * (kc + Kc_[c + 1]) * wx;
            sw += w;
            acc += w * V[c + 1];
        } else if (L.bchi[0] == FLD_BC_DIRICHLET) sw += T(2) * kc * wx;
        // y faces
        if (gy > 0 || yper) {
            const T w = T(0.5) * (kc + Kc_[c - W]) * wy;
            sw += w;
            acc += w * V[c - W];
        } else if (L.bclo[1] == FLD_BC_DIRICHLET) sw += T(2) * kc * wy;
        if (gy < ny - 1 || yper) {
            const T w = T(0.5) * (kc + Kc_[c + W]) * wy;
            sw += w;
            acc += w * V[c + W];
        } else if (L.bchi[1] == FLD_BC_DIRICHLET) sw += T(2) * kc * wy;
        // z faces
        if (three) {
            if (gz > 0 || zper) {
                const T w = T(0.5) * (kc + Km[c]) * wz;
                sw += w;
                acc += w * Vm[c];
            } else if (L.bclo[2] == FLD_BC_DIRICHLET) sw += T(2) * kc * wz;
            if (gz < nz - 1 || zper) {
                const T w = T(0.5) * (kc + Kq[c]) * wz;
                sw += w;
                acc += w * Vp[c];
            } else if (L.bchi[2] == FLD_BC_DIRICHLET) sw += T(2) * kc * wz;
        }
        return (bval + acc) / (T(1) + sw);
    };

    // red-updated values of plane m on the tile and its 1-cell ring
    auto red_plane = [&](int m) {
        const int gz = zmap(m);
        if (gz < 0) return;
        const T* X0 = Xs + ((m + 3) % 3) * XP;
        const T* Xm = Xs + ((m + 2) % 3) * XP;
        const T* Xq = Xs + ((m + 1) % 3) * XP;
        const T* K0 = Ks + ((m + 4) % 4) * XP;
        const T* Km = Ks + ((m + 3) % 4) * XP;
        const T* Kq = Ks + ((m + 5) % 4) * XP;
        const T* B0 = Bs + ((m + 2) % 2) * RP;
        T* R0 = Rs + ((m + 3) % 3) * RP;
        for (int e = tid; e < RP; e += NT) {
            const int ry = e / RW, rx = e - ry * RW;
            const int gx = wrap_idx(tx0 - 1 + rx, nx, xper);
            const int gy = wrap_idx(ty0 - 1 + ry, ny, yper);
            const int c = (ry + 1) * XW + rx + 1;
            T v = X0[c];
            if (gx >= 0 && gy >= 0 && ((gx + gy + gz) & 1) == 0)
                v = update(gx, gy, gz, X0, Xm, Xq, K0, Km, Kq, c, XW, B0[e]);
            R0[e] = v;
        }
    };

    // black half-sweep of plane m on the tile, written to xout
    auto black_plane = [&](int m) {
        const int gz = zmap(m);
        const T* R0 = Rs + ((m + 3) % 3) * RP;
        const T* Rm = Rs + ((m + 2) % 3) * RP;
        const T* Rq = Rs + ((m + 1) % 3) * RP;
        const T* K0 = Ks + ((m + 4) % 4) * XP;
        const T* Km = Ks + ((m + 3) % 4) * XP;
        const T* Kq = Ks + ((m + 5) % 4) * XP;
        const T* B0 = Bs + ((m + 2) % 2) * RP;
        const long long zb = (long long)gz * plane;
        for (int e = tid; e < TX * TY; e += NT) {
            const int ly = e / TX, lx = e - ly * TX;
            const int gx = tx0 + lx, gy = ty0 + ly;
            if (gx >= nx || gy >= ny) continue;
            const int cr = (ly + 1) * RW + lx + 1;      // index in the halo-1 planes
            const int ck = (ly + 2) * XW + lx + 2;      // index in the halo-2 planes
            T v = R0[cr];
            if (((gx + gy + gz) & 1) == 1) {
                // neighbours from the red-updated planes, coefficients from K: the two
                // plane layouts differ, so pass K re-based to the R layout
                const T kc = K0[ck];
                T sw = T(0), acc = T(0);
                if (gx > 0 || xper) {
                    const T w = T(0.5) * (kc + K0[ck - 1]) * wx;
                    sw += w;
                    acc += w * R0[cr - 1];
                } else if (L.bclo[0] == FLD_BC_DIRICHLET) sw += T(2) * kc * wx;
                if (gx < nx - 1 || xper) {
                    const T w = T(0.5) * (kc + K0[ck + 1]) * wx;
                    sw += w;
                    acc += w * R0[cr + 1];
                } else if (L.bchi[0] == FLD_BC_DIRICHLET) sw += T(2) * kc * wx;
                if (gy > 0 || yper) {
                    const T w = T(0.5) * (kc + K0[ck - XW]) * wy;
                    sw += w;
                    acc += w * R0[cr - RW];
                } else if (L.bclo[1] == FLD_BC_DIRICHLET) sw += T(2) * kc * wy;
                if (gy < ny - 1 || yper) {
                    const T w = T(0.5) * (kc + K0[ck + XW]) * wy;
                    sw += w;
                    acc += w * R0[cr + RW];
                } else if (L.bchi[1] == FLD_BC_DIRICHLET) sw += T(2) * kc * wy;
                if (three) {
                    if (gz > 0 || zper) {
                        const T w = T(0.5) * (kc + Km[ck]) * wz;
                        sw += w;
                        acc += w * Rm[cr];
                    } else if (L.bclo[2] == FLD_BC_DIRICHLET) sw += T(2) * kc * wz;
                    if (gz < nz - 1 || zper) {
                        const T w = T(0.5) * (kc + Kq[ck]) * wz;
                        sw += w;
                        acc += w * Rq[cr];
                    } else if (L.bchi[2] == FLD_BC_DIRICHLET) sw += T(2) * kc * wz;
                }
                v = (B0[cr] + acc) / (T(1) + sw);
            }
            xout[zb + (long long)gy * nx + gx] = v;
        }
    };

    // pipeline: red plane m needs x, K at m-1..m+1 and b at m; black plane m-1 needs
    // red planes m-2..m, K at m-2..m and b at m-1
    load_xk(z0 - 2);
    load_xk(z0 - 1);
    for (int m = z0 - 1; m <= z1; ++m) {
        load_xk(m + 1);
        load_b(m);
        __syncthreads();
        red_plane(m);
        __syncthreads();
        if (m - 1 >= z0) black_plane(m - 1);
        __syncthreads();
    }
}

template <typename T>
static size_t rb_smem(int tx, int ty) {
    return sizeof(T) * (size_t)(7 * (tx + 4) * (ty + 4) + 5 * (tx + 2) * (ty + 2));
}

template <typename T>
bool rb_sweep_supported(const Lvl& L) {
    return L.ndim >= 2 && L.n[0] >= 8;
}

template <typename T>
void launch_rb_sweep(const Lvl& L, const T* xin, T* xout, const T* b, const T* K, cudaStream_t s) {
    constexpr int TX = 64, TY = 8;
    const int tiles = ((L.n[0] + TX - 1) / TX) * ((L.n[1] + TY - 1) / TY);
    const int cz = (L.ndim == 3) ? std::max(8, std::min(L.n[2], 32)) : 1;
    const int zch = (L.n[2] + cz - 1) / cz;
    const size_t sm = rb_smem<T>(TX, TY);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_rb_sweep<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
        attr_set = true;
    }
    k_rb_sweep<T, TX, TY><<<tiles * zch, TX * TY, sm, s>>>(L, xin, xout, b, K, cz);
}

template bool rb_sweep_supported<float>(const Lvl&);
template bool rb_sweep_supported<double>(const Lvl&);
template void launch_rb_sweep<float>(const Lvl&, const float*, float*, const float*, const float*,
                                     cudaStream_t);
template void launch_rb_sweep<double>(const Lvl&, const double*, double*, const double*,
                                      const double*, cudaStream_t);

}  // namespace fld
