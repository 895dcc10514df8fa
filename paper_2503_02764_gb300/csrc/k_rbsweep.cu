// One full red-black Gauss-Seidel sweep of a 3D FP32 level (red cells, then black cells)
// in a single pass over memory, out of place: xout = sweep(xin).
//
// Each block owns a tile of ZM_TX x TY cells of the x-y plane and marches along z over a
// chunk of planes [z0, z1). Thread (tp, ty) owns the cell pair (tx0 + 2 tp, +1) of row
// ty0 + ty: one red and one black cell, so both colour phases keep every lane busy, and a
// warp is one tile row (64 cells, 256 contiguous bytes).
//
// Shared memory holds a ring of ZM_R planes of x, K and b, each with a 2-row halo in y
// and a 4-column (one 16-byte chunk) halo in x, filled by cp.async ZM_D planes ahead of
// use. Step m evaluates the red cells of plane m in place in the shared copy, on the tile
// and on its 1-cell ring (the ring values are recomputed rather than exchanged between
// blocks), then the black cells of plane m-1, which need shared data only, and stores
// plane m-1 of xout. Per sweep each cell's x, K and b are read once from global memory
// and xout written once: 16 B per cell, against ~29 B for two in-place half sweeps,
// whose red and black cells share every sector.
//
// The updates are those of the half-sweep kernels: red cells take (b + acc)/(1 + sw) of
// the input iterate, black cells that of the red-updated one, with the same face weights
// (K_p + K_q) w_d / 2 summed in the same order. Boundary faces are encoded in the halo
// instead of branches: x and b are 0 outside the domain, and K of the ghost next to a wall
// is -K of the wall cell (Neumann: the face weight vanishes) or 3 K (Dirichlet: the face
// weight becomes the half-cell 2 K w_d of the operator; the wall value itself lives in b).
// Periodic axes wrap. Same-colour cells must never meet across a periodic wrap, so odd
// periodic extents are left to the other smoothers, as for the in-place half sweeps.
#include <algorithm>
#include <mutex>

#include "fld_internal.cuh"

namespace fld {

namespace {

constexpr int ZM_TXP = 32;                 // cell pairs per tile row (one warp)
constexpr int ZM_TX = 2 * ZM_TXP;          // tile width in cells
constexpr int ZM_XL = 4;                   // halo columns on each side: one 16-byte chunk
constexpr int ZM_XW = ZM_TX + 2 * ZM_XL;   // shared row length
constexpr int ZM_CPR = ZM_XW / 4;          // 16-byte chunks per shared row
constexpr int ZM_D = 2;                    // planes in flight ahead of use
constexpr int ZM_R = ZM_D + 4;             // ring depth: planes m-2 .. m+1+D

template <int TY>
struct ZmShape {
    static constexpr int NROW = TY + 4;
    static constexpr int PL = ZM_XW * NROW;     // floats per plane and field
    static constexpr int NCH = NROW * ZM_CPR;   // 16-byte chunks per plane and field
    static constexpr int NT = ZM_TXP * TY;      // threads per block
    static constexpr size_t SMEM = sizeof(float) * 3 * ZM_R * PL;
    static_assert(NCH <= NT, "one copy chunk per thread");
};

// Where coordinate g of an axis of extent n lands: the cell index (periodic axes wrap),
// -1 for the ghost next to the low wall, -2 for the ghost next to the high wall, -3
// farther out (only ever a neighbour of ghosts, which are never updated).
__device__ __forceinline__ int zm_axis(int g, int n, bool per) {
    if (g >= 0 && g < n) return g;
    if (per) {
        g %= n;
        return g < 0 ? g + n : g;
    }
    if (g == -1) return -1;
    if (g == n) return -2;
    return -3;
}

// K factor of the ghost cell next to a wall of this kind.
__device__ __forceinline__ float zm_ghost_factor(int bc) {
    return bc == FLD_BC_DIRICHLET ? 3.0f : -1.0f;
}

__device__ __forceinline__ void zm_cp16(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void zm_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void zm_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// (b + acc)/(1 + sw) of the cell at shared offset c; S0/K0 hold its plane, Sm/Km the one
// below, Sp/Kp the one above; h* = w_d / 2.
__device__ __forceinline__ float zm_relax(const float* S0, const float* K0, const float* Sm,
                                          const float* Km, const float* Sp, const float* Kp,
                                          int c, float bv, float hx, float hy, float hz) {
    const float kc = K0[c];
    float f = (kc + K0[c - 1]) * hx;
    float sw = f;
    float acc = f * S0[c - 1];
    f = (kc + K0[c + 1]) * hx;
    sw += f;
    acc = fmaf(f, S0[c + 1], acc);
    f = (kc + K0[c - ZM_XW]) * hy;
    sw += f;
    acc = fmaf(f, S0[c - ZM_XW], acc);
    f = (kc + K0[c + ZM_XW]) * hy;
    sw += f;
    acc = fmaf(f, S0[c + ZM_XW], acc);
    f = (kc + Km[c]) * hz;
    sw += f;
    acc = fmaf(f, Sm[c], acc);
    f = (kc + Kp[c]) * hz;
    sw += f;
    acc = fmaf(f, Sp[c], acc);
    return __fdividef(bv + acc, 1.0f + sw);
}

}  // namespace

template <int TY, int MINB>
__global__ void __launch_bounds__(ZM_TXP * TY, MINB)
k_rb_zmarch(Lvl L, const float* __restrict__ xin, float* __restrict__ xout,
            const float* __restrict__ b, const float* __restrict__ K, int cz) {
    using SH = ZmShape<TY>;
    constexpr int PL = SH::PL;
    extern __shared__ __align__(16) float zsm[];

    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int tilesx = (nx + ZM_TX - 1) / ZM_TX, tilesy = (ny + TY - 1) / TY;
    int bid = blockIdx.x;
    const int tx0 = (bid % tilesx) * ZM_TX;
    bid /= tilesx;
    const int ty0 = (bid % tilesy) * TY;
    bid /= tilesy;
    const int z0 = bid * cz, z1 = min(z0 + cz, nz);
    const bool xper = L.bclo[0] == FLD_BC_PERIODIC;
    const bool yper = L.bclo[1] == FLD_BC_PERIODIC;
    const bool zper = L.bclo[2] == FLD_BC_PERIODIC;
    const float hx = 0.5f * L.wf[0], hy = 0.5f * L.wf[1], hz = 0.5f * L.wf[2];
    const long long plane = (long long)nx * ny;
    const int tid = threadIdx.x;

    // ---- this thread's 16-byte copy chunk of every plane (same x-y footprint each plane)
    // mode 0: four cells, copied; 1: x-ghost chunk left of x = 0 (its element 3 is the
    // ghost); 2: x-ghost chunk right of x = nx - 1 (element 0); 3: y-ghost row (all four);
    // 4: nothing but zeros; 5: no chunk.
    int cmode = 5, soff = 0;
    long long goff = 0;        // plane offset of the copied cells / of the mirrored cells
    float gfac = 0.0f;
    if (tid < SH::NCH) {
        const int r = tid / ZM_CPR, ch = tid - r * ZM_CPR;
        soff = r * ZM_XW + 4 * ch;
        const int gy = zm_axis(ty0 - 2 + r, ny, yper);
        const int rawx = tx0 - ZM_XL + 4 * ch;
        const int gx = zm_axis(rawx, nx, xper);
        if (gy >= 0 && gx >= 0) {
            cmode = 0;
            goff = (long long)gy * nx + gx;
        } else if (gy >= 0 && rawx == -4 && !xper) {
            cmode = 1;
            goff = (long long)gy * nx;
            gfac = zm_ghost_factor(L.bclo[0]);
        } else if (gy >= 0 && rawx == nx && !xper) {
            cmode = 2;
            goff = (long long)gy * nx + nx - 1;
            gfac = zm_ghost_factor(L.bchi[0]);
        } else if (gx >= 0 && (gy == -1 || gy == -2)) {
            cmode = 3;
            goff = (long long)(gy == -1 ? 0 : ny - 1) * nx + gx;
            gfac = zm_ghost_factor(gy == -1 ? L.bclo[1] : L.bchi[1]);
        } else {
            cmode = 4;
        }
    }

    auto slot = [](int m) { return (m + ZM_R) % ZM_R; };
    auto Sp = [&](int m) { return zsm + slot(m) * 3 * PL; };

    // Copy plane m (raw z coordinate, may lie outside [0, nz)) into its ring slot.
    auto issue = [&](int m) {
        if (cmode < 5 && m <= z1 + 1) {
            float* Sd = Sp(m) + soff;
            float* Kd = Sd + PL;
            float* Bd = Kd + PL;
            const int gz = zm_axis(m, nz, zper);
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gz >= 0 && cmode == 0) {
                const long long o = gz * plane + goff;
                zm_cp16(Sd, xin + o);
                zm_cp16(Kd, K + o);
                zm_cp16(Bd, b + o);
            } else {
                // ghosts: x = b = 0 and K = factor * K of the mirrored wall cell
                float4 k4 = z4;
                if (gz >= 0 && cmode == 1) {
                    k4.w = gfac * K[gz * plane + goff];
                } else if (gz >= 0 && cmode == 2) {
                    k4.x = gfac * K[gz * plane + goff];
                } else if (gz >= 0 && cmode == 3) {
                    const float4 v = *reinterpret_cast<const float4*>(K + gz * plane + goff);
                    k4 = make_float4(gfac * v.x, gfac * v.y, gfac * v.z, gfac * v.w);
                } else if ((gz == -1 || gz == -2) && cmode == 0) {
                    const float f = zm_ghost_factor(gz == -1 ? L.bclo[2] : L.bchi[2]);
                    const long long o = (long long)(gz == -1 ? 0 : nz - 1) * plane + goff;
                    const float4 v = *reinterpret_cast<const float4*>(K + o);
                    k4 = make_float4(f * v.x, f * v.y, f * v.z, f * v.w);
                }
                *reinterpret_cast<float4*>(Sd) = z4;
                *reinterpret_cast<float4*>(Kd) = k4;
                *reinterpret_cast<float4*>(Bd) = z4;
            }
        }
        zm_commit();
    };

    // ---- the interior pair of this thread
    const int tp = tid & (ZM_TXP - 1), ty = tid / ZM_TXP;
    const int gx = tx0 + 2 * tp, gy = ty0 + ty;
    const bool active = gx < nx && gy < ny;
    const int c0 = (ty + 2) * ZM_XW + ZM_XL + 2 * tp;

    // ---- the ring cell pair of this thread: cells at distance 1 outside the active
    // rectangle [0, ax) x [0, ay) of the tile whose red value a black interior cell reads.
    // Row pairs (lx = 2k - 1, 2k) on ly = -1 and ly = ay; column pairs (ly = 2k, 2k + 1)
    // on lx = -1 and lx = ax. Exactly one cell of a pair is red on any plane.
    const int ax = min(ZM_TX, nx - tx0), ay = min(TY, ny - ty0);
    const int nrow = (ax + 2) / 2, ncol = (ay + 1) / 2;
    int rc0 = -1, rc1 = -1;    // shared offsets of the two candidates (-1: not a cell)
    int rpar = 0;              // parity of gx + gy of candidate 0
    {
        int lx0 = 0, ly0 = 0, dx = 0, dy = 0;
        bool has = true, colseg = false;
        if (tid < nrow) {
            lx0 = 2 * tid - 1; ly0 = -1; dx = 1;
        } else if (tid < 2 * nrow) {
            lx0 = 2 * (tid - nrow) - 1; ly0 = ay; dx = 1;
        } else if (tid < 2 * nrow + ncol) {
            lx0 = -1; ly0 = 2 * (tid - 2 * nrow); dy = 1; colseg = true;
        } else if (tid < 2 * nrow + 2 * ncol) {
            lx0 = ax; ly0 = 2 * (tid - 2 * nrow - ncol); dy = 1; colseg = true;
        } else {
            has = false;
        }
        if (has) {
            rpar = (tx0 + lx0 + ty0 + ly0) & 1;
            for (int q = 0; q < 2; ++q) {
                const int lx = lx0 + q * dx, ly = ly0 + q * dy;
                const bool cell = zm_axis(tx0 + lx, nx, xper) >= 0 &&
                                  zm_axis(ty0 + ly, ny, yper) >= 0;
                const int off = (cell && !(colseg && ly >= ay)) ? (ly + 2) * ZM_XW + ZM_XL + lx : -1;
                if (q == 0) rc0 = off; else rc1 = off;
            }
        }
    }

    // red cells of plane m (global index gz) on the tile and its ring, in shared memory
    auto red = [&](int m, int gz) {
        float* S0 = Sp(m);
        const float* K0 = S0 + PL;
        const float* B0 = K0 + PL;
        const float* Sm = Sp(m - 1);
        const float* Km = Sm + PL;
        const float* Sq = Sp(m + 1);
        const float* Kq = Sq + PL;
        if (active) {
            const int c = c0 + ((gy + gz) & 1);
            S0[c] = zm_relax(S0, K0, Sm, Km, Sq, Kq, c, B0[c], hx, hy, hz);
        }
        const int q = (rpar + gz) & 1;      // candidate 0 red when gx + gy + gz is even
        const int c = q ? rc1 : rc0;
        if (c >= 0) S0[c] = zm_relax(S0, K0, Sm, Km, Sq, Kq, c, B0[c], hx, hy, hz);
    };

    // black cells of plane m (global index gz): relax from the red-updated values and
    // store the cell pair of xout
    auto black = [&](int m, int gz) {
        if (!active) return;
        const float* S0 = Sp(m);
        const float* K0 = S0 + PL;
        const float* B0 = K0 + PL;
        const float* Sm = Sp(m - 1);
        const float* Km = Sm + PL;
        const float* Sq = Sp(m + 1);
        const float* Kq = Sq + PL;
        const int qb = (gy + gz + 1) & 1;   // which cell of the pair is black
        const float v = zm_relax(S0, K0, Sm, Km, Sq, Kq, c0 + qb, B0[c0 + qb], hx, hy, hz);
        const float2 out = qb ? make_float2(S0[c0], v) : make_float2(v, S0[c0 + 1]);
        *reinterpret_cast<float2*>(xout + gz * plane + (long long)gy * nx + gx) = out;
    };

    // ---- the march. Step m: planes <= m + 1 have landed; red(m), then black(m - 1).
    // The copy of plane m + 1 + D goes into the slot of plane m - 3, last read by
    // black(m - 2) in the previous step.
    for (int m = z0 - 2; m <= z0 - 1 + ZM_D; ++m) issue(m);
    for (int m = z0 - 1; m <= z1; ++m) {
        zm_wait<ZM_D - 1>();
        __syncthreads();
        issue(m + 1 + ZM_D);
        const int gz = zm_axis(m, nz, zper);
        if (gz >= 0) red(m, gz);
        __syncthreads();
        if (m - 1 >= z0) black(m - 1, m - 1);
    }
    zm_wait<0>();
}

namespace {

constexpr int ZM_TY = 16, ZM_MINB = 2;

int g_zm_slots = 0;   // resident blocks of the sweep kernel on the whole GPU

// z-chunk length: enough blocks for one full wave on every SM (the tiles times the
// chunks), chunks of at least 8 planes so the 2-plane overlap stays small.
int zm_chunk(const Lvl& L) {
    const int tiles = ((L.n[0] + ZM_TX - 1) / ZM_TX) * ((L.n[1] + ZM_TY - 1) / ZM_TY);
    const int nch = std::max(1, std::max(g_zm_slots, 1) / std::max(1, tiles));
    const int cz = (L.n[2] + nch - 1) / nch;
    return std::min(L.n[2], std::max(8, cz));
}

}  // namespace

// FP32 3D levels whose x extent is a whole number of 16-byte chunks and whose periodic
// extents are even; everything else (and FP64) uses the half-sweep smoothers.
template <typename T>
bool rb_sweep_supported(const Lvl& L) {
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
        if (L.ndim != 3 || L.n[0] % 4 != 0 || L.n[0] < 16) return false;
        for (int d = 0; d < 3; ++d)
            if (L.bclo[d] == FLD_BC_PERIODIC && (L.n[d] & 1)) return false;
        return true;
    }
}

template <typename T>
void launch_rb_sweep(const Lvl& L, const T* xin, T* xout, const T* b, const T* K,
                     cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        constexpr size_t sm = ZmShape<ZM_TY>::SMEM;
        const int cz = zm_chunk(L);
        const int tiles = ((L.n[0] + ZM_TX - 1) / ZM_TX) * ((L.n[1] + ZM_TY - 1) / ZM_TY);
        const int nch = (L.n[2] + cz - 1) / cz;
        k_rb_zmarch<ZM_TY, ZM_MINB><<<tiles * nch, ZM_TXP * ZM_TY, sm, s>>>(L, xin, xout, b, K,
                                                                             cz);
    }
}

// Opt the kernel into its shared-memory size and count its resident blocks: once per
// process, outside any stream capture (called when a handle is created).
void prepare_rb_sweep() {
    static std::once_flag once;
    std::call_once(once, [] {
        constexpr size_t sm = ZmShape<ZM_TY>::SMEM;
        cudaFuncSetAttribute(k_rb_zmarch<ZM_TY, ZM_MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int dev = 0, nsm = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rb_zmarch<ZM_TY, ZM_MINB>,
                                                      ZM_TXP * ZM_TY, sm);
        g_zm_slots = std::max(1, nsm) * std::max(1, occ);
    });
}

template bool rb_sweep_supported<float>(const Lvl&);
template bool rb_sweep_supported<double>(const Lvl&);
template void launch_rb_sweep<float>(const Lvl&, const float*, float*, const float*, const float*,
                                     cudaStream_t);
template void launch_rb_sweep<double>(const Lvl&, const double*, double*, const double*,
                                      const double*, cudaStream_t);

}  // namespace fld
