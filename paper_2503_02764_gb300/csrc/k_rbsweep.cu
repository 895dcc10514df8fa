// One full red-black Gauss-Seidel sweep of a 3D FP32 level (red cells, then black cells)
// in a single pass over memory, out of place: xout = sweep(xin).
//
// Each block owns a tile of TX x TY cells of the x-y plane and marches along z over a
// chunk of planes [z0, z1). Lane l of warp w owns the two cells (x, y0) and (x, y0 + 1)
// of one column pair, x = tx0 + 32 (w % WX) + l, y0 = ty0 + 2 (w / WX): one red and one
// black cell, so both colour phases keep every lane busy. Within a warp the red cells
// alternate between the two rows; with a shared row pitch of 8 (mod 32) words those 32
// scalar accesses fall in 32 distinct banks, as do those of every neighbour.
//
// Shared memory holds a ring of ZM_R planes of x, K and b, each with a 2-row halo in y
// and a 4-column (one 16-byte chunk) halo in x, filled by cp.async ZM_D planes ahead of
// use. Step k evaluates the red cells of plane k in place in the shared copy, on the tile
// and on its 1-cell ring (the ring values are recomputed rather than exchanged between
// blocks), and the black cells of plane k-2, which need the red values of planes k-3 ..
// k-1 only, so the two share one barrier per step; it stores plane k-2 of xout. Per sweep
// each cell's x, K and b are read once from global memory and xout written once: 16 B
// per cell, against ~29 B for two in-place half sweeps, whose red and black cells share
// every sector.
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
#include <atomic>
#include <mutex>

#include "fld_internal.cuh"

namespace fld {

namespace {

constexpr int ZM_XL = 4;         // halo columns on each side: one 16-byte chunk
constexpr int ZM_D = 2;          // planes in flight ahead of use
constexpr int ZM_R = ZM_D + 5;   // ring depth: planes k-3 .. k+1+D

template <int TX, int TY>
struct ZmShape {
    static constexpr int XW = TX + 2 * ZM_XL;   // shared row pitch (words)
    static constexpr int NROW = TY + 4;
    static constexpr int PL = XW * NROW;        // floats per plane and field
    static constexpr int CPR = XW / 4;          // 16-byte chunks per shared row
    static constexpr int NCH = NROW * CPR;      // chunks per plane and field
    static constexpr int WX = TX / 32;          // warps across the tile width
    static constexpr int NT = 32 * WX * (TY / 2);
    static constexpr size_t SMEM = sizeof(float) * 3 * ZM_R * PL;
    static_assert(TX % 32 == 0 && TY % 2 == 0, "tile of whole warps and row pairs");
    static_assert(XW % 32 == 8 || XW % 32 == 24, "row pitch giving conflict-free lanes");
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

// (b + acc)/(1 + sw) of one cell: z points at the shared array, o0 is the cell's offset
// in the slot of its plane (x at +0, K at +PL, b at +2 PL), om and op the offsets of the
// same cell in the slots of the planes below and above; XW is the row pitch; h* = w_d / 2.
// Every access is one shared load at an immediate offset from o0, om or op.
template <int XW, int PL>
__device__ __forceinline__ float zm_relax(const float* z, int o0, int om, int op, float hx,
                                          float hy, float hz) {
    const float kc = z[o0 + PL];
    float f = (kc + z[o0 + PL - 1]) * hx;
    float sw = f;
    float acc = f * z[o0 - 1];
    f = (kc + z[o0 + PL + 1]) * hx;
    sw += f;
    acc = fmaf(f, z[o0 + 1], acc);
    f = (kc + z[o0 + PL - XW]) * hy;
    sw += f;
    acc = fmaf(f, z[o0 - XW], acc);
    f = (kc + z[o0 + PL + XW]) * hy;
    sw += f;
    acc = fmaf(f, z[o0 + XW], acc);
    f = (kc + z[om + PL]) * hz;
    sw += f;
    acc = fmaf(f, z[om], acc);
    f = (kc + z[op + PL]) * hz;
    sw += f;
    acc = fmaf(f, z[op], acc);
    return __fdividef(z[o0 + 2 * PL] + acc, 1.0f + sw);
}

}  // namespace

template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(ZmShape<TX, TY>::NT, MINB)
k_rb_zmarch(Lvl L, const float* __restrict__ xin, float* __restrict__ xout,
            const float* __restrict__ b, const float* __restrict__ K, int cz) {
    using SH = ZmShape<TX, TY>;
    constexpr int PL = SH::PL, XW = SH::XW, CPR = SH::CPR;
    extern __shared__ __align__(16) float zsm[];

    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int tilesx = (nx + TX - 1) / TX, tilesy = (ny + TY - 1) / TY;
    int bid = blockIdx.x;
    const int tx0 = (bid % tilesx) * TX;
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
        const int r = tid / CPR, ch = tid - r * CPR;
        soff = r * XW + 4 * ch;
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

    // Copy plane m (raw z coordinate, may lie outside [0, nz)) into the ring slot at
    // offset `slot` of the shared array.
    auto issue = [&](int m, int slot) {
        if (cmode < 5 && m <= z1 + 1) {
            float* Sd = zsm + slot + soff;
            float* Kd = Sd + PL;
            float* Bd = Kd + PL;
            const int gz = zm_axis(m, nz, zper);
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gz >= 0 && cmode == 0) {
                const long long o = fld_span(gz * plane + goff, 4, L.ncell);
                zm_cp16(Sd, xin + o);
                zm_cp16(Kd, K + o);
                zm_cp16(Bd, b + o);
            } else {
                // ghosts: x = b = 0 and K = factor * K of the mirrored wall cell
                float4 k4 = z4;
                if (gz >= 0 && cmode == 1) {
                    k4.w = gfac * K[fld_at(gz * plane + goff, L.ncell)];
                } else if (gz >= 0 && cmode == 2) {
                    k4.x = gfac * K[fld_at(gz * plane + goff, L.ncell)];
                } else if (gz >= 0 && cmode == 3) {
                    const float4 v = *reinterpret_cast<const float4*>(
                        K + fld_span(gz * plane + goff, 4, L.ncell));
                    k4 = make_float4(gfac * v.x, gfac * v.y, gfac * v.z, gfac * v.w);
                } else if ((gz == -1 || gz == -2) && cmode == 0) {
                    const float f = zm_ghost_factor(gz == -1 ? L.bclo[2] : L.bchi[2]);
                    const long long o = fld_span((long long)(gz == -1 ? 0 : nz - 1) * plane + goff,
                                                 4, L.ncell);
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

    // ---- the interior column pair of this thread
    const int lane = tid & 31, w = tid >> 5;
    const int lx = 32 * (w % SH::WX) + lane, ly0 = 2 * (w / SH::WX);
    const int gx = tx0 + lx, gy0 = ty0 + ly0;
    const bool act0 = gx < nx && gy0 < ny, act1 = gx < nx && gy0 + 1 < ny;
    const int c0 = (ly0 + 2) * XW + ZM_XL + lx;

    // ---- the ring cell pair of this thread: cells at distance 1 outside the active
    // rectangle [0, ax) x [0, ay) of the tile whose red value a black interior cell reads.
    // Row pairs (lx = 2k - 1, 2k) on ly = -1 and ly = ay; column pairs (ly = 2k, 2k + 1)
    // on lx = -1 and lx = ax. Exactly one cell of a pair is red on any plane.
    const int ax = min(TX, nx - tx0), ay = min(TY, ny - ty0);
    const int nrow = (ax + 2) / 2, ncol = (ay + 1) / 2;
    int rc0 = -1, rc1 = -1;    // shared offsets of the two candidates (-1: not a cell)
    int rpar = 0;              // parity of gx + gy of candidate 0
    {
        int qx0 = 0, qy0 = 0, dx = 0, dy = 0;
        bool has = true, colseg = false;
        if (tid < nrow) {
            qx0 = 2 * tid - 1; qy0 = -1; dx = 1;
        } else if (tid < 2 * nrow) {
            qx0 = 2 * (tid - nrow) - 1; qy0 = ay; dx = 1;
        } else if (tid < 2 * nrow + ncol) {
            qx0 = -1; qy0 = 2 * (tid - 2 * nrow); dy = 1; colseg = true;
        } else if (tid < 2 * nrow + 2 * ncol) {
            qx0 = ax; qy0 = 2 * (tid - 2 * nrow - ncol); dy = 1; colseg = true;
        } else {
            has = false;
        }
        if (has) {
            rpar = (tx0 + qx0 + ty0 + qy0) & 1;
            for (int q = 0; q < 2; ++q) {
                const int qx = qx0 + q * dx, qy = qy0 + q * dy;
                const bool cell = zm_axis(tx0 + qx, nx, xper) >= 0 &&
                                  zm_axis(ty0 + qy, ny, yper) >= 0;
                const int off = (cell && !(colseg && qy >= ay)) ? (qy + 2) * XW + ZM_XL + qx : -1;
                if (q == 0) rc0 = off; else rc1 = off;
            }
        }
    }

    // Ring slot offsets of planes k-3 .. k+3 at step k (x at +0, K at +PL, b at +2 PL);
    // each step rotates them by one, the slot of k-3 coming back as that of k+4.
    auto slot_of = [&](int m) { return ((m + 2 * ZM_R) % ZM_R) * 3 * PL; };
    int pm3 = slot_of(z0 - 4), pm2 = slot_of(z0 - 3), pm1 = slot_of(z0 - 2), p00 = slot_of(z0 - 1);
    int pp1 = slot_of(z0), pp2 = slot_of(z0 + 1), pp3 = slot_of(z0 + 2);
    static_assert(ZM_D == 2 && ZM_R == 7, "the rotation below holds planes k-3 .. k+3");
    const bool ring_warp = (tid & ~31) < 2 * nrow + 2 * ncol;   // warp-uniform
    float* xo = xout + (long long)gy0 * nx + gx;

    // ---- the march. Step k: planes <= k + 1 have landed; red(k) on the tile and its ring
    // (in place in the shared copy) and black(k - 2), which reads planes k - 3 .. k - 1
    // only. Both are evaluated unconditionally (so their arithmetic interleaves) and only
    // the stores are predicated. The copy of plane k + 3 goes into the slot of plane k - 4,
    // last read by black(k - 3) in the previous step.
    issue(z0 - 2, pm1);
    issue(z0 - 1, p00);
    issue(z0, pp1);
    issue(z0 + 1, pp2);
    for (int k = z0 - 1; k <= z1 + 1; ++k) {
        zm_wait<ZM_D - 1>();
        __syncthreads();
        issue(k + 3, pp3);
        const bool do_red = k <= z1 && zm_axis(k, nz, zper) >= 0;
        const bool do_black = k - 2 >= z0;
        // red(k): the red row of the pair (parity of gz = parity of k: periodic extents
        // are even, ghost planes are not updated)
        const int q = (gx + gy0 + k) & 1;
        const int cr = c0 + q * XW, cb = cr + (1 - 2 * q) * XW;
        const float vr = zm_relax<XW, PL>(zsm, p00 + cr, pm1 + cr, pp1 + cr, hx, hy, hz);
        // black(k - 2): the other row of the pair at plane k - 2 (same parity as k)
        const float vb = zm_relax<XW, PL>(zsm, pm2 + cb, pm3 + cb, pm1 + cb, hx, hy, hz);
        const float vrb = zsm[pm2 + cr];             // its red cell, updated two steps ago
        if (ring_warp) {
            const bool rsel = (rpar + k) & 1;
            const int cg = rsel ? rc1 : rc0;
            const int cq = cg >= 0 ? cg : c0;
            const float vg = zm_relax<XW, PL>(zsm, p00 + cq, pm1 + cq, pp1 + cq, hx, hy, hz);
            if (do_red && cg >= 0) zsm[p00 + cg] = vg;
        }
        if (do_red && (q ? act1 : act0)) zsm[p00 + cr] = vr;
        if (do_black) {
            // the pair's plane k - 2 (its row span checked in the debug build)
            float* o = xo + (long long)(k - 2) * plane;
            if (act0) o = xout + fld_span(o - xout, act1 ? nx + 1 : 1, L.ncell);
            if (act0) o[0] = q ? vb : vrb;
            if (act1) o[nx] = q ? vrb : vb;
        }
        const int t = pm3;
        pm3 = pm2; pm2 = pm1; pm1 = p00; p00 = pp1; pp1 = pp2; pp2 = pp3; pp3 = t;
    }
    zm_wait<0>();
}

namespace {

constexpr int ZM_TX = 32, ZM_TY = 16, ZM_MINB = 3;
using ZmMain = ZmShape<ZM_TX, ZM_TY>;

constexpr int ZM_MAXDEV = 64;
// resident blocks of the sweep kernel on the whole GPU, per device (0: not prepared yet)
std::atomic<int> g_zm_slots[ZM_MAXDEV];
std::mutex g_zm_mutex;

int zm_slots() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= ZM_MAXDEV) return 1;
    return std::max(1, g_zm_slots[dev].load(std::memory_order_relaxed));
}

// z-chunk length. A block of a chunk of cz planes marches cz + 3 steps, and the blocks
// (tiles times chunks) run in waves of the resident slots, so the sweep takes about
// waves x (cz + 3) step times: the chunk length minimises that, from chunks of at least 8
// planes (2 on levels of at most 64^3 cells, which are bound by the march's per-plane
// latency, not by traffic) up to the whole extent. At 256^3 it picks 37 planes (7 chunks,
// two full waves); at 128^3 10 planes (one wave of 416 blocks, where 8 planes made 512
// blocks, a second wave of 56).
int zm_chunk(const Lvl& L) {
    const long long tiles = ((L.n[0] + ZM_TX - 1) / ZM_TX) * ((L.n[1] + ZM_TY - 1) / ZM_TY);
    const long long slots = zm_slots();
    const int nz = L.n[2];
    const int minc = std::min(nz, L.ncell <= (1LL << 18) ? 2 : 8);
    int best = nz;
    long long best_cost = -1;
    for (int cz = minc; cz <= nz; ++cz) {
        const long long nch = (nz + cz - 1) / cz;
        if (cz > minc && (nz + cz - 2) / (cz - 1) == nch) continue;   // same chunk count
        const long long waves = (tiles * nch + slots - 1) / slots;
        const long long cost = waves * (cz + 3);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = cz;
        }
    }
    return best;
}

}  // namespace

// FP32 3D levels whose x extent is a whole number of 16-byte chunks and whose periodic
// extents are even; everything else (and FP64) uses the half-sweep smoothers.
template <typename T>
bool rb_sweep_supported(const Lvl& L) {
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
        // the arithmetic face mean only (the harmonic one takes the half sweeps)
        if (L.fm || L.ndim != 3 || L.n[0] % 4 != 0 || L.n[0] < 16) return false;
        for (int d = 0; d < 3; ++d)
            if (L.bclo[d] == FLD_BC_PERIODIC && (L.n[d] & 1)) return false;
        return true;
    }
}

template <typename T>
void launch_rb_sweep(const Lvl& L, const T* xin, T* xout, const T* b, const T* K,
                     cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        const int cz = zm_chunk(L);
        const int tiles = ((L.n[0] + ZM_TX - 1) / ZM_TX) * ((L.n[1] + ZM_TY - 1) / ZM_TY);
        const int nch = (L.n[2] + cz - 1) / cz;
        k_rb_zmarch<ZM_TX, ZM_TY, ZM_MINB>
            <<<tiles * nch, ZmMain::NT, ZmMain::SMEM, s>>>(L, xin, xout, b, K, cz);
    }
}

// Opt the kernel into its shared-memory size and count its resident blocks, once per
// device (the attribute is a per-device setting), with that device current and outside
// any stream capture (called when a handle is created).
void prepare_rb_sweep() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= ZM_MAXDEV) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lock(g_zm_mutex);
    if (g_zm_slots[dev].load() > 0) return;
    cudaFuncSetAttribute(k_rb_zmarch<ZM_TX, ZM_TY, ZM_MINB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZmMain::SMEM);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rb_zmarch<ZM_TX, ZM_TY, ZM_MINB>,
                                                  ZmMain::NT, ZmMain::SMEM);
    g_zm_slots[dev].store(num_sms() * std::max(1, occ));
}

template bool rb_sweep_supported<float>(const Lvl&);
template bool rb_sweep_supported<double>(const Lvl&);
template void launch_rb_sweep<float>(const Lvl&, const float*, float*, const float*, const float*,
                                     cudaStream_t);
template void launch_rb_sweep<double>(const Lvl&, const double*, double*, const double*,
                                      const double*, cudaStream_t);

}  // namespace fld
