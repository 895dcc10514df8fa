// Grid transfers between a 3D level and its coarse level when every axis halves exactly
// (even fine extents, C.n = F.n / 2): one thread per coarse cell handles its 2 x 2 x 2
// children. The fine rows of a warp's 32 coarse cells are 64 contiguous values, read and
// written as pairs; the values the children share with their neighbours come from the
// neighbouring threads' lines in L1.
//
// Restriction: coarse b = mean over the 8 children of the fine residual b - A x, with A
// the level operator (face weights (K_p + K_q) w_d / 2; a Neumann face has weight 0, a
// Dirichlet face the half-cell 2 K_p w_d, both folded into a ghost K = -K_p or 3 K_p and
// ghost x = 0 in registers). Prolongation: x += the cell-centred trilinear interpolant of
// the coarse correction, 3/4 of the parent and 1/4 of the coarse neighbour on the child's
// side along each axis, a missing neighbour at a wall being the parent mirrored (+e for
// Neumann, -e for Dirichlet). Levels outside this shape use the general kernels.
#include "fld_device.cuh"

namespace fld {

namespace {

// Fine index of the neighbour at offset `d` (-1 or +1) of fine cell `i` on an axis of
// extent n: the index, or -1 beyond a non-periodic wall.
__device__ __forceinline__ int tr_nb(int i, int d, int n, bool per) {
    const int j = i + d;
    if (j >= 0 && j < n) return j;
    if (!per) return -1;
    return j < 0 ? j + n : j - n;
}

__device__ __forceinline__ float tr_factor(int bc) { return bc == FLD_BC_DIRICHLET ? 3.f : -1.f; }

template <typename T>
struct Pair {
    T v[2];
};

template <typename T>
__device__ __forceinline__ Pair<T> ld2(const T* p) {
    Pair<T> r;
    if constexpr (sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        r.v[0] = v.x;
        r.v[1] = v.y;
    } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        r.v[0] = v.x;
        r.v[1] = v.y;
    }
    return r;
}

template <typename T>
__device__ __forceinline__ void st2(T* p, T a, T b) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
    }
}

}  // namespace

bool transfer3_ok(const Lvl& F, const Lvl& C) {
    if (F.ndim != 3) return false;
    for (int d = 0; d < 3; ++d)
        if (F.n[d] != 2 * C.n[d]) return false;
    return true;
}

template <typename T>
__global__ void k_resid_restrict3(Lvl F, Lvl C, const T* __restrict__ x, const T* __restrict__ b,
                                  const T* __restrict__ K, T* __restrict__ bc) {
    const int I = blockIdx.x * 32 + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int Kc = blockIdx.z;
    if (I >= C.n[0] || J >= C.n[1]) return;
    const int nx = F.n[0], ny = F.n[1], nz = F.n[2];
    const long long sy = nx, sz = (long long)nx * ny;
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * Kc;
    const T hx = T(0.5) * wgt<T>(F, 0), hy = T(0.5) * wgt<T>(F, 1), hz = T(0.5) * wgt<T>(F, 2);
    // neighbours outside the 2x2x2 block on each axis (below, above)
    const int xl = tr_nb(i0, -1, nx, F.bclo[0] == FLD_BC_PERIODIC);
    const int xr = tr_nb(i0 + 1, 1, nx, F.bclo[0] == FLD_BC_PERIODIC);
    const int yl = tr_nb(j0, -1, ny, F.bclo[1] == FLD_BC_PERIODIC);
    const int yr = tr_nb(j0 + 1, 1, ny, F.bclo[1] == FLD_BC_PERIODIC);
    const int zl = tr_nb(k0, -1, nz, F.bclo[2] == FLD_BC_PERIODIC);
    const int zr = tr_nb(k0 + 1, 1, nz, F.bclo[2] == FLD_BC_PERIODIC);
    const T fxl = (T)tr_factor(F.bclo[0]), fxr = (T)tr_factor(F.bchi[0]);
    const T fyl = (T)tr_factor(F.bclo[1]), fyr = (T)tr_factor(F.bchi[1]);
    const T fzl = (T)tr_factor(F.bclo[2]), fzr = (T)tr_factor(F.bchi[2]);

    T s = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const long long pz = (long long)(k0 + c) * sz;
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const long long row = fld_span(pz + (long long)(j0 + bb) * sy, nx, F.ncell);
            const Pair<T> xv = ld2(x + row + i0), kv = ld2(K + row + i0), bv = ld2(b + row + i0);
            // x-neighbours of the pair
            const T xlv = xl >= 0 ? x[row + xl] : T(0);
            const T klv = xl >= 0 ? K[row + xl] : fxl * kv.v[0];
            const T xrv = xr >= 0 ? x[row + xr] : T(0);
            const T krv = xr >= 0 ? K[row + xr] : fxr * kv.v[1];
            // y-neighbours (row j0 - 1 for bb = 0, j0 + 2 for bb = 1; the other is the pair)
            const int jo = bb ? yr : yl;
            const T fy = bb ? fyr : fyl;
            Pair<T> xyo, kyo;
            if (jo >= 0) {
                const long long ry = fld_span(pz + (long long)jo * sy, nx, F.ncell);
                xyo = ld2(x + ry + i0);
                kyo = ld2(K + ry + i0);
            } else {
                xyo.v[0] = xyo.v[1] = T(0);
                kyo.v[0] = fy * kv.v[0];
                kyo.v[1] = fy * kv.v[1];
            }
            const long long rowi = fld_span(pz + (long long)(j0 + 1 - bb) * sy, nx, F.ncell);   // the pair's other row
            const Pair<T> xyi = ld2(x + rowi + i0), kyi = ld2(K + rowi + i0);
            // z-neighbours (plane k0 - 1 for c = 0, k0 + 2 for c = 1; the other is the pair)
            const int ko = c ? zr : zl;
            const T fz = c ? fzr : fzl;
            Pair<T> xzo, kzo;
            if (ko >= 0) {
                const long long ro = fld_span((long long)ko * sz + (long long)(j0 + bb) * sy, nx, F.ncell) + i0;
                xzo = ld2(x + ro);
                kzo = ld2(K + ro);
            } else {
                xzo.v[0] = xzo.v[1] = T(0);
                kzo.v[0] = fz * kv.v[0];
                kzo.v[1] = fz * kv.v[1];
            }
            const long long rzi = fld_span((long long)(k0 + 1 - c) * sz + (long long)(j0 + bb) * sy, nx, F.ncell) + i0;
            const Pair<T> xzi = ld2(x + rzi), kzi = ld2(K + rzi);
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const T kc = kv.v[a];
                // faces in the order x-, x+, y-, y+, z-, z+
                const T kxm = a ? kv.v[0] : klv, xxm = a ? xv.v[0] : xlv;
                const T kxp = a ? krv : kv.v[1], xxp = a ? xrv : xv.v[1];
                const T kym = bb ? kyi.v[a] : kyo.v[a], xym = bb ? xyi.v[a] : xyo.v[a];
                const T kyp = bb ? kyo.v[a] : kyi.v[a], xyp = bb ? xyo.v[a] : xyi.v[a];
                const T kzm = c ? kzi.v[a] : kzo.v[a], xzm = c ? xzi.v[a] : xzo.v[a];
                const T kzp = c ? kzo.v[a] : kzi.v[a], xzp = c ? xzo.v[a] : xzi.v[a];
                T f = (kc + kxm) * hx;
                T sw = f, acc = f * xxm;
                f = (kc + kxp) * hx;
                sw += f;
                acc += f * xxp;
                f = (kc + kym) * hy;
                sw += f;
                acc += f * xym;
                f = (kc + kyp) * hy;
                sw += f;
                acc += f * xyp;
                f = (kc + kzm) * hz;
                sw += f;
                acc += f * xzm;
                f = (kc + kzp) * hz;
                sw += f;
                acc += f * xzp;
                s += bv.v[a] - (T(1) + sw) * xv.v[a] + acc;
            }
        }
    }
    bc[fld_at(((long long)Kc * C.n[1] + J) * C.n[0] + I, C.ncell)] = s * T(0.125);
}

// The same restriction right after a red-black smoothing sweep, which ends with the black
// cells (x + y + z odd) relaxed against their updated red neighbours: their residual is
// zero up to the rounding of that relaxation, so only the four red children of a coarse
// cell, (0,0,0), (1,1,0), (1,0,1) and (0,1,1) in (x, y, z) offsets, enter the mean. Each
// red child's six neighbours are three black siblings and three cells outside the block
// (one per axis, on its side), read as single values.
template <typename T>
__global__ void k_restrict_red3(Lvl F, Lvl C, const T* __restrict__ x, const T* __restrict__ b,
                                const T* __restrict__ K, T* __restrict__ bc) {
    const int I = blockIdx.x * 32 + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int Kc = blockIdx.z;
    if (I >= C.n[0] || J >= C.n[1]) return;
    const int nx = F.n[0], ny = F.n[1], nz = F.n[2];
    const long long sy = nx, sz = (long long)nx * ny;
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * Kc;
    const T hx = T(0.5) * wgt<T>(F, 0), hy = T(0.5) * wgt<T>(F, 1), hz = T(0.5) * wgt<T>(F, 2);
    const int xo[2] = {tr_nb(i0, -1, nx, F.bclo[0] == FLD_BC_PERIODIC),
                       tr_nb(i0 + 1, 1, nx, F.bclo[0] == FLD_BC_PERIODIC)};
    const int yo[2] = {tr_nb(j0, -1, ny, F.bclo[1] == FLD_BC_PERIODIC),
                       tr_nb(j0 + 1, 1, ny, F.bclo[1] == FLD_BC_PERIODIC)};
    const int zo[2] = {tr_nb(k0, -1, nz, F.bclo[2] == FLD_BC_PERIODIC),
                       tr_nb(k0 + 1, 1, nz, F.bclo[2] == FLD_BC_PERIODIC)};
    const T fx[2] = {(T)tr_factor(F.bclo[0]), (T)tr_factor(F.bchi[0])};
    const T fy[2] = {(T)tr_factor(F.bclo[1]), (T)tr_factor(F.bchi[1])};
    const T fz[2] = {(T)tr_factor(F.bclo[2]), (T)tr_factor(F.bchi[2])};

    // x and K of the eight children, rows (bb, c) read as pairs
    Pair<T> xv[2][2], kv[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const long long row =
                fld_span((long long)(k0 + c) * sz + (long long)(j0 + bb) * sy, nx, F.ncell) + i0;
            xv[c][bb] = ld2(x + row);
            kv[c][bb] = ld2(K + row);
        }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const int a = bb ^ c;                       // the red child of row (bb, c)
            const long long row =
                fld_span((long long)(k0 + c) * sz + (long long)(j0 + bb) * sy, nx, F.ncell);
            const T kc = kv[c][bb].v[a], xc = xv[c][bb].v[a];
            const T bv = b[row + i0 + a];
            // outside neighbours: x on side a, y on side bb, z on side c
            T xxo, kxo, xyo, kyo, xzo, kzo;
            if (xo[a] >= 0) {
                xxo = x[row + xo[a]];
                kxo = K[row + xo[a]];
            } else {
                xxo = T(0);
                kxo = fx[a] * kc;
            }
            if (yo[bb] >= 0) {
                const long long r = fld_span((long long)(k0 + c) * sz + (long long)yo[bb] * sy, nx,
                                             F.ncell) + i0 + a;
                xyo = x[r];
                kyo = K[r];
            } else {
                xyo = T(0);
                kyo = fy[bb] * kc;
            }
            if (zo[c] >= 0) {
                const long long r = fld_span((long long)zo[c] * sz + (long long)(j0 + bb) * sy, nx,
                                             F.ncell) + i0 + a;
                xzo = x[r];
                kzo = K[r];
            } else {
                xzo = T(0);
                kzo = fz[c] * kc;
            }
            // black siblings: across x in the same row, across y in row (1 - bb, c), across z
            // in row (bb, 1 - c), each at offset 1 - a, a, a of its pair
            const T xxi = xv[c][bb].v[1 - a], kxi = kv[c][bb].v[1 - a];
            const T xyi = xv[c][1 - bb].v[a], kyi = kv[c][1 - bb].v[a];
            const T xzi = xv[1 - c][bb].v[a], kzi = kv[1 - c][bb].v[a];
            // faces in the order x-, x+, y-, y+, z-, z+ (the side-0 neighbour is the lower)
            const T kxm = a ? kxi : kxo, xxm = a ? xxi : xxo;
            const T kxp = a ? kxo : kxi, xxp = a ? xxo : xxi;
            const T kym = bb ? kyi : kyo, xym = bb ? xyi : xyo;
            const T kyp = bb ? kyo : kyi, xyp = bb ? xyo : xyi;
            const T kzm = c ? kzi : kzo, xzm = c ? xzi : xzo;
            const T kzp = c ? kzo : kzi, xzp = c ? xzo : xzi;
            T f = (kc + kxm) * hx;
            T sw = f, acc = f * xxm;
            f = (kc + kxp) * hx;
            sw += f;
            acc += f * xxp;
            f = (kc + kym) * hy;
            sw += f;
            acc += f * xym;
            f = (kc + kyp) * hy;
            sw += f;
            acc += f * xyp;
            f = (kc + kzm) * hz;
            sw += f;
            acc += f * xzm;
            f = (kc + kzp) * hz;
            sw += f;
            acc += f * xzp;
            s += bv - (T(1) + sw) * xc + acc;
        }
    bc[fld_at(((long long)Kc * C.n[1] + J) * C.n[0] + I, C.ncell)] = s * T(0.125);
}

template <typename T>
__global__ void k_prolong3(Lvl F, Lvl C, T* __restrict__ xf, const T* __restrict__ xc) {
    const int I = blockIdx.x * 32 + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int Kc = blockIdx.z;
    if (I >= C.n[0] || J >= C.n[1]) return;
    const int cx = C.n[0], cy = C.n[1], cz = C.n[2];
    // coarse neighbour indices and mirror signs per axis: [0] below, [1] the parent, [2] above
    int ix[3], iy[3], iz[3];
    T sx[3], sy[3], sz[3];
    {
        const int n[3] = {cx, cy, cz};
        const int c[3] = {I, J, Kc};
        int* idx[3] = {ix, iy, iz};
        T* sg[3] = {sx, sy, sz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const bool per = F.bclo[d] == FLD_BC_PERIODIC;
            idx[d][1] = c[d];
            sg[d][1] = T(1);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int o = e ? c[d] + 1 : c[d] - 1;
                const int bc = e ? F.bchi[d] : F.bclo[d];
                int j = o;
                T sgn = T(1);
                if (o < 0 || o >= n[d]) {
                    if (per) {
                        j = o < 0 ? o + n[d] : o - n[d];
                    } else {
                        j = c[d];
                        sgn = bc == FLD_BC_DIRICHLET ? T(-1) : T(1);
                    }
                }
                idx[d][e ? 2 : 0] = j;
                sg[d][e ? 2 : 0] = sgn;
            }
        }
    }
    // interpolate along x, then y, then z: child a of an axis takes 3/4 of the parent and
    // 1/4 of the neighbour on its side (a = 0: below, a = 1: above)
    T vx[3][3][2];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const T* r = xc + fld_span(((long long)iz[dz] * cy + iy[dy]) * cx, cx, C.ncell);
            const T s = sz[dz] * sy[dy];
            const T e0 = s * sx[0] * r[ix[0]], e1 = s * r[ix[1]], e2 = s * sx[2] * r[ix[2]];
            vx[dz][dy][0] = T(0.75) * e1 + T(0.25) * e0;
            vx[dz][dy][1] = T(0.75) * e1 + T(0.25) * e2;
        }
    T vy[3][2][2];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            vy[dz][0][a] = T(0.75) * vx[dz][1][a] + T(0.25) * vx[dz][0][a];
            vy[dz][1][a] = T(0.75) * vx[dz][1][a] + T(0.25) * vx[dz][2][a];
        }
    const int nx = F.n[0];
    const long long sy2 = nx, sz2 = (long long)nx * F.n[1];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const T v0 = T(0.75) * vy[1][bb][0] + T(0.25) * vy[c ? 2 : 0][bb][0];
            const T v1 = T(0.75) * vy[1][bb][1] + T(0.25) * vy[c ? 2 : 0][bb][1];
            T* p = xf + fld_span((long long)(2 * Kc + c) * sz2 + (long long)(2 * J + bb) * sy2, nx, F.ncell) + 2 * I;
            const Pair<T> old = ld2(p);
            st2(p, old.v[0] + v0, old.v[1] + v1);
        }
}

template <typename T>
void launch_resid_restrict3(const Lvl& F, const Lvl& C, const T* x, const T* b, const T* K, T* bc,
                            bool red_only, cudaStream_t s) {
    dim3 block(32, 4);
    dim3 grid((C.n[0] + 31) / 32, (C.n[1] + 3) / 4, C.n[2]);
    if (red_only)
        k_restrict_red3<T><<<grid, block, 0, s>>>(F, C, x, b, K, bc);
    else
        k_resid_restrict3<T><<<grid, block, 0, s>>>(F, C, x, b, K, bc);
}

template <typename T>
void launch_prolong3(const Lvl& F, const Lvl& C, T* xf, const T* xc, cudaStream_t s) {
    dim3 block(32, 4);
    dim3 grid((C.n[0] + 31) / 32, (C.n[1] + 3) / 4, C.n[2]);
    k_prolong3<T><<<grid, block, 0, s>>>(F, C, xf, xc);
}

template void launch_resid_restrict3<float>(const Lvl&, const Lvl&, const float*, const float*,
                                            const float*, float*, bool, cudaStream_t);
template void launch_resid_restrict3<double>(const Lvl&, const Lvl&, const double*, const double*,
                                             const double*, double*, bool, cudaStream_t);
template void launch_prolong3<float>(const Lvl&, const Lvl&, float*, const float*, cudaStream_t);
template void launch_prolong3<double>(const Lvl&, const Lvl&, double*, const double*, cudaStream_t);

}  // namespace fld
