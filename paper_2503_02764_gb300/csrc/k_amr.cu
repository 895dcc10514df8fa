// Kernels of the composite-grid diffusion solve (fld_amr_*): a coarse block of cells H_d
// with one box refined by 2 in every axis (cells h_d = H_d / 2). The unknowns are the
// coarse cells outside the box and every fine cell; for each, in volume-normalised flux
// form,
//   (A x)_p = x_p + sum_faces c_f (x_p - x_q) + sum_Dirichlet c_w x_p,
//   c_f = dt a_f / V_p,  a_f = (D_p + D_q)/2 * area_f / dist_f,
// with dist_f = H_d (coarse-coarse), h_d (fine-fine), 3 h_d / 2 (a fine cell and the coarse
// cell across the box's edge, one coarse face meeting 2^(d-1) fine faces), and a Dirichlet
// wall at half a cell. Each face flux enters both its cells with opposite signs
// (conservative). Along each axis the box lies strictly inside the block or spans it (then
// the axis's walls apply to the fine cells).
//
// The solve (fld_amr_api.cu) is a two-level scheme: red-black Gauss-Seidel on the
// composite grid (coarse cells, then fine cells, each in two colours), the composite
// residual, its restriction to the whole coarse block (a covered coarse cell takes the
// mean of its fine cells' residuals, the volume-weighted restriction of the flux form),
// the coarse correction by the uniform multigrid solver on the coarse block (covered
// cells carry the mean of their fine cells' D) and its piecewise-constant prolongation.
// FP64 throughout; one thread per cell.
#include "fld_amr.cuh"
#include "fld_device.cuh"

namespace fld {

namespace {

__device__ __forceinline__ int amr_ncoarse_cells(const AmrGeom& G) {
    return G.nc[0] * G.nc[1] * G.nc[2];
}
__device__ __forceinline__ int amr_nfine_cells(const AmrGeom& G) {
    return G.nf[0] * G.nf[1] * G.nf[2];
}
__device__ __forceinline__ int cidx(const AmrGeom& G, const int* c) {
    return (c[2] * G.nc[1] + c[1]) * G.nc[0] + c[0];
}
__device__ __forceinline__ int fidx(const AmrGeom& G, const int* f) {
    return (f[2] * G.nf[1] + f[1]) * G.nf[0] + f[0];
}
__device__ __forceinline__ bool covered(const AmrGeom& G, const int* c) {
    for (int d = 0; d < G.nd; ++d)
        if (c[d] < G.lo[d] || c[d] >= G.hi[d]) return false;
    return true;
}
__device__ __forceinline__ bool spans(const AmrGeom& G, int d) {
    return G.lo[d] == 0 && G.hi[d] == G.nc[d];
}

// Face value of a Dirichlet wall of the coarse block for coarse cell c (axis d, side s):
// the face array over the two other axes, the lower one fastest.
__device__ __forceinline__ double wall_value(const AmrGeom& G, const double* Ebc, int d, int s,
                                             const int* c) {
    const long long off = G.bcoff[2 * d + s];
    const long long f = d == 0 ? (long long)c[2] * G.nc[1] + c[1]
                      : d == 1 ? (long long)c[2] * G.nc[0] + c[0]
                               : (long long)c[1] * G.nc[0] + c[0];
    return Ebc[off + f];
}

// Operator row of coarse cell c (uncovered): diag = 1 + sum c_f (+ walls), off = sum c_f x_q,
// wall = sum c_w E_b (the right-hand side's wall term).
__device__ void coarse_row(const AmrGeom& G, const double* Dc, const double* Df,
                           const double* xc, const double* xf, const double* Ebc, const int* c,
                           double& diag, double& off, double& wall) {
    const double Dp = Dc[cidx(G, c)];
    diag = 1.0;
    off = 0.0;
    wall = 0.0;
    for (int d = 0; d < G.nd; ++d) {
        const double H2 = G.H[d] * G.H[d];
        for (int s = 0; s < 2; ++s) {
            int q[3] = {c[0], c[1], c[2]};
            q[d] += s ? 1 : -1;
            if (q[d] < 0 || q[d] >= G.nc[d]) {
                const int kind = s ? G.bchi[d] : G.bclo[d];
                if (kind == FLD_BC_PERIODIC) {
                    q[d] = (q[d] + G.nc[d]) % G.nc[d];
                } else {
                    if (kind == FLD_BC_DIRICHLET) {
                        const double cw = G.dt * 2.0 * Dp / H2;
                        diag += cw;
                        if (Ebc) wall += cw * wall_value(G, Ebc, d, s, c);
                    }
                    continue;
                }
            }
            if (!covered(G, q)) {
                const double cf = G.dt * 0.5 * (Dp + Dc[cidx(G, q)]) / H2;
                diag += cf;
                off += cf * xc[cidx(G, q)];
                continue;
            }
            // the box's edge: the 2^(nd-1) fine cells of the layer facing c
            int f0[3] = {0, 0, 0};
            for (int e = 0; e < G.nd; ++e) f0[e] = 2 * (c[e] - G.lo[e]);
            f0[d] = s ? 0 : G.nf[d] - 1;
            const double w = G.dt * 0.5 / (0.75 * H2 * (double)(1 << (G.nd - 1)));
            const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
            const int n1 = t1 < G.nd ? 2 : 1, n2 = t2 < G.nd ? 2 : 1;
            for (int b = 0; b < n2; ++b)
                for (int a = 0; a < n1; ++a) {
                    int f[3] = {f0[0], f0[1], f0[2]};
                    f[t1] += a;
                    f[t2] += b;
                    const int fi = fidx(G, f);
                    const double cf = w * (Dp + Df[fi]);
                    diag += cf;
                    off += cf * xf[fi];
                }
        }
    }
}

// Operator row of fine cell f.
__device__ void fine_row(const AmrGeom& G, const double* Dc, const double* Df, const double* xc,
                         const double* xf, const double* Ebc, const int* f, double& diag,
                         double& off, double& wall) {
    const double Dp = Df[fidx(G, f)];
    diag = 1.0;
    off = 0.0;
    wall = 0.0;
    for (int d = 0; d < G.nd; ++d) {
        const double h2 = 0.25 * G.H[d] * G.H[d];
        for (int s = 0; s < 2; ++s) {
            int g[3] = {f[0], f[1], f[2]};
            g[d] += s ? 1 : -1;
            if (g[d] >= 0 && g[d] < G.nf[d]) {
                const double cf = G.dt * 0.5 * (Dp + Df[fidx(G, g)]) / h2;
                diag += cf;
                off += cf * xf[fidx(G, g)];
                continue;
            }
            if (spans(G, d)) {
                const int kind = s ? G.bchi[d] : G.bclo[d];
                if (kind == FLD_BC_PERIODIC) {
                    g[d] = (g[d] + G.nf[d]) % G.nf[d];
                    const double cf = G.dt * 0.5 * (Dp + Df[fidx(G, g)]) / h2;
                    diag += cf;
                    off += cf * xf[fidx(G, g)];
                } else if (kind == FLD_BC_DIRICHLET) {
                    const double cw = G.dt * 2.0 * Dp / h2;
                    diag += cw;
                    if (Ebc) {
                        int c[3] = {0, 0, 0};
                        for (int e = 0; e < 3; ++e) c[e] = e < G.nd ? G.lo[e] + f[e] / 2 : 0;
                        wall += cw * wall_value(G, Ebc, d, s, c);
                    }
                }
                continue;
            }
            // the coarse cell across the box's edge
            int c[3] = {0, 0, 0};
            for (int e = 0; e < 3; ++e) c[e] = e < G.nd ? G.lo[e] + f[e] / 2 : 0;
            c[d] += s ? 1 : -1;
            const int ci = cidx(G, c);
            const double cf = G.dt * 0.5 * (Dp + Dc[ci]) / (1.5 * h2);
            diag += cf;
            off += cf * xc[ci];
        }
    }
}

__device__ __forceinline__ void coarse_coord(const AmrGeom& G, int p, int* c) {
    c[0] = p % G.nc[0];
    const int q = p / G.nc[0];
    c[1] = q % G.nc[1];
    c[2] = q / G.nc[1];
}
__device__ __forceinline__ void fine_coord(const AmrGeom& G, int p, int* f) {
    f[0] = p % G.nf[0];
    const int q = p / G.nf[0];
    f[1] = q % G.nf[1];
    f[2] = q / G.nf[1];
}

// b = E + wall terms (unknown cells); DH = Dc (uncovered) or the mean of the fine D
__global__ void k_amr_setup(AmrGeom G, const double* __restrict__ Dc,
                            const double* __restrict__ Df, const double* __restrict__ Ec,
                            const double* __restrict__ Ef, const double* __restrict__ Ebc,
                            double* __restrict__ bc, double* __restrict__ bf,
                            double* __restrict__ DH) {
    const int nC = amr_ncoarse_cells(G), nF = amr_nfine_cells(G);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nC + nF; p += gridDim.x * blockDim.x) {
        double diag, off, wall;
        if (p < nC) {
            int c[3];
            coarse_coord(G, p, c);
            if (covered(G, c)) {
                double s = 0.0;
                const int n1 = G.nd > 1 ? 2 : 1, n2 = G.nd > 2 ? 2 : 1;
                for (int z = 0; z < n2; ++z)
                    for (int y = 0; y < n1; ++y)
                        for (int x = 0; x < 2; ++x) {
                            const int f[3] = {2 * (c[0] - G.lo[0]) + x,
                                              G.nd > 1 ? 2 * (c[1] - G.lo[1]) + y : 0,
                                              G.nd > 2 ? 2 * (c[2] - G.lo[2]) + z : 0};
                            s += Df[fidx(G, f)];
                        }
                DH[p] = s / (double)(2 * n1 * n2);
                bc[p] = 0.0;
            } else {
                coarse_row(G, Dc, Df, Ec, Ef, Ebc, c, diag, off, wall);
                DH[p] = Dc[p];
                bc[p] = Ec[p] + wall;
            }
        } else {
            int f[3];
            fine_coord(G, p - nC, f);
            fine_row(G, Dc, Df, Ec, Ef, Ebc, f, diag, off, wall);
            bf[p - nC] = Ef[p - nC] + wall;
        }
    }
}

// one colour of one grid: phase 0/1 coarse cells of colour 0/1, 2/3 fine cells
__global__ void k_amr_smooth(AmrGeom G, int phase, const double* __restrict__ Dc,
                             const double* __restrict__ Df, const double* __restrict__ bc,
                             const double* __restrict__ bf, double* xc, double* xf) {
    const bool fine = phase >= 2;
    const int colour = phase & 1;
    const int n = fine ? amr_nfine_cells(G) : amr_ncoarse_cells(G);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        int c[3];
        if (fine) fine_coord(G, p, c);
        else coarse_coord(G, p, c);
        if (((c[0] + c[1] + c[2]) & 1) != colour) continue;
        double diag, off, wall;
        if (fine) {
            fine_row(G, Dc, Df, xc, xf, nullptr, c, diag, off, wall);
            xf[p] = (bf[p] + off) / diag;
        } else {
            if (covered(G, c)) continue;
            coarse_row(G, Dc, Df, xc, xf, nullptr, c, diag, off, wall);
            xc[p] = (bc[p] + off) / diag;
        }
    }
}

// composite residual r = b - A x (covered coarse cells: the mean of their fine cells'
// residuals, the restriction) and partial sums of r^2 over the unknowns
__global__ void k_amr_resid(AmrGeom G, const double* __restrict__ Dc,
                            const double* __restrict__ Df, const double* __restrict__ bc,
                            const double* __restrict__ bf, const double* __restrict__ xc,
                            const double* __restrict__ xf, double* __restrict__ rc,
                            double* __restrict__ rf, double* __restrict__ partials) {
    __shared__ double sh[32];
    const int nC = amr_ncoarse_cells(G), nF = amr_nfine_cells(G);
    double acc = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nC + nF; p += gridDim.x * blockDim.x) {
        double diag, off, wall;
        if (p < nC) {
            int c[3];
            coarse_coord(G, p, c);
            if (covered(G, c)) continue;
            coarse_row(G, Dc, Df, xc, xf, nullptr, c, diag, off, wall);
            const double r = bc[p] + off - diag * xc[p];
            rc[p] = r;
            acc = fma(r, r, acc);
        } else {
            int f[3];
            fine_coord(G, p - nC, f);
            fine_row(G, Dc, Df, xc, xf, nullptr, f, diag, off, wall);
            const double r = bf[p - nC] + off - diag * xf[p - nC];
            rf[p - nC] = r;
            acc = fma(r, r, acc);
        }
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// covered coarse cells: the mean of their fine cells (of v)
__global__ void k_amr_average(AmrGeom G, const double* __restrict__ vf, double* vc) {
    const int nC = amr_ncoarse_cells(G);
    const int n1 = G.nd > 1 ? 2 : 1, n2 = G.nd > 2 ? 2 : 1;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nC; p += gridDim.x * blockDim.x) {
        int c[3];
        coarse_coord(G, p, c);
        if (!covered(G, c)) continue;
        double s = 0.0;
        for (int z = 0; z < n2; ++z)
            for (int y = 0; y < n1; ++y)
                for (int x = 0; x < 2; ++x) {
                    const int f[3] = {2 * (c[0] - G.lo[0]) + x,
                                      G.nd > 1 ? 2 * (c[1] - G.lo[1]) + y : 0,
                                      G.nd > 2 ? 2 * (c[2] - G.lo[2]) + z : 0};
                    s += vf[fidx(G, f)];
                }
        vc[p] = s / (double)(2 * n1 * n2);
    }
}

// x += e on the composite grid: uncovered coarse cells directly, fine cells from their
// parent (piecewise constant)
__global__ void k_amr_correct(AmrGeom G, const double* __restrict__ e, double* xc, double* xf) {
    const int nC = amr_ncoarse_cells(G), nF = amr_nfine_cells(G);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nC + nF; p += gridDim.x * blockDim.x) {
        if (p < nC) {
            int c[3];
            coarse_coord(G, p, c);
            if (!covered(G, c)) xc[p] += e[p];
        } else {
            int f[3];
            fine_coord(G, p - nC, f);
            int c[3] = {0, 0, 0};
            for (int d = 0; d < 3; ++d) c[d] = d < G.nd ? G.lo[d] + f[d] / 2 : 0;
            xf[p - nC] += e[cidx(G, c)];
        }
    }
}

int amr_blocks(long long n) {
    const long long nb = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(nb, (long long)num_sms() * 16));
}

}  // namespace

void launch_amr_setup(const AmrGeom& G, const double* Dc, const double* Df, const double* Ec,
                      const double* Ef, const double* Ebc, double* bc, double* bf, double* DH,
                      cudaStream_t s) {
    const long long n = (long long)G.nc[0] * G.nc[1] * G.nc[2] + (long long)G.nf[0] * G.nf[1] * G.nf[2];
    k_amr_setup<<<amr_blocks(n), 256, 0, s>>>(G, Dc, Df, Ec, Ef, Ebc, bc, bf, DH);
}

void launch_amr_smooth(const AmrGeom& G, int phase, const double* Dc, const double* Df,
                       const double* bc, const double* bf, double* xc, double* xf,
                       cudaStream_t s) {
    const long long n = phase >= 2 ? (long long)G.nf[0] * G.nf[1] * G.nf[2]
                                   : (long long)G.nc[0] * G.nc[1] * G.nc[2];
    k_amr_smooth<<<amr_blocks(n), 256, 0, s>>>(G, phase, Dc, Df, bc, bf, xc, xf);
}

int launch_amr_resid(const AmrGeom& G, const double* Dc, const double* Df, const double* bc,
                     const double* bf, const double* xc, const double* xf, double* rc, double* rf,
                     double* partials, int nblocks, cudaStream_t s) {
    const long long n = (long long)G.nc[0] * G.nc[1] * G.nc[2] + (long long)G.nf[0] * G.nf[1] * G.nf[2];
    const int nb = std::min(nblocks, amr_blocks(n));
    k_amr_resid<<<nb, 256, 0, s>>>(G, Dc, Df, bc, bf, xc, xf, rc, rf, partials);
    return nb;
}

void launch_amr_average(const AmrGeom& G, const double* vf, double* vc, cudaStream_t s) {
    k_amr_average<<<amr_blocks((long long)G.nc[0] * G.nc[1] * G.nc[2]), 256, 0, s>>>(G, vf, vc);
}

void launch_amr_correct(const AmrGeom& G, const double* e, double* xc, double* xf,
                        cudaStream_t s) {
    const long long n = (long long)G.nc[0] * G.nc[1] * G.nc[2] + (long long)G.nf[0] * G.nf[1] * G.nf[2];
    k_amr_correct<<<amr_blocks(n), 256, 0, s>>>(G, e, xc, xf);
}

}  // namespace fld
