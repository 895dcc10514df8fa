// Declarations shared by the composite-grid solve's kernels (k_amr.cu) and its host side
// (fld_amr_api.cu).
#pragma once
#include <algorithm>

#include "fld_internal.cuh"

namespace fld {

// Geometry of a coarse block with one box refined by 2 (axes beyond nd have n = 1).
struct AmrGeom {
    int nd;
    int nc[3];              // coarse cells per axis
    int nf[3];              // fine cells per axis: 2 (hi - lo)
    int lo[3], hi[3];       // the box in coarse indices (hi exclusive)
    int bclo[3], bchi[3];
    double H[3];            // coarse cell sizes
    double dt;
    long long bcoff[6];     // offset of each Dirichlet face block in E_bc (-1: none)
};

void launch_amr_setup(const AmrGeom& G, const double* Dc, const double* Df, const double* Ec,
                      const double* Ef, const double* Ebc, double* bc, double* bf, double* DH,
                      cudaStream_t s);
void launch_amr_smooth(const AmrGeom& G, int phase, const double* Dc, const double* Df,
                       const double* bc, const double* bf, double* xc, double* xf,
                       cudaStream_t s);
int launch_amr_resid(const AmrGeom& G, const double* Dc, const double* Df, const double* bc,
                     const double* bf, const double* xc, const double* xf, double* rc, double* rf,
                     double* partials, int nblocks, cudaStream_t s);
void launch_amr_average(const AmrGeom& G, const double* vf, double* vc, cudaStream_t s);
void launch_amr_correct(const AmrGeom& G, const double* e, double* xc, double* xf,
                        cudaStream_t s);

}  // namespace fld
