// The ARS3 IMEX Runge-Kutta scheme the paper combines its explicit and implicit terms with
// (Sect. 3): the ARS(2,3,3) tableaux of Ascher, Ruuth and Spiteri (1997, "Implicit-explicit
// Runge-Kutta methods for time-dependent partial differential equations", Sect. 2.7), and
// the implicit solve of one of its stages around the substep (include/fld.h,
// fld_ars3_tableau, fld_ars3_stage).
#include <cmath>
#include <cstring>

#include "fld_internal.cuh"

using namespace fld;

namespace {

// F_E = (E - E_pred) / (a dt), F_e = rho c_v (T - T_pred) / (a dt); the predictors arrive in
// F_E and F_e
__global__ void k_stage_increments(long long n, double inv_adt, double cv,
                                   const double* __restrict__ rho, const double* __restrict__ T,
                                   const double* __restrict__ E, double* __restrict__ FE,
                                   double* __restrict__ Fe) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        if (FE) FE[p] = (E[p] - FE[p]) * inv_adt;
        if (Fe) Fe[p] = rho[p] * cv * (T[p] - Fe[p]) * inv_adt;
    }
}

double ars3_gamma() { return (3.0 + std::sqrt(3.0)) / 6.0; }

}  // namespace

extern "C" {

void fld_ars3_tableau(double a_ex[9], double a_im[9], double b[3], double c[3]) {
    const double g = ars3_gamma();
    const double ex[9] = {0.0, 0.0, 0.0, g, 0.0, 0.0, g - 1.0, 2.0 * (1.0 - g), 0.0};
    const double im[9] = {0.0, 0.0, 0.0, 0.0, g, 0.0, 0.0, 1.0 - 2.0 * g, g};
    const double bb[3] = {0.0, 0.5, 0.5};
    const double cc[3] = {0.0, g, 1.0 - g};
    if (a_ex) memcpy(a_ex, ex, sizeof(ex));
    if (a_im) memcpy(a_im, im, sizeof(im));
    if (b) memcpy(b, bb, sizeof(bb));
    if (c) memcpy(c, cc, sizeof(cc));
}

fld_status fld_ars3_stage(fld_handle* h, const fld_consts* k, const fld_opacity* op, double dt,
                          int stage, const double* rho, double* T, double* E, const double* E_bc,
                          double* F_E, double* F_e, fld_stats* stats, void* stream) {
    if (!h || !k || !rho || !T || !E || !(dt > 0) || !std::isfinite(dt) ||
        (stage != 1 && stage != 2))
        return FLD_ERR_ARG;
    const long long n = fld_handle_cells(h);
    cudaStream_t s = (cudaStream_t)stream;
    // the implicit stage: the substep over a_ss dt from the predictor
    const double adt = ars3_gamma() * dt;
    if (F_E && cudaMemcpyAsync(F_E, E, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return FLD_ERR_CUDA;
    if (F_e && cudaMemcpyAsync(F_e, T, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return FLD_ERR_CUDA;
    const fld_status rs = fld_step(h, k, op, adt, rho, T, E, E_bc, stats, stream);
    if (rs != FLD_OK && rs != FLD_ERR_NOT_CONVERGED) return rs;
    if (F_E || F_e) {
        const long long nb = std::min<long long>((n + 255) / 256, (long long)num_sms() * 32);
        k_stage_increments<<<(int)nb, 256, 0, s>>>(n, 1.0 / adt, k->R_gas / (k->gamma - 1.0), rho,
                                                   T, E, F_E, F_e);
        note_launches(1);
        if (cudaGetLastError() != cudaSuccess) return FLD_ERR_CUDA;
    }
    return rs;
}

}  // extern "C"
