// Device parameters and launchers of the one-dimensional radiation-MHD wave step.
#pragma once

#include <algorithm>

#include "fld_internal.cuh"

namespace fld {

struct Wave1dDev {
    int n, nd;                  // cells, driven cells at the left end
    double dx, gamma, Bx, R_gas;
    double W0[8], hat[8];       // driving wave W0 + hat sin(k x - omega t), primitive
    double k, omega;
};

void launch_w1_prim(const Wave1dDev& P, const double* U, double* rho, double* vx, double* T,
                    double* T0, double* E, cudaStream_t s);
void launch_w1_iface(const Wave1dDev& P, const double* U, double t, double* Fi, cudaStream_t s);
void launch_w1_stage(const Wave1dDev& P, const double* U0, const double* Uin, double* Uout,
                     const double* Fi, const double* fr, const double* vfr, const double* pt,
                     double a, double b, double dt, double t_stage, cudaStream_t s);
void launch_w1_post(const Wave1dDev& P, double* U, const double* rho, const double* T0,
                    const double* T, const double* E, double t, cudaStream_t s);
void launch_w1_speed(const Wave1dDev& P, const double* U, unsigned long long* out,
                     cudaStream_t s);
// the IMEX (ARS3) step's pieces: explicit right-hand side, stage combination, implicit
// increment of a stage
void launch_w1_rhs(const Wave1dDev& P, const double* Fi, const double* fr, const double* vfr,
                   const double* pt, double* Lout, cudaStream_t s);
void launch_w1_comb(const Wave1dDev& P, const double* U0, const double* L1, const double* L2,
                    const double* L3, double c1, double c2, double c3, const double* G2,
                    const double* G3, double d2, double d3, double dt, double* Uout,
                    double t_stage, cudaStream_t s);
void launch_w1_incr(const Wave1dDev& P, const double* Ua, const double* Ub, double inv_tau,
                    double* G, cudaStream_t s);

}  // namespace fld
