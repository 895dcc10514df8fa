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

}  // namespace fld
