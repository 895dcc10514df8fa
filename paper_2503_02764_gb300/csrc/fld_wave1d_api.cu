// Host side of the one-dimensional radiation-MHD wave step (include/fld.h): three SSP
// Runge-Kutta stages of the hyperbolic update with the explicit coupling terms, then the
// FLD substep of a 1D handle, then the exchange's energy fed back to the gas.
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <new>
#include <vector>

#include "fld_wave1d.cuh"

using namespace fld;

struct fld_wave1d {
    fld_wave1d_params p;
    Wave1dDev dev;
    fld_handle* h = nullptr;
    std::vector<void*> allocs;
    double *A = nullptr, *B = nullptr, *Fi = nullptr;
    double *rho = nullptr, *vx = nullptr, *T = nullptr, *T0 = nullptr, *E = nullptr;
    double *fr = nullptr, *vfr = nullptr, *pt = nullptr, *ebc = nullptr;
    // ARS3 IMEX stages: explicit right-hand sides, predictor, implicit increments (e, E)
    double *L1 = nullptr, *L2 = nullptr, *L3 = nullptr, *Pp = nullptr, *G2 = nullptr,
           *G3 = nullptr;
    unsigned long long* smax = nullptr;
};

namespace {

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

bool params_ok(const fld_wave1d_params* p) {
    if (!p || p->n < 8 || p->n_driven < 0 || p->n_driven > p->n - 4) return false;
    if (!finite_pos(p->dx) || !(p->gamma > 1) || !std::isfinite(p->gamma) ||
        !finite_pos(p->R_gas) || !std::isfinite(p->Bx) || !finite_pos(p->E_right) ||
        !std::isfinite(p->k) || !std::isfinite(p->omega))
        return false;
    if (!finite_pos(p->consts.c) || !finite_pos(p->consts.a_r)) return false;
    if (p->scheme != 0 && p->scheme != 1) return false;
    if (p->radiation != 0 && p->radiation != 1) return false;
    for (int v = 0; v < 8; ++v)
        if (!std::isfinite(p->W0[v]) || !std::isfinite(p->hat[v])) return false;
    // the driving wave keeps rho, p and E positive
    for (int v : {0, 6, 7})
        if (!(p->W0[v] - std::fabs(p->hat[v]) > 0)) return false;
    return true;
}

void destroy(fld_wave1d* w) {
    if (!w) return;
    for (void* q : w->allocs) cudaFree(q);
    if (w->h) fld_destroy(w->h);
    delete w;
}

bool dal(fld_wave1d* w, double** q, long long n) {
    void* m = nullptr;
    if (cudaMalloc(&m, sizeof(double) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    w->allocs.push_back(m);
    *q = (double*)m;
    return true;
}

fld_consts step_consts(const fld_wave1d* w) {
    fld_consts k = w->p.consts;
    k.gamma = w->p.gamma;
    k.R_gas = w->p.R_gas;
    return k;
}

// one Runge-Kutta stage: Uout = a U0 + b (Uin + dt L(Uin)) at time t_in, driven at t_out
fld_status stage(fld_wave1d* w, const double* U0, const double* Uin, double* Uout, double a,
                 double b, double dt, double t_in, double t_out, cudaStream_t s) {
    const Wave1dDev& P = w->dev;
    const fld_consts k = step_consts(w);
    if (w->p.radiation) {
        launch_w1_prim(P, Uin, w->rho, w->vx, w->T, nullptr, w->E, s);
        fld_status rc = fld_coupling(w->h, &k, &w->p.opacity, w->E, w->rho, w->T, w->ebc, w->vx,
                                     nullptr, w->fr, nullptr, w->vfr, w->pt, s);
        if (rc != FLD_OK) return rc;
    }
    launch_w1_iface(P, Uin, t_in, w->Fi, s);
    launch_w1_stage(P, U0, Uin, Uout, w->Fi, w->fr, w->vfr, w->pt, a, b, dt, t_out, s);
    note_launches(3);
    return cudaGetLastError() == cudaSuccess ? FLD_OK : FLD_ERR_CUDA;
}

// the explicit right-hand side L(Uin) at time t (hyperbolic fluxes with the driven left
// ghosts at t, plus the coupling terms)
fld_status explicit_rhs(fld_wave1d* w, const double* Uin, double t, double* Lout,
                        cudaStream_t s) {
    const Wave1dDev& P = w->dev;
    const fld_consts k = step_consts(w);
    if (w->p.radiation) {
        launch_w1_prim(P, Uin, w->rho, w->vx, w->T, nullptr, w->E, s);
        fld_status rc = fld_coupling(w->h, &k, &w->p.opacity, w->E, w->rho, w->T, w->ebc, w->vx,
                                     nullptr, w->fr, nullptr, w->vfr, w->pt, s);
        if (rc != FLD_OK) return rc;
    }
    launch_w1_iface(P, Uin, t, w->Fi, s);
    launch_w1_rhs(P, w->Fi, w->fr, w->vfr, w->pt, Lout, s);
    note_launches(3);
    return cudaGetLastError() == cudaSuccess ? FLD_OK : FLD_ERR_CUDA;
}

// an implicit stage: Uout = the FLD substep over tau from the predictor Pin (the gas energy
// takes the exchange's change of T_g; driven cells at t_drive), G its increment / tau
fld_status implicit_stage(fld_wave1d* w, const double* Pin, double* Uout, double* G, double tau,
                          double t_drive, fld_stats* stats, cudaStream_t s) {
    const long long n = w->p.n;
    if (cudaMemcpyAsync(Uout, Pin, sizeof(double) * 8 * n, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return FLD_ERR_CUDA;
    if (!w->p.radiation)   // no implicit terms: the stage value is the predictor
        return cudaMemsetAsync(G, 0, sizeof(double) * 2 * n, s) == cudaSuccess ? FLD_OK
                                                                               : FLD_ERR_CUDA;
    launch_w1_prim(w->dev, Uout, w->rho, w->vx, w->T, w->T0, w->E, s);
    note_launches(1);
    const fld_consts k = step_consts(w);
    const fld_status rc = fld_step(w->h, &k, &w->p.opacity, tau, w->rho, w->T, w->E, w->ebc,
                                   stats, s);
    if (rc != FLD_OK && rc != FLD_ERR_NOT_CONVERGED) return rc;
    launch_w1_post(w->dev, Uout, w->rho, w->T0, w->T, w->E, t_drive, s);
    launch_w1_incr(w->dev, Uout, Pin, 1.0 / tau, G, s);
    note_launches(2);
    return cudaGetLastError() == cudaSuccess ? rc : FLD_ERR_CUDA;
}

// One ARS(2,3,3) step (Ascher, Ruuth and Spiteri 1997; the ARS3 of Sect. 3), gamma =
// (3 + sqrt 3)/6: P1 = U + dt gamma L1; U2 = substep(P1, gamma dt); P2 = U + dt ((gamma - 1)
// L1 + 2 (1 - gamma) L2) + dt (1 - 2 gamma) G2; U3 = substep(P2, gamma dt); U += dt/2 (L2 +
// L3) + dt/2 (G2 + G3), L_s the explicit right-hand side at stage s, G_s the implicit
// increments; predictors and stage values take the driving wave at their stage times.
fld_status step_ars3(fld_wave1d* w, double* U, double t, double dt, fld_stats* stats,
                     cudaStream_t s) {
    const double g = (3.0 + std::sqrt(3.0)) / 6.0;
    const Wave1dDev& P = w->dev;
    fld_status rc = explicit_rhs(w, U, t, w->L1, s);
    if (rc != FLD_OK) return rc;
    launch_w1_comb(P, U, w->L1, nullptr, nullptr, g, 0.0, 0.0, nullptr, nullptr, 0.0, 0.0, dt,
                   w->Pp, t + g * dt, s);
    note_launches(1);
    fld_status rs = implicit_stage(w, w->Pp, w->A, w->G2, g * dt, t + g * dt, stats, s);
    if (rs != FLD_OK && rs != FLD_ERR_NOT_CONVERGED) return rs;
    rc = explicit_rhs(w, w->A, t + g * dt, w->L2, s);
    if (rc != FLD_OK) return rc;
    launch_w1_comb(P, U, w->L1, w->L2, nullptr, g - 1.0, 2.0 * (1.0 - g), 0.0, w->G2, nullptr,
                   1.0 - 2.0 * g, 0.0, dt, w->Pp, t + (1.0 - g) * dt, s);
    note_launches(1);
    const fld_status rs3 = implicit_stage(w, w->Pp, w->B, w->G3, g * dt, t + (1.0 - g) * dt,
                                          stats, s);
    if (rs3 != FLD_OK && rs3 != FLD_ERR_NOT_CONVERGED) return rs3;
    if (rs3 != FLD_OK) rs = rs3;
    rc = explicit_rhs(w, w->B, t + (1.0 - g) * dt, w->L3, s);
    if (rc != FLD_OK) return rc;
    launch_w1_comb(P, U, nullptr, w->L2, w->L3, 0.0, 0.5, 0.5, w->G2, w->G3, 0.5, 0.5, dt, U,
                   t + dt, s);
    note_launches(1);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return FLD_ERR_CUDA;
    return rs;
}

}  // namespace

extern "C" {

fld_status fld_wave1d_create(fld_wave1d** out, const fld_wave1d_params* p) {
    if (!out) return FLD_ERR_ARG;
    *out = nullptr;
    if (!params_ok(p)) return FLD_ERR_ARG;
    fld_wave1d* w = new (std::nothrow) fld_wave1d();
    if (!w) return FLD_ERR_NOMEM;
    w->p = *p;
    Wave1dDev& D = w->dev;
    D.n = p->n;
    D.nd = p->n_driven;
    D.dx = p->dx;
    D.gamma = p->gamma;
    D.Bx = p->Bx;
    D.R_gas = p->R_gas;
    for (int v = 0; v < 8; ++v) {
        D.W0[v] = p->W0[v];
        D.hat[v] = p->hat[v];
    }
    D.k = p->k;
    D.omega = p->omega;
    fld_grid g;
    memset(&g, 0, sizeof(g));
    g.ndim = 1;
    g.n[0] = p->n;
    g.n[1] = g.n[2] = 1;
    g.h[0] = p->dx;
    g.h[1] = g.h[2] = 1.0;
    g.bc_lo[0] = FLD_BC_NEUMANN;
    g.bc_hi[0] = FLD_BC_DIRICHLET;
    fld_status rc = fld_create(&w->h, &g, &p->opts);
    if (rc != FLD_OK) {
        w->h = nullptr;
        destroy(w);
        return rc;
    }
    const long long n = p->n;
    bool ok = dal(w, &w->A, 8 * n) && dal(w, &w->B, 8 * n) && dal(w, &w->Fi, 8 * (n + 1)) &&
              dal(w, &w->rho, n) && dal(w, &w->vx, n) && dal(w, &w->T, n) && dal(w, &w->T0, n) &&
              dal(w, &w->E, n) && dal(w, &w->fr, n) && dal(w, &w->vfr, n) && dal(w, &w->pt, n) &&
              dal(w, &w->ebc, 1);
    if (ok && p->scheme == 1)
        ok = dal(w, &w->L1, 8 * n) && dal(w, &w->L2, 8 * n) && dal(w, &w->L3, 8 * n) &&
             dal(w, &w->Pp, 8 * n) && dal(w, &w->G2, 2 * n) && dal(w, &w->G3, 2 * n);
    double* sm = nullptr;
    ok = ok && dal(w, &sm, 1);
    w->smax = (unsigned long long*)sm;
    if (!ok) {
        destroy(w);
        return FLD_ERR_NOMEM;
    }
    // the coupling sources stay zero without radiation
    if (cudaMemset(w->fr, 0, sizeof(double) * n) != cudaSuccess ||
        cudaMemset(w->vfr, 0, sizeof(double) * n) != cudaSuccess ||
        cudaMemset(w->pt, 0, sizeof(double) * n) != cudaSuccess ||
        cudaMemcpy(w->ebc, &p->E_right, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        destroy(w);
        return FLD_ERR_CUDA;
    }
    *out = w;
    return FLD_OK;
}

fld_status fld_wave1d_destroy(fld_wave1d* w) {
    if (!w) return FLD_ERR_ARG;
    cudaDeviceSynchronize();
    destroy(w);
    return FLD_OK;
}

fld_status fld_wave1d_max_dt(fld_wave1d* w, const double* U, double cfl, double* dt,
                             void* stream) {
    if (!w || !U || !dt || !finite_pos(cfl)) return FLD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(w->smax, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return FLD_ERR_CUDA;
    launch_w1_speed(w->dev, U, w->smax, s);
    note_launches(1);
    unsigned long long bits = 0;
    if (cudaMemcpyAsync(&bits, w->smax, sizeof(bits), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FLD_ERR_CUDA;
    double vmax;
    memcpy(&vmax, &bits, sizeof(vmax));
    if (!finite_pos(vmax)) return FLD_ERR_DOMAIN;
    *dt = cfl * w->p.dx / vmax;
    return FLD_OK;
}

fld_status fld_wave1d_step(fld_wave1d* w, double* U, double t, double dt, fld_stats* stats,
                           void* stream) {
    if (!w || !U || !finite_pos(dt) || !std::isfinite(t)) return FLD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (w->p.scheme == 1) return step_ars3(w, U, t, dt, stats, s);
    // SSP-RK3: U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1));
    //          U3 = 1/3 U + 2/3 (U2 + dt L(U2)), written over U
    fld_status rc = stage(w, U, U, w->A, 0.0, 1.0, dt, t, t + dt, s);
    if (rc == FLD_OK) rc = stage(w, U, w->A, w->B, 0.75, 0.25, dt, t + dt, t + 0.5 * dt, s);
    if (rc == FLD_OK)
        rc = stage(w, U, w->B, U, 1.0 / 3.0, 2.0 / 3.0, dt, t + 0.5 * dt, t + dt, s);
    if (rc != FLD_OK) return rc;
    if (!w->p.radiation) {
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return FLD_ERR_CUDA;
        return FLD_OK;
    }
    // FLD substep on (rho, T_g, E), then e += rho R_gas (T' - T) / (gamma - 1), E = E'
    launch_w1_prim(w->dev, U, w->rho, w->vx, w->T, w->T0, w->E, s);
    note_launches(1);
    const fld_consts k = step_consts(w);
    rc = fld_step(w->h, &k, &w->p.opacity, dt, w->rho, w->T, w->E, w->ebc, stats, s);
    if (rc != FLD_OK && rc != FLD_ERR_NOT_CONVERGED) return rc;
    launch_w1_post(w->dev, U, w->rho, w->T0, w->T, w->E, t + dt, s);
    note_launches(1);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return FLD_ERR_CUDA;
    return rc;
}

}  // extern "C"
