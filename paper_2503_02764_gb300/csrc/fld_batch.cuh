// Batched substep: per-problem descriptors and the persistent kernel's launcher.
#pragma once
#include "fld_internal.cuh"

namespace fld {

constexpr int BMAXL = 16;   // multigrid levels per batched problem

// Device-resident descriptor of one batched problem.
struct BProb {
    Lvl lv[BMAXL];          // level geometry (level 0 = the problem's grid)
    long long o32[BMAXL];   // offset (floats) of level l's FP32 arrays x, b, K, t in the
                            // problem's FP32 workspace (x at o32, b at +n, K +2n, t +3n)
    double kdown[BMAXL];    // K_{l+1} = mean(K_l children) * kdown[l]
    int nlev;
    double h[3];            // cell sizes (x, y, z)
    long long cell_off;     // first cell of the problem in the concatenated fields
    long long ebc_off;      // first Dirichlet face value in the concatenated faces (-1: none)
    long long bc_off[6];    // Dirichlet face blocks within the problem's faces (-1: none)
    long long ws_d;         // offset (doubles) of the problem's FP64 workspace: D, then
                            // the FP64 refinement's x, b and K (4 n doubles)
    long long ws_f;         // offset (floats) of the problem's FP32 workspace
};

// Per-call data of one problem (uploaded each step).
struct BDyn {
    double dt;              // time step
    Opacity op;             // opacity law
};

struct BatchParams {
    double c, a_r, cv;      // speed of light, radiation constant, R_gas/(gamma - 1)
    double tol;
    int max_cycles, nu1, nu2, coarse_sweeps, limiter, inner;
    int fp64;               // 1: FP64 refinement, limiter and exchange; 0: double-FP32
};

struct BatchStat {
    int cycles;
    double rel_resid;       // final relative residual (-1 on a domain error)
    double rel_resid0;      // before the first cycle
};

int batch_threads_supported(int nt);
int batch_cluster_supported(int cs);
// groups (clusters of cs blocks of nt threads) that can be resident at once
int batch_max_groups(int nt, int cs);
void launch_batch_step(int nt, int cs, int ngroups, const BProb* probs, const BDyn* dyn,
                       const int* order, int nprob, int* queue, const BatchParams& prm,
                       const double* rho, double* T, double* E, const double* Ebc, double* wsd,
                       float* wsf, BatchStat* stats, unsigned* err, cudaStream_t s);

}  // namespace fld
