/*
 * fld.h - C ABI of the GB300 flux-limited-diffusion (FLD) radiation substep.
 *
 * The substep (paper: arXiv 2503.02764, Sect. 2 and Sect. 3) advances the
 * radiation energy density E and the gas temperature T of a Cartesian block by
 * one time step dt:
 *
 *   1. limiter  (Eqs. fld_R, fld_lambda, fld_F; gradient stencil of Sect. 3)
 *        R = |grad E| / (kappa rho E),  lambda = (2 + R)/(6 + 3R + R^2),
 *        D = c lambda / (kappa rho), cell-centred, grad E by the 4th-order
 *        5-point central difference per axis;
 *   2. diffuse  (the div F term of Eq. mhd_r_e with F = -D grad E, treated
 *        implicitly as Sect. 3 describes): backward Euler
 *        (I - dt div D grad) E^{n+1} = E^n on cell-centred finite volumes,
 *        face D = mean of the two cell values (arithmetic, or harmonic as an
 *        option), solved by geometric multigrid V-cycles (1D grids: a direct
 *        tridiagonal solve) to a relative residual ||b - A x||_2 / ||b||_2 <= tol;
 *   3. exchange (Eqs. heating, qdot; implicit quartic of Sect. 3): backward
 *        Euler on de/dt = +qdot, dE/dt = -qdot, qdot = c kappa rho (E - a_r T^4),
 *        e = rho R_gas T / (gamma - 1) (Eqs. energy_density, ideal_gas_law).
 *
 * Around the substep: its explicit coupling terms (fld_coupling), a batched
 * substep over many independent grids in one launch (fld_step_batched), an
 * allocation-free solve (fld_diffuse_static), a 1D radiation-MHD step that
 * runs the substep inside a hyperbolic update (fld_wave1d_*), the implicit stage
 * of the ARS3 IMEX scheme (fld_ars3_*), the diffusion solve on a coarse block
 * with a refined box (fld_amr_*), and the bounds flags of the debug build
 * (fld_debug_flags).
 *
 * Layout: every field is a contiguous float64 array of n[0]*n[1]*n[2] cells,
 * x fastest: index = (k * n[1] + j) * n[0] + i. Absent axes have n = 1.
 *
 * Memory: field pointers are DEVICE pointers owned by the caller. The handle
 * owns its workspace (the multigrid level pyramid, scratch and reduction
 * buffers), allocated once in fld_create and freed in fld_destroy; only the
 * create calls (fld_create, fld_batch_create, fld_wave1d_create, fld_amr_create)
 * allocate device memory.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream). Work is enqueued on it. fld_diffuse and fld_step read the residual
 * norm back once per V-cycle, so they return only after the solve on `stream`
 * has finished; fld_limiter and fld_exchange return at once (asynchronous).
 *
 * Errors: every call returns an fld_status and never throws. Argument errors
 * are detected on the host before any work is enqueued. Device-side errors
 * (a cell with non-positive or non-finite E, rho, T or kappa) set a flag in the
 * handle; calls that synchronise (fld_diffuse, fld_step) report it, and
 * fld_get_status synchronises `stream` and reports/clears it for the others.
 * A cell that fails the domain check is left unchanged.
 */
#ifndef FLD_H
#define FLD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FLD_OK = 0,
    FLD_ERR_ARG = 1,            /* invalid argument: null pointer, size, enum or option */
    FLD_ERR_DOMAIN = 2,         /* a cell had E, rho, T or kappa <= 0 or non-finite     */
    FLD_ERR_NOT_CONVERGED = 3,  /* max_cycles V-cycles did not reach tol; E holds the
                                   last iterate                                        */
    FLD_ERR_TIMEOUT = 4,        /* reserved for a bounded device-side wait; no kernel of
                                   this library waits on another block, so none returns it */
    FLD_ERR_CUDA = 5,           /* a CUDA runtime call failed                          */
    FLD_ERR_NOMEM = 6           /* device allocation failed in a create call           */
} fld_status;

/* boundary kinds, per axis side */
enum { FLD_BC_PERIODIC = 0, FLD_BC_NEUMANN = 1, FLD_BC_DIRICHLET = 2 };
/* opacity laws: kappa = kappa0 (CONST), kappa0 rho^a_rho T^a_T (POWER), or kappa0 times
   10 to a bilinear interpolant of a table of log10 kappa over (log10 rho, log10 T) (TABLE;
   the paper uses constant opacities and names tables as the next step, Sect. 5) */
enum { FLD_OPACITY_CONST = 0, FLD_OPACITY_POWER = 1, FLD_OPACITY_TABLE = 2 };
/* limiter: Levermore-Pomraning (Eq. fld_lambda), the diffusion limit lambda = 1/3, or
   Minerbo's limiter (named in Sect. 2, published closed form) */
enum { FLD_LIMITER_LP = 0, FLD_LIMITER_DIFFUSION = 1, FLD_LIMITER_MINERBO = 2 };
/* precision mode of a handle (solve, limiter and exchange):
   FP64      FP64 V-cycles; FP64 limiter and exchange.
   MIXED     FP32 V-cycles (smoothing, restriction, prolongation) inside iterative
             refinement whose residual and correction are FP64; the coarsest-level solve
             is FP64 arithmetic (in every mode). Limiter and exchange are FP64 as in FP64
             mode.
   MIXED_DF  as MIXED, but the refinement's iterate, right-hand side, coefficients,
             residual and correction are carried as double-FP32 pairs (48-bit significand,
             error-free transformations) between reading E and writing it back, and the
             limiter (gradient, R, lambda, D) and the exchange (coefficients, the Newton
             step that polishes the FP32 root, E') run in the same double-FP32 arithmetic:
             FP64-grade accuracy (relative error ~1e-14) at FP32 instruction cost, since
             FP64 issues at a small fraction of the FP32 rate on this GPU. Cells whose
             values leave the FP32 exponent window take the FP64 routines, and the solve's
             values must stay within that window after its power-of-two scaling (|S E|
             well inside 1e-30..1e30).
   In FP64 and MIXED the FP64 limiter and exchange seed their reciprocals, square roots
   and the quartic's root in FP32 and refine them by FP64 Newton steps. */
enum { FLD_PREC_FP64 = 0, FLD_PREC_MIXED = 1, FLD_PREC_MIXED_DF = 2 };

/* Physical constants in the caller's units: speed of light c, radiation
   constant a_r, adiabatic index gamma and R_gas = k_B / (mu m_p). */
typedef struct { double c, a_r, gamma, R_gas; } fld_consts;

/* Uniform Cartesian block. ndim in {1,2,3}; n[d] >= 2 for d < ndim and n[d] = 1
   otherwise; h[d] > 0 the cell size along axis d; bc_lo/bc_hi the boundary kind
   of each side (periodic must be set on both sides of an axis). A Dirichlet
   side takes face values from the E_bc array (see fld_limiter). */
typedef struct {
    int ndim;
    int n[3];
    double h[3];
    int bc_lo[3], bc_hi[3];
} fld_grid;

/* Opacity law, read on the host at each call (kappa0 > 0 and finite in every kind).
   POWER uses a_rho and a_T. TABLE uses the table fields:
     table     device array of n_rho * n_T float64, caller-owned, read by the call's
               kernels (keep it alive and unchanged until they finish): log10 kappa at
               log10 rho = log_rho0 + i dlog_rho, log10 T = log_T0 + j dlog_T stored at
               [j * n_rho + i] (rho fastest);
     n_rho, n_T >= 2 with n_rho * n_T < 2^31; dlog_rho, dlog_T > 0, all four finite.
   A cell's (log10 rho, log10 T) is clamped to the table's range (outside it the edge
   values hold) and log10 kappa interpolated bilinearly between the four nodes around
   it, in FP64. TABLE is taken by fld_limiter, fld_coupling, fld_exchange and fld_step
   (which then read T); fld_step_batched returns FLD_ERR_ARG for it. The other kinds
   ignore the table fields (zero them). */
typedef struct {
    int kind;
    double kappa0, a_rho, a_T;
    const double* table;
    int n_rho, n_T;
    double log_rho0, dlog_rho, log_T0, dlog_T;
} fld_opacity;

/* Solver options; fld_default_opts fills sensible values. */
typedef struct {
    int precision;      /* FLD_PREC_FP64, FLD_PREC_MIXED or FLD_PREC_MIXED_DF        */
    double tol;         /* stop when ||b - A x||_2 <= tol ||b||_2                    */
    int max_cycles;     /* V-cycle limit (outer refinement steps in MIXED)          */
    int nu1, nu2;       /* red-black Gauss-Seidel sweeps before / after coarse corr. */
    int coarse_sweeps;  /* red-black sweeps of the coarsest-level solve             */
    int limiter;        /* FLD_LIMITER_LP, _DIFFUSION (lambda = 1/3) or _MINERBO    */
    int block;          /* threads per block of the row-mapped kernels (0 = default) */
    int smoother;       /* 0: in-place red and black half sweeps (levels with no odd
                           periodic extent; others as 1); 1: two out-of-place half
                           sweeps; 2: one z-marching pass per sweep (3D FP32 levels
                           with nx a multiple of 4, nx >= 16, even periodic extents;
                           others as 0). The levels from 8^3 cells down run in one
                           single-block launch whatever the smoother.                  */
    int graph;          /* single grid: replay the FP32 V-cycle from a CUDA graph
                           captured on first use; batched step: capture the step on
                           the first call with given field pointers and replay it       */
    int cluster;        /* batched step: blocks per problem (1, 2, 4 or 8, a thread-block
                           cluster when > 1); 0 = chosen from the largest problem      */
    int inner;          /* MIXED/MIXED_DF: FP32 V-cycles per refinement step (the later
                           ones continue from the previous correction); 0 means 1      */
    int direct1d;       /* 1D grids: 1 solves the tridiagonal system directly (parallel
                           cyclic reduction in FP64, a dozen launches; stats report one
                           cycle), 0 runs V-cycles as in 2D and 3D                      */
    int diag;           /* diagnostics filled into fld_stats by fld_diffuse and fld_step
                           when a stats pointer is given: FLD_DIAG_ENERGY adds the total
                           energy before and after (two reductions), FLD_DIAG_TIMES the
                           per-phase times (CUDA events on the stream); 0 = none        */
    int face_mean;      /* face coefficient w_f of the diffusion operator from the two
                           cell values D_i, D_j: FLD_FACE_ARITH (D_i + D_j)/2, the
                           default, or FLD_FACE_HARM 2 D_i D_j/(D_i + D_j), which keeps
                           the flux through layers of unequal D that of resistances in
                           series. HARM is taken by FP64 and MIXED handles (their fine
                           levels then use the generic half-sweep smoother and residual
                           kernels, not the z-marching ones), not by MIXED_DF, the
                           batched step or the composite grid (FLD_ERR_ARG)            */
    int prolong;        /* V-cycle prolongation of the coarse correction:
                           FLD_PROLONG_LINEAR (bi/trilinear, cell-centred: 3/4 parent +
                           1/4 neighbour per coarsened axis, walls mirrored), the
                           default, or FLD_PROLONG_CONSTANT (the parent's value). The
                           choice changes the convergence rate, not the solution.
                           CONSTANT runs the generic prolongation kernel; the batched
                           step takes LINEAR only                                      */
    int limiter_df;     /* 1: the limiter (fld_limiter, and the limiter of fld_step) runs
                           in double-FP32 as in MIXED_DF (gradient from FP32 pairs of E,
                           R, lambda, D; relative error ~1e-14) whatever the precision
                           mode, the solve and the exchange keeping theirs; 0 (default):
                           the limiter of the precision mode                           */
    int resid_update;   /* MIXED on 3D grids with the arithmetic face mean: 1 (default)
                           forms the first refinement residual after the FP32 solve of
                           E^n in FP64 and the later ones as r - A e, A e evaluated in FP32
                           on the level's FP32 coefficients (x + e stays FP64), with a
                           per-cell bound on that update's rounding accumulated beside it;
                           the solve stops when ||r|| plus the accumulated bound is below
                           tol ||b|| (rel_resid reports that sum, an upper bound on the
                           true relative residual), and takes a full FP64 residual
                           whenever the bound alone passes tol/2 or the recursive residual
                           is below tol while the sum is not. 0: every refinement residual
                           in FP64. Ignored by the other modes and grids                */
    int truncate;       /* V-cycle depth from the operator (every precision, 2D and 3D):
                           1 (default) ends the V-cycle at the first level below the finest
                           on which at most 4 red-black sweeps from zero reduce the error to
                           1e-2, and solves that level by them. The bound comes from the
                           call's largest K = dt D / h_x^2: on level l the off-diagonal row
                           sums are at most s_l = 2 K_l sum_d w_d (K_l the largest K rescaled
                           to the level's spacing), a sweep contracts by about
                           (s_l/(1 + s_l))^2. Diffusion steps of a few explicit time steps
                           then skip the coarse levels whose operator is close to the
                           identity. 0: every level down to the coarsest (the single-block
                           tail and its dense solve). The batched step keeps every level */
} fld_opts;

enum { FLD_DIAG_ENERGY = 1, FLD_DIAG_TIMES = 2 };
enum { FLD_FACE_ARITH = 0, FLD_FACE_HARM = 1 };
enum { FLD_PROLONG_LINEAR = 0, FLD_PROLONG_CONSTANT = 1 };

/* Per-solve statistics (optional output). resid_hist[i] is the relative
   residual after i cycles (resid_hist[0] before the first), for i < 64. levels: the
   levels the solve's V-cycles used (fewer than the pyramid's with the truncate option;
   1 for a direct 1D solve).
   With FLD_DIAG_ENERGY in the handle's diag option: energy_before / energy_after are the
   sums over the block of the energy per cell times the cell volume (prod h[d], d < ndim),
   before the call and after it: E for fld_diffuse, rho c_v T + E (c_v = R_gas/(gamma-1),
   the gas internal energy of Eq. energy_density plus the radiation energy) for fld_step.
   With periodic and Neumann walls the two agree to the solve's tolerance (the discrete
   diffusion operator and the exchange conserve energy); Dirichlet walls let energy in or
   out. With FLD_DIAG_TIMES: t_ms = {limiter, diffusion solve, exchange, whole call} in
   milliseconds between CUDA events on the call's stream (fld_diffuse fills the solve and
   the whole call). Unrequested fields are zero. */
typedef struct {
    int cycles;
    double rel_resid;
    double resid_hist[64];
    int levels;
    double energy_before, energy_after;
    double t_ms[4];
} fld_stats;

typedef struct fld_handle fld_handle;

/* Fill *o with defaults: FP64, tol 1e-10, 50 cycles, V(2,2), 32 coarse sweeps,
   Levermore-Pomraning limiter, direct 1D solves. */
void fld_default_opts(fld_opts* o);

/* Create a handle bound to grid *g with options *o; allocates the workspace on
   the current CUDA device. Returns FLD_ERR_ARG for an invalid grid or options,
   FLD_ERR_NOMEM if an allocation fails (nothing is leaked). */
fld_status fld_create(fld_handle** h, const fld_grid* g, const fld_opts* o);

/* Free the handle and its workspace (NULL is accepted). */
fld_status fld_destroy(fld_handle* h);

/* Bounds flags of the debug build. The library compiled with FLD_DEBUG (the build step's
   libfld_gb300_debug.so) checks the computed indices of its stencil, gradient, residual,
   sweep and transfer kernels: an index outside its array raises a flag in a device word
   and is replaced by 0 (the kernel carries on; nothing traps). Returns the flags raised
   since the last call (0: none) and clears them, synchronising the device; -1 from the
   normal build, which carries no checks. */
int fld_debug_flags(void);

/* Replace the handle's options (the grid and workspace are kept). */
fld_status fld_set_opts(fld_handle* h, const fld_opts* o);

/* Limiter (Eqs. fld_R, fld_lambda, fld_F; Sect. 3 gradient).
   In:  E, rho, T (device, ncell float64 each; T is only read by a POWER or TABLE
        opacity and may be NULL for a CONST one),
        E_bc (device float64, may be NULL when no side is Dirichlet): the
        Dirichlet face values packed side after side in the order x-lo, x-hi,
        y-lo, y-hi, z-lo, z-hi (Dirichlet sides only), each face row-major over
        the two other axes (the lower axis fastest).
   Out: D (device, ncell float64) the cell diffusion coefficient c lambda/(kappa rho);
        lambda (device, ncell float64, may be NULL) the limiter value.
   Ghost values for the gradient: periodic wrap; Neumann even mirror
   (E_-1 = E_0, E_-2 = E_1); Dirichlet odd reflection (E_-k = 2 E_b - E_{k-1}).
   |grad E| = 0 gives lambda = 1/3. FP64 arithmetic, or double-FP32 on a MIXED_DF handle
   (relative error ~1e-14 in D). Asynchronous. */
fld_status fld_limiter(fld_handle* h, const fld_consts* k, const fld_opacity* op,
                       const double* E, const double* rho, const double* T,
                       const double* E_bc, double* D, double* lambda, void* stream);

/* Explicit coupling terms of the limiter pass (Sect. 3, which adds them explicitly):
   from the same gradient, R and lambda as fld_limiter (the handle's limiter option),
     F   = -D grad E = -(c lambda/(kappa rho)) grad E             (Eq. fld_F),
     f_r = rho kappa F / c = -lambda grad E                         (Eq. rad_force),
     f   = lambda + lambda^2 R^2                                    (Eq. fld_f),
   and, given the velocity v, the work of the radiation force v . f_r and the photon
   tiring term P : grad v = sum_ij P_ij d_j v_i with P = E f_tensor (Eq. fld_P),
   f_tensor = ((1 - f) I + (3f - 1) n n)/2, n = grad E/|grad E| (Eq.
   fld_Eddington_tensor; n n drops out where grad E = 0, since f = 1/3 there). grad v
   uses the same 5-point stencil; velocity ghosts wrap on periodic axes and mirror evenly
   (zero gradient) at walls.
   In:  E, rho, T, E_bc as for fld_limiter; v (device float64, ndim * ncell, component d
        at v + d * ncell, may be NULL).
   Out (device float64, each may be NULL): F and fr (ndim * ncell, component-major like v),
        f_edd (ncell), vfr and ptire (ncell; need v).
   FLD_ERR_ARG for a missing required input; invalid cells set the domain flag and keep
   their outputs unchanged. FP64 arithmetic. Asynchronous. */
fld_status fld_coupling(fld_handle* h, const fld_consts* k, const fld_opacity* op,
                        const double* E, const double* rho, const double* T,
                        const double* E_bc, const double* v, double* F, double* fr,
                        double* f_edd, double* vfr, double* ptire, void* stream);

/* Backward-Euler diffusion step: solves A E^{n+1} = E^n + g in place,
     (A x)_i = x_i + sum_faces (dt/h_d^2) w_f (x_i - x_j),  w_f = (D_i + D_j)/2
   (2 D_i D_j/(D_i + D_j) with the face_mean option FLD_FACE_HARM), a Dirichlet face adding (dt/h_d^2) 2 D_i (x_i - E_b) (g holds the E_b part),
   a Neumann face nothing.
   In:  dt > 0; D (device, ncell float64, > 0); E_bc as for fld_limiter.
   In/out: E (device, ncell float64): E^n on entry, E^{n+1} on return (the last
   iterate on FLD_ERR_NOT_CONVERGED).
   stats may be NULL. Returns after the solve has finished on `stream`. */
fld_status fld_diffuse(fld_handle* h, double dt, const double* D, const double* E_bc,
                       double* E, fld_stats* stats, void* stream);

/* Gas-radiation exchange, cell by cell (Eqs. heating, qdot): with
   chi = dt c kappa rho, c_v = R_gas/(gamma - 1), e = rho c_v T, solves
   rho c_v T' + (chi/(1+chi)) a_r T'^4 = e + chi E/(1+chi) for the unique positive
   T' and sets E' = (E + chi a_r T'^4)/(1 + chi). kappa = kappa(rho, T) on entry.
   The root is found by Newton iterations in FP32 on a scaled form of the quartic, then
   polished by one Newton step in FP64 (double-FP32 on a MIXED_DF handle).
   In: rho (device float64). In/out: T, E (device float64). Asynchronous. */
fld_status fld_exchange(fld_handle* h, const fld_consts* k, const fld_opacity* op, double dt,
                        const double* rho, double* T, double* E, void* stream);

/* The whole substep: limiter -> diffuse -> exchange, the opacity frozen at
   (rho, T^n) for all three. The handle's scratch holds D. Returns after the
   step has finished on `stream`. A solve that stops at max_cycles still
   completes the substep from its last iterate and the call returns
   FLD_ERR_NOT_CONVERGED; any other error returns before the exchange. */
fld_status fld_step(fld_handle* h, const fld_consts* k, const fld_opacity* op, double dt,
                    const double* rho, double* T, double* E, const double* E_bc,
                    fld_stats* stats, void* stream);

/* ---------------------------------------------------------------- batched substep
   Many independent problems of uneven sizes advanced by one substep each in ONE
   persistent kernel launch (512 uneven 2D problems is the intended scale):
   every block takes the next problem from a queue ordered by decreasing cell count
   and runs limiter -> multigrid solve -> exchange on it, so no block ever waits on
   another. The solve runs FP32 V-cycles inside iterative refinement whose residual,
   correction, limiter and exchange are FP64 (o->precision FLD_PREC_MIXED, or
   FLD_PREC_FP64, which keeps the FP32 V-cycles) or double-FP32 (FLD_PREC_MIXED_DF);
   o->block (256, 512 or 1024; 0 = 512) is the block size and o->cluster the number of blocks that share one problem
   (a thread-block cluster synchronised by the hardware cluster barrier);
   o->nu1/nu2/coarse_sweeps/tol/max_cycles/limiter apply.
   Layout: the fields of all problems are concatenated in problem order (problem p
   starts at the sum of the cell counts of problems 0..p-1), each in the layout of
   fld_limiter; Dirichlet faces likewise concatenated problem after problem. */
typedef struct fld_batch fld_batch;

typedef struct {
    int cycles;             /* refinement cycles used                               */
    double rel_resid;       /* final ||b - A x|| / ||b|| (-1 after a domain error)   */
    double rel_resid0;      /* the same before the first cycle                      */
} fld_batch_stat;

/* grids: host array of nprob grids (each as for fld_create, at most 2^27 cells).
   Allocates the per-problem descriptors and workspace once. */
fld_status fld_batch_create(fld_batch** b, int nprob, const fld_grid* grids, const fld_opts* o);
fld_status fld_batch_destroy(fld_batch* b);
fld_status fld_batch_set_opts(fld_batch* b, const fld_opts* o);
/* Total number of cells of the batch (length of the concatenated fields). */
long long fld_batch_cells(const fld_batch* b);

/* One substep of every problem (Sect. 2/3 as for fld_step): k shared; ops[p] and dt[p]
   (host arrays) per problem; rho, T, E, E_bc device arrays as described above.
   With o->graph the launch sequence is captured into a CUDA graph on the first call
   with these field pointers and replayed by later calls. stats (host, nprob entries)
   may be NULL. Returns after the step has finished on `stream`: FLD_ERR_DOMAIN if a
   problem held an invalid value (it is left unchanged), FLD_ERR_NOT_CONVERGED if a
   problem missed tol within max_cycles (its E and T hold the last iterate's step). */
fld_status fld_step_batched(fld_batch* b, const fld_consts* k, const fld_opacity* ops,
                            const double* dt, const double* rho, double* T, double* E,
                            const double* E_bc, fld_batch_stat* stats, void* stream);

/* Synchronise `stream` and return (and clear) any device-side error flag. */
fld_status fld_get_status(fld_handle* h, void* stream);

/* Number of multigrid levels of the handle's pyramid. */
int fld_num_levels(const fld_handle* h);

/* ---------------------------------------------------------------- profiling
   While profiling is on, every kernel the handle launches is bracketed by a pair of
   CUDA events on its stream (up to `capacity` launches; later ones are counted but
   not timed). fld_prof_read synchronises the device, fills up to `cap` entries, one
   per (kernel, level), and returns the number of entries; enabling again resets
   the record. The events are created in fld_prof_enable, never in the timed path. */
typedef struct {
    char name[24];          /* kernel family, e.g. "smooth32", "resid64", "exchange" */
    int level;              /* multigrid level (0 = the caller's grid)              */
    long long launches;     /* launches timed                                       */
    long long cells;        /* cells processed over those launches                  */
    double ms;              /* summed event time                                    */
} fld_prof_entry;

fld_status fld_prof_enable(fld_handle* h, int on, int capacity);
int fld_prof_read(fld_handle* h, fld_prof_entry* out, int cap);

/* Number of kernels launched by this library in this process so far. */
long long fld_launch_count(void);

/* ---------------------------------------------------------------- no-allocation solve
   fld_diffuse_static: the same backward-Euler multigrid solve as fld_diffuse, for callers
   that cannot allocate device memory themselves or through a handle: host codes that hand
   every byte of the GPU to their own memory pool at start-up, so that cudaMalloc would
   fail, or real-time loops that must never enter the CUDA allocator. The paper has no
   counterpart; this is a property of the library, not of the method.
   The workspace lives in one 16 MiB array defined in the library as a file-scope
   __device__ variable: every GPU on which the library is loaded keeps those 16 MiB until
   the process exits, and no call allocates or frees device or pinned host memory. Grids
   of up to 131072 cells are accepted in any precision mode; larger grids return
   FLD_ERR_ARG with a message on stderr.
   Arguments and results are those of fld_diffuse plus the grid and options a handle would
   hold (o may be NULL for the defaults; its graph option is ignored, every kernel is
   launched directly); D, E_bc and E are caller-owned device arrays as above. The first
   call on a device looks up the array's device address (cudaGetSymbolAddress) with that
   device current; make that first call before any stream capture. The call reads the
   residual back to the host once per V-cycle, each time synchronising `stream`, and
   synchronises `stream` once more before it returns: it returns after all of its GPU work
   has finished. Every call reuses the same array, which keeps the previous call's contents
   (the call clears what must start at zero). Two calls in flight on the GPU at once would
   race on the array; a lock held for the whole call, together with that final
   synchronisation, keeps calls from several host threads from overlapping. */
fld_status fld_diffuse_static(const fld_grid* g, const fld_opts* o, double dt, const double* D,
                              const double* E_bc, double* E, fld_stats* stats, void* stream);

/* ---------------------------------------------------------------- 1D RMHD wave step
   One step of the one-dimensional radiation-MHD problem of the paper's linear-wave tests
   (Sect. 4.3) with the scheme of Sect. 3, for the travelling radiation-damped waves:
   With scheme 0 (first-order split):
   1. the hyperbolic terms (left-hand sides of Eqs. mhd_mass, mhd_mom, mhd_energy,
      mhd_mag and the advection term of Eq. mhd_r_e) plus the explicit coupling terms
      (radiation force f_r = -lambda grad E, its work v . f_r, photon tiring P : grad v,
      as fld_coupling computes them) by the three-stage SSP Runge-Kutta scheme of Shu and
      Osher, with HLL interface fluxes (signal speeds v_x -+ the gas fast magnetosonic
      speed) and third-order WENO reconstruction (Jiang-Shu weights, epsilon 1e-6 on
      smoothness indicators divided by the largest square of the stencil's four cells)
      of the primitive variables;
   2. the FLD substep (as fld_step: limiter, backward-Euler diffusion, implicit exchange)
      on (rho, T_g = p / (rho R_gas), E); the exchange's change of T_g is added to the
      total gas energy.
   With scheme 1 the same explicit right-hand side (hyperbolic terms and coupling terms)
   and the same substep (as the implicit operator) are combined by the ARS3 IMEX scheme,
   the paper's (Sect. 3): three explicit evaluations and two substeps over gamma dt per
   step (the stage equations are those of fld_ars3_tableau).
   Units are the caller's; the magnetic field is in Heaviside-Lorentz form (magnetic
   pressure B^2/2) with B_x constant.
   State U: caller-owned device float64 array [8][n] (variable-major): rho, rho v_x,
   rho v_y, rho v_z, B_y, B_z, e (total gas energy: p/(gamma-1) + rho v^2/2 + B^2/2), E.
   Boundaries: the first n_driven cells and the two left ghost cells take the driving
   wave W0 + hat sin(k x - omega t) (primitive variables rho, v_x, v_y, v_z, B_y, B_z, p,
   E; cell centres x = (i + 1/2) dx) at every Runge-Kutta stage and after the substep;
   on the right, zero gradient for every variable and a Dirichlet face value E_right
   for E in the diffusion solve and the gradient; E's gradient takes an even mirror on
   the left. */
typedef struct {
    int n;                      /* cells, >= 8                                          */
    int n_driven;               /* driven cells at the left end, 0 .. n - 4            */
    double dx, gamma, Bx, R_gas;
    fld_consts consts;          /* c, a_r (gamma and R_gas as above)                    */
    fld_opacity opacity;
    double E_right;             /* Dirichlet face value of E on the right, > 0           */
    double W0[8], hat[8];       /* driving wave, primitive variables                    */
    double k, omega;
    fld_opts opts;              /* options of the FLD substep (limiter, precision, tol)  */
    int scheme;                 /* 0: SSP-RK3 then the FLD substep over dt (first-order
                                   split); 1: the ARS3 IMEX scheme (fld_ars3_tableau): the
                                   hyperbolic and coupling terms explicit, the substep as
                                   its two implicit stages over gamma dt                 */
    int radiation;              /* 1: as above; 0: ideal MHD (no coupling terms, no
                                   substep: the scheme's own damping, for reference)       */
} fld_wave1d_params;

typedef struct fld_wave1d fld_wave1d;

/* Allocates the 1D FLD handle and the step's device scratch (about 30 n doubles). */
fld_status fld_wave1d_create(fld_wave1d** w, const fld_wave1d_params* p);
fld_status fld_wave1d_destroy(fld_wave1d* w);
/* cfl dx / max_i (|v_x| + c_f) over the cells of U (device); synchronises `stream`. */
fld_status fld_wave1d_max_dt(fld_wave1d* w, const double* U, double cfl, double* dt,
                             void* stream);
/* Advances U (device, in place) from t to t + dt. Returns after the step has finished on
   `stream`, with fld_step's status (FLD_ERR_NOT_CONVERGED when the diffusion solve
   stopped at max_cycles: the step is still completed; FLD_ERR_DOMAIN when a cell left
   the physical domain: U holds the stage where it happened). stats may be NULL. */
fld_status fld_wave1d_step(fld_wave1d* w, double* U, double t, double dt, fld_stats* stats,
                           void* stream);

/* ---------------------------------------------------------------- IMEX stages
   The paper advances the explicit terms (hyperbolic fluxes, the coupling terms of
   fld_coupling) and the implicit ones (this substep) together with the ARS3 IMEX Runge-
   Kutta scheme (Sect. 3): ARS(2,3,3) of Ascher, Ruuth and Spiteri (1997), with
   gamma = (3 + sqrt 3)/6,
     explicit  A_ex = [[0, 0, 0], [gamma, 0, 0], [gamma - 1, 2 (1 - gamma), 0]],
     implicit  A_im = [[0, 0, 0], [0, gamma, 0], [0, 1 - 2 gamma, gamma]],
     b = [0, 1/2, 1/2] (both), c = [0, gamma, 1 - gamma]  (row-major 3 x 3 arrays).
   For dU/dt = F_ex(U) + F_im(U) the stages are U_1 = U^n and, for s = 1, 2,
     U_{s+1} = P_s + gamma dt F_im(U_{s+1}),
     P_s = U^n + dt sum_{j<=s} A_ex[s][j] F_ex(U_j) + dt sum_{1<=j<=s} A_im[s][j] F_im(U_j),
   then U^{n+1} = U^n + dt sum_j b[j] (F_ex(U_j) + F_im(U_j)). A host code forms F_ex and the
   predictors P_s; fld_ars3_stage makes the implicit solve of stage s: the substep
   (fld_step) over gamma dt from the predictor, F_im being the substep's diffusion and
   exchange. */
void fld_ars3_tableau(double a_ex[9], double a_im[9], double b[3], double c[3]);
/* Stage s (1 or 2) of ARS3 on the handle's grid. In: rho; T, E hold the predictor P_s (gas
   temperature and radiation energy density; device float64). Out: T, E the stage value
   U_{s+1}; F_E, F_e (device float64, ncell, each may be NULL) the implicit increments
   F_im(U_{s+1}) of E and of the gas energy rho c_v T, (U_{s+1} - P_s)/(gamma dt). dt is
   the full step (the substep runs over gamma dt). Returns fld_step's status. */
fld_status fld_ars3_stage(fld_handle* h, const fld_consts* k, const fld_opacity* op, double dt,
                          int stage, const double* rho, double* T, double* E,
                          const double* E_bc, double* F_E, double* F_e, fld_stats* stats,
                          void* stream);

/* ---------------------------------------------------------------- composite grid
   Backward-Euler diffusion (the solve of fld_diffuse) on a block-structured composite grid:
   a coarse block (the fld_grid, cells h[d]) with one box of it refined by 2 in every axis
   (cells h[d]/2), the smallest case of the block-adaptive hierarchy whose implicit div F
   the paper solves with its octree multigrid library (Sect. 3; AMR by Loehner's criterion).
   The unknowns are the coarse cells outside the box and every fine cell; for each, of
   volume V_p,
     (A x)_p = x_p + (dt/V_p) sum_faces a_f (x_p - x_q) + Dirichlet walls at half a cell,
     a_f = (D_p + D_q)/2 * area_f / dist_f,
   dist_f the distance of the two cell centres along the face normal: h between coarse
   cells, h/2 between fine cells, 3h/4 between a fine cell and the coarse cell across the
   box's edge (one coarse face meets 2^(ndim-1) fine faces). Each face flux enters both
   its cells with opposite signs: the step conserves sum V E on periodic and Neumann blocks.
   Along each axis the box lies at least one coarse cell inside the walls or spans the
   axis (the axis's walls then bound the fine cells; a fine Dirichlet face takes the value
   of the coarse face it lies in). Periodic extents of the coarse block must be even.
   The solve: red-black Gauss-Seidel on the composite grid, and the composite residual
   restricted to the whole block (a covered coarse cell takes the mean of its fine cells')
   as the right-hand side of a correction solved by the block's own multigrid (covered
   cells carrying the mean of their fine cells' D), prolonged piecewise constant; repeated
   until ||b - A x||_2 <= tol ||b||_2 over the unknowns (o->tol, o->max_cycles; the other
   options go to the block's solver). FP64 composite arithmetic. */
typedef struct {
    int lo[3], hi[3];       /* the refined box in coarse cell indices (hi exclusive);
                               lo = 0, hi = 1 on absent axes */
} fld_patch;

typedef struct fld_amr fld_amr;

/* Allocates the composite workspace and a handle for the coarse block. FLD_ERR_ARG for an
   invalid grid, options or box (a box touching one wall without spanning the axis, odd
   periodic extents). */
fld_status fld_amr_create(fld_amr** a, const fld_grid* coarse, const fld_patch* patch,
                          const fld_opts* o);
fld_status fld_amr_destroy(fld_amr* a);
/* One step. In: dt > 0; Dc (device, the coarse block's cells, float64, layout of
   fld_limiter) and Df (device, the box's fine cells: 2 (hi - lo) per axis, same layout):
   cell diffusion coefficients (> 0); E_bc: the coarse block's Dirichlet face values as
   for fld_limiter (may be NULL without Dirichlet sides). In/out: Ec, Ef (device, same
   layouts): E^n on entry (covered coarse cells ignored), E^{n+1} on return, covered coarse
   cells set to the mean of their fine cells. stats may be NULL (cycles = two-level
   iterations). Returns after the solve has finished on `stream`. */
fld_status fld_amr_diffuse(fld_amr* a, double dt, const double* Dc, const double* Df,
                           const double* E_bc, double* Ec, double* Ef, fld_stats* stats,
                           void* stream);

/* Static string for a status code. */
const char* fld_strerror(fld_status s);

#ifdef __cplusplus
}
#endif
#endif /* FLD_H */
