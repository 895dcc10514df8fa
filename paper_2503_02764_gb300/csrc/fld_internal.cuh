// Internal declarations shared by the FLD CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fld.h"

namespace fld {

// Device error bits (OR-ed into the handle's status word).
enum : unsigned { ERRBIT_DOMAIN = 1u, ERRBIT_TIMEOUT = 2u, ERRBIT_NOTCONV = 4u };

// Bounds-checked indexing for the debug build (FLD_DEBUG defined at compile time; the
// library's build step makes it with FLD_DEBUG=1 in the environment). fld_at(i, n) is i
// when 0 <= i < n; otherwise it raises a flag in a device word the host reads with
// fld_debug_flags() and returns 0, so the access stays inside the array and the kernel
// carries on (no trap). Without FLD_DEBUG it is i itself. The word's address is held in
// a constant of each translation unit, set for all of them when a handle is created.
void debug_register(void (*attach)(unsigned*));
void debug_attach_all();
#ifdef FLD_DEBUG
static __constant__ unsigned* fld_dbg_word;
// registers, at load time, the setter of this translation unit's copy (internal linkage)
static void fld_debug_attach_here(unsigned* w) {
    cudaMemcpyToSymbol(fld_dbg_word, &w, sizeof(w));
}
static int fld_debug_register_here() {
    debug_register(&fld_debug_attach_here);
    return 0;
}
static int fld_debug_registered = fld_debug_register_here();
__device__ __forceinline__ long long fld_at(long long i, long long n) {
    if (i >= 0 && i < n) return i;
    if (fld_dbg_word) atomicOr(fld_dbg_word, 1u);
    return 0;
}
// the same for the span [i, i + len) of one vector access
__device__ __forceinline__ long long fld_span(long long i, long long len, long long n) {
    if (i >= 0 && i + len <= n) return i;
    if (fld_dbg_word) atomicOr(fld_dbg_word, 1u);
    return 0;
}
#else
__device__ __forceinline__ long long fld_at(long long i, long long) { return i; }
__device__ __forceinline__ long long fld_span(long long i, long long, long long) { return i; }
#endif

// One multigrid level of a uniform block. The operator at this level is
//   (A x)_p = x_p + sum_faces 0.5 (K_p + K_q) w_d (x_p - x_q) + sum_dirichlet 2 K_p w_d x_p
// with K = dt D / H_x^2 (stored per cell) and w_d = (H_x / H_d)^2.
struct Lvl {
    int n[3];       // nx, ny, nz (1 for absent axes)
    int ndim;
    int bclo[3];
    int bchi[3];
    double w[3];    // axis weights (H_x / H_d)^2
    float wf[3];    // the same in FP32 (FP32 kernels never touch FP64 values)
    long long ncell;
    int fm;         // face coefficient from the two cell values: 0 arithmetic, 1 harmonic mean
    int pk;         // prolongation onto this level: 0 (bi/tri)linear, 1 piecewise constant
};

// Twice the face coefficient between two cells with cell coefficients a and b: a + b
// (arithmetic mean, fm = 0) or 4ab/(a + b) (harmonic mean, fm = 1; zero when a + b is not
// positive). The flag is uniform over a launch.
template <typename T>
__host__ __device__ __forceinline__ T fsum2(T a, T b, int fm) {
    const T s = a + b;
    if (fm == 0) return s;
    return s > T(0) ? T(4) * a * b / s : T(0);
}
// the face coefficient itself: (a + b)/2 or 2ab/(a + b)
template <typename T>
__host__ __device__ __forceinline__ T fmean(T a, T b, int fm) { return T(0.5) * fsum2(a, b, fm); }

// Axis weight in the kernel's arithmetic type.
template <typename T>
__host__ __device__ __forceinline__ T wgt(const Lvl& L, int d);
template <>
__host__ __device__ __forceinline__ double wgt<double>(const Lvl& L, int d) { return L.w[d]; }
template <>
__host__ __device__ __forceinline__ float wgt<float>(const Lvl& L, int d) { return L.wf[d]; }

// Opacity law evaluated in FP64: kappa0 (kind 0) or kappa0 rho^a T^b (kind 1).
struct Opacity {
    int kind;
    double kappa0, a_rho, a_T;
    const double* tab;           // TABLE: log10 kappa, [j * nr + i]
    int nr, nt;
    double lr0, ilr, lt0, ilt;   // first node and inverse spacing in log10 rho, log10 T
};

// v > 0 and finite, tested on the bit pattern (integer pipe, not the FP64 one).
__device__ __forceinline__ bool pos_finite(double v) {
    const long long b = __double_as_longlong(v);
    return b > 0 && b < 0x7FF0000000000000LL;
}

// Format conversions for FP32 seeds in integer arithmetic (a conversion instruction runs
// on the FP64 pipe of this GPU, at the FP64 rate):
// f32_near_pos: the FP32 number nearest to v (ties rounded up), for 2^-126 <= v < 2^127:
//   the double's exponent rebiased and its significand rounded to 24 bits, a carry moving
//   it to the next binade;
// f64_of_pos:   the exact FP64 value of a positive normal FP32 number.
__device__ __forceinline__ float f32_near_pos(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return __uint_as_float((unsigned)((b + (1ull << 28)) >> 29) - (896u << 23));
}
__device__ __forceinline__ double f64_of_pos(float f) {
    return __longlong_as_double(
        (long long)(((unsigned long long)__float_as_uint(f) + (896ull << 23)) << 29));
}

// 1/sqrt(t) for 0 < t within the FP32 normal range: FP32 seed refined by Newton-Raphson
// on f(y) = 1/y^2 - t, y <- y (3/2 - t y^2 / 2); each step squares the relative error
// (~2^-22 -> ~2^-44 -> rounding). `steps` = 1 or 2.
__device__ __forceinline__ double rsqrt_nr(double t, int steps) {
    double y = f64_of_pos(rsqrtf(f32_near_pos(t)));
    const double ht = 0.5 * t;
    y = y * fma(-ht, y * y, 1.5);
    if (steps > 1) y = y * fma(-ht, y * y, 1.5);
    return y;
}

// 1/a for 0 < a within the FP32 normal range (and 1/a too): FP32 reciprocal seed refined
// by Newton-Raphson on f(y) = 1/y - a, y <- y + y (1 - a y); each step squares the
// relative error.
__device__ __forceinline__ double rcp_nr(double a) {
    double y = f64_of_pos(__frcp_rn(f32_near_pos(a)));
    double e = fma(-a, y, 1.0);
    y = fma(y, e, y);
    e = fma(-a, y, 1.0);
    return fma(y, e, y);
}

// n / d for n >= 0 and 0 < d within the FP32 normal range (and 1/d too): one Newton-
// Raphson step on the FP32 reciprocal, the quotient, and one correction from its exact
// remainder n - d q (Markstein's scheme): within a unit of rounding, five FP64 operations.
__device__ __forceinline__ double div_nr(double n, double d) {
    double y = f64_of_pos(__frcp_rn(f32_near_pos(d)));
    y = fma(y, fma(-d, y, 1.0), y);
    const double q = n * y;
    return fma(fma(-d, q, n), y, q);
}

// sqrt(t) for 0 < t within the FP32 normal range: from the FP32 reciprocal square root
// y0, s = t y0 corrected twice by s <- s + (t - s^2) y0 / 2 (a Newton step for s^2 = t
// with the derivative's inverse taken from the seed): relative error 1.5 e0^2 after the
// first, rounding after the second; five FP64 operations.
__device__ __forceinline__ double sqrt_nr(double t) {
    const float y0 = rsqrtf(f32_near_pos(t));
    const double hy = f64_of_pos(0.5f * y0);
    double s = t * f64_of_pos(y0);
    s = fma(fma(-s, s, t), hy, s);
    return fma(fma(-s, s, t), hy, s);
}

// |v| within [2^-99, 2^99] (safely inside the FP32 normal range), tested on the
// exponent bits with integer operations.
__device__ __forceinline__ bool in_f32_range(double v) {
    const int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF) - 1023;
    return e > -100 && e < 99;
}

// kappa0 10^(bilinear interpolant of the log10 kappa table) at (log10 rho, log10 T), the
// coordinates clamped to the table; fmax/fmin also send a NaN coordinate to the first
// node, so every read stays inside the nr x nt array (nr, nt >= 2 on the host). Out of
// line, with scalar arguments, so the kernels' register allocation for the other laws
// is what it is without tables.
static __device__ __noinline__ double opacity_table(const double* __restrict__ tab, int nr,
                                                    int nt, double lr0, double ilr, double lt0,
                                                    double ilt, double kappa0, double rho,
                                                    double T) {
    double x = (log10(rho) - lr0) * ilr;
    double y = (log10(T) - lt0) * ilt;
    x = fmin(fmax(x, 0.0), (double)(nr - 1));
    y = fmin(fmax(y, 0.0), (double)(nt - 1));
    const int i = min((int)x, nr - 2), j = min((int)y, nt - 2);
    const double fx = x - i, fy = y - j;
    const double* t = tab + (long long)j * nr + i;
    const double lo = fma(fx, t[1] - t[0], t[0]);
    const double hi = fma(fx, t[nr + 1] - t[nr], t[nr]);
    return kappa0 * exp10(fma(fy, hi - lo, lo));
}

// kTables = false compiles the table law out (callers that never receive it)
template <bool kTables = true>
__device__ __forceinline__ double opacity_eval(const Opacity& op, double rho, double T) {
    if (op.kind == FLD_OPACITY_CONST) return op.kappa0;
    if (kTables && op.kind == FLD_OPACITY_TABLE)
        return opacity_table(op.tab, op.nr, op.nt, op.lr0, op.ilr, op.lt0, op.ilt, op.kappa0,
                             rho, T);
    const double fr = (op.a_rho == 1.0) ? rho : pow(rho, op.a_rho);
    double ft;
    if (op.a_T == 0.0) {
        ft = 1.0;
    } else if (op.a_T == -3.5) {            // Kramers-like law: T^-3.5 = (T^-1/2)^7
        if (in_f32_range(T)) {
            const double y = rsqrt_nr(T, 2);
            const double y2 = y * y;
            ft = y2 * y2 * y2 * y;
        } else {
            ft = 1.0 / (T * T * T * sqrt(T));
        }
    } else {
        ft = pow(T, op.a_T);
    }
    return op.kappa0 * fr * ft;
}

// (hi, lo) FP32 pair nearest to a double, on the host
inline void split_host(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// ----------------------------------------------------------------- host helpers
// Streaming multiprocessors of the current device, queried once per device; grid caps
// and the residual-norm grid are sized from it.
int num_sms();
int make_levels(const fld_grid& g, Lvl* lv, double* kdown, int maxl);
bool grid_valid(const fld_grid* g);
void note_launches(long long n);   // adds to fld_launch_count
bool opts_valid(const fld_opts* o);
long long fld_handle_cells(const fld_handle* h);   // cells of the handle's grid

// ----------------------------------------------------------------- launchers
// pointwise / limiter (k_pointwise.cu)
// kr (nullable) in the exchange: kappa rho per cell, frozen by the limiter of the same
// substep (which writes it when its own kr is non-null); without it kappa is evaluated
void launch_exchange(long long n, const double* rho, double* T, double* E, Opacity op,
                     double dtc, double a_r, double cv, int use_df, unsigned* err, cudaStream_t s,
                     const double* kr = nullptr);
void launch_limiter(const Lvl& L, const double* h, const double* E, const double* rho,
                    const double* T, const double* E_bc, const long long* bc_off, Opacity op,
                    double c, int mode, int use_df, double* D, double* lam, unsigned* err,
                    cudaStream_t s, float* Eh = nullptr, float* El = nullptr,
                    double* kr = nullptr);
// explicit coupling terms of the limiter pass (nullable outputs; v, vfr and pt together)
void launch_coupling(const Lvl& L, const double* h, const double* E, const double* rho,
                     const double* T, const double* E_bc, const long long* bc_off, Opacity op,
                     double c, int mode, const double* v, double* F, double* fr, double* fe,
                     double* vfr, double* pt, unsigned* err, cudaStream_t s);
// E split into FP32 (hi, lo) pairs (the double-FP32 limiter's input; Eh, El: n floats each).
void launch_split_df(long long n, const double* v, float* hi, float* lo, cudaStream_t s);

// multigrid (k_mg.cu)
// kmax (nullable): the FP32 bits of the largest K, folded in by atomicMax (zero it first)
void launch_prep_level0(const Lvl& L, double kscale, const double* D, const double* E,
                        const double* E_bc, const long long* bc_off, double* K64, float* K32,
                        double* b, unsigned* err, unsigned* kmax, cudaStream_t s);
template <typename T>
void launch_restrict_K(const Lvl& F, const Lvl& C, double scale, const T* Kf, T* Kc,
                       cudaStream_t s);
template <typename T>
void launch_smooth(const Lvl& L, int color, const T* xin, T* xout, const T* b, const T* K,
                   int block, cudaStream_t s);
// in-place half sweep of one colour (no odd periodic extent)
template <typename T>
bool rb_half_supported(const Lvl& L);
template <typename T>
void launch_rb_half(const Lvl& L, int color, T* x, const T* b, const T* K, cudaStream_t s);
// fused red+black sweep, xin -> xout (2D/3D levels with nx >= 8)
template <typename T>
bool rb_sweep_supported(const Lvl& L);
template <typename T>
void launch_rb_sweep(const Lvl& L, const T* xin, T* xout, const T* b, const T* K, cudaStream_t s);
void prepare_rb_sweep();
// The coarse end of a V-cycle in one single-block launch: the levels from the first with at
// most TAIL_MAX_CELLS cells to the coarsest (which must hold at most TAIL_MAX_DENSE cells).
constexpr long long TAIL_MAX_CELLS = 512;
constexpr int TAIL_MAX_DENSE = 64;
constexpr int TAIL_MAX_LEVELS = 10;
template <typename T>
struct TailLevels {
    Lvl L[TAIL_MAX_LEVELS];
    T* x[TAIL_MAX_LEVELS];
    T* b[TAIL_MAX_LEVELS];
    T* K[TAIL_MAX_LEVELS];
    T* tmp[TAIL_MAX_LEVELS];
    int n;          // levels in the tail, the last one the coarsest
    int nu1, nu2;
};
template <typename T>
void launch_vcycle_tail(const TailLevels<T>& t, cudaStream_t s);
// dynamic shared memory of a tail (4 arrays of every level) and its cap; the dense
// coarsest solve adds 33 KB of static shared memory
constexpr size_t TAIL_SMEM_MAX = 180 * 1024;
template <typename T>
size_t tail_smem_bytes(const Lvl* lv, int n);
void prepare_vcycle_tail();

// 3D transfers when every axis halves exactly (one thread per coarse cell).
bool transfer3_ok(const Lvl& F, const Lvl& C);
// red_only: the level was just smoothed by a red-black sweep (black last), so only the
// red children's residuals are summed (the black ones vanish up to rounding)
template <typename T>
void launch_resid_restrict3(const Lvl& F, const Lvl& C, const T* x, const T* b, const T* K, T* bc,
                            bool red_only, cudaStream_t s);
template <typename T>
void launch_prolong3(const Lvl& F, const Lvl& C, T* xf, const T* xc, cudaStream_t s);
template <typename T>
void launch_resid_restrict(const Lvl& F, const Lvl& C, const T* x, const T* b, const T* K,
                           T* bc, int block, bool red_only, cudaStream_t s);
template <typename T>
void launch_prolong(const Lvl& F, const Lvl& C, T* xf, const T* xc, int block, cudaStream_t s);
template <typename T>
void launch_coarse_solve(const Lvl& L, T* x, const T* b, const T* K, int sweeps, cudaStream_t s);
void launch_resid64(const Lvl& L, const double* x, const double* b, const double* K,
                    float* r32, double* partials, int nblocks, int block, cudaStream_t s);
void launch_add_correction(long long n, double* x, const float* e, cudaStream_t s);
// direct solve of a 1D level's system by parallel cyclic reduction (k_tridiag.cu), and one
// step of iterative refinement of x with it; w holds 12 n + 1 doubles; both return the
// kernels launched
int launch_tridiag_solve(const Lvl& L, const double* K, const double* rhs, double* x, double* w,
                         cudaStream_t s);
int launch_tridiag_refine(const Lvl& L, const double* K, const double* rhs, double* x, double* w,
                          cudaStream_t s);
// FP64 residual on 3D levels with each face flux evaluated once (k_resid64.cu): r = b - A x
// (x + e written to xo first when e is given), r32 its FP32 image (nullable), partial sums
// of r^2; returns the partials written (<= nblocks). resid64z_ok: the level is 3D and its
// tiles fit the partial-sum slots.
bool resid64z_ok(const Lvl& L, int nblocks);
// FP32 residual of the FP64 iterate (the mixed refinement's first correction): r32 and
// partial sums of r^2, z-marching tiles on 3D levels (where resid64z_ok holds), else one
// block per row; returns the number of partial sums written (<= nblocks)
int launch_resid32_init(const Lvl& L, const double* x, const double* b, const float* K,
                        float* r32, double* partials, int nblocks, cudaStream_t s);
int launch_resid64z(const Lvl& L, const double* x, const float* e, double* xo, const double* b,
                    const double* K, float* r32, double* partials, int nblocks, cudaStream_t s);
// Recursive refinement residual (k_resupd.cu): xo = x + e, r32 <- r32 - A e in FP32 on the
// level's FP32 coefficients, sums of (rs r)^2 in partials[0, n) and of (bs beta)^2 in
// partials[n, 2n), beta the per-cell rounding bound of the update, the largest absolute
// row sum of A in partials[2n, 3n); returns n (<= nblocks).
// resid_update_ok: the level is 3D, arithmetic face mean, its tiles fit the slots.
bool resid_update_ok(const Lvl& L, int nblocks);
int launch_resid_update(const Lvl& L, const double* x, const float* e, double* xo,
                        const float* K, float* r32, double* partials, int nblocks, float rs,
                        float bs, cudaStream_t s);
// its reductions in one launch: the two sums and the largest row sum (partials[2n, 3n))
void launch_finish_update(const double* partials, int nparts, double* out0, double* out1,
                          double* out2, cudaStream_t s);

// double-FP32 refinement (k_df.cu): half axis weights w_d/2 as (hi, lo) pairs
struct DfW {
    float hh[3], hl[3];
};
void launch_df_setup(long long n, double S, const double* E, const double* b, const double* K,
                     float* xh, float* xl, float* bh, float* bl, float* Kh, float* Kl,
                     cudaStream_t s);
void launch_df_finish(long long n, double invS, const float* xh, const float* xl, double* E,
                      cudaStream_t s);
int launch_df_resid(const Lvl& L, const DfW& wd, const float* xh, const float* xl, const float* e,
                     const float* bh, const float* bl, const float* Kh, const float* Kl, float* oh,
                     float* ol, float* r32, double* partials, int nblocks, int block,
                     cudaStream_t s);
void launch_sumsq(long long n, const double* v, double* partials, int nblocks, cudaStream_t s);
void launch_finish_sum(const double* partials, int nparts, double* out, cudaStream_t s);
// partial sums of c_v rho T + E over n cells (E alone when rho is null), nblocks partials
void launch_energy_sum(long long n, const double* rho, const double* T, const double* E, double cv,
                       double* partials, int nblocks, cudaStream_t s);

}  // namespace fld
