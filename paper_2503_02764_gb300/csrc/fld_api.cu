// Host side of the C ABI declared in include/fld.h: handle and workspace, the
// multigrid level pyramid, the V-cycle driver (FP64, or FP32 cycles inside FP64
// iterative refinement) and the substep composition limiter -> diffuse -> exchange.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fld_internal.cuh"

using namespace fld;

namespace {

constexpr int MAX_LEVELS = 24;
constexpr long long COARSE_TARGET = 8;    // stop coarsening at or below this many cells
constexpr int NORM_BLOCKS_PER_SM = 8;    // residual-norm grid: 8 blocks per SM
constexpr int NORM_THREADS = 256;

template <typename T>
struct LevelBufs {
    T* x = nullptr;
    T* b = nullptr;
    T* K = nullptr;
    T* tmp = nullptr;
};

struct DevScalars {       // read back together after each cycle
    double sum;
    unsigned err;
    unsigned kmax;        // FP32 bits of the largest level-0 K of the solve
    double energy[2];     // diagnostics: total energy before and after a call
    double drift;         // recursive residual: sum of the squared scaled rounding bound
    double amax;          //   and the largest absolute row sum of the level-0 operator
};

std::atomic<long long> g_launches{0};

// Event-bracketed launch record (profiling on).
struct ProfRec {
    const char* name;
    int level;
    long long cells;
};

struct Prof {
    bool on = false;
    int cap = 0;
    int used = 0;
    std::vector<cudaEvent_t> ev;     // 2 per record
    std::vector<ProfRec> rec;
};

}  // namespace

namespace fld {
// Level pyramid of a grid: an axis with n >= 4 halves to ceil(n/2) (cell size reset to
// L/n), until <= COARSE_TARGET cells remain or no axis can coarsen. Returns the number
// of levels; kdown[l] rescales the averaged K of level l to level l+1's spacing.
int make_levels(const fld_grid& g, Lvl* lv, double* kdown, int maxl) {
    Lvl L{};
    double H[3], len[3];
    for (int d = 0; d < 3; ++d) {
        L.n[d] = g.n[d];
        L.bclo[d] = d < g.ndim ? g.bc_lo[d] : FLD_BC_PERIODIC;
        L.bchi[d] = d < g.ndim ? g.bc_hi[d] : FLD_BC_PERIODIC;
        H[d] = d < g.ndim ? g.h[d] : 1.0;
        len[d] = H[d] * g.n[d];
    }
    L.ndim = g.ndim;
    int nl = 0;
    for (;;) {
        L.ncell = (long long)L.n[0] * L.n[1] * L.n[2];
        for (int d = 0; d < 3; ++d) {
            L.w[d] = d < g.ndim ? (H[0] / H[d]) * (H[0] / H[d]) : 0.0;
            L.wf[d] = (float)L.w[d];
        }
        lv[nl++] = L;
        bool can = false;
        for (int d = 0; d < g.ndim; ++d) can |= L.n[d] >= 4;
        if (!can || L.ncell <= COARSE_TARGET || nl == maxl) break;
        const double Hx_old = H[0];
        for (int d = 0; d < g.ndim; ++d) {
            if (L.n[d] >= 4) {
                L.n[d] = (L.n[d] + 1) / 2;
                H[d] = len[d] / L.n[d];
            }
        }
        kdown[nl - 1] = (Hx_old / H[0]) * (Hx_old / H[0]);
    }
    return nl;
}
int num_sms() {
    constexpr int MAXDEV = 64;
    static std::atomic<int> cache[MAXDEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = (dev >= 0 && dev < MAXDEV) ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;
    }
    if (dev >= 0 && dev < MAXDEV) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}
// launches made outside this file's launch wrapper (the wave step's kernels)
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Debug build: every translation unit registers the setter of its copy of the debug
// word's address when the library loads; the word is allocated and handed to all of them
// on the first handle creation.
namespace {
std::vector<void (*)(unsigned*)>& debug_setters() {
    static std::vector<void (*)(unsigned*)> v;
    return v;
}
unsigned* g_debug_word = nullptr;
std::mutex g_debug_mu;
}  // namespace
void debug_register(void (*attach)(unsigned*)) { debug_setters().push_back(attach); }
void debug_attach_all() {
#ifdef FLD_DEBUG
    std::lock_guard<std::mutex> lock(g_debug_mu);
    if (g_debug_word) return;
    if (cudaMalloc(&g_debug_word, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        g_debug_word = nullptr;
        return;
    }
    cudaMemset(g_debug_word, 0, sizeof(unsigned));
    for (auto f : debug_setters()) f(g_debug_word);
    cudaDeviceSynchronize();
#endif
}
}  // namespace fld

struct fld_handle {
    fld_grid g;
    fld_opts o;
    int nlev = 0;
    Lvl lv[MAX_LEVELS];
    double kscale_down[MAX_LEVELS];   // K_{l+1} = mean(K_l) * kscale_down[l]
    long long bc_off[6];
    long long ncell = 0;
    LevelBufs<double> d64[MAX_LEVELS];
    LevelBufs<float> d32[MAX_LEVELS];
    float* dfx[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // iterate (hi, lo), ping-pong
    float* dfb[2] = {nullptr, nullptr};                            // right-hand side (hi, lo)
    float* dfK[2] = {nullptr, nullptr};                            // coefficient K (hi, lo)
    double* Dscratch = nullptr;
    double* krscratch = nullptr;     // kappa rho of the substep (limiter -> exchange)
    double* triw = nullptr;          // 1D grids: the direct solve's workspace (12 n + 1)
    double* partials = nullptr;
    int norm_blocks = 0;              // blocks (and partial sums) of the norm kernels
    DevScalars* scal = nullptr;       // device
    DevScalars* hscal = nullptr;      // pinned host
    std::vector<void*> allocs;
    Prof prof;
    // CUDA graph of the FP32 V-cycle (handle-owned buffers only), replayed per cycle
    cudaStream_t gs = nullptr;
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    cudaGraphExec_t vgraph = nullptr;
    int vgraph_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long vgraph_nodes = 0;
    // first level of the single-launch V-cycle tail (-1: none); set when the levels are built
    int tail_start = -1;
    // levels the V-cycles of the current solve use (the last one solved by vsweeps
    // red-black sweeps when vdepth < nlev); set per solve from the largest K
    int vdepth = 0;
    int vsweeps = 0;
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};   // per-phase times (diag)
};

namespace {

fld_status cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return FLD_OK;
    fprintf(stderr, "fld: CUDA error: %s\n", cudaGetErrorString(e));
    return FLD_ERR_CUDA;
}

#define FLD_CK(call)                                          \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_);          \
    } while (0)

}  // namespace

bool fld::grid_valid(const fld_grid* g) {
    if (!g || g->ndim < 1 || g->ndim > 3) return false;
    long long n = 1;
    for (int d = 0; d < 3; ++d) {
        if (d < g->ndim) {
            if (g->n[d] < 2 || !(g->h[d] > 0) || !std::isfinite(g->h[d])) return false;
            for (int s = 0; s < 2; ++s) {
                int k = s ? g->bc_hi[d] : g->bc_lo[d];
                if (k < FLD_BC_PERIODIC || k > FLD_BC_DIRICHLET) return false;
            }
            if ((g->bc_lo[d] == FLD_BC_PERIODIC) != (g->bc_hi[d] == FLD_BC_PERIODIC)) return false;
        } else if (g->n[d] != 1) {
            return false;
        }
        n *= g->n[d];
    }
    return n < (1LL << 31);
}

namespace {

bool grid_ok(const fld_grid* g) { return fld::grid_valid(g); }

bool opts_ok(const fld_opts* o) { return fld::opts_valid(o); }

}  // namespace

bool fld::opts_valid(const fld_opts* o) {
    return o && (o->precision == FLD_PREC_FP64 || o->precision == FLD_PREC_MIXED ||
                 o->precision == FLD_PREC_MIXED_DF) && o->tol > 0 &&
           o->max_cycles >= 1 && o->nu1 >= 0 && o->nu2 >= 0 && (o->nu1 + o->nu2) >= 1 &&
           o->coarse_sweeps >= 1 &&
           (o->limiter == FLD_LIMITER_LP || o->limiter == FLD_LIMITER_DIFFUSION ||
            o->limiter == FLD_LIMITER_MINERBO) &&
           (o->block == 0 || (o->block >= 32 && o->block <= 1024 && o->block % 32 == 0)) &&
           (o->smoother >= 0 && o->smoother <= 2) &&
           (o->cluster == 0 || o->cluster == 1 || o->cluster == 2 || o->cluster == 4 ||
            o->cluster == 8) &&
           (o->inner >= 0 && o->inner <= 8) && (o->direct1d == 0 || o->direct1d == 1) &&
           (o->diag >= 0 && o->diag <= (FLD_DIAG_ENERGY | FLD_DIAG_TIMES)) &&
           (o->face_mean == FLD_FACE_ARITH ||
            (o->face_mean == FLD_FACE_HARM && o->precision != FLD_PREC_MIXED_DF)) &&
           (o->prolong == FLD_PROLONG_LINEAR || o->prolong == FLD_PROLONG_CONSTANT) &&
           (o->limiter_df == 0 || o->limiter_df == 1) &&
           (o->resid_update == 0 || o->resid_update == 1) &&
           (o->truncate == 0 || o->truncate == 1);
}

namespace {

Opacity to_op(const fld_opacity* op) {
    Opacity o;
    o.kind = op->kind;
    o.kappa0 = op->kappa0;
    o.a_rho = op->a_rho;
    o.a_T = op->a_T;
    o.tab = nullptr;
    o.nr = o.nt = 0;
    o.lr0 = o.ilr = o.lt0 = o.ilt = 0.0;
    if (op->kind == FLD_OPACITY_TABLE) {
        o.a_rho = o.a_T = 0.0;
        o.tab = op->table;
        o.nr = op->n_rho;
        o.nt = op->n_T;
        o.lr0 = op->log_rho0;
        o.ilr = 1.0 / op->dlog_rho;
        o.lt0 = op->log_T0;
        o.ilt = 1.0 / op->dlog_T;
    }
    return o;
}

bool table_ok(const fld_opacity* op) {
    return op->table && op->n_rho >= 2 && op->n_T >= 2 &&
           (long long)op->n_rho * op->n_T < (1LL << 31) && op->dlog_rho > 0 &&
           op->dlog_T > 0 && std::isfinite(op->dlog_rho) && std::isfinite(op->dlog_T) &&
           std::isfinite(op->log_rho0) && std::isfinite(op->log_T0) &&
           std::isfinite(1.0 / op->dlog_rho) && std::isfinite(1.0 / op->dlog_T);
}

bool op_ok(const fld_opacity* op) {
    if (!op || !(op->kappa0 > 0) || !std::isfinite(op->kappa0)) return false;
    if (op->kind == FLD_OPACITY_CONST) return true;
    if (op->kind == FLD_OPACITY_POWER)
        return std::isfinite(op->a_rho) && std::isfinite(op->a_T);
    return op->kind == FLD_OPACITY_TABLE && table_ok(op);
}

bool consts_ok(const fld_consts* k) {
    return k && k->c > 0 && k->a_r > 0 && k->gamma > 1 && k->R_gas > 0 && std::isfinite(k->c) &&
           std::isfinite(k->a_r) && std::isfinite(k->gamma) && std::isfinite(k->R_gas);
}

bool has_dirichlet(const fld_grid& g) {
    for (int d = 0; d < g.ndim; ++d)
        if (g.bc_lo[d] == FLD_BC_DIRICHLET || g.bc_hi[d] == FLD_BC_DIRICHLET) return true;
    return false;
}

void build_levels(fld_handle* h) {
    h->nlev = fld::make_levels(h->g, h->lv, h->kscale_down, MAX_LEVELS);
    for (int l = 0; l < h->nlev; ++l) {
        h->lv[l].fm = h->o.face_mean;
        h->lv[l].pk = h->o.prolong;
    }
    // the tail starts at the first level small enough for one block (cells, and all its
    // levels in shared memory even in FP64), if the coarsest level takes the dense solve
    // and at least two levels remain
    h->tail_start = -1;
    if (h->lv[h->nlev - 1].ncell > TAIL_MAX_DENSE) return;
    for (int l = 0; l + 1 < h->nlev; ++l)
        if (h->lv[l].ncell <= TAIL_MAX_CELLS && h->nlev - l <= TAIL_MAX_LEVELS &&
            tail_smem_bytes<double>(h->lv + l, h->nlev - l) <= TAIL_SMEM_MAX) {
            h->tail_start = l;
            break;
        }
}

// Depth of the V-cycles of one solve. On level l the operator is I plus a part whose
// off-diagonal row sums are at most s_l = 2 Kmax_l sum_d w_d (Kmax_l <= Kmax times the
// K rescalings down to l: restriction averages K), so the Jacobi iteration contracts by
// at most rho_l = s_l / (1 + s_l) and a red-black sweep by about rho_l^2. The V-cycle
// stops at the first level below the finest where TRUNC_MAX_SWEEPS such sweeps or fewer
// reduce the error to TRUNC_EPS, and solves that level by them; with no such level above
// the single-block tail (or the coarsest level) it runs to the coarsest level.
constexpr double TRUNC_EPS = 0.01;
constexpr int TRUNC_MAX_SWEEPS = 4;

void choose_depth(fld_handle* h, double kmax) {
    h->vdepth = h->nlev;
    h->vsweeps = 0;
    if (!h->o.truncate || !(kmax >= 0.0) || !std::isfinite(kmax)) return;
    const int stop = h->tail_start >= 0 ? h->tail_start : h->nlev - 1;
    double kl = kmax * (1.0 + 1e-6);        // the maximum was taken in FP32
    for (int c = 1; c < stop; ++c) {
        kl *= h->kscale_down[c - 1];
        double ws = 0.0;
        for (int d = 0; d < h->lv[c].ndim; ++d) ws += h->lv[c].w[d];
        const double sw = 2.0 * kl * ws;
        const double rho = sw / (1.0 + sw);
        const int n = rho > 0.0 ? (int)std::ceil(std::log(TRUNC_EPS) / (2.0 * std::log(rho)))
                                : 1;
        if (n >= 1 && n <= TRUNC_MAX_SWEEPS) {
            h->vdepth = c + 1;
            h->vsweeps = n;
            return;
        }
    }
}

template <typename T>
fld_status dalloc(fld_handle* h, T** p, long long n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (size_t)std::max<long long>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FLD_ERR_NOMEM;
    }
    h->allocs.push_back(q);
    *p = (T*)q;
    return FLD_OK;
}

void free_all(fld_handle* h) {
    for (cudaEvent_t& e : h->tev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->hscal) cudaFreeHost(h->hscal);
    h->hscal = nullptr;
}

int blk(const fld_handle* h) { return h->o.block ? h->o.block : 256; }

// Launch `f` (which enqueues exactly one kernel on s), counting it and, when
// profiling is on, bracketing it with events.
template <typename F>
void run(fld_handle* h, const char* name, int level, long long cells, cudaStream_t s, F&& f) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    Prof& P = h->prof;
    const bool timed = P.on && P.used < P.cap;
    if (timed) cudaEventRecord(P.ev[2 * P.used], s);
    f();
    if (timed) {
        cudaEventRecord(P.ev[2 * P.used + 1], s);
        P.rec[P.used] = ProfRec{name, level, cells};
        ++P.used;
    }
}

void prof_free(fld_handle* h) {
    for (cudaEvent_t e : h->prof.ev) cudaEventDestroy(e);
    h->prof.ev.clear();
    h->prof.rec.clear();
    h->prof.cap = h->prof.used = 0;
    h->prof.on = false;
}

// -------------------------------------------------- smoothing: `n` red-black sweeps of
// the iterate in `cur` (B.x or B.tmp; `oth` is the other buffer). The first `fused` of
// them use the single-pass out-of-place kernel, each moving the iterate to the other
// buffer (the two pointers swap). The rest run in place: two half-sweep launches, or,
// where those do not apply (odd periodic extents) or smoother 1 asks for it, the
// out-of-place half-sweep pair cur -> oth -> cur.
template <typename T>
void smooth(fld_handle* h, LevelBufs<T>& B, int l, int n, int fused, T*& cur, T*& oth,
            cudaStream_t s) {
    const Lvl& L = h->lv[l];
    const bool f32 = sizeof(T) == 4;
    const int bs = blk(h);
    for (int i = 0; i < fused; ++i) {
        run(h, f32 ? "rbsweep32" : "rbsweep64", l, L.ncell, s,
            [&] { launch_rb_sweep<T>(L, cur, oth, B.b, B.K, s); });
        std::swap(cur, oth);
    }
    int left = n - fused;
    if (h->o.smoother != 1 && rb_half_supported<T>(L)) {
        const char* nm = f32 ? "rbhalf32" : "rbhalf64";
        for (; left > 0; --left) {
            run(h, nm, l, L.ncell, s, [&] { launch_rb_half<T>(L, 0, cur, B.b, B.K, s); });
            run(h, nm, l, L.ncell, s, [&] { launch_rb_half<T>(L, 1, cur, B.b, B.K, s); });
        }
    }
    const char* sm = f32 ? "smooth32" : "smooth64";
    for (; left > 0; --left) {
        run(h, sm, l, L.ncell, s, [&] { launch_smooth<T>(L, 0, cur, oth, B.b, B.K, bs, s); });
        run(h, sm, l, L.ncell, s, [&] { launch_smooth<T>(L, 1, oth, cur, B.b, B.K, bs, s); });
    }
}

// -------------------------------------------------- V-cycle on level l (x_l in/out)
template <typename T>
void vcycle(fld_handle* h, LevelBufs<T>* P, int l, cudaStream_t s) {
    const Lvl& L = h->lv[l];
    LevelBufs<T>& B = P[l];
    const bool f32 = sizeof(T) == 4;
    if (l == h->nlev - 1) {
        run(h, f32 ? "coarse32" : "coarse64", l, L.ncell, s,
            [&] { launch_coarse_solve<T>(L, B.x, B.b, B.K, h->o.coarse_sweeps, s); });
        return;
    }
    if (l == h->vdepth - 1) {
        // the truncated coarsest level: vsweeps red-black sweeps from x = 0 (an even
        // number of them single-pass, so the iterate ends in B.x)
        T* cur = B.x;
        T* oth = B.tmp;
        const int n = h->vsweeps;
        const int f = (h->o.smoother == 2 && rb_sweep_supported<T>(L)) ? (n & ~1) : 0;
        smooth<T>(h, B, l, n, f, cur, oth, s);
        return;
    }
    if (l == h->tail_start) {
        // the rest of the V-cycle (a few thousand cells at most) in one launch
        TailLevels<T> t{};
        t.n = h->nlev - l;
        t.nu1 = h->o.nu1;
        t.nu2 = h->o.nu2;
        for (int q = 0; q < t.n; ++q) {
            t.L[q] = h->lv[l + q];
            t.x[q] = P[l + q].x;
            t.b[q] = P[l + q].b;
            t.K[q] = P[l + q].K;
            t.tmp[q] = P[l + q].tmp;
        }
        run(h, f32 ? "tail32" : "tail64", l, L.ncell, s, [&] { launch_vcycle_tail<T>(t, s); });
        return;
    }
    const int bs = blk(h);
    // fused sweeps swap the buffers, so an even number of them brings the iterate back
    // to B.x; with an odd nu1 + nu2 the last sweep of the cycle runs in place
    const int nu1 = h->o.nu1, nu2 = h->o.nu2;
    int f1 = 0, f2 = 0;
    if (h->o.smoother == 2 && rb_sweep_supported<T>(L)) {
        f1 = nu1;
        f2 = nu2;
        if ((nu1 + nu2) & 1) (nu2 > 0 ? f2 : f1) -= 1;
    }
    T* cur = B.x;
    T* oth = B.tmp;
    smooth<T>(h, B, l, nu1, f1, cur, oth, s);
    const Lvl& C = h->lv[l + 1];
    run(h, f32 ? "resid_restrict32" : "resid_restrict64", l, L.ncell, s,
        [&] { launch_resid_restrict<T>(L, C, cur, B.b, B.K, P[l + 1].b, bs, nu1 > 0, s); });
    if (l + 1 < h->nlev - 1) cudaMemsetAsync(P[l + 1].x, 0, sizeof(T) * C.ncell, s);
    vcycle<T>(h, P, l + 1, s);
    run(h, f32 ? "prolong32" : "prolong64", l, L.ncell, s,
        [&] { launch_prolong<T>(L, C, cur, P[l + 1].x, bs, s); });
    smooth<T>(h, B, l, nu2, f2, cur, oth, s);
}

template <typename T>
void restrict_pyramid(fld_handle* h, LevelBufs<T>* P, cudaStream_t s) {
    for (int l = 0; l + 1 < h->nlev; ++l)
        run(h, "restrict_K", l, h->lv[l + 1].ncell, s, [&] {
            launch_restrict_K<T>(h->lv[l], h->lv[l + 1], h->kscale_down[l], P[l].K, P[l + 1].K, s);
        });
}

fld_status read_scalars(fld_handle* h, cudaStream_t s, double* sum, unsigned* err) {
    FLD_CK(cudaMemcpyAsync(h->hscal, h->scal, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    FLD_CK(cudaStreamSynchronize(s));
    *sum = h->hscal->sum;
    *err = h->hscal->err;
    return FLD_OK;
}

// relative residual of x at level 0 (FP64), optional FP32 copy of the residual. With e
// (3D levels, where the z-marching kernel applies) the iterate is first corrected: x + e is
// written to xo and the residual is that of xo.
fld_status residual(fld_handle* h, const double* x, const float* e, double* xo, float* r32,
                    cudaStream_t s, double* rr, unsigned* err) {
    const Lvl& L = h->lv[0];
    int nparts = h->norm_blocks;
    if (resid64z_ok(L, h->norm_blocks)) {
        run(h, e ? "resid64x" : "resid64", 0, L.ncell, s, [&] {
            nparts = launch_resid64z(L, x, e, xo, h->d64[0].b, h->d64[0].K, r32, h->partials,
                                     h->norm_blocks, s);
        });
    } else {
        run(h, "resid64", 0, L.ncell, s, [&] {
            launch_resid64(L, x, h->d64[0].b, h->d64[0].K, r32, h->partials, h->norm_blocks,
                           NORM_THREADS, s);
        });
    }
    run(h, "finish_sum", 0, nparts, s,
        [&] { launch_finish_sum(h->partials, nparts, &h->scal->sum, s); });
    FLD_CK(cudaGetLastError());
    return read_scalars(h, s, rr, err);
}

// The recursive refinement residual at level 0 (3D, MIXED): xo = x + e (e the FP32 V-cycles'
// correction), r32 <- r32 - A e in FP32; *rr = ||r||^2, *dd = ||beta||^2 (beta the per-cell
// bound on the update's rounding) and *amax the largest absolute row sum of A. The kernel
// forms beta' = 2^20 beta and squares rs r and bs beta' = 2^-20 rs beta' = rs beta, rs a power
// of two.
fld_status residual_update(fld_handle* h, const double* x, double* xo, double rs, double bs,
                           cudaStream_t s, double* rr, double* dd, double* amax,
                           unsigned* err) {
    const Lvl& L = h->lv[0];
    int nparts = 0;
    run(h, "resid_upd", 0, L.ncell, s, [&] {
        nparts = launch_resid_update(L, x, h->d32[0].x, xo, h->d32[0].K, h->d32[0].b,
                                     h->partials, h->norm_blocks, (float)rs, (float)bs, s);
    });
    run(h, "finish_sum", 0, nparts, s, [&] {
        launch_finish_update(h->partials, nparts, &h->scal->sum, &h->scal->drift,
                             &h->scal->amax, s);
    });
    FLD_CK(cudaGetLastError());
    double sum;
    const fld_status rc = read_scalars(h, s, &sum, err);
    if (rc != FLD_OK) return rc;
    *rr = sum / (rs * rs);
    *dd = h->hscal->drift / (rs * rs);     // (bs beta')^2 / rs^2 = (2^-20 beta')^2
    *amax = h->hscal->amax;
    return FLD_OK;
}

void graph_free(fld_handle* h) {
    if (h->vgraph) cudaGraphExecDestroy(h->vgraph);
    if (h->gev_in) cudaEventDestroy(h->gev_in);
    if (h->gev_out) cudaEventDestroy(h->gev_out);
    if (h->gs) cudaStreamDestroy(h->gs);
    h->vgraph = nullptr;
    h->gev_in = h->gev_out = nullptr;
    h->gs = nullptr;
}

// e32 = 0, then `inner` FP32 V-cycles on level 0 (each later one continues from the
// correction so far: its restriction sees the FP32 residual r32 - A e32). With graphs on (and profiling off) the
// sequence is captured once per option set on a handle-owned stream and replayed;
// the caller's stream and that stream are ordered through events.
fld_status vcycle32(fld_handle* h, cudaStream_t s) {
    const long long n0 = h->lv[0].ncell;
    const int inner = h->o.inner > 0 ? h->o.inner : 1;
    if (!h->o.graph || h->prof.on) {
        FLD_CK(cudaMemsetAsync(h->d32[0].x, 0, sizeof(float) * n0, s));
        for (int c = 0; c < inner; ++c) vcycle<float>(h, h->d32, 0, s);
        return FLD_OK;
    }
    const int key[8] = {h->o.nu1, h->o.nu2, h->o.smoother, h->o.block, h->o.coarse_sweeps,
                        inner, h->vdepth, h->vsweeps};
    if (!h->gs) {
        FLD_CK(cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking));
        FLD_CK(cudaEventCreateWithFlags(&h->gev_in, cudaEventDisableTiming));
        FLD_CK(cudaEventCreateWithFlags(&h->gev_out, cudaEventDisableTiming));
    }
    if (!h->vgraph || memcmp(key, h->vgraph_key, sizeof(key)) != 0) {
        if (h->vgraph) cudaGraphExecDestroy(h->vgraph);
        h->vgraph = nullptr;
        cudaGraph_t g = nullptr;
        const long long before = g_launches.load();
        FLD_CK(cudaStreamBeginCapture(h->gs, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(h->d32[0].x, 0, sizeof(float) * n0, h->gs);
        for (int c = 0; c < inner; ++c) vcycle<float>(h, h->d32, 0, h->gs);
        FLD_CK(cudaStreamEndCapture(h->gs, &g));
        h->vgraph_nodes = g_launches.load() - before;
        g_launches.fetch_sub(h->vgraph_nodes);       // counted per replay below
        cudaError_t e = cudaGraphInstantiate(&h->vgraph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->vgraph = nullptr;
            return cuda_fail(e);
        }
        memcpy(h->vgraph_key, key, sizeof(key));
    }
    FLD_CK(cudaEventRecord(h->gev_in, s));
    FLD_CK(cudaStreamWaitEvent(h->gs, h->gev_in, 0));
    FLD_CK(cudaGraphLaunch(h->vgraph, h->gs));
    g_launches.fetch_add(h->vgraph_nodes);
    FLD_CK(cudaEventRecord(h->gev_out, h->gs));
    FLD_CK(cudaStreamWaitEvent(s, h->gev_out, 0));
    return FLD_OK;
}

// Mixed refinement with the residual and the correction in double-FP32: the scaled
// iterate S x, S b and K live as (hi, lo) FP32 pairs for the duration of the solve;
// E is read at the start and written at the end.
fld_status diffuse_df(fld_handle* h, double* E, double bsum, fld_stats* st, cudaStream_t s) {
    const Lvl& L0 = h->lv[0];
    const long long n = L0.ncell;
    int ex = 0;
    const double rms = bsum > 0 ? std::sqrt(bsum / (double)n) : 1.0;
    std::frexp(rms, &ex);
    const double S = std::ldexp(1.0, -ex);        // power of two: exact scaling
    const double bnorm = std::sqrt(bsum) * S;
    DfW wd;
    for (int d = 0; d < 3; ++d) {
        const double wh = 0.5 * L0.w[d];
        wd.hh[d] = (float)wh;
        wd.hl[d] = (float)(wh - (double)wd.hh[d]);
    }
    run(h, "df_setup", 0, n, s, [&] {
        launch_df_setup(n, S, E, h->d64[0].b, h->d64[0].K, h->dfx[0][0], h->dfx[0][1], h->dfb[0],
                        h->dfb[1], h->dfK[0], h->dfK[1], s);
    });
    int cur = 0;
    auto resid = [&](const float* e, double* rr) -> fld_status {
        float* oh = e ? h->dfx[cur ^ 1][0] : nullptr;
        float* ol = e ? h->dfx[cur ^ 1][1] : nullptr;
        int nparts = h->norm_blocks;
        run(h, "resid_df", 0, n, s, [&] {
            nparts = launch_df_resid(L0, wd, h->dfx[cur][0], h->dfx[cur][1], e, h->dfb[0],
                                     h->dfb[1], h->dfK[0], h->dfK[1], oh, ol, h->d32[0].b,
                                     h->partials, h->norm_blocks, NORM_THREADS, s);
        });
        if (e) cur ^= 1;
        run(h, "finish_sum", 0, nparts, s,
            [&] { launch_finish_sum(h->partials, nparts, &h->scal->sum, s); });
        FLD_CK(cudaGetLastError());
        unsigned err;
        return read_scalars(h, s, rr, &err);
    };
    double r2;
    fld_status rc = resid(nullptr, &r2);
    if (rc != FLD_OK) return rc;
    double rel = bnorm > 0 ? std::sqrt(r2) / bnorm : 0.0;
    if (st) {
        memset(st, 0, sizeof(*st));
        st->resid_hist[0] = rel;
        st->levels = h->vdepth;
    }
    int cyc = 0;
    while (rel > h->o.tol && cyc < h->o.max_cycles && std::isfinite(rel)) {
        rc = vcycle32(h, s);
        if (rc != FLD_OK) return rc;
        rc = resid(h->d32[0].x, &r2);
        if (rc != FLD_OK) return rc;
        rel = std::sqrt(r2) / bnorm;
        ++cyc;
        if (st && cyc < 64) st->resid_hist[cyc] = rel;
    }
    run(h, "df_finish", 0, n, s, [&] {
        launch_df_finish(n, 1.0 / S, h->dfx[cur][0], h->dfx[cur][1], E, s);
    });
    FLD_CK(cudaGetLastError());
    if (st) {
        st->cycles = cyc;
        st->rel_resid = rel;
    }
    if (!std::isfinite(rel)) return FLD_ERR_DOMAIN;
    return rel <= h->o.tol ? FLD_OK : FLD_ERR_NOT_CONVERGED;
}

fld_status diffuse_impl(fld_handle* h, double dt, const double* D, const double* E_bc, double* E,
                        fld_stats* st, cudaStream_t s) {
    const Lvl& L0 = h->lv[0];
    const bool dfmode = h->o.precision == FLD_PREC_MIXED_DF;
    const bool mixed = h->o.precision == FLD_PREC_MIXED || dfmode;
    const double kscale = dt / (h->g.h[0] * h->g.h[0]);
    // 1D grids with direct1d: the tridiagonal system solved directly (no pyramid needed)
    const bool direct = h->g.ndim == 1 && h->o.direct1d && h->triw;
    // the largest K decides the V-cycle depth (read back with the norm of b)
    const bool want_kmax = !direct && h->o.truncate;
    if (want_kmax) FLD_CK(cudaMemsetAsync(&h->scal->kmax, 0, sizeof(unsigned), s));
    run(h, "prep", 0, L0.ncell, s, [&] {
        launch_prep_level0(L0, kscale, D, E, E_bc, h->bc_off, h->d64[0].K,
                           mixed ? h->d32[0].K : nullptr, h->d64[0].b, &h->scal->err,
                           want_kmax ? &h->scal->kmax : nullptr, s);
    });
    if (!direct) {
        if (mixed) restrict_pyramid<float>(h, h->d32, s);
        else restrict_pyramid<double>(h, h->d64, s);
    }
    run(h, "sumsq", 0, L0.ncell, s,
        [&] { launch_sumsq(L0.ncell, h->d64[0].b, h->partials, h->norm_blocks, s); });
    run(h, "finish_sum", 0, h->norm_blocks, s,
        [&] { launch_finish_sum(h->partials, h->norm_blocks, &h->scal->sum, s); });
    FLD_CK(cudaGetLastError());
    double bsum;
    unsigned err;
    fld_status rc = read_scalars(h, s, &bsum, &err);
    if (rc != FLD_OK) return rc;
    if (err) {
        cudaMemsetAsync(&h->scal->err, 0, sizeof(unsigned), s);
        return FLD_ERR_DOMAIN;
    }
    const double bnorm = std::sqrt(bsum);
    if (want_kmax) {
        unsigned kb = h->hscal->kmax;
        float kf;
        memcpy(&kf, &kb, sizeof(kf));
        choose_depth(h, (double)kf);
    } else {
        choose_depth(h, -1.0);
    }
    if (direct) {
        // the reduction, then refinement steps with it while the FP64 residual is above
        // tol (each one a cycle; rounding of the reduction grows with dt D / h^2)
        if (st) {
            // the residual of E^n, as the V-cycle path reports it
            double r0;
            rc = residual(h, E, nullptr, nullptr, nullptr, s, &r0, &err);
            if (rc != FLD_OK) return rc;
            memset(st, 0, sizeof(*st));
            st->resid_hist[0] = bnorm > 0 ? std::sqrt(r0) / bnorm : 0.0;
            st->levels = 1;
        }
        int nl = 0;
        run(h, "tridiag", 0, L0.ncell, s,
            [&] { nl = launch_tridiag_solve(L0, h->d64[0].K, h->d64[0].b, E, h->triw, s); });
        g_launches.fetch_add(nl - 1, std::memory_order_relaxed);
        double rel = 0.0;
        int cyc = 1;
        for (;;) {
            double r2;
            rc = residual(h, E, nullptr, nullptr, nullptr, s, &r2, &err);
            if (rc != FLD_OK) return rc;
            rel = bnorm > 0 ? std::sqrt(r2) / bnorm : 0.0;
            if (st && cyc < 64) st->resid_hist[cyc] = rel;
            if (!(rel > h->o.tol) || cyc >= h->o.max_cycles || !std::isfinite(rel)) break;
            run(h, "tridiag_refine", 0, L0.ncell, s, [&] {
                nl = launch_tridiag_refine(L0, h->d64[0].K, h->d64[0].b, E, h->triw, s);
            });
            g_launches.fetch_add(nl - 1, std::memory_order_relaxed);
            ++cyc;
        }
        if (st) {
            st->cycles = cyc;
            st->rel_resid = rel;
        }
        if (!std::isfinite(rel)) return FLD_ERR_DOMAIN;
        return rel <= h->o.tol ? FLD_OK : FLD_ERR_NOT_CONVERGED;
    }
    if (dfmode) return diffuse_df(h, E, bsum, st, s);
    h->d64[0].x = E;
    double r2;
    if (mixed) {
        // the first correction's right-hand side: the FP32 residual of E^n (the refinement
        // starts from an FP32 solve); every later residual, which decides convergence, is
        // FP64
        int nparts = 0;
        run(h, "resid32", 0, L0.ncell, s, [&] {
            nparts = launch_resid32_init(L0, E, h->d64[0].b, h->d32[0].K, h->d32[0].b,
                                         h->partials, h->norm_blocks, s);
        });
        run(h, "finish_sum", 0, nparts, s,
            [&] { launch_finish_sum(h->partials, nparts, &h->scal->sum, s); });
        FLD_CK(cudaGetLastError());
        rc = read_scalars(h, s, &r2, &err);
        // an FP32 residual at the tolerance is confirmed in FP64 before the solve stops
        if (rc == FLD_OK && !(bnorm > 0 && std::sqrt(r2) / bnorm > h->o.tol))
            rc = residual(h, E, nullptr, nullptr, h->d32[0].b, s, &r2, &err);
    } else {
        rc = residual(h, E, nullptr, nullptr, nullptr, s, &r2, &err);
    }
    if (rc != FLD_OK) return rc;
    double rel = bnorm > 0 ? std::sqrt(r2) / bnorm : 0.0;
    if (st) {
        memset(st, 0, sizeof(*st));
        st->resid_hist[0] = rel;
        st->levels = h->vdepth;
    }
    // mixed refinement on 3D levels: the correction is added inside the residual kernel,
    // out of place, the iterate alternating between E and the level-0 FP64 scratch (free
    // in this mode); it ends in E
    const bool fused = mixed && resid64z_ok(L0, h->norm_blocks);
    // after the first FP64 residual, the later ones may be updated recursively (r - A e in
    // FP32) while the accumulated rounding bound `drift` stays below tol/2 ||b||; the scale
    // of the squared sums is 2^-k with 2^k near the RMS of b
    const bool upd = fused && h->o.resid_update && resid_update_ok(L0, h->norm_blocks);
    int sk = 0;
    if (bnorm > 0 && std::isfinite(bnorm))
        sk = std::max(-100, std::min(100, -std::ilogb(bnorm / std::sqrt((double)L0.ncell))));
    const double rs = std::ldexp(1.0, sk), bs = std::ldexp(1.0, sk - 20);
    const double tolb = h->o.tol * bnorm;
    bool have64 = false;
    double drift = 0.0;
    double* cur = E;
    double* oth = h->d64[0].tmp;
    int cyc = 0;
    rc = FLD_OK;
    while (rel > h->o.tol && cyc < h->o.max_cycles && std::isfinite(rel)) {
        if (fused) {
            rc = vcycle32(h, s);
            if (rc != FLD_OK) break;
            if (upd && have64 && drift <= 0.5 * tolb) {
                double d2 = 0.0, amax = 0.0;
                rc = residual_update(h, cur, oth, rs, bs, s, &r2, &d2, &amax, &err);
                std::swap(cur, oth);
                if (rc != FLD_OK) break;
                // the update's FP32 rounding, and that of x + e in FP64 moved through A
                // (||A||_2 <= its largest row sum, FP32-rounded: 1.01; ||x + e||_2 <= ||b||_2)
                drift += std::sqrt(d2) + 1.01 * std::ldexp(amax, -53) * bnorm;
                // the recursive residual passes and its bound does not: the FP64 residual
                // of the same iterate decides
                if (std::sqrt(r2) <= tolb && std::sqrt(r2) + drift > tolb) {
                    rc = residual(h, cur, nullptr, nullptr, h->d32[0].b, s, &r2, &err);
                    drift = 0.0;
                }
            } else {
                rc = residual(h, cur, h->d32[0].x, oth, h->d32[0].b, s, &r2, &err);
                std::swap(cur, oth);
                have64 = true;
                drift = 0.0;
            }
        } else if (mixed) {
            rc = vcycle32(h, s);
            if (rc != FLD_OK) break;
            run(h, "add_correction", 0, L0.ncell, s,
                [&] { launch_add_correction(L0.ncell, E, h->d32[0].x, s); });
            rc = residual(h, E, nullptr, nullptr, h->d32[0].b, s, &r2, &err);
        } else {
            vcycle<double>(h, h->d64, 0, s);
            rc = residual(h, E, nullptr, nullptr, nullptr, s, &r2, &err);
        }
        if (rc != FLD_OK) break;
        rel = (std::sqrt(r2) + drift) / bnorm;
        ++cyc;
        if (st && cyc < 64) st->resid_hist[cyc] = rel;
    }
    if (cur != E) {
        const cudaError_t ce =
            cudaMemcpyAsync(E, cur, sizeof(double) * L0.ncell, cudaMemcpyDeviceToDevice, s);
        if (rc == FLD_OK && ce != cudaSuccess) rc = cuda_fail(ce);
    }
    if (rc != FLD_OK) return rc;
    if (st) {
        st->cycles = cyc;
        st->rel_resid = rel;
    }
    if (!std::isfinite(rel)) return FLD_ERR_DOMAIN;
    return rel <= h->o.tol ? FLD_OK : FLD_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" {

void fld_default_opts(fld_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = FLD_PREC_FP64;
    o->tol = 1e-10;
    o->max_cycles = 50;
    o->nu1 = 2;
    o->nu2 = 2;
    o->coarse_sweeps = 32;
    o->limiter = FLD_LIMITER_LP;
    o->block = 0;
    o->smoother = 0;
    o->graph = 1;
    o->cluster = 0;
    o->inner = 1;
    o->direct1d = 1;
    o->resid_update = 1;
    o->truncate = 1;
}

fld_status fld_create(fld_handle** out, const fld_grid* g, const fld_opts* o) {
    if (!out) return FLD_ERR_ARG;
    *out = nullptr;
    if (!grid_ok(g)) return FLD_ERR_ARG;
    fld_opts def;
    fld_default_opts(&def);
    if (!o) o = &def;
    if (!opts_ok(o)) return FLD_ERR_ARG;
    fld_handle* h = new (std::nothrow) fld_handle();
    if (!h) return FLD_ERR_NOMEM;
    h->g = *g;
    h->o = *o;
    build_levels(h);
    h->ncell = h->lv[0].ncell;
    // Dirichlet face offsets (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi)
    long long off = 0;
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
            const int kind = s ? g->bc_hi[d] : g->bc_lo[d];
            if (d < g->ndim && kind == FLD_BC_DIRICHLET) {
                h->bc_off[2 * d + s] = off;
                off += h->ncell / g->n[d];
            } else {
                h->bc_off[2 * d + s] = -1;
            }
        }
    fld_status rc = FLD_OK;
    const long long n0 = h->ncell;
    rc = rc ? rc : dalloc(h, &h->d64[0].b, n0);
    rc = rc ? rc : dalloc(h, &h->d64[0].K, n0);
    rc = rc ? rc : dalloc(h, &h->d64[0].tmp, n0);
    for (int l = 1; l < h->nlev && !rc; ++l) {
        const long long n = h->lv[l].ncell;
        rc = rc ? rc : dalloc(h, &h->d64[l].x, n);
        rc = rc ? rc : dalloc(h, &h->d64[l].b, n);
        rc = rc ? rc : dalloc(h, &h->d64[l].K, n);
        rc = rc ? rc : dalloc(h, &h->d64[l].tmp, n);
    }
    for (int l = 0; l < h->nlev && !rc; ++l) {
        const long long n = h->lv[l].ncell;
        rc = rc ? rc : dalloc(h, &h->d32[l].x, n);
        rc = rc ? rc : dalloc(h, &h->d32[l].b, n);
        rc = rc ? rc : dalloc(h, &h->d32[l].K, n);
        rc = rc ? rc : dalloc(h, &h->d32[l].tmp, n);
    }
    for (int q = 0; q < 2 && !rc; ++q) {
        rc = rc ? rc : dalloc(h, &h->dfx[q][0], n0);
        rc = rc ? rc : dalloc(h, &h->dfx[q][1], n0);
        rc = rc ? rc : dalloc(h, &h->dfb[q], n0);
        rc = rc ? rc : dalloc(h, &h->dfK[q], n0);
    }
    rc = rc ? rc : dalloc(h, &h->Dscratch, n0);
    rc = rc ? rc : dalloc(h, &h->krscratch, n0);
    if (g->ndim == 1) rc = rc ? rc : dalloc(h, &h->triw, 12 * n0 + 1);
    h->norm_blocks = NORM_BLOCKS_PER_SM * num_sms();
    rc = rc ? rc : dalloc(h, &h->partials, 3LL * h->norm_blocks);
    rc = rc ? rc : dalloc(h, &h->scal, 1);
    if (!rc && cudaMallocHost(&h->hscal, sizeof(DevScalars)) != cudaSuccess) {
        cudaGetLastError();
        rc = FLD_ERR_NOMEM;
    }
    if (!rc && cudaMemset(h->scal, 0, sizeof(DevScalars)) != cudaSuccess) rc = FLD_ERR_CUDA;
    for (int q = 0; q < 4 && !rc; ++q)
        if (cudaEventCreate(&h->tev[q]) != cudaSuccess) {
            h->tev[q] = nullptr;
            rc = FLD_ERR_CUDA;
        }
    if (!rc) {
        prepare_rb_sweep();
        prepare_vcycle_tail();
        debug_attach_all();
    }
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = FLD_ERR_CUDA;
    if (rc) {
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return FLD_OK;
}

int fld_debug_flags(void) {
#ifdef FLD_DEBUG
    std::lock_guard<std::mutex> lock(g_debug_mu);
    if (!g_debug_word) return 0;
    unsigned v = 0;
    if (cudaMemcpy(&v, g_debug_word, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaMemset(g_debug_word, 0, sizeof(unsigned));
    return (int)v;
#else
    return -1;
#endif
}

fld_status fld_destroy(fld_handle* h) {
    if (!h) return FLD_OK;
    cudaDeviceSynchronize();
    prof_free(h);
    graph_free(h);
    free_all(h);
    delete h;
    return FLD_OK;
}

fld_status fld_set_opts(fld_handle* h, const fld_opts* o) {
    if (!h || !opts_ok(o)) return FLD_ERR_ARG;
    const bool lv_changed = o->face_mean != h->o.face_mean || o->prolong != h->o.prolong;
    h->o = *o;
    if (lv_changed) {
        // the levels carry the face mean and the prolongation kind, and a captured V-cycle
        // holds them by value
        FLD_CK(cudaDeviceSynchronize());
        graph_free(h);
        for (int l = 0; l < h->nlev; ++l) {
            h->lv[l].fm = o->face_mean;
            h->lv[l].pk = o->prolong;
        }
    }
    return FLD_OK;
}

int fld_num_levels(const fld_handle* h) { return h ? h->nlev : 0; }

namespace {
// diagnostics: the energy sum of the block into energy[slot] (device), cell volume applied on
// the host when read
void energy_sum(fld_handle* h, const double* rho, const double* T, const double* E, double cv,
                int slot, cudaStream_t s) {
    run(h, "energy_sum", 0, h->ncell, s, [&] {
        launch_energy_sum(h->ncell, rho, T, E, cv, h->partials, h->norm_blocks, s);
    });
    run(h, "finish_sum", 0, h->norm_blocks, s, [&] {
        launch_finish_sum(h->partials, h->norm_blocks, &h->scal->energy[slot], s);
    });
}

double cell_volume(const fld_handle* h) {
    double v = 1.0;
    for (int d = 0; d < h->g.ndim; ++d) v *= h->g.h[d];
    return v;
}

bool want(const fld_handle* h, const fld_stats* st, int bit) { return st && (h->o.diag & bit); }

// copies the diagnostics out of the scalars read back last (the stream is synchronised)
void fill_diag(fld_handle* h, fld_stats* st, int phases) {
    if (want(h, st, FLD_DIAG_ENERGY)) {
        const double v = cell_volume(h);
        st->energy_before = h->hscal->energy[0] * v;
        st->energy_after = h->hscal->energy[1] * v;
    }
    if (want(h, st, FLD_DIAG_TIMES)) {
        float ms = 0.f;
        // phases: 3 = limiter, solve, exchange (events 0..3); 1 = solve (events 0, 3)
        if (phases == 3) {
            for (int q = 0; q < 3; ++q)
                if (cudaEventElapsedTime(&ms, h->tev[q], h->tev[q + 1]) == cudaSuccess)
                    st->t_ms[q] = ms;
        }
        if (cudaEventElapsedTime(&ms, h->tev[0], h->tev[3]) == cudaSuccess) {
            st->t_ms[3] = ms;
            if (phases == 1) st->t_ms[1] = ms;
        }
        cudaGetLastError();
    }
}

// the limiter of a handle; kr (nullable) receives kappa rho for the exchange of the same step
fld_status limiter_impl(fld_handle* h, const fld_consts* k, const fld_opacity* op, const double* E,
                        const double* rho, const double* T, const double* E_bc, double* D,
                        double* lambda, double* kr, cudaStream_t s) {
    // double-FP32 limiter (MIXED_DF, or the limiter_df option): E split once into FP32
    // pairs (the level-0 FP32 buffers are free until the solve), so the limiter forms the
    // gradient without FP64 arithmetic
    const bool dfmode = h->o.precision == FLD_PREC_MIXED_DF || h->o.limiter_df;
    const bool split = dfmode && h->o.limiter != FLD_LIMITER_DIFFUSION;
    float* Eh = split ? h->d32[0].x : nullptr;
    float* El = split ? h->d32[0].tmp : nullptr;
    if (split)
        run(h, "split_df", 0, h->ncell, s, [&] { launch_split_df(h->ncell, E, Eh, El, s); });
    run(h, "limiter", 0, h->ncell, s, [&] {
        launch_limiter(h->lv[0], h->g.h, E, rho, T, E_bc, h->bc_off, to_op(op), k->c, h->o.limiter,
                       dfmode, D, lambda, &h->scal->err, s, Eh, El, kr);
    });
    FLD_CK(cudaGetLastError());
    return FLD_OK;
}

fld_status exchange_impl(fld_handle* h, const fld_consts* k, const fld_opacity* op, double dt,
                         const double* rho, double* T, double* E, const double* kr,
                         cudaStream_t s) {
    run(h, "exchange", 0, h->ncell, s, [&] {
        launch_exchange(h->ncell, rho, T, E, to_op(op), dt * k->c, k->a_r,
                        k->R_gas / (k->gamma - 1.0), h->o.precision == FLD_PREC_MIXED_DF,
                        &h->scal->err, s, kr);
    });
    FLD_CK(cudaGetLastError());
    return FLD_OK;
}
}  // namespace

fld_status fld_limiter(fld_handle* h, const fld_consts* k, const fld_opacity* op, const double* E,
                       const double* rho, const double* T, const double* E_bc, double* D,
                       double* lambda, void* stream) {
    if (!h || !consts_ok(k) || !op_ok(op) || !E || !rho || !D) return FLD_ERR_ARG;
    if (op->kind != FLD_OPACITY_CONST && !T) return FLD_ERR_ARG;
    if (has_dirichlet(h->g) && !E_bc && h->o.limiter != FLD_LIMITER_DIFFUSION) return FLD_ERR_ARG;
    return limiter_impl(h, k, op, E, rho, T, E_bc, D, lambda, nullptr, (cudaStream_t)stream);
}

fld_status fld_coupling(fld_handle* h, const fld_consts* k, const fld_opacity* op,
                        const double* E, const double* rho, const double* T, const double* E_bc,
                        const double* v, double* F, double* fr, double* f_edd, double* vfr,
                        double* ptire, void* stream) {
    if (!h || !consts_ok(k) || !op_ok(op) || !E || !rho) return FLD_ERR_ARG;
    if (op->kind != FLD_OPACITY_CONST && !T) return FLD_ERR_ARG;
    if (has_dirichlet(h->g) && !E_bc) return FLD_ERR_ARG;
    if ((vfr || ptire) && !v) return FLD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    run(h, "coupling", 0, h->ncell, s, [&] {
        launch_coupling(h->lv[0], h->g.h, E, rho, T, E_bc, h->bc_off, to_op(op), k->c,
                        h->o.limiter, v, F, fr, f_edd, vfr, ptire, &h->scal->err, s);
    });
    FLD_CK(cudaGetLastError());
    return FLD_OK;
}

fld_status fld_diffuse(fld_handle* h, double dt, const double* D, const double* E_bc, double* E,
                       fld_stats* stats, void* stream) {
    if (!h || !D || !E || !(dt > 0) || !std::isfinite(dt)) return FLD_ERR_ARG;
    if (has_dirichlet(h->g) && !E_bc) return FLD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool en = want(h, stats, FLD_DIAG_ENERGY), tm = want(h, stats, FLD_DIAG_TIMES);
    if (!en && !tm) return diffuse_impl(h, dt, D, E_bc, E, stats, s);
    if (tm) FLD_CK(cudaEventRecord(h->tev[0], s));
    if (en) energy_sum(h, nullptr, nullptr, E, 0.0, 0, s);
    const fld_status rs = diffuse_impl(h, dt, D, E_bc, E, stats, s);
    if (rs != FLD_OK && rs != FLD_ERR_NOT_CONVERGED) return rs;
    if (en) energy_sum(h, nullptr, nullptr, E, 0.0, 1, s);
    if (tm) FLD_CK(cudaEventRecord(h->tev[3], s));
    double sum;
    unsigned err;
    const fld_status rc = read_scalars(h, s, &sum, &err);
    if (rc) return rc;
    fill_diag(h, stats, 1);
    return rs;
}

fld_status fld_exchange(fld_handle* h, const fld_consts* k, const fld_opacity* op, double dt,
                        const double* rho, double* T, double* E, void* stream) {
    if (!h || !consts_ok(k) || !op_ok(op) || !rho || !T || !E || !(dt >= 0) || !std::isfinite(dt))
        return FLD_ERR_ARG;
    return exchange_impl(h, k, op, dt, rho, T, E, nullptr, (cudaStream_t)stream);
}

fld_status fld_step(fld_handle* h, const fld_consts* k, const fld_opacity* op, double dt,
                    const double* rho, double* T, double* E, const double* E_bc, fld_stats* stats,
                    void* stream) {
    if (!h || !consts_ok(k) || !op_ok(op) || !rho || !T || !E || !(dt > 0) || !std::isfinite(dt))
        return FLD_ERR_ARG;
    if (has_dirichlet(h->g) && !E_bc) return FLD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool en = want(h, stats, FLD_DIAG_ENERGY), tm = want(h, stats, FLD_DIAG_TIMES);
    const double cv = k->R_gas / (k->gamma - 1.0);
    if (tm) FLD_CK(cudaEventRecord(h->tev[0], s));
    if (en) energy_sum(h, rho, T, E, cv, 0, s);
    // the limiter freezes kappa rho at (rho, T^n) for the exchange (one opacity evaluation
    // per cell and step)
    fld_status rc = limiter_impl(h, k, op, E, rho, T, E_bc, h->Dscratch, nullptr, h->krscratch, s);
    if (rc) return rc;
    if (tm) FLD_CK(cudaEventRecord(h->tev[1], s));
    // a solve that stopped at max_cycles still completes the substep from its last iterate
    // (the status reports it); any other failure stops here
    const fld_status rs = diffuse_impl(h, dt, h->Dscratch, E_bc, E, stats, s);
    if (rs != FLD_OK && rs != FLD_ERR_NOT_CONVERGED) return rs;
    if (tm) FLD_CK(cudaEventRecord(h->tev[2], s));
    rc = exchange_impl(h, k, op, dt, rho, T, E, h->krscratch, s);
    if (rc) return rc;
    if (en) energy_sum(h, rho, T, E, cv, 1, s);
    if (tm) FLD_CK(cudaEventRecord(h->tev[3], s));
    rc = fld_get_status(h, stream);
    if (!rc) fill_diag(h, stats, 3);
    return rc ? rc : rs;
}

}  // extern "C"

long long fld::fld_handle_cells(const fld_handle* h) { return h ? h->ncell : 0; }

extern "C" {

fld_status fld_get_status(fld_handle* h, void* stream) {
    if (!h) return FLD_ERR_ARG;
    double sum;
    unsigned err;
    fld_status rc = read_scalars(h, (cudaStream_t)stream, &sum, &err);
    if (rc) return rc;
    if (err) {
        FLD_CK(cudaMemsetAsync(&h->scal->err, 0, sizeof(unsigned), (cudaStream_t)stream));
        FLD_CK(cudaStreamSynchronize((cudaStream_t)stream));
        if (err & ERRBIT_TIMEOUT) return FLD_ERR_TIMEOUT;
        return FLD_ERR_DOMAIN;
    }
    return FLD_OK;
}

fld_status fld_prof_enable(fld_handle* h, int on, int capacity) {
    if (!h || capacity < 0) return FLD_ERR_ARG;
    FLD_CK(cudaDeviceSynchronize());
    prof_free(h);
    if (!on) return FLD_OK;
    Prof& P = h->prof;
    P.ev.resize(2 * (size_t)capacity);
    for (auto& e : P.ev) FLD_CK(cudaEventCreate(&e));
    P.rec.resize(capacity);
    P.cap = capacity;
    P.used = 0;
    P.on = true;
    return FLD_OK;
}

int fld_prof_read(fld_handle* h, fld_prof_entry* out, int cap) {
    if (!h || !out || cap <= 0) return 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return 0;
    Prof& P = h->prof;
    int nout = 0;
    for (int r = 0; r < P.used; ++r) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, P.ev[2 * r], P.ev[2 * r + 1]);
        int slot = -1;
        for (int q = 0; q < nout; ++q)
            if (out[q].level == P.rec[r].level && strcmp(out[q].name, P.rec[r].name) == 0) slot = q;
        if (slot < 0) {
            if (nout == cap) continue;
            slot = nout++;
            memset(&out[slot], 0, sizeof(out[slot]));
            strncpy(out[slot].name, P.rec[r].name, sizeof(out[slot].name) - 1);
            out[slot].level = P.rec[r].level;
        }
        out[slot].launches += 1;
        out[slot].cells += P.rec[r].cells;
        out[slot].ms += ms;
    }
    return nout;
}

long long fld_launch_count(void) { return g_launches.load(); }

const char* fld_strerror(fld_status s) {
    switch (s) {
        case FLD_OK: return "ok";
        case FLD_ERR_ARG: return "invalid argument";
        case FLD_ERR_DOMAIN: return "non-positive or non-finite field value";
        case FLD_ERR_NOT_CONVERGED: return "multigrid did not reach the tolerance";
        case FLD_ERR_TIMEOUT: return "bounded device wait expired";
        case FLD_ERR_CUDA: return "CUDA runtime error";
        case FLD_ERR_NOMEM: return "device allocation failed";
    }
    return "unknown status";
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free solve
// fld_diffuse_static: the diffusion solve with its whole workspace (level pyramid,
// scratch, reduction buffers, status word) carved from one fixed device array that the
// library defines, so the call itself never allocates device or pinned memory.
namespace {
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)16 << 20;   // 16 MiB on every GPU using it
constexpr long long STATIC_MAX_CELLS = 131072;                // fits the worst-case pyramid
constexpr int STATIC_MAX_DEVICES = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

namespace {
unsigned char* g_static_base[STATIC_MAX_DEVICES];   // device address of the array, per device
fld_handle g_static_handle;                         // host bookkeeping, rebuilt per call
DevScalars g_static_host_scalars;                   // pageable host copy of the device scalars
std::mutex g_static_mutex;
}  // namespace

extern "C" fld_status fld_diffuse_static(const fld_grid* g, const fld_opts* o, double dt,
                                         const double* D, const double* E_bc, double* E,
                                         fld_stats* stats, void* stream) {
    if (!grid_ok(g) || !D || !E || !(dt > 0) || !std::isfinite(dt)) return FLD_ERR_ARG;
    fld_opts def;
    fld_default_opts(&def);
    if (!o) o = &def;
    if (!opts_ok(o)) return FLD_ERR_ARG;
    const long long ncell = (long long)g->n[0] * g->n[1] * g->n[2];
    if (ncell > STATIC_MAX_CELLS) {
        fprintf(stderr, "fld_diffuse_static: %lld cells exceed the %lld-cell limit of the "
                        "static workspace\n", ncell, STATIC_MAX_CELLS);
        return FLD_ERR_ARG;
    }
    if (has_dirichlet(*g) && !E_bc) return FLD_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    int dev = 0;
    FLD_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= STATIC_MAX_DEVICES) return FLD_ERR_ARG;
    if (!g_static_base[dev]) {
        // once per device, with that device current: the host-side symbol is only a
        // stand-in, the kernels need the device address
        void* p = nullptr;
        FLD_CK(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_base[dev] = (unsigned char*)p;
    }
    fld_handle& h = g_static_handle;
    h.g = *g;
    h.o = *o;
    h.o.graph = 0;        // graph capture and instantiation allocate: launch directly
    h.o.direct1d = 0;     // V-cycles in every dimension (the workspace holds no direct solver)
    prepare_rb_sweep();   // kernel attributes only (no device memory)
    prepare_vcycle_tail();
    build_levels(&h);
    h.ncell = h.lv[0].ncell;
    long long off = 0;
    for (int d = 0; d < 3; ++d)
        for (int sd = 0; sd < 2; ++sd) {
            const int kind = sd ? g->bc_hi[d] : g->bc_lo[d];
            if (d < g->ndim && kind == FLD_BC_DIRICHLET) {
                h.bc_off[2 * d + sd] = off;
                off += h.ncell / g->n[d];
            } else {
                h.bc_off[2 * d + sd] = -1;
            }
        }
    size_t used = 0;
    bool fits = true;
    auto take = [&](size_t bytes) -> unsigned char* {
        used = (used + 255) & ~(size_t)255;
        if (used + bytes > STATIC_SCRATCH_BYTES) {
            fits = false;
            return nullptr;
        }
        unsigned char* q = g_static_base[dev] + used;
        used += bytes;
        return q;
    };
    const long long n0 = h.ncell;
    h.d64[0].b = (double*)take(8 * n0);
    h.d64[0].K = (double*)take(8 * n0);
    h.d64[0].tmp = (double*)take(8 * n0);
    for (int l = 1; l < h.nlev; ++l) {
        const long long n = h.lv[l].ncell;
        h.d64[l].x = (double*)take(8 * n);
        h.d64[l].b = (double*)take(8 * n);
        h.d64[l].K = (double*)take(8 * n);
        h.d64[l].tmp = (double*)take(8 * n);
    }
    for (int l = 0; l < h.nlev; ++l) {
        const long long n = h.lv[l].ncell;
        h.d32[l].x = (float*)take(4 * n);
        h.d32[l].b = (float*)take(4 * n);
        h.d32[l].K = (float*)take(4 * n);
        h.d32[l].tmp = (float*)take(4 * n);
    }
    for (int q = 0; q < 2; ++q) {
        h.dfx[q][0] = (float*)take(4 * n0);
        h.dfx[q][1] = (float*)take(4 * n0);
        h.dfb[q] = (float*)take(4 * n0);
        h.dfK[q] = (float*)take(4 * n0);
    }
    h.norm_blocks = NORM_BLOCKS_PER_SM * num_sms();
    h.partials = (double*)take(24 * (size_t)h.norm_blocks);
    h.scal = (DevScalars*)take(sizeof(DevScalars));
    if (!fits) return FLD_ERR_ARG;
    h.Dscratch = nullptr;
    h.hscal = &g_static_host_scalars;
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear the status word and sums
    FLD_CK(cudaMemsetAsync(h.scal, 0, sizeof(DevScalars), s));
    const fld_status rc = diffuse_impl(&h, dt, D, E_bc, E, stats, s);
    // the write-back of the double-FP32 iterate is enqueued after the last read-back: wait
    // for it, so that no kernel of this call still uses the array once the lock is released
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    return rc;
}
