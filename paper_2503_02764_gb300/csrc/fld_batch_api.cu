// Host side of the batched substep (fld_batch_* and fld_step_batched in include/fld.h):
// per-problem level pyramids and workspace offsets, the size-ordered work queue, and
// the CUDA-graph capture of the step's launch sequence.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "fld_batch.cuh"

using namespace fld;

struct fld_batch {
    int nprob = 0;
    fld_opts o{};
    std::vector<fld_grid> grids;
    std::vector<BProb> hp;
    long long ncell = 0, nface = 0, wsd_n = 0, wsf_n = 0;
    BProb* dprobs = nullptr;
    BDyn* ddyn = nullptr;
    BDyn* hdyn = nullptr;          // pinned staging of the per-call data
    int* dorder = nullptr;
    int* dqueue = nullptr;
    BatchStat* dstats = nullptr;
    BatchStat* hstats = nullptr;   // pinned
    unsigned* derr = nullptr;
    unsigned* herr = nullptr;      // pinned
    double* wsd = nullptr;
    float* wsf = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    unsigned char gkey[256];
    size_t gkey_len = 0;
};

namespace {

fld_status batch_fail(cudaError_t e) {
    fprintf(stderr, "fld_batch: CUDA error: %s\n", cudaGetErrorString(e));
    return FLD_ERR_CUDA;
}

#define BCK(call)                                      \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return batch_fail(e_); \
    } while (0)

void batch_free(fld_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    void* dev[] = {b->dprobs, b->ddyn, b->dorder, b->dqueue, b->dstats, b->derr, b->wsd, b->wsf};
    for (void* p : dev)
        if (p) cudaFree(p);
    void* host[] = {b->hdyn, b->hstats, b->herr};
    for (void* p : host)
        if (p) cudaFreeHost(p);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->cs) cudaStreamDestroy(b->cs);
}

int block_threads(const fld_opts& o) { return o.block ? o.block : 512; }

bool batch_opts_ok(const fld_opts* o) {
    // the batched kernels use the arithmetic face mean and linear prolongation
    return fld::opts_valid(o) && o->face_mean == FLD_FACE_ARITH &&
           o->prolong == FLD_PROLONG_LINEAR &&
           (o->block == 0 || batch_threads_supported(o->block));
}

// blocks per problem: the option, or the smallest cluster giving the largest problem
// at most 64 cells per thread
int cluster_size(const fld_batch* b, int nt) {
    if (b->o.cluster) return b->o.cluster;
    long long mx = 0;
    for (const BProb& P : b->hp) mx = std::max(mx, P.lv[0].ncell);
    int cs = 1;
    while (cs < 8 && mx > 64LL * cs * nt) cs *= 2;
    return cs;
}

// enqueue the step's launch sequence on b->cs
void enqueue(fld_batch* b, const BatchParams& prm, const double* rho, double* T, double* E,
             const double* Ebc, int nt, int cl, int ngroups) {
    cudaMemcpyAsync(b->ddyn, b->hdyn, sizeof(BDyn) * b->nprob, cudaMemcpyHostToDevice, b->cs);
    cudaMemsetAsync(b->dqueue, 0, sizeof(int), b->cs);
    cudaMemsetAsync(b->derr, 0, sizeof(unsigned), b->cs);
    launch_batch_step(nt, cl, ngroups, b->dprobs, b->ddyn, b->dorder, b->nprob, b->dqueue, prm,
                      rho, T, E, Ebc, b->wsd, b->wsf, b->dstats, b->derr, b->cs);
    cudaMemcpyAsync(b->hstats, b->dstats, sizeof(BatchStat) * b->nprob, cudaMemcpyDeviceToHost,
                    b->cs);
    cudaMemcpyAsync(b->herr, b->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, b->cs);
}

}  // namespace

extern "C" {

fld_status fld_batch_create(fld_batch** out, int nprob, const fld_grid* grids, const fld_opts* o) {
    if (!out || nprob < 1 || !grids) return FLD_ERR_ARG;
    *out = nullptr;
    fld_opts def;
    fld_default_opts(&def);
    if (!o) o = &def;
    if (!batch_opts_ok(o)) return FLD_ERR_ARG;
    for (int p = 0; p < nprob; ++p) {
        if (!fld::grid_valid(&grids[p])) return FLD_ERR_ARG;
        if ((long long)grids[p].n[0] * grids[p].n[1] * grids[p].n[2] > (1LL << 27)) return FLD_ERR_ARG;
    }
    fld_batch* b = new (std::nothrow) fld_batch();
    if (!b) return FLD_ERR_NOMEM;
    b->nprob = nprob;
    b->o = *o;
    b->grids.assign(grids, grids + nprob);
    b->hp.resize(nprob);
    for (int p = 0; p < nprob; ++p) {
        const fld_grid& g = grids[p];
        BProb& P = b->hp[p];
        memset(&P, 0, sizeof(P));
        P.nlev = make_levels(g, P.lv, P.kdown, BMAXL);
        for (int d = 0; d < 3; ++d) P.h[d] = d < g.ndim ? g.h[d] : 1.0;
        const long long n0 = P.lv[0].ncell;
        P.cell_off = b->ncell;
        b->ncell += n0;
        long long nf = 0;
        for (int d = 0; d < 3; ++d)
            for (int s = 0; s < 2; ++s) {
                const int kind = s ? g.bc_hi[d] : g.bc_lo[d];
                if (d < g.ndim && kind == FLD_BC_DIRICHLET) {
                    P.bc_off[2 * d + s] = nf;
                    nf += n0 / g.n[d];
                } else {
                    P.bc_off[2 * d + s] = -1;
                }
            }
        P.ebc_off = nf ? b->nface : -1;
        b->nface += nf;
        P.ws_d = b->wsd_n;
        b->wsd_n += 4 * n0;                   // D, and the FP64 refinement's x, b, K
        long long f = 6 * n0;                 // double-FP32 x, b, K (hi and lo)
        for (int l = 0; l < P.nlev; ++l) {
            P.o32[l] = f;
            f += 4 * P.lv[l].ncell;           // x, b, K, t per level
        }
        P.ws_f = b->wsf_n;
        b->wsf_n += f;
    }
    std::vector<int> order(nprob);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return b->hp[a].lv[0].ncell > b->hp[c].lv[0].ncell;
    });
    bool ok = true;
    auto dal = [&](void** p, size_t bytes) {
        if (ok && cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        }
    };
    auto hal = [&](void** p, size_t bytes) {
        if (ok && cudaMallocHost(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        }
    };
    dal((void**)&b->dprobs, sizeof(BProb) * nprob);
    dal((void**)&b->ddyn, sizeof(BDyn) * nprob);
    dal((void**)&b->dorder, sizeof(int) * nprob);
    dal((void**)&b->dqueue, sizeof(int));
    dal((void**)&b->dstats, sizeof(BatchStat) * nprob);
    dal((void**)&b->derr, sizeof(unsigned));
    dal((void**)&b->wsd, sizeof(double) * b->wsd_n);
    dal((void**)&b->wsf, sizeof(float) * b->wsf_n);
    hal((void**)&b->hdyn, sizeof(BDyn) * nprob);
    hal((void**)&b->hstats, sizeof(BatchStat) * nprob);
    hal((void**)&b->herr, sizeof(unsigned));
    if (ok && cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) != cudaSuccess) ok = false;
    if (ok && cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (ok && cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (ok && cudaMemcpy(b->dprobs, b->hp.data(), sizeof(BProb) * nprob, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
    if (ok && cudaMemcpy(b->dorder, order.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        delete b;
        return FLD_ERR_NOMEM;
    }
    *out = b;
    return FLD_OK;
}

fld_status fld_batch_destroy(fld_batch* b) {
    if (!b) return FLD_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
    return FLD_OK;
}

fld_status fld_batch_set_opts(fld_batch* b, const fld_opts* o) {
    if (!b || !batch_opts_ok(o)) return FLD_ERR_ARG;
    b->o = *o;
    return FLD_OK;
}

long long fld_batch_cells(const fld_batch* b) { return b ? b->ncell : 0; }

fld_status fld_step_batched(fld_batch* b, const fld_consts* k, const fld_opacity* ops,
                            const double* dt, const double* rho, double* T, double* E,
                            const double* E_bc, fld_batch_stat* stats, void* stream) {
    if (!b || !k || !ops || !dt || !rho || !T || !E) return FLD_ERR_ARG;
    if (!(k->c > 0 && k->a_r > 0 && k->gamma > 1 && k->R_gas > 0)) return FLD_ERR_ARG;
    if (b->nface > 0 && !E_bc) return FLD_ERR_ARG;
    for (int p = 0; p < b->nprob; ++p) {
        if (!(dt[p] > 0) || !std::isfinite(dt[p])) return FLD_ERR_ARG;
        if (!(ops[p].kind == FLD_OPACITY_CONST || ops[p].kind == FLD_OPACITY_POWER) ||
            !(ops[p].kappa0 > 0))
            return FLD_ERR_ARG;
        b->hdyn[p].dt = dt[p];
        b->hdyn[p].op = Opacity{};
        b->hdyn[p].op.kind = ops[p].kind;
        b->hdyn[p].op.kappa0 = ops[p].kappa0;
        b->hdyn[p].op.a_rho = ops[p].a_rho;
        b->hdyn[p].op.a_T = ops[p].a_T;
    }
    BatchParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.c = k->c;
    prm.a_r = k->a_r;
    prm.cv = k->R_gas / (k->gamma - 1.0);
    prm.tol = b->o.tol;
    prm.max_cycles = b->o.max_cycles;
    prm.nu1 = b->o.nu1;
    prm.nu2 = b->o.nu2;
    prm.coarse_sweeps = b->o.coarse_sweeps;
    prm.limiter = b->o.limiter;
    prm.inner = b->o.inner > 0 ? b->o.inner : 1;
    prm.fp64 = b->o.precision == FLD_PREC_MIXED_DF ? 0 : 1;
    const int nt = block_threads(b->o);
    const int cl = cluster_size(b, nt);
    const int maxg = batch_max_groups(nt, cl);
    if (maxg < 1) return FLD_ERR_ARG;          // this block/cluster shape cannot be resident
    const int ngroups = std::min(b->nprob, maxg);
    cudaStream_t s = (cudaStream_t)stream;
    BCK(cudaEventRecord(b->ev_in, s));
    BCK(cudaStreamWaitEvent(b->cs, b->ev_in, 0));
    if (b->o.graph) {
        unsigned char key[256];
        size_t kl = 0;
        auto put = [&](const void* v, size_t n) {
            memcpy(key + kl, v, n);
            kl += n;
        };
        put(&rho, sizeof(rho));
        put(&T, sizeof(T));
        put(&E, sizeof(E));
        put(&E_bc, sizeof(E_bc));
        put(&prm, sizeof(prm));
        put(&nt, sizeof(nt));
        put(&cl, sizeof(cl));
        put(&ngroups, sizeof(ngroups));
        if (!b->gexec || kl != b->gkey_len || memcmp(key, b->gkey, kl) != 0) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            BCK(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
            enqueue(b, prm, rho, T, E, E_bc, nt, cl, ngroups);
            BCK(cudaStreamEndCapture(b->cs, &g));
            cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->gexec = nullptr;
                return batch_fail(e);
            }
            memcpy(b->gkey, key, kl);
            b->gkey_len = kl;
        }
        BCK(cudaGraphLaunch(b->gexec, b->cs));
    } else {
        enqueue(b, prm, rho, T, E, E_bc, nt, cl, ngroups);
        BCK(cudaGetLastError());
    }
    BCK(cudaEventRecord(b->ev_out, b->cs));
    BCK(cudaStreamWaitEvent(s, b->ev_out, 0));
    BCK(cudaEventSynchronize(b->ev_out));
    if (stats)
        for (int p = 0; p < b->nprob; ++p) {
            stats[p].cycles = b->hstats[p].cycles;
            stats[p].rel_resid = b->hstats[p].rel_resid;
            stats[p].rel_resid0 = b->hstats[p].rel_resid0;
        }
    const unsigned err = *b->herr;
    if (err & ERRBIT_DOMAIN) return FLD_ERR_DOMAIN;
    if (err & ERRBIT_NOTCONV) return FLD_ERR_NOT_CONVERGED;
    return FLD_OK;
}

}  // extern "C"
