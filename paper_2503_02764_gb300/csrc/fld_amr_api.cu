// Host side of the composite-grid diffusion solve (include/fld.h, fld_amr_*): a coarse
// block with one box refined by 2, solved by a two-level scheme whose coarse correction is
// the uniform multigrid solver of a handle on the coarse block (k_amr.cu has the operator).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fld_amr.cuh"

using namespace fld;

struct fld_amr {
    fld_grid g;
    fld_patch patch;
    fld_opts o;
    AmrGeom G;
    fld_handle* hc = nullptr;         // coarse block: the correction solves
    long long nC = 0, nF = 0;
    int nblk = 0;
    double *bc = nullptr, *bf = nullptr, *rc = nullptr, *rf = nullptr;
    double *eH = nullptr, *DH = nullptr, *zero_faces = nullptr, *partials = nullptr;
    double *sum = nullptr, *hsum = nullptr;   // device scalar, pinned host copy
    std::vector<void*> allocs;
};

namespace {

constexpr int AMR_SWEEPS = 2;          // composite red-black sweeps after each correction
constexpr double AMR_COARSE_TOL = 1e-6;

bool dal(fld_amr* a, double** q, long long n) {
    void* m = nullptr;
    if (cudaMalloc(&m, sizeof(double) * (size_t)std::max<long long>(n, 1)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    a->allocs.push_back(m);
    *q = (double*)m;
    return true;
}

void destroy(fld_amr* a) {
    if (!a) return;
    for (void* q : a->allocs) cudaFree(q);
    if (a->hsum) cudaFreeHost(a->hsum);
    if (a->hc) fld_destroy(a->hc);
    delete a;
}

fld_status ck(cudaError_t e) {
    if (e == cudaSuccess) return FLD_OK;
    fprintf(stderr, "fld: CUDA error: %s\n", cudaGetErrorString(e));
    return FLD_ERR_CUDA;
}

// sum of the partials on the device, read back (synchronises the stream)
fld_status reduce(fld_amr* a, int nparts, cudaStream_t s, double* out) {
    launch_finish_sum(a->partials, nparts, a->sum, s);
    note_launches(1);
    fld_status rc = ck(cudaMemcpyAsync(a->hsum, a->sum, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (rc) return rc;
    rc = ck(cudaStreamSynchronize(s));
    *out = *a->hsum;
    return rc;
}

}  // namespace

extern "C" {

fld_status fld_amr_create(fld_amr** out, const fld_grid* g, const fld_patch* patch,
                          const fld_opts* o) {
    if (!out) return FLD_ERR_ARG;
    *out = nullptr;
    if (!grid_valid(g) || !patch) return FLD_ERR_ARG;
    fld_opts def;
    fld_default_opts(&def);
    if (!o) o = &def;
    // the composite operator uses the arithmetic face mean
    if (!opts_valid(o) || o->face_mean != FLD_FACE_ARITH) return FLD_ERR_ARG;
    AmrGeom G;
    memset(&G, 0, sizeof(G));
    G.nd = g->ndim;
    long long nF = 1;
    for (int d = 0; d < 3; ++d) {
        G.nc[d] = g->n[d];
        if (d < g->ndim) {
            const int n = g->n[d], lo = patch->lo[d], hi = patch->hi[d];
            const bool full = lo == 0 && hi == n;
            const bool inside = lo >= 1 && lo < hi && hi <= n - 1;
            if (!(full || inside)) return FLD_ERR_ARG;
            // the composite red-black sweep needs even periodic extents
            if (g->bc_lo[d] == FLD_BC_PERIODIC && (n & 1)) return FLD_ERR_ARG;
            G.lo[d] = lo;
            G.hi[d] = hi;
            G.nf[d] = 2 * (hi - lo);
            G.bclo[d] = g->bc_lo[d];
            G.bchi[d] = g->bc_hi[d];
            G.H[d] = g->h[d];
        } else {
            G.lo[d] = 0;
            G.hi[d] = 1;
            G.nf[d] = 1;
            G.bclo[d] = G.bchi[d] = FLD_BC_PERIODIC;
            G.H[d] = 1.0;
        }
        nF *= G.nf[d];
    }
    if (nF >= (1LL << 31)) return FLD_ERR_ARG;
    long long off = 0, nfaces = 0;
    const long long nC = (long long)g->n[0] * g->n[1] * g->n[2];
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
            const int kind = s ? g->bc_hi[d] : g->bc_lo[d];
            if (d < g->ndim && kind == FLD_BC_DIRICHLET) {
                G.bcoff[2 * d + s] = off;
                off += nC / g->n[d];
            } else {
                G.bcoff[2 * d + s] = -1;
            }
        }
    nfaces = off;
    fld_amr* a = new (std::nothrow) fld_amr();
    if (!a) return FLD_ERR_NOMEM;
    a->g = *g;
    a->patch = *patch;
    a->o = *o;
    a->G = G;
    a->nC = nC;
    a->nF = nF;
    a->nblk = num_sms() * 8;
    fld_opts oc = *o;
    oc.tol = AMR_COARSE_TOL;
    oc.max_cycles = 30;
    fld_status rc = fld_create(&a->hc, g, &oc);
    if (rc != FLD_OK) {
        a->hc = nullptr;
        destroy(a);
        return rc;
    }
    bool ok = dal(a, &a->bc, nC) && dal(a, &a->bf, nF) && dal(a, &a->rc, nC) &&
              dal(a, &a->rf, nF) && dal(a, &a->eH, nC) && dal(a, &a->DH, nC) &&
              dal(a, &a->zero_faces, nfaces) && dal(a, &a->partials, a->nblk) &&
              dal(a, &a->sum, 1);
    if (ok && cudaMallocHost(&a->hsum, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        a->hsum = nullptr;
        ok = false;
    }
    if (!ok) {
        destroy(a);
        return FLD_ERR_NOMEM;
    }
    if (cudaMemset(a->zero_faces, 0, sizeof(double) * (size_t)std::max<long long>(nfaces, 1)) !=
            cudaSuccess ||
        cudaMemset(a->rc, 0, sizeof(double) * nC) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        destroy(a);
        return FLD_ERR_CUDA;
    }
    *out = a;
    return FLD_OK;
}

fld_status fld_amr_destroy(fld_amr* a) {
    if (!a) return FLD_OK;
    cudaDeviceSynchronize();
    destroy(a);
    return FLD_OK;
}

fld_status fld_amr_diffuse(fld_amr* a, double dt, const double* Dc, const double* Df,
                           const double* E_bc, double* Ec, double* Ef, fld_stats* st,
                           void* stream) {
    if (!a || !Dc || !Df || !Ec || !Ef || !(dt > 0) || !std::isfinite(dt)) return FLD_ERR_ARG;
    bool dir = false;
    for (int q = 0; q < 6; ++q) dir |= a->G.bcoff[q] >= 0;
    if (dir && !E_bc) return FLD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    AmrGeom& G = a->G;
    G.dt = dt;
    launch_amr_setup(G, Dc, Df, Ec, Ef, E_bc, a->bc, a->bf, a->DH, s);
    launch_sumsq(a->nC, a->bc, a->partials, a->nblk, s);
    note_launches(2);
    double b2c = 0.0, b2f = 0.0;
    fld_status rc = reduce(a, a->nblk, s, &b2c);
    if (rc) return rc;
    launch_sumsq(a->nF, a->bf, a->partials, a->nblk, s);
    note_launches(1);
    rc = reduce(a, a->nblk, s, &b2f);
    if (rc) return rc;
    const double bnorm = std::sqrt(b2c + b2f);
    if (st) {
        memset(st, 0, sizeof(*st));
        st->levels = fld_num_levels(a->hc) + 1;
    }
    int cyc = 0;
    double rel = 0.0;
    for (;;) {
        const int nb = launch_amr_resid(G, Dc, Df, a->bc, a->bf, Ec, Ef, a->rc, a->rf,
                                        a->partials, a->nblk, s);
        note_launches(1);
        double r2;
        rc = reduce(a, nb, s, &r2);
        if (rc) return rc;
        rel = bnorm > 0 ? std::sqrt(r2) / bnorm : 0.0;
        if (st && cyc < 64) st->resid_hist[cyc] = rel;
        if (!(rel > a->o.tol) || cyc >= a->o.max_cycles || !std::isfinite(rel)) break;
        // coarse correction: the restricted residual on the whole block, solved by the
        // block's multigrid (homogeneous walls), added on the composite grid
        launch_amr_average(G, a->rf, a->rc, s);
        rc = ck(cudaMemcpyAsync(a->eH, a->rc, sizeof(double) * a->nC, cudaMemcpyDeviceToDevice,
                                s));
        if (rc) return rc;
        note_launches(1);
        const fld_status cs = fld_diffuse(a->hc, dt, a->DH, a->zero_faces, a->eH, nullptr, stream);
        if (cs != FLD_OK && cs != FLD_ERR_NOT_CONVERGED) return cs;
        launch_amr_correct(G, a->eH, Ec, Ef, s);
        note_launches(1);
        for (int i = 0; i < AMR_SWEEPS; ++i)
            for (int ph = 0; ph < 4; ++ph) launch_amr_smooth(G, ph, Dc, Df, a->bc, a->bf, Ec, Ef, s);
        note_launches(4 * AMR_SWEEPS);
        ++cyc;
    }
    // covered coarse cells: the mean of their fine cells
    launch_amr_average(G, Ef, Ec, s);
    note_launches(1);
    rc = ck(cudaGetLastError());
    if (rc) return rc;
    rc = ck(cudaStreamSynchronize(s));
    if (rc) return rc;
    if (st) {
        st->cycles = cyc;
        st->rel_resid = rel;
    }
    if (!std::isfinite(rel)) return FLD_ERR_DOMAIN;
    return rel <= a->o.tol ? FLD_OK : FLD_ERR_NOT_CONVERGED;
}

}  // extern "C"
