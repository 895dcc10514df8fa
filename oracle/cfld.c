/*
 * cfld.c - plain C restatement of the FLD radiation substep, the timed CPU baseline.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle. Built by the package's build step
 * into oracle/_build/libcfld.so and loaded through oracle/cfld.py by the tests (which pin
 * it to oracle/fld.py) and by the benchmark's CPU-baseline leg; the library never uses
 * it. FP64 throughout; loops over planes run on OpenMP threads when it is built with
 * OpenMP.
 *
 * The same definitions as oracle/fld.py (paper: Sect. 2 and Sect. 3):
 *   limiter   grad E by the 4th-order 5-point central difference per axis (Sect. 3),
 *             R = |grad E| / (kappa rho E) (Eq. fld_R), lambda = (2 + R)/(6 + 3R + R^2)
 *             (Eq. fld_lambda), D = c lambda / (kappa rho) (Eq. fld_F); ghost values:
 *             periodic wrap, Neumann even mirror, Dirichlet odd reflection about E_b;
 *   diffuse   backward Euler on the div F term of Eq. mhd_r_e:
 *             (A x)_p = x_p + sum_faces (dt/h_d^2) (D_p + D_q)/2 (x_p - x_q)
 *                       + sum_Dirichlet (dt/h_d^2) 2 D_p (x_p - E_b) = E^n_p,
 *             solved to ||b - A x||_2 <= tol ||b||_2 by a plain geometric-multigrid
 *             V-cycle (red-black Gauss-Seidel, averaging restriction, piecewise-constant
 *             prolongation, many sweeps on the coarsest level; an axis is halved while
 *             its extent is even and >= 4) or by Jacobi-preconditioned conjugate
 *             gradients;
 *   exchange  backward Euler on de/dt = +qdot, dE/dt = -qdot (Eqs. heating, qdot):
 *             alpha T' + beta T'^4 = q with alpha = rho c_v, beta = a_r chi/(1 + chi),
 *             q = alpha T + chi E/(1 + chi), chi = dt c kappa rho, by Newton from the
 *             upper bound min(q/alpha, (q/beta)^(1/4)) (monotone for this convex
 *             increasing quartic), then E' = (E + chi a_r T'^4)/(1 + chi);
 *   the substep: limiter -> diffuse -> exchange, kappa frozen at (rho, T^n).
 * Arrays are x fastest; absent axes have n = 1; Dirichlet face values are packed side
 * after side (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi), each face row-major over the two
 * other axes (lower axis fastest).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXLEV 24
enum { PER = 0, NEU = 1, DIR = 2 };

typedef struct {
    int n[3];
    long long nc;
    double w[3];        /* dt / H_d^2 at this level (0 for absent axes) */
    int lo[3], hi[3];
    double *x, *b, *K, *r;
} lvl_t;

typedef struct {
    int ndim;
    int nlev;
    lvl_t L[MAXLEV];
    int serial;         /* an odd periodic extent: same-colour cells touch, sweep serially */
} mg_t;

int cfld_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static long long idx(const int* n, int i, int j, int k) {
    return ((long long)k * n[1] + j) * n[0] + i;
}

/* neighbour of cell c along axis d at offset s (+-1): its index, or -1 at a wall */
static long long nbr(const lvl_t* L, int i, int j, int k, int d, int s) {
    int c[3] = {i, j, k};
    int m = c[d] + s;
    if (m < 0 || m >= L->n[d]) {
        if ((s < 0 ? L->lo[d] : L->hi[d]) != PER) return -1;
        m = (m + L->n[d]) % L->n[d];
    }
    c[d] = m;
    return idx(L->n, c[0], c[1], c[2]);
}

/* off-diagonal sum  sum_q w_f x_q  and the diagonal 1 + sum_f w_f (+ Dirichlet) at cell p */
static void row(const lvl_t* L, int ndim, const double* x, int i, int j, int k, double* diag,
                double* off) {
    const long long p = idx(L->n, i, j, k);
    double dg = 1.0, of = 0.0;
    for (int d = 0; d < ndim; ++d)
        for (int s = -1; s <= 1; s += 2) {
            const long long q = nbr(L, i, j, k, d, s);
            if (q >= 0) {
                const double wf = L->w[d] * 0.5 * (L->K[p] + L->K[q]);
                dg += wf;
                of += wf * x[q];
            } else if ((s < 0 ? L->lo[(d)] : L->hi[d]) == DIR) {
                dg += 2.0 * L->w[d] * L->K[p];
            }
        }
    *diag = dg;
    *off = of;
}

static void gs_colour(mg_t* M, lvl_t* L, int colour) {
    const int nz = L->n[2], ny = L->n[1], nx = L->n[0];
#pragma omp parallel for schedule(static) if (!M->serial)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = (colour + j + k) & 1; i < nx; i += 2) {
                double dg, of;
                row(L, M->ndim, L->x, i, j, k, &dg, &of);
                const long long p = idx(L->n, i, j, k);
                L->x[p] = (L->b[p] + of) / dg;
            }
}

static void smooth(mg_t* M, lvl_t* L, int sweeps) {
    for (int s = 0; s < sweeps; ++s) {
        gs_colour(M, L, 0);
        gs_colour(M, L, 1);
    }
}

/* r = b - A x; returns ||r||_2^2 */
static double residual(mg_t* M, lvl_t* L) {
    const int nz = L->n[2], ny = L->n[1], nx = L->n[0];
    double s2 = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s2)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double dg, of;
                row(L, M->ndim, L->x, i, j, k, &dg, &of);
                const long long p = idx(L->n, i, j, k);
                const double r = L->b[p] - (dg * L->x[p] - of);
                L->r[p] = r;
                s2 += r * r;
            }
    return s2;
}

/* coarse-cell children range along each axis */
static int halves(const lvl_t* F, const lvl_t* C, int d) { return F->n[d] != C->n[d]; }

static void restrict_to(const lvl_t* F, lvl_t* C, const double* src, double* dst) {
    const int hx = halves(F, C, 0), hy = halves(F, C, 1), hz = halves(F, C, 2);
    const double inv = 1.0 / (double)((1 << hx) * (1 << hy) * (1 << hz));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < C->n[2]; ++k)
        for (int j = 0; j < C->n[1]; ++j)
            for (int i = 0; i < C->n[0]; ++i) {
                double s = 0.0;
                for (int c = 0; c <= hz; ++c)
                    for (int b = 0; b <= hy; ++b)
                        for (int a = 0; a <= hx; ++a)
                            s += src[idx(F->n, (i << hx) + a, (j << hy) + b, (k << hz) + c)];
                dst[idx(C->n, i, j, k)] = s * inv;
            }
}

static void prolong_add(lvl_t* F, const lvl_t* C) {
    const int hx = halves(F, C, 0), hy = halves(F, C, 1), hz = halves(F, C, 2);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < F->n[2]; ++k)
        for (int j = 0; j < F->n[1]; ++j)
            for (int i = 0; i < F->n[0]; ++i)
                F->x[idx(F->n, i, j, k)] += C->x[idx(C->n, i >> hx, j >> hy, k >> hz)];
}

static void vcycle(mg_t* M, int l, int nu1, int nu2) {
    lvl_t* L = &M->L[l];
    if (l == M->nlev - 1) {
        smooth(M, L, 64);
        return;
    }
    lvl_t* C = &M->L[l + 1];
    smooth(M, L, nu1);
    residual(M, L);
    restrict_to(L, C, L->r, C->b);
    memset(C->x, 0, sizeof(double) * C->nc);
    vcycle(M, l + 1, nu1, nu2);
    prolong_add(L, C);
    smooth(M, L, nu2);
}

static int mg_build(mg_t* M, int ndim, const int* n, const double* h, const int* lo,
                    const int* hi, double dt, const double* D) {
    memset(M, 0, sizeof(*M));
    M->ndim = ndim;
    lvl_t L;
    memset(&L, 0, sizeof(L));
    for (int d = 0; d < 3; ++d) {
        L.n[d] = n[d];
        L.lo[d] = d < ndim ? lo[d] : PER;
        L.hi[d] = d < ndim ? hi[d] : PER;
        L.w[d] = d < ndim ? dt / (h[d] * h[d]) : 0.0;
        if (d < ndim && lo[d] == PER && (n[d] & 1)) M->serial = 1;
    }
    for (;;) {
        L.nc = (long long)L.n[0] * L.n[1] * L.n[2];
        L.x = calloc(L.nc, sizeof(double));
        L.b = calloc(L.nc, sizeof(double));
        L.K = calloc(L.nc, sizeof(double));
        L.r = calloc(L.nc, sizeof(double));
        if (!L.x || !L.b || !L.K || !L.r) return -1;
        M->L[M->nlev++] = L;
        int can = 0;
        for (int d = 0; d < ndim; ++d) can |= (L.n[d] >= 4 && !(L.n[d] & 1));
        if (!can || L.nc <= 64 || M->nlev == MAXLEV) break;
        for (int d = 0; d < ndim; ++d)
            if (L.n[d] >= 4 && !(L.n[d] & 1)) {
                L.n[d] /= 2;
                L.w[d] /= 4.0;
            }
    }
    memcpy(M->L[0].K, D, sizeof(double) * M->L[0].nc);
    for (int l = 0; l + 1 < M->nlev; ++l)
        restrict_to(&M->L[l], &M->L[l + 1], M->L[l].K, M->L[l + 1].K);
    return 0;
}

static void mg_free(mg_t* M) {
    for (int l = 0; l < M->nlev; ++l) {
        free(M->L[l].x);
        free(M->L[l].b);
        free(M->L[l].K);
        free(M->L[l].r);
    }
}

/* b = E + Dirichlet face terms 2 (dt/h_d^2) D_p E_b */
static void rhs(const lvl_t* L, int ndim, const double* E, const double* D, const double* Ebc,
                double* b) {
    memcpy(b, E, sizeof(double) * L->nc);
    long long off = 0;
    for (int d = 0; d < ndim; ++d)
        for (int s = 0; s < 2; ++s) {
            if ((s ? L->hi[d] : L->lo[d]) != DIR) continue;
            const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
            for (int v = 0; v < L->n[a2]; ++v)
                for (int u = 0; u < L->n[a1]; ++u) {
                    int c[3];
                    c[d] = s ? L->n[d] - 1 : 0;
                    c[a1] = u;
                    c[a2] = v;
                    const long long p = idx(L->n, c[0], c[1], c[2]);
                    b[p] += 2.0 * L->w[d] * D[p] * Ebc[off + (long long)v * L->n[a1] + u];
                }
            off += (long long)L->n[a1] * L->n[a2];
        }
}

static double norm2(const double* v, long long n) {
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (long long p = 0; p < n; ++p) s += v[p] * v[p];
    return s;
}

/* Solve A E^{n+1} = E^n + g in place. method 0: V(nu1, nu2) cycles; 1: Jacobi-PCG.
   Returns 0 (converged), 1 (not converged within max_it), -1 (allocation). */
int cfld_diffuse(int ndim, const int* n, const double* h, const int* lo, const int* hi,
                 const double* Ebc, double dt, const double* D, double* E, int method,
                 double tol, int max_it, int nu1, int nu2, double* rel_out, int* it_out) {
    mg_t M;
    if (mg_build(&M, ndim, n, h, lo, hi, dt, D)) {
        mg_free(&M);
        return -1;
    }
    lvl_t* L = &M.L[0];
    const long long nc = L->nc;
    rhs(L, ndim, E, D, Ebc, L->b);
    memcpy(L->x, E, sizeof(double) * nc);
    const double bn = sqrt(norm2(L->b, nc));
    double rel = sqrt(residual(&M, L)) / (bn > 0 ? bn : 1.0);
    int it = 0;
    if (method == 0) {
        while (rel > tol && it < max_it) {
            vcycle(&M, 0, nu1, nu2);
            rel = sqrt(residual(&M, L)) / bn;
            ++it;
        }
    } else {
        double *z = malloc(sizeof(double) * nc), *pv = malloc(sizeof(double) * nc),
               *Ap = malloc(sizeof(double) * nc), *dinv = malloc(sizeof(double) * nc);
        if (!z || !pv || !Ap || !dinv) {
            free(z), free(pv), free(Ap), free(dinv);
            mg_free(&M);
            return -1;
        }
        double rz = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rz)
        for (int k = 0; k < L->n[2]; ++k)
            for (int j = 0; j < L->n[1]; ++j)
                for (int i = 0; i < L->n[0]; ++i) {
                    double dg, of;
                    row(L, ndim, L->x, i, j, k, &dg, &of);
                    const long long p = idx(L->n, i, j, k);
                    dinv[p] = 1.0 / dg;
                    z[p] = dinv[p] * L->r[p];
                    pv[p] = z[p];
                    rz += L->r[p] * z[p];
                }
        while (rel > tol && it < max_it) {
            double pAp = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : pAp)
            for (int k = 0; k < L->n[2]; ++k)
                for (int j = 0; j < L->n[1]; ++j)
                    for (int i = 0; i < L->n[0]; ++i) {
                        double dg, of;
                        row(L, ndim, pv, i, j, k, &dg, &of);
                        const long long p = idx(L->n, i, j, k);
                        Ap[p] = dg * pv[p] - of;
                        pAp += pv[p] * Ap[p];
                    }
            const double alpha = rz / pAp;
            double rz1 = 0.0, rr = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rz1, rr)
            for (long long p = 0; p < nc; ++p) {
                L->x[p] += alpha * pv[p];
                L->r[p] -= alpha * Ap[p];
                z[p] = dinv[p] * L->r[p];
                rz1 += L->r[p] * z[p];
                rr += L->r[p] * L->r[p];
            }
            const double beta = rz1 / rz;
            rz = rz1;
#pragma omp parallel for schedule(static)
            for (long long p = 0; p < nc; ++p) pv[p] = z[p] + beta * pv[p];
            rel = sqrt(rr) / bn;
            ++it;
        }
        free(z), free(pv), free(Ap), free(dinv);
    }
    memcpy(E, L->x, sizeof(double) * nc);
    mg_free(&M);
    if (rel_out) *rel_out = rel;
    if (it_out) *it_out = it;
    return rel <= tol ? 0 : 1;
}

/* kappa: kind 0 kappa0, kind 1 kappa0 rho^a_rho T^a_T */
static double opacity(int kind, double k0, double ar, double at, double rho, double T) {
    return kind == 0 ? k0 : k0 * pow(rho, ar) * pow(T, at);
}

/* E at offset o (|o| <= 2) along axis d with the ghost rules */
static double fetch(const int* n, const int* lo, const int* hi, const double* E,
                    const double* Ebc, const long long* boff, int i, int j, int k, int d, int o) {
    int c[3] = {i, j, k};
    const int m = c[d] + o;
    if (m >= 0 && m < n[d]) {
        c[d] = m;
        return E[idx(n, c[0], c[1], c[2])];
    }
    const int side = m < 0 ? 0 : 1;
    const int kind = side ? hi[d] : lo[d];
    if (kind == PER) c[d] = (m + n[d]) % n[d];
    else c[d] = side ? 2 * n[d] - 1 - m : -m - 1;
    const double v = E[idx(n, c[0], c[1], c[2])];
    if (kind != DIR) return v;
    /* the face array over the two other axes, the lower one fastest */
    const long long f = d == 0 ? (long long)k * n[1] + j
                      : d == 1 ? (long long)k * n[0] + i
                               : (long long)j * n[0] + i;
    return 2.0 * Ebc[boff[2 * d + side] + f] - v;
}

void cfld_limiter(int ndim, const int* n, const double* h, const int* lo, const int* hi,
                  const double* Ebc, double c, int kind, double k0, double ar, double at,
                  const double* E, const double* rho, const double* T, double* D) {
    long long boff[6], off = 0;
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
            boff[2 * d + s] = -1;
            if (d < ndim && (s ? hi[d] : lo[d]) == DIR) {
                boff[2 * d + s] = off;
                off += (long long)n[0] * n[1] * n[2] / n[d];
            }
        }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                const long long p = idx(n, i, j, k);
                const double kr = opacity(kind, k0, ar, at, rho[p], T[p]) * rho[p];
                double g2 = 0.0;
                for (int d = 0; d < ndim; ++d) {
                    const double em2 = fetch(n, lo, hi, E, Ebc, boff, i, j, k, d, -2);
                    const double em1 = fetch(n, lo, hi, E, Ebc, boff, i, j, k, d, -1);
                    const double ep1 = fetch(n, lo, hi, E, Ebc, boff, i, j, k, d, 1);
                    const double ep2 = fetch(n, lo, hi, E, Ebc, boff, i, j, k, d, 2);
                    const double g = (em2 - 8.0 * em1 + 8.0 * ep1 - ep2) / (12.0 * h[d]);
                    g2 += g * g;
                }
                const double R = sqrt(g2) / (kr * E[p]);
                const double lam = (2.0 + R) / (6.0 + 3.0 * R + R * R);
                D[p] = c * lam / kr;
            }
}

void cfld_exchange(long long nc, double dt, double c, double a_r, double gamma, double R_gas,
                   int kind, double k0, double ar, double at, const double* rho, double* T,
                   double* E) {
    const double cv = R_gas / (gamma - 1.0);
#pragma omp parallel for schedule(static)
    for (long long p = 0; p < nc; ++p) {
        const double chi = dt * c * opacity(kind, k0, ar, at, rho[p], T[p]) * rho[p];
        const double alpha = rho[p] * cv;
        const double w = chi / (1.0 + chi);
        const double beta = a_r * w;
        const double q = alpha * T[p] + w * E[p];
        double x = q / alpha;
        if (beta > 0.0) {
            const double x4 = sqrt(sqrt(q / beta));
            if (x4 < x) x = x4;
        }
        for (int it = 0; it < 100; ++it) {
            const double x2 = x * x;
            const double dx = (beta * x2 * x2 + alpha * x - q) / (4.0 * beta * x2 * x + alpha);
            x -= dx;
            if (fabs(dx) <= 4e-16 * x) break;
        }
        E[p] = (E[p] + chi * a_r * x * x * x * x) / (1.0 + chi);
        T[p] = x;
    }
}

/* limiter -> diffuse -> exchange; returns cfld_diffuse's status */
int cfld_step(int ndim, const int* n, const double* h, const int* lo, const int* hi,
              const double* Ebc, double dt, double c, double a_r, double gamma, double R_gas,
              int kind, double k0, double ar, double at, const double* rho, double* T,
              double* E, int method, double tol, int max_it, int nu1, int nu2,
              double* rel_out, int* it_out) {
    const long long nc = (long long)n[0] * n[1] * n[2];
    double* D = malloc(sizeof(double) * nc);
    if (!D) return -1;
    cfld_limiter(ndim, n, h, lo, hi, Ebc, c, kind, k0, ar, at, E, rho, T, D);
    const int st = cfld_diffuse(ndim, n, h, lo, hi, Ebc, dt, D, E, method, tol, max_it, nu1, nu2,
                                rel_out, it_out);
    /* T still holds T^n here: the exchange evaluates kappa at (rho, T^n) */
    if (st >= 0) cfld_exchange(nc, dt, c, a_r, gamma, R_gas, kind, k0, ar, at, rho, T, E);
    free(D);
    return st;
}
