/*
 * FP64 oracle of the acoustic leapfrog with a shaped stencil, a sponge layer,
 * point-source injection and receiver sampling, plus its exact discrete
 * adjoint and the gradient with respect to m = 1/v^2.
 *
 * TEST INFRASTRUCTURE ONLY: called from tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline leg through ctypes.  Shares no code with the CUDA
 * library.
 *
 * Discretisation (paper Section 3.1 Eq. wave_eq with the damping term
 * eta u_t, Eq. time_derivative1 in time, Eq. spacexz_derivative2_sym in
 * space), on the padded grid with the field zero outside it:
 *
 *   u^{n+1} = [ 2 u^n - (1 - g) u^{n-1} + k * sum_o w_o u^n(x+o) + a^n ] / (1 + g)
 *
 * k = (v tau / h)^2 per node, g = eta tau / 2 per node, w_o the stencil weights
 * (the Laplacian is (1/h^2) sum_o w_o u(x+o)), a^n = tau^2 s(t^n) / h^dim at a
 * source node.  trace[n][r] = u^{n+1} at receiver r (after injection).
 *
 * Adjoint (Lagrangian with multipliers lambda^{n+1} on each step equation,
 * J = 1/2 sum ||trace - d_obs||^2, r^n = dJ/dtrace^n):
 *   lambda^j = S^T r^{j-1} + 2 nu^{j+1} + sum_o w_o (k nu^{j+1})(x+o) - (1 - g) nu^{j+2},
 *   nu^j = lambda^j / (1 + g),   j = nt .. 1,  nu^{nt+1} = nu^{nt+2} = 0,
 * and dJ/dm(x) = -(k/m)(x) sum_{n} nu^{n+1}(x) sum_o w_o u^n(x+o).
 * The raw correlation G(x) = sum_n nu^{n+1}(x) sum_o w_o u^n(x+o) is returned;
 * the caller applies -(k/m) and folds the padding.  adj_trace[n][i] =
 * nu^{n+1} at node adj_idx[i] is d<r, trace>/d a^n for a source there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t nz, ny, nx;
    int npts;
    const int *off;      /* [npts][3] = (dz, dy, dx) */
    const double *w;     /* [npts] */
} grid_t;

/* sum_o w_o f(x+o), zero outside the padded grid */
static double apply_stencil(const grid_t *g, const double *f, int64_t z, int64_t y, int64_t x)
{
    double s = 0.0;
    for (int k = 0; k < g->npts; ++k) {
        int64_t zz = z + g->off[3 * k], yy = y + g->off[3 * k + 1], xx = x + g->off[3 * k + 2];
        if (zz < 0 || zz >= g->nz || yy < 0 || yy >= g->ny || xx < 0 || xx >= g->nx) continue;
        s += g->w[k] * f[(zz * g->ny + yy) * g->nx + xx];
    }
    return s;
}

/* one forward step: u_prev <- u^{n+1} (overwrites u^{n-1}), optional
 * lap_out <- sum_o w_o u^n */
static void forward_step(const grid_t *g, const double *kap, const double *gam,
                         const double *u_cur, double *u_prev, double *lap_out,
                         int nsrc, const int64_t *src_idx, const double *amp_n,
                         int nthreads)
{
    const int64_t nz = g->nz, ny = g->ny, nx = g->nx;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t i = (z * ny + y) * nx + x;
                double lap = apply_stencil(g, u_cur, z, y, x);
                if (lap_out) lap_out[i] = lap;
                u_prev[i] = 2.0 * u_cur[i] - (1.0 - gam[i]) * u_prev[i] + kap[i] * lap;
            }
    for (int s = 0; s < nsrc; ++s) u_prev[src_idx[s]] += amp_n[s];
    const int64_t n = nz * ny * nx;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t i = 0; i < n; ++i) u_prev[i] /= (1.0 + gam[i]);
}

int oracle_forward(int64_t nz, int64_t ny, int64_t nx,
                   const double *kap, const double *gam,
                   int npts, const int *off, const double *w,
                   int nt, int nsrc, const int64_t *src_idx, const double *src_amp,
                   int nrec, const int64_t *rec_idx, double *traces,
                   double *u_prev, double *u_cur, int nthreads)
{
    grid_t g = {nz, ny, nx, npts, off, w};
    for (int n = 0; n < nt; ++n) {
        forward_step(&g, kap, gam, u_cur, u_prev, NULL, nsrc, src_idx,
                     src_amp ? src_amp + (int64_t)n * nsrc : NULL, nthreads);
        double *t = u_prev; u_prev = u_cur; u_cur = t;       /* u_cur = u^{n+1} */
        if (traces)
            for (int r = 0; r < nrec; ++r) traces[(int64_t)n * nrec + r] = u_cur[rec_idx[r]];
    }
    /* buffers were swapped nt times: the caller's u_cur must end as u^{nt} */
    if (nt % 2 == 1) {
        int64_t n = nz * ny * nx;
        for (int64_t i = 0; i < n; ++i) { double t = u_prev[i]; u_prev[i] = u_cur[i]; u_cur[i] = t; }
    }
    return 0;
}

/* Gradient: forward with checkpoints every `seg` steps, then segments in
 * reverse: recompute the segment's u^n, run the adjoint recurrence backwards
 * and accumulate G.  With seg >= nt everything is stored (one segment). */
int oracle_gradient(int64_t nz, int64_t ny, int64_t nx,
                    const double *kap, const double *gam,
                    int npts, const int *off, const double *w,
                    int nt, int nsrc, const int64_t *src_idx, const double *src_amp,
                    int nrec, const int64_t *rec_idx, const double *resid,
                    int nadj, const int64_t *adj_idx, double *adj_trace,
                    double *G, int seg, int nthreads)
{
    grid_t g = {nz, ny, nx, npts, off, w};
    const int64_t n = nz * ny * nx;
    if (seg < 1) seg = 1;
    if (seg > nt) seg = nt;
    const int nseg = (nt + seg - 1) / seg;
    /* checkpoint s holds (u^{s*seg}, u^{s*seg-1}) */
    double *ck = (double *)calloc((size_t)(2 * nseg) * n, sizeof(double));
    double *a = (double *)calloc(n, sizeof(double)), *b = (double *)calloc(n, sizeof(double));
    double *useg = (double *)malloc((size_t)(seg + 1) * n * sizeof(double));
    double *nu1 = (double *)calloc(n, sizeof(double)), *nu2 = (double *)calloc(n, sizeof(double));
    double *tmp = (double *)malloc(n * sizeof(double)), *lam = (double *)malloc(n * sizeof(double));
    if (!ck || !a || !b || !useg || !nu1 || !nu2 || !tmp || !lam) return -6;
    memset(G, 0, n * sizeof(double));
    /* forward sweep: a = u^{n-1}, b = u^n */
    for (int s = 0, k = 0; k < nt; ++k) {
        if (k % seg == 0) {
            memcpy(ck + (size_t)(2 * s) * n, b, n * sizeof(double));
            memcpy(ck + (size_t)(2 * s + 1) * n, a, n * sizeof(double));
            ++s;
        }
        forward_step(&g, kap, gam, b, a, NULL, nsrc, src_idx,
                     src_amp ? src_amp + (int64_t)k * nsrc : NULL, nthreads);
        double *t = a; a = b; b = t;
    }
    /* nu1 = nu^{j+1}, nu2 = nu^{j+2}; start j = nt with both zero */
    for (int s = nseg - 1; s >= 0; --s) {
        int k0 = s * seg, k1 = k0 + seg < nt ? k0 + seg : nt;
        memcpy(b, ck + (size_t)(2 * s) * n, n * sizeof(double));
        memcpy(a, ck + (size_t)(2 * s + 1) * n, n * sizeof(double));
        memcpy(useg, b, n * sizeof(double));                 /* u^{k0} */
        for (int k = k0; k < k1 - 1; ++k) {                  /* u^{k0+1} .. u^{k1-1} */
            forward_step(&g, kap, gam, b, a, NULL, nsrc, src_idx,
                         src_amp ? src_amp + (int64_t)k * nsrc : NULL, nthreads);
            double *t = a; a = b; b = t;
            memcpy(useg + (size_t)(k - k0 + 1) * n, b, n * sizeof(double));
        }
        for (int j = k1; j > k0; --j) {                      /* adjoint step j uses u^{j-1} */
#pragma omp parallel for num_threads(nthreads) schedule(static)
            for (int64_t i = 0; i < n; ++i) tmp[i] = kap[i] * nu1[i];
#pragma omp parallel for num_threads(nthreads) schedule(static)
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x) {
                        int64_t i = (z * ny + y) * nx + x;
                        lam[i] = 2.0 * nu1[i] + apply_stencil(&g, tmp, z, y, x) - (1.0 - gam[i]) * nu2[i];
                    }
            for (int r = 0; r < nrec; ++r) lam[rec_idx[r]] += resid[(int64_t)(j - 1) * nrec + r];
            /* shift: nu2 <- nu^{j+1}, nu1 <- nu^{j} */
            double *t = nu2; nu2 = nu1; nu1 = t;
#pragma omp parallel for num_threads(nthreads) schedule(static)
            for (int64_t i = 0; i < n; ++i) nu1[i] = lam[i] / (1.0 + gam[i]);
            if (adj_trace)
                for (int q = 0; q < nadj; ++q) adj_trace[(int64_t)(j - 1) * nadj + q] = nu1[adj_idx[q]];
            const double *un = useg + (size_t)(j - 1 - k0) * n;  /* u^{j-1} */
#pragma omp parallel for num_threads(nthreads) schedule(static)
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x) {
                        int64_t i = (z * ny + y) * nx + x;
                        G[i] += nu1[i] * apply_stencil(&g, un, z, y, x);
                    }
        }
    }
    free(ck); free(a); free(b); free(useg); free(nu1); free(nu2); free(tmp); free(lam);
    return 0;
}
