/*
 * FP64 CPU oracle of the MFV/MFM hydro step (arXiv:2211.12243, "Mesh-free
 * hydrodynamics in pkdgrav3 for galaxy formation simulations", §2.3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header or constant table with
 * the CUDA library.
 *
 * Everything is plain double precision, compiled with -ffp-contract=off so
 * that no multiply-add is fused behind the reader's back.  Loops over
 * particles are parallelised with OpenMP; each particle's arithmetic is
 * exactly the sequential definition.
 *
 * Layout of every array: structure of arrays, particle index = the caller's
 * order.  Periodic box [0,Lx) x [0,Ly) x [0,Lz).
 *
 * Readings of the paper taken here where it is silent:
 *   - Kernel: Wendland C2 (default) or cubic spline, compact radius H = h.
 *   - W(r_ij) in E_i and grad_i uses the evaluating particle's own h_i; the
 *     j-term of A_ij uses h_j.
 *   - The gradient weight is omega_j (Lanson & Vila form, §2.3.3).
 *   - The self term is part of omega^-1 (Eq. 6) and absent from E and grad.
 *   - Smoothing length: safeguarded Newton on Eq. 18 with bisection fallback.
 *   - N_cond > crit  =>  N_NGB,i *= grow, density redone for i (§2.3.5).
 *   - Conditioned Barth-Jespersen limiter and pairwise limiter: the forms of
 *     Hopkins (2015) eqs. B3 and B4 that §2.3.6 cites (a reading: the paper
 *     does not print them; the tests pin these forms by closed forms and
 *     invariants).
 *   - Half-step predictor in the particle (Lagrangian) frame.
 *   - Riemann: exact (Toro 2009) with Toro's adaptive initial guess, or HLLC.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* configuration                                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    double gamma;        /* adiabatic index */
    int kernel;          /* 0 = Wendland C2, 1 = cubic spline */
    double n_ngb;        /* target neighbour number, Eq. 18 */
    int scheme;          /* 0 = MFV, 1 = MFM (§2.3.3, last paragraphs) */
    int riemann;         /* 0 = exact iterative (Toro), 1 = HLLC */
    int limiter;         /* 1 = conditioned BJ + pairwise limiters, 0 = off */
    int time_extrap;     /* 1 = half-step predictor (Eq. 16), 0 = off */
    double ncond_crit;   /* N_cond threshold, §2.3.5 (100) */
    double ngb_grow;     /* N_NGB growth factor, §2.3.5 (1.2) */
    int max_ngb_grow;    /* growth rounds before giving up (5) */
    double psi1, psi2;   /* pairwise limiter, §2.3.6 (0.5, 0.25) */
    double beta_min, beta_max; /* conditioned BJ (1, 2) */
    double c_cfl;        /* CFL factor, Eq. 31 */
    double alpha1;       /* total-energy switch, §2.3.7 (1/100) */
    double h_tol;        /* relative Newton tolerance on h */
    double p_tol;        /* relative Newton tolerance on p* */
    int max_h_iter;      /* cap on the h iteration */
    int max_newton;      /* cap on the Riemann Newton iteration */
    int entropy;         /* 1 = entropy switch of §2.3.7 (entropic function evolved) */
    double alpha2, alpha3; /* entropy switch thresholds, §2.3.7 (1/1000 each) */
} orc_config;

typedef struct {
    int64_t newton_iters;     /* Riemann Newton iterations summed over faces */
    int64_t faces;            /* Riemann problems solved */
    int64_t vacuum;           /* faces with vacuum generation (zero flux) */
    int64_t bisect_fallback;  /* faces that needed bisection */
    int64_t first_order;      /* faces that fell back to cell-centred states */
    int64_t pairs;            /* unordered flux pairs */
} orc_flux_stats;

enum { ORC_OK = 0, ORC_ENOCONV_H = -4, ORC_ENCOND = -5, ORC_ERIEMANN = -6 };

/* ------------------------------------------------------------------------ */
/* kernels, §2.3.2 (compact support r < H, unit normalisation)               */
/* ------------------------------------------------------------------------ */

/* W(r, H) in three dimensions.  Wendland C2 (Dehnen & Aly 2012):
 *   W = 21/(2 pi H^3) (1-q)^4 (1+4q),  q = r/H < 1.
 * Cubic spline (M4, compact radius H):
 *   W = 8/(pi H^3) {1 - 6q^2 + 6q^3  (q <= 1/2);  2(1-q)^3  (q <= 1)}.     */
double orc_kernel_W(int kernel, double r, double H)
{
    double q = r / H;
    if (q >= 1.0) return 0.0;
    if (kernel == 0) {
        double t = 1.0 - q;
        return 21.0 / (2.0 * M_PI * H * H * H) * (t * t * t * t) * (1.0 + 4.0 * q);
    }
    double s = 8.0 / (M_PI * H * H * H);
    if (q <= 0.5) return s * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
    double t = 1.0 - q;
    return s * 2.0 * t * t * t;
}

/* dW/dH at fixed r (needed for the Newton step on h). */
double orc_kernel_dWdH(int kernel, double r, double H)
{
    double q = r / H;
    if (q >= 1.0) return 0.0;
    /* W = c/H^3 f(q); dW/dH = -3 W/H + c/H^3 f'(q) (-q/H) */
    double fprime, c, f;
    if (kernel == 0) {
        double t = 1.0 - q;
        c = 21.0 / (2.0 * M_PI);
        f = t * t * t * t * (1.0 + 4.0 * q);
        fprime = -4.0 * t * t * t * (1.0 + 4.0 * q) + 4.0 * t * t * t * t;
    } else {
        c = 8.0 / M_PI;
        if (q <= 0.5) {
            f = 1.0 - 6.0 * q * q + 6.0 * q * q * q;
            fprime = -12.0 * q + 18.0 * q * q;
        } else {
            double t = 1.0 - q;
            f = 2.0 * t * t * t;
            fprime = -6.0 * t * t;
        }
    }
    double H3 = H * H * H;
    return -3.0 * c * f / (H3 * H) + c * fprime * (-q / H) / H3;
}

/* ------------------------------------------------------------------------ */
/* periodic geometry                                                         */
/* ------------------------------------------------------------------------ */

/* Minimum-image separation along one axis: d = xj - xi folded once into
 * [-L/2, L/2] (positions lie in [0, L), so one fold suffices). */
static double orc_fold(double d, double L)
{
    if (d > 0.5 * L) return d - L;
    if (d < -0.5 * L) return d + L;
    return d;
}

/* dx = x_j - x_i (minimum image), r^2 = (dx^2 + dy^2) + dz^2 */
static double orc_sep(const double *x, const double *y, const double *z,
                      const double L[3], int64_t i, int64_t j, double d[3])
{
    d[0] = orc_fold(x[j] - x[i], L[0]);
    d[1] = orc_fold(y[j] - y[i], L[1]);
    d[2] = orc_fold(z[j] - z[i], L[2]);
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* ------------------------------------------------------------------------ */
/* neighbour search (§2.2.3 defines the set; this is a plain search for it)  */
/* ------------------------------------------------------------------------ */

/* A uniform cell grid used only to avoid the O(N^2) scan; it never changes
 * which particles are found: every j with r_ij < R_i is in one of the
 * 27 cells around i because the cell side is >= max R.  When fewer than
 * three cells fit along an axis the search degrades to a scan of all cells
 * along that axis. */
typedef struct {
    int n[3];
    double L[3];
    int64_t *start;  /* [ncell+1] */
    int64_t *item;   /* particle ids grouped by cell, ascending within cell */
} orc_grid;

static int orc_cell_coord(double x, double L, int n)
{
    int c = (int)(x / L * n);
    if (c < 0) c = 0;
    if (c >= n) c = n - 1;
    return c;
}

static void orc_grid_build(orc_grid *g, int64_t n, const double *x, const double *y,
                           const double *z, const double L[3], double rmax)
{
    for (int a = 0; a < 3; a++) {
        g->L[a] = L[a];
        int c = (int)floor(L[a] / rmax);
        if (c < 1) c = 1;
        if (c > 1024) c = 1024;
        g->n[a] = c;
    }
    int64_t ncell = (int64_t)g->n[0] * g->n[1] * g->n[2];
    g->start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    g->item = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *cell = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int cx = orc_cell_coord(x[i], L[0], g->n[0]);
        int cy = orc_cell_coord(y[i], L[1], g->n[1]);
        int cz = orc_cell_coord(z[i], L[2], g->n[2]);
        cell[i] = ((int64_t)cx * g->n[1] + cy) * g->n[2] + cz;
        g->start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) g->start[c + 1] += g->start[c];
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    memcpy(fill, g->start, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) g->item[fill[cell[i]]++] = i;
    free(fill);
    free(cell);
}

static void orc_grid_free(orc_grid *g)
{
    free(g->start);
    free(g->item);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* All j with r_ij^2 < R^2 (j = i included), ascending j.  Grows *buf. */
static int64_t orc_gather(const orc_grid *g, const double *x, const double *y,
                          const double *z, int64_t i, double R,
                          int64_t **buf, int64_t *cap)
{
    int64_t cnt = 0;
    int ci[3] = {orc_cell_coord(x[i], g->L[0], g->n[0]),
                 orc_cell_coord(y[i], g->L[1], g->n[1]),
                 orc_cell_coord(z[i], g->L[2], g->n[2])};
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        if (g->n[a] < 3) { lo[a] = 0; hi[a] = g->n[a] - 1; }
        else { lo[a] = ci[a] - 1; hi[a] = ci[a] + 1; }
    }
    double R2 = R * R;
    for (int a = lo[0]; a <= hi[0]; a++)
        for (int b = lo[1]; b <= hi[1]; b++)
            for (int c = lo[2]; c <= hi[2]; c++) {
                int aa = (a + g->n[0]) % g->n[0];
                int bb = (b + g->n[1]) % g->n[1];
                int cc = (c + g->n[2]) % g->n[2];
                int64_t cell = ((int64_t)aa * g->n[1] + bb) * g->n[2] + cc;
                for (int64_t k = g->start[cell]; k < g->start[cell + 1]; k++) {
                    int64_t j = g->item[k];
                    double d[3];
                    double r2 = orc_sep(x, y, z, g->L, i, j, d);
                    if (r2 < R2) {
                        if (cnt == *cap) {
                            *cap = *cap * 2 + 64;
                            *buf = (int64_t *)realloc(*buf, (size_t)*cap * sizeof(int64_t));
                        }
                        (*buf)[cnt++] = j;
                    }
                }
            }
    qsort(*buf, (size_t)cnt, sizeof(int64_t), cmp_i64);
    return cnt;
}

/* Gather lists {j : r_ij^2 < hs_i^2}, j = i included, rows ascending.
 * Brute force O(N^2) when use_grid == 0.  off[n+1]; idx[cap].
 * Returns the total number of entries (which may exceed cap: nothing is
 * written past cap and the caller retries with a larger buffer). */
int64_t orc_neighbours(int64_t n, const double *x, const double *y, const double *z,
                       const double *L, const double *hs, int use_grid,
                       int64_t cap, int64_t *off, int32_t *idx)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    double rmax = 0.0;
    for (int64_t i = 0; i < n; i++) if (hs[i] > rmax) rmax = hs[i];
    orc_grid g;
    if (use_grid) orc_grid_build(&g, n, x, y, z, L, rmax);
    /* pass 1: counts */
    #pragma omp parallel
    {
        int64_t *buf = NULL, bcap = 0;
        #pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            if (use_grid) {
                cnt[i] = orc_gather(&g, x, y, z, i, hs[i], &buf, &bcap);
            } else {
                int64_t c = 0;
                double h2 = hs[i] * hs[i];
                for (int64_t j = 0; j < n; j++) {
                    double d[3];
                    if (orc_sep(x, y, z, L, i, j, d) < h2) c++;
                }
                cnt[i] = c;
            }
        }
        free(buf);
    }
    off[0] = 0;
    for (int64_t i = 0; i < n; i++) off[i + 1] = off[i] + cnt[i];
    int64_t total = off[n];
    if (total <= cap) {
        #pragma omp parallel
        {
            int64_t *buf = NULL, bcap = 0;
            #pragma omp for schedule(dynamic, 256)
            for (int64_t i = 0; i < n; i++) {
                if (use_grid) {
                    int64_t c = orc_gather(&g, x, y, z, i, hs[i], &buf, &bcap);
                    for (int64_t k = 0; k < c; k++) idx[off[i] + k] = (int32_t)buf[k];
                } else {
                    int64_t c = 0;
                    double h2 = hs[i] * hs[i];
                    for (int64_t j = 0; j < n; j++) {
                        double d[3];
                        if (orc_sep(x, y, z, L, i, j, d) < h2) idx[off[i] + c++] = (int32_t)j;
                    }
                }
            }
            free(buf);
        }
    }
    if (use_grid) orc_grid_free(&g);
    free(cnt);
    return total;
}

/* ------------------------------------------------------------------------ */
/* density and smoothing length, §2.3.2 (Eqs. 5-7) and §2.3.5 (Eq. 18)       */
/* ------------------------------------------------------------------------ */

/* g(h) = (4 pi/3) h^3 sum_j W(r_ij, h) - N  and dg/dh over a candidate set */
static void orc_density_residual(const orc_config *c, const double *x, const double *y,
                                 const double *z, const double L[3], int64_t i,
                                 const int64_t *cand, int64_t nc, double h, double N,
                                 double *g, double *dg, double *sumW)
{
    double s = 0.0, ds = 0.0;
    for (int64_t k = 0; k < nc; k++) {
        double d[3];
        double r = sqrt(orc_sep(x, y, z, L, i, cand[k], d));
        s += orc_kernel_W(c->kernel, r, h);
        ds += orc_kernel_dWdH(c->kernel, r, h);
    }
    double v = 4.0 * M_PI / 3.0;
    *g = v * h * h * h * s - N;
    *dg = v * (3.0 * h * h * s + h * h * h * ds);
    *sumW = s;
}

/* Solve Eq. 18 for h_i with n_i = omega_i^-1 (Eq. 6) for the particles with
 * active[i] != 0 (all when active == NULL).  h holds the initial guess on
 * entry.  Output: h, omega = 1/sum_j W(r_ij, h_i) (self included).
 * Safeguarded Newton: the root is bracketed by [lo, hi]; a Newton proposal
 * outside the bracket is replaced by bisection.  Converged when the last
 * correction is below h_tol * h; that correction is applied.
 * iters[i] (optional) receives the iteration count.  Returns ORC_OK or
 * ORC_ENOCONV_H (h left unconverged for at least one particle). */
int orc_density(const orc_config *c, int64_t n, const double *x, const double *y,
                const double *z, const double *L, const double *n_ngb_i,
                const int32_t *active, double *h, double *omega, int32_t *iters)
{
    double hmax_guess = 0.0;
    for (int64_t i = 0; i < n; i++) if (h[i] > hmax_guess) hmax_guess = h[i];
    orc_grid g;
    /* cell side: generous, the search radius below is re-widened as needed */
    orc_grid_build(&g, n, x, y, z, L, 2.0 * hmax_guess);
    int status = ORC_OK;
    #pragma omp parallel
    {
        int64_t *buf = NULL, bcap = 0;
        #pragma omp for schedule(dynamic, 128)
        for (int64_t i = 0; i < n; i++) {
            if (active && !active[i]) continue;
            double N = n_ngb_i ? n_ngb_i[i] : c->n_ngb;
            double hh = h[i];
            double R = 1.5 * hh;              /* candidate radius */
            int64_t nc;
            if (R > 2.0 * hmax_guess) nc = -1;  /* grid too fine: brute force */
            else nc = orc_gather(&g, x, y, z, i, R, &buf, &bcap);
            if (nc < 0) {
                nc = 0;
                for (int64_t j = 0; j < n; j++) {
                    double d[3];
                    if (orc_sep(x, y, z, L, i, j, d) < R * R) {
                        if (nc == bcap) { bcap = 2 * bcap + 64; buf = (int64_t *)realloc(buf, (size_t)bcap * sizeof(int64_t)); }
                        buf[nc++] = j;
                    }
                }
            }
            double lo = 0.0, hi = -1.0;  /* hi < 0: no upper bracket yet */
            int it, conv = 0;
            double gv = 0, dg = 0, sw = 0;
            for (it = 1; it <= c->max_h_iter; it++) {
                if (hh >= R) {
                    /* widen the candidate set so that every r < hh is present */
                    R = 1.5 * hh;
                    nc = 0;
                    for (int64_t j = 0; j < n; j++) {
                        double d[3];
                        if (orc_sep(x, y, z, L, i, j, d) < R * R) {
                            if (nc == bcap) { bcap = 2 * bcap + 64; buf = (int64_t *)realloc(buf, (size_t)bcap * sizeof(int64_t)); }
                            buf[nc++] = j;
                        }
                    }
                }
                orc_density_residual(c, x, y, z, L, i, buf, nc, hh, N, &gv, &dg, &sw);
                if (gv == 0.0) { conv = 1; break; }
                if (gv < 0.0) { if (hh > lo) lo = hh; }
                else { if (hi < 0.0 || hh < hi) hi = hh; }
                double hn;
                if (dg > 0.0) hn = hh - gv / dg; else hn = -1.0;
                if (hn > 0.0 && fabs(hn - hh) <= c->h_tol * hh) {
                    /* converged: the Newton correction is below tolerance */
                    hh = hn;
                    conv = 1;
                    break;
                }
                if (hi < 0.0) {
                    /* no upper bound known: Newton, but at most doubling */
                    if (!(hn > lo) || hn > 2.0 * hh) hn = 2.0 * hh;
                } else if (!(hn > lo && hn < hi)) {
                    hn = 0.5 * (lo + hi);
                }
                double step = fabs(hn - hh);
                hh = hn;
                if (step <= c->h_tol * hh) { conv = 1; break; }
            }
            /* final state: omega from the accepted h */
            if (hh >= R) {
                R = 1.5 * hh;
                nc = 0;
                for (int64_t j = 0; j < n; j++) {
                    double d[3];
                    if (orc_sep(x, y, z, L, i, j, d) < R * R) {
                        if (nc == bcap) { bcap = 2 * bcap + 64; buf = (int64_t *)realloc(buf, (size_t)bcap * sizeof(int64_t)); }
                        buf[nc++] = j;
                    }
                }
            }
            orc_density_residual(c, x, y, z, L, i, buf, nc, hh, N, &gv, &dg, &sw);
            h[i] = hh;
            omega[i] = 1.0 / sw;
            if (iters) iters[i] = it;
            if (!conv) {
                #pragma omp atomic write
                status = ORC_ENOCONV_H;
            }
        }
        free(buf);
    }
    orc_grid_free(&g);
    return status;
}

/* ------------------------------------------------------------------------ */
/* primitive variables, Eq. 2 and §2.3.7 (Eqs. 23-24)                         */
/* ------------------------------------------------------------------------ */

/* rho = m/omega (= m omega^-1, §2.3.2), v = P/m, and the pressure from the
 * total energy (Eq. 23) when U_i > alpha1 (E_grav,i + E_kin,i), else from
 * the separately integrated internal energy U_i (p = (gamma-1) U_i / omega_i).
 * E_kin = P.P / 2m; E_grav = m |a_grav| h (§2.3.7), zero without an
 * acceleration (acc NULL; h may then be NULL too).  The total energy route
 * also requires E - E_kin > 0.  acc: 3 per particle (ax, ay, az). */
void orc_primitives(const orc_config *c, int64_t n, const double *m, const double *px,
                    const double *py, const double *pz, const double *E, const double *U,
                    const double *omega, const double *h, const double *acc, const double *A,
                    const double *ekmax, int32_t *src, double *rho, double *vx, double *vy,
                    double *vz, double *p)
{
    for (int64_t i = 0; i < n; i++) {
        rho[i] = m[i] / omega[i];
        vx[i] = px[i] / m[i];
        vy[i] = py[i] / m[i];
        vz[i] = pz[i] / m[i];
        double ekin = (px[i] * px[i] + py[i] * py[i] + pz[i] * pz[i]) / (2.0 * m[i]);
        double egrav = 0.0;
        if (acc) {
            const double *a = acc + 3 * i;
            egrav = m[i] * sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) * h[i];
        }
        double therm = U[i];
        int from = 2;   /* 0 total energy, 1 entropy, 2 internal energy */
        if (U[i] > c->alpha1 * (egrav + ekin) && E[i] - ekin > 0.0) {
            therm = E[i] - ekin;
            from = 0;
        } else if (c->entropy && A && A[i] > 0.0 &&
                   (U[i] < c->alpha2 * (ekmax[i] + U[i]) || U[i] < c->alpha3 * egrav)) {
            from = 1;
        }
        if (from == 1)
            p[i] = A[i] * pow(rho[i], c->gamma);   /* the entropic function p = A rho^gamma */
        else
            p[i] = therm * (c->gamma - 1.0) / omega[i];
        if (src) src[i] = from;
    }
}

/* The largest kinetic energy of particle i relative to a neighbour,
 * max_j (1/2) m_i |v_j - v_i|^2 over j != i with r_ij < h_i (§2.3.7: the
 * smoothness measure of the entropy switch; 0 without neighbours). */
void orc_ekin_max(int64_t n, const double *x, const double *y, const double *z,
                  const double *L, const double *h, const double *m, const double *px,
                  const double *py, const double *pz, double *out)
{
    int64_t *off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t tot = orc_neighbours(n, x, y, z, L, h, 1, 0, off, NULL);
    int32_t *idx = (int32_t *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
    orc_neighbours(n, x, y, z, L, h, 1, tot, off, idx);
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        const double vix = px[i] / m[i], viy = py[i] / m[i], viz = pz[i] / m[i];
        double best = 0.0;
        for (int64_t k = off[i]; k < off[i + 1]; k++) {
            const int64_t j = idx[k];
            if (j == i) continue;
            const double dx = px[j] / m[j] - vix, dy = py[j] / m[j] - viy, dz = pz[j] / m[j] - viz;
            const double e = 0.5 * m[i] * ((dx * dx + dy * dy) + dz * dz);
            if (e > best) best = e;
        }
        out[i] = best;
    }
    free(idx);
    free(off);
}

/* ------------------------------------------------------------------------ */
/* E matrix, its inverse and the condition number (Eqs. 10, 11, 19)           */
/* ------------------------------------------------------------------------ */

/* 3x3 symmetric inverse by cofactors.  E and B are full row-major 3x3. */
static int orc_inv3(const double E[9], double B[9])
{
    double c00 = E[4] * E[8] - E[5] * E[7];
    double c01 = E[5] * E[6] - E[3] * E[8];
    double c02 = E[3] * E[7] - E[4] * E[6];
    double det = E[0] * c00 + E[1] * c01 + E[2] * c02;
    if (!(det != 0.0) || !isfinite(det)) return -1;
    double id = 1.0 / det;
    B[0] = c00 * id;
    B[1] = (E[2] * E[7] - E[1] * E[8]) * id;
    B[2] = (E[1] * E[5] - E[2] * E[4]) * id;
    B[3] = c01 * id;
    B[4] = (E[0] * E[8] - E[2] * E[6]) * id;
    B[5] = (E[2] * E[3] - E[0] * E[5]) * id;
    B[6] = c02 * id;
    B[7] = (E[1] * E[6] - E[0] * E[7]) * id;
    B[8] = (E[0] * E[4] - E[1] * E[3]) * id;
    return 0;
}

/* For every particle i: E_i^{ab} = sum_{j != i, r<h_i} omega_j dx^b dx^a W(r,h_i)
 * (Eq. 11 with mu(x_i,x_j) = (x_j - x_i) W(r_ij, h_i), weight omega_j),
 * B_i = E_i^-1 and N_cond,i = (1/3) sqrt(||B|| ||E||), ||A|| = sum A_ab^2
 * (Eq. 19).  B is stored as 6 unique entries (xx, xy, xz, yy, yz, zz);
 * E likewise when E_out is not NULL.  A singular E gives N_cond = +inf and
 * B = 0. */
void orc_matrices(const orc_config *c, int64_t n, const double *x, const double *y,
                  const double *z, const double *L, const double *h, const double *omega,
                  double *B6, double *E6_out, double *ncond)
{
    double hmax = 0.0;
    for (int64_t i = 0; i < n; i++) if (h[i] > hmax) hmax = h[i];
    orc_grid g;
    orc_grid_build(&g, n, x, y, z, L, hmax);
    #pragma omp parallel
    {
        int64_t *buf = NULL, bcap = 0;
        #pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            int64_t nc = orc_gather(&g, x, y, z, i, h[i], &buf, &bcap);
            double E[9] = {0};
            for (int64_t k = 0; k < nc; k++) {
                int64_t j = buf[k];
                if (j == i) continue;
                double d[3];
                double r = sqrt(orc_sep(x, y, z, L, i, j, d));
                double w = omega[j] * orc_kernel_W(c->kernel, r, h[i]);
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) E[3 * a + b] += w * d[b] * d[a];
            }
            double B[9];
            double nrmE = 0.0, nrmB = 0.0;
            if (orc_inv3(E, B) != 0) {
                for (int a = 0; a < 9; a++) B[a] = 0.0;
                ncond[i] = INFINITY;
            } else {
                for (int a = 0; a < 9; a++) { nrmE += E[a] * E[a]; nrmB += B[a] * B[a]; }
                ncond[i] = sqrt(nrmB * nrmE) / 3.0;
            }
            B6[6 * i + 0] = B[0]; B6[6 * i + 1] = B[1]; B6[6 * i + 2] = B[2];
            B6[6 * i + 3] = B[4]; B6[6 * i + 4] = B[5]; B6[6 * i + 5] = B[8];
            if (E6_out) {
                E6_out[6 * i + 0] = E[0]; E6_out[6 * i + 1] = E[1]; E6_out[6 * i + 2] = E[2];
                E6_out[6 * i + 3] = E[4]; E6_out[6 * i + 4] = E[5]; E6_out[6 * i + 5] = E[8];
            }
        }
        free(buf);
    }
    orc_grid_free(&g);
}

static void orc_B9(const double *B6, int64_t i, double B[9])
{
    const double *b = B6 + 6 * i;
    B[0] = b[0]; B[1] = b[1]; B[2] = b[2];
    B[3] = b[1]; B[4] = b[3]; B[5] = b[4];
    B[6] = b[2]; B[7] = b[4]; B[8] = b[5];
}

/* ------------------------------------------------------------------------ */
/* gradients and slope limiter (Eq. 10, §2.3.6 Eqs. 20-22)                    */
/* ------------------------------------------------------------------------ */

/* Gradients of the five primitives f in (rho, vx, vy, vz, p):
 *   grad f_i = B_i sum_{j != i, r<h_i} omega_j (f_j - f_i) (x_j - x_i) W(r_ij, h_i)
 * Conditioned Barth-Jespersen factor alpha_i (Hopkins 2015 eq. B3):
 *   f_max/min = extremes of f over i and its neighbours,
 *   D+ / D-   = largest / smallest of (1/2)(x_j - x_i).grad f_i over j,
 *   beta_i    = max(beta_min, beta_max min(1, (ncrit/N_cond,i)^2)),
 *   alpha     = min(1, beta_i min((f_max - f_i)/D+, (f_min - f_i)/D-))
 *   (a ratio is +inf when its denominator has the wrong sign or is 0).
 * limiter == 0 gives alpha = 1.
 * The signal velocity of Eq. 32 is collected over the same neighbours:
 *   v_sig,i = max_j (c_i + c_j - min(0, (x_i-x_j).(v_i-v_j)/|x_i-x_j|)).
 * grad[15 i + 3 f + a], alpha[5 i + f], vsig[i] (optional). */
void orc_gradients(const orc_config *c, int64_t n, const double *x, const double *y,
                   const double *z, const double *L, const double *h, const double *omega,
                   const double *rho, const double *vx, const double *vy, const double *vz,
                   const double *p, const double *B6, const double *ncond,
                   double *grad, double *alpha, double *vsig)
{
    double hmax = 0.0;
    for (int64_t i = 0; i < n; i++) if (h[i] > hmax) hmax = h[i];
    orc_grid g;
    orc_grid_build(&g, n, x, y, z, L, hmax);
    const double *F[5] = {rho, vx, vy, vz, p};
    #pragma omp parallel
    {
        int64_t *buf = NULL, bcap = 0;
        #pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            int64_t nc = orc_gather(&g, x, y, z, i, h[i], &buf, &bcap);
            double S[5][3] = {{0}};
            double fmax[5], fmin[5];
            for (int f = 0; f < 5; f++) fmax[f] = fmin[f] = F[f][i];
            double ci = sqrt(c->gamma * p[i] / rho[i]);
            double vs = 0.0;
            for (int64_t k = 0; k < nc; k++) {
                int64_t j = buf[k];
                if (j == i) continue;
                double d[3];
                double r = sqrt(orc_sep(x, y, z, L, i, j, d));
                double w = omega[j] * orc_kernel_W(c->kernel, r, h[i]);
                for (int f = 0; f < 5; f++) {
                    double df = F[f][j] - F[f][i];
                    for (int a = 0; a < 3; a++) S[f][a] += w * df * d[a];
                    if (F[f][j] > fmax[f]) fmax[f] = F[f][j];
                    if (F[f][j] < fmin[f]) fmin[f] = F[f][j];
                }
                double cj = sqrt(c->gamma * p[j] / rho[j]);
                double wdot = (d[0] * (vx[j] - vx[i]) + d[1] * (vy[j] - vy[i]) + d[2] * (vz[j] - vz[i])) / r;
                double s = ci + cj - (wdot < 0.0 ? wdot : 0.0);
                if (s > vs) vs = s;
            }
            if (vsig) vsig[i] = vs;
            double B[9];
            orc_B9(B6, i, B);
            double G[5][3];
            for (int f = 0; f < 5; f++)
                for (int a = 0; a < 3; a++)
                    G[f][a] = B[3 * a + 0] * S[f][0] + B[3 * a + 1] * S[f][1] + B[3 * a + 2] * S[f][2];
            for (int f = 0; f < 5; f++)
                for (int a = 0; a < 3; a++) grad[15 * i + 3 * f + a] = G[f][a];
            if (!c->limiter) {
                for (int f = 0; f < 5; f++) alpha[5 * i + f] = 1.0;
                continue;
            }
            double dplus[5], dminus[5];
            for (int f = 0; f < 5; f++) { dplus[f] = 0.0; dminus[f] = 0.0; }
            for (int64_t k = 0; k < nc; k++) {
                int64_t j = buf[k];
                if (j == i) continue;
                double d[3];
                orc_sep(x, y, z, L, i, j, d);
                for (int f = 0; f < 5; f++) {
                    double e = 0.5 * (d[0] * G[f][0] + d[1] * G[f][1] + d[2] * G[f][2]);
                    if (e > dplus[f]) dplus[f] = e;
                    if (e < dminus[f]) dminus[f] = e;
                }
            }
            double ratio = c->ncond_crit / ncond[i];
            double beta = c->beta_max * (ratio * ratio < 1.0 ? ratio * ratio : 1.0);
            if (beta < c->beta_min) beta = c->beta_min;
            for (int f = 0; f < 5; f++) {
                double rp = INFINITY, rm = INFINITY;
                if (dplus[f] > 0.0) rp = (fmax[f] - F[f][i]) / dplus[f];
                if (dminus[f] < 0.0) rm = (fmin[f] - F[f][i]) / dminus[f];
                double a = beta * (rp < rm ? rp : rm);
                alpha[5 * i + f] = a < 1.0 ? a : 1.0;
            }
        }
        free(buf);
    }
    orc_grid_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Riemann solvers                                                           */
/* ------------------------------------------------------------------------ */

/* Toro (2009) ch. 4: pressure function of one side and its derivative. */
static void orc_fK(double p, double rk, double pk, double ck, double g,
                   double *f, double *df)
{
    if (p > pk) {   /* shock */
        double A = 2.0 / ((g + 1.0) * rk);
        double Bk = (g - 1.0) / (g + 1.0) * pk;
        double q = sqrt(A / (p + Bk));
        *f = (p - pk) * q;
        *df = q * (1.0 - 0.5 * (p - pk) / (Bk + p));
    } else {        /* rarefaction */
        double pr = p / pk;
        *f = 2.0 * ck / (g - 1.0) * (pow(pr, (g - 1.0) / (2.0 * g)) - 1.0);
        *df = 1.0 / (rk * ck) * pow(pr, -(g + 1.0) / (2.0 * g));
    }
}

/* Toro's adaptive initial guess (Toro 2009 §9.5): PVRS when the pressure
 * ratio is small and the PVRS value lies between the data, otherwise the
 * two-rarefaction value (expansion) or the two-shock value. */
double orc_riemann_guess(double rl, double ul, double pl, double rr, double ur,
                         double pr, double g)
{
    double cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
    double ppv = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
    if (ppv < 0.0) ppv = 0.0;
    double pmin = pl < pr ? pl : pr, pmax = pl > pr ? pl : pr;
    if (pmax / pmin <= 2.0 && ppv >= pmin && ppv <= pmax) return ppv;
    if (ppv < pmin) {
        double z = (g - 1.0) / (2.0 * g);
        double pq = pow(pl / pr, z);
        double um = (pq * ul / cl + ur / cr + 2.0 / (g - 1.0) * (pq - 1.0)) / (pq / cl + 1.0 / cr);
        double tl = 1.0 + 0.5 * (g - 1.0) * (ul - um) / cl;
        double tr = 1.0 + 0.5 * (g - 1.0) * (um - ur) / cr;
        return 0.5 * (pl * pow(tl, 1.0 / z) + pr * pow(tr, 1.0 / z));
    }
    double gl = sqrt((2.0 / ((g + 1.0) * rl)) / ((g - 1.0) / (g + 1.0) * pl + ppv));
    double gr = sqrt((2.0 / ((g + 1.0) * rr)) / ((g - 1.0) / (g + 1.0) * pr + ppv));
    return (gl * pl + gr * pr - (ur - ul)) / (gl + gr);
}

/* Star pressure and velocity of the exact Riemann problem.  Newton from
 * p0 (p0 <= 0: Toro's adaptive guess), stopping when the relative change
 * 2|p_new-p|/(p_new+p) < tol, followed by one more Newton step.  After
 * max_newton iterations without convergence, bisection on a bracket of the
 * monotone pressure function.  Returns 1 on vacuum generation (p*, u* set to
 * 0), 0 otherwise.  *iters = Newton iterations taken (excluding the polish
 * step), *bisect = 1 if the bracket fallback ran. */
int orc_riemann_star(double rl, double ul, double pl, double rr, double ur, double pr,
                     double g, double p0, double tol, int max_newton,
                     double *pstar, double *ustar, int *iters, int *bisect)
{
    double cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
    double du = ur - ul;
    *iters = 0;
    *bisect = 0;
    if (2.0 / (g - 1.0) * (cl + cr) <= du) {
        *pstar = 0.0;
        *ustar = 0.0;
        return 1;
    }
    double p = p0 > 0.0 ? p0 : orc_riemann_guess(rl, ul, pl, rr, ur, pr, g);
    const double pfloor = 1e-300;
    if (!(p > pfloor)) p = pfloor;
    int conv = 0;
    double fl, dfl, fr, dfr;
    for (int k = 1; k <= max_newton; k++) {
        orc_fK(p, rl, pl, cl, g, &fl, &dfl);
        orc_fK(p, rr, pr, cr, g, &fr, &dfr);
        double pn = p - (fl + fr + du) / (dfl + dfr);
        if (!(pn > pfloor)) pn = pfloor;
        double ch = 2.0 * fabs(pn - p) / (pn + p);
        p = pn;
        *iters = k;
        if (ch < tol) { conv = 1; break; }
    }
    if (conv) {
        orc_fK(p, rl, pl, cl, g, &fl, &dfl);
        orc_fK(p, rr, pr, cr, g, &fr, &dfr);
        double pn = p - (fl + fr + du) / (dfl + dfr);
        if (pn > pfloor) p = pn;
    } else {
        /* f is increasing in p; f(0+) < 0 when there is no vacuum */
        double lo = 0.0, hi = pl > pr ? pl : pr;
        for (;;) {
            orc_fK(hi, rl, pl, cl, g, &fl, &dfl);
            orc_fK(hi, rr, pr, cr, g, &fr, &dfr);
            if (fl + fr + du > 0.0) break;
            lo = hi;
            hi *= 2.0;
        }
        for (int k = 0; k < 200; k++) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            orc_fK(mid, rl, pl, cl, g, &fl, &dfl);
            orc_fK(mid, rr, pr, cr, g, &fr, &dfr);
            if (fl + fr + du > 0.0) hi = mid; else lo = mid;
        }
        p = 0.5 * (lo + hi);
        *bisect = 1;
    }
    orc_fK(p, rl, pl, cl, g, &fl, &dfl);
    orc_fK(p, rr, pr, cr, g, &fr, &dfr);
    *pstar = p;
    *ustar = 0.5 * (ul + ur) + 0.5 * (fr - fl);
    return 0;
}

/* Sample the exact solution at x/t = 0 (Toro 2009 §4.5).  Returns the state
 * (rho, u, p) there and side = -1 when the point lies left of the contact,
 * +1 when right. */
void orc_riemann_sample(double rl, double ul, double pl, double rr, double ur, double pr,
                        double g, double ps, double us, double *rho, double *u,
                        double *p, int *side)
{
    double cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
    double gm = (g - 1.0) / (g + 1.0);
    if (0.0 <= us) {
        *side = -1;
        if (ps > pl) {   /* left shock */
            double sl = ul - cl * sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g));
            if (0.0 <= sl) { *rho = rl; *u = ul; *p = pl; }
            else { *rho = rl * (ps / pl + gm) / (gm * ps / pl + 1.0); *u = us; *p = ps; }
        } else {         /* left rarefaction */
            double shl = ul - cl;
            if (0.0 <= shl) { *rho = rl; *u = ul; *p = pl; }
            else {
                double cml = cl * pow(ps / pl, (g - 1.0) / (2.0 * g));
                double stl = us - cml;
                if (0.0 > stl) { *rho = rl * pow(ps / pl, 1.0 / g); *u = us; *p = ps; }
                else {  /* inside the fan */
                    double cc = 2.0 / (g + 1.0) + gm / cl * ul;
                    *rho = rl * pow(cc, 2.0 / (g - 1.0));
                    *u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul);
                    *p = pl * pow(cc, 2.0 * g / (g - 1.0));
                }
            }
        }
    } else {
        *side = 1;
        if (ps > pr) {   /* right shock */
            double sr = ur + cr * sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g));
            if (0.0 >= sr) { *rho = rr; *u = ur; *p = pr; }
            else { *rho = rr * (ps / pr + gm) / (gm * ps / pr + 1.0); *u = us; *p = ps; }
        } else {         /* right rarefaction */
            double shr = ur + cr;
            if (0.0 >= shr) { *rho = rr; *u = ur; *p = pr; }
            else {
                double cmr = cr * pow(ps / pr, (g - 1.0) / (2.0 * g));
                double str = us + cmr;
                if (0.0 <= str) { *rho = rr * pow(ps / pr, 1.0 / g); *u = us; *p = ps; }
                else {
                    double cc = 2.0 / (g + 1.0) - gm / cr * ur;
                    *rho = rr * pow(cc, 2.0 / (g - 1.0));
                    *u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur);
                    *p = pr * pow(cc, 2.0 * g / (g - 1.0));
                }
            }
        }
    }
}

/* HLLC (Toro 2009 ch. 10) with the pressure-based wave-speed estimates of
 * §10.6.  One-dimensional problem along the face normal with transverse
 * velocities wl, wr (3-vectors, normal part removed) carried passively.
 * Returns the face-frame flux density (mass, momentum 3-vector, energy) at
 * x/t = 0, plus the star pressure and contact speed. */
void orc_hllc(double rl, double ul, double pl, const double wl[3],
              double rr, double ur, double pr, const double wr[3],
              const double nhat[3], double g, double F[5], double *pstar, double *sstar)
{
    double cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
    double ppv = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
    if (ppv < 0.0) ppv = 0.0;
    double ql = ppv <= pl ? 1.0 : sqrt(1.0 + (g + 1.0) / (2.0 * g) * (ppv / pl - 1.0));
    double qr = ppv <= pr ? 1.0 : sqrt(1.0 + (g + 1.0) / (2.0 * g) * (ppv / pr - 1.0));
    double sl = ul - cl * ql, sr = ur + cr * qr;
    double ss = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) /
                (rl * (sl - ul) - rr * (sr - ur));
    *sstar = ss;
    *pstar = pl + rl * (sl - ul) * (ss - ul);
    /* conserved state and physical flux along n of each side */
    double w2l = wl[0] * wl[0] + wl[1] * wl[1] + wl[2] * wl[2];
    double w2r = wr[0] * wr[0] + wr[1] * wr[1] + wr[2] * wr[2];
    double El = pl / (g - 1.0) + 0.5 * rl * (ul * ul + w2l);
    double Er = pr / (g - 1.0) + 0.5 * rr * (ur * ur + w2r);
    double Ul[5], Ur[5], Fl[5], Fr[5];
    /* components: mass, normal momentum, energy; transverse handled below */
    Ul[0] = rl; Ul[1] = rl * ul; Ul[2] = El;
    Ur[0] = rr; Ur[1] = rr * ur; Ur[2] = Er;
    Fl[0] = rl * ul; Fl[1] = rl * ul * ul + pl; Fl[2] = ul * (El + pl);
    Fr[0] = rr * ur; Fr[1] = rr * ur * ur + pr; Fr[2] = ur * (Er + pr);
    double fm, fn, fe, wt[3];
    if (0.0 <= sl) {
        fm = Fl[0]; fn = Fl[1]; fe = Fl[2];
        for (int a = 0; a < 3; a++) wt[a] = wl[a];
    } else if (0.0 <= ss) {
        double k = rl * (sl - ul) / (sl - ss);
        double us0 = k, us1 = k * ss, us2 = k * (El / rl + (ss - ul) * (ss + pl / (rl * (sl - ul))));
        fm = Fl[0] + sl * (us0 - Ul[0]);
        fn = Fl[1] + sl * (us1 - Ul[1]);
        fe = Fl[2] + sl * (us2 - Ul[2]);
        for (int a = 0; a < 3; a++) wt[a] = wl[a];
    } else if (0.0 <= sr) {
        double k = rr * (sr - ur) / (sr - ss);
        double us0 = k, us1 = k * ss, us2 = k * (Er / rr + (ss - ur) * (ss + pr / (rr * (sr - ur))));
        fm = Fr[0] + sr * (us0 - Ur[0]);
        fn = Fr[1] + sr * (us1 - Ur[1]);
        fe = Fr[2] + sr * (us2 - Ur[2]);
        for (int a = 0; a < 3; a++) wt[a] = wr[a];
    } else {
        fm = Fr[0]; fn = Fr[1]; fe = Fr[2];
        for (int a = 0; a < 3; a++) wt[a] = wr[a];
    }
    /* transverse momentum is advected with the mass flux of the upwind side
     * (the HLLC star states keep each side's transverse velocity) */
    F[0] = fm;
    for (int a = 0; a < 3; a++) F[1 + a] = fn * nhat[a] + fm * wt[a];
    F[4] = fe;
}

/* ------------------------------------------------------------------------ */
/* fluxes, §2.3.3 (A_ij after Eq. 13), §2.3.4 (Eqs. 15-16), §2.3.6           */
/* ------------------------------------------------------------------------ */

static int sgn(double v) { return (v > 0.0) - (v < 0.0); }

/* Pairwise limiter (Hopkins 2015 eq. B4, psi1, psi2 of §2.3.6) applied to
 * the face value e extrapolated from the side whose cell value is a, the
 * other side's cell value being b.  The bracket [lo - psi1 d, hi + psi1 d]
 * is shrunk so as not to change sign only for positive quantities
 * (positive != 0: density, pressure); velocities use the plain bracket so
 * that the limiter commutes with a Galilean boost. */
double orc_pair_limit(double e, double a, double b, double psi1, double psi2, int positive)
{
    if (a == b) return a;
    double d = fabs(a - b);
    double mean = 0.5 * (a + b);
    double d1 = psi1 * d, d2 = psi2 * d;
    double lo = a < b ? a : b, hi = a > b ? a : b;
    double lo_x, hi_x;
    if (!positive || sgn(lo - d1) == sgn(lo)) lo_x = lo - d1;
    else lo_x = (lo == 0.0) ? 0.0 : lo / (1.0 + d1 / fabs(lo));
    if (!positive || sgn(hi + d1) == sgn(hi)) hi_x = hi + d1;
    else hi_x = (hi == 0.0) ? 0.0 : hi / (1.0 + d1 / fabs(hi));
    if (a < b) {
        double t = e < mean + d2 ? e : mean + d2;
        return t > lo_x ? t : lo_x;
    }
    double t = e > mean - d2 ? e : mean - d2;
    return t < hi_x ? t : hi_x;
}

/* Neumaier-compensated accumulator */
typedef struct { double s, c; } orc_ksum;
static void ks_add(orc_ksum *k, double v)
{
    double t = k->s + v;
    if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
    else k->c += (v - t) + k->s;
    k->s = t;
}

/* Per-face computation for the unordered pair (i, j), oriented i -> j.
 * Returns c = dt |A_ij| F (mass, momentum 3, energy) in the lab frame:
 * particle i loses c, particle j gains c.  tl, tr: the times over which the
 * predictor advances the i and j states (dt/2 for a global step; under
 * individual timesteps the time since the particle's state was taken plus
 * half the face's step). */
static void orc_face(const orc_config *c, int64_t i, int64_t j, const double d[3], double r,
                     const double *h, const double *omega, const double *B6,
                     const double *Wp[5], const double *grad, const double *alpha, double dt,
                     double tl, double tr, const double *pguess, double cflux[5],
                     orc_flux_stats *st, double *face_out)
{
    double g = c->gamma;
    /* face vector A_ij = omega_i omega_j [B_i dx W(r,h_i) + B_j dx W(r,h_j)] */
    double Bi[9], Bj[9];
    orc_B9(B6, i, Bi);
    orc_B9(B6, j, Bj);
    double wi = orc_kernel_W(c->kernel, r, h[i]);
    double wj = orc_kernel_W(c->kernel, r, h[j]);
    double A[3];
    for (int a = 0; a < 3; a++) {
        double ti = Bi[3 * a + 0] * d[0] + Bi[3 * a + 1] * d[1] + Bi[3 * a + 2] * d[2];
        double tj = Bj[3 * a + 0] * d[0] + Bj[3 * a + 1] * d[1] + Bj[3 * a + 2] * d[2];
        A[a] = omega[i] * omega[j] * (ti * wi + tj * wj);
    }
    double Amag = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    for (int k = 0; k < 5; k++) cflux[k] = 0.0;
    if (!(Amag > 0.0)) return;
    double nh[3] = {A[0] / Amag, A[1] / Amag, A[2] / Amag};

    /* cell states and limited gradients */
    double Wi[5], Wj[5], Gi[5][3], Gj[5][3];
    for (int f = 0; f < 5; f++) {
        Wi[f] = Wp[f][i];
        Wj[f] = Wp[f][j];
        for (int a = 0; a < 3; a++) {
            Gi[f][a] = alpha[5 * i + f] * grad[15 * i + 3 * f + a];
            Gj[f][a] = alpha[5 * j + f] * grad[15 * j + 3 * f + a];
        }
    }
    /* spatial extrapolation to the midpoint, Eqs. 20-21 */
    double L_[5], R_[5];
    for (int f = 0; f < 5; f++) {
        L_[f] = Wi[f] + 0.5 * (d[0] * Gi[f][0] + d[1] * Gi[f][1] + d[2] * Gi[f][2]);
        R_[f] = Wj[f] - 0.5 * (d[0] * Gj[f][0] + d[1] * Gj[f][1] + d[2] * Gj[f][2]);
        if (c->limiter) {
            int pos = (f == 0 || f == 4);
            L_[f] = orc_pair_limit(L_[f], Wi[f], Wj[f], c->psi1, c->psi2, pos);
            R_[f] = orc_pair_limit(R_[f], Wj[f], Wi[f], c->psi1, c->psi2, pos);
        }
    }
    /* half-step predictor in each particle's own frame (Eq. 16):
     * d rho/dt = -rho div v, dv/dt = -grad p / rho, dp/dt = -gamma p div v */
    if (c->time_extrap) {
        double divi = Gi[1][0] + Gi[2][1] + Gi[3][2];
        double divj = Gj[1][0] + Gj[2][1] + Gj[3][2];
        L_[0] -= tl * Wi[0] * divi;
        R_[0] -= tr * Wj[0] * divj;
        for (int a = 0; a < 3; a++) {
            L_[1 + a] -= tl * Gi[4][a] / Wi[0];
            R_[1 + a] -= tr * Gj[4][a] / Wj[0];
        }
        L_[4] -= tl * g * Wi[4] * divi;
        R_[4] -= tr * g * Wj[4] * divj;
    }
    if (!(L_[0] > 0.0 && L_[4] > 0.0 && R_[0] > 0.0 && R_[4] > 0.0)) {
        for (int f = 0; f < 5; f++) { L_[f] = Wi[f]; R_[f] = Wj[f]; }
        st->first_order++;
    }
    /* boost to the frame of the face, project on n.  The fluxes are those of
     * the half step (Eq. 16), so the face moves with the mean of the two
     * particles' velocities at the half step: each velocity advanced by the
     * predictor's acceleration -grad p / rho over tl (resp. tr), the same
     * times as the face states (with the predictor off: the velocities at
     * the step's start). */
    double vf[3];
    for (int a = 0; a < 3; a++) {
        double vi = Wi[1 + a], vj = Wj[1 + a];
        if (c->time_extrap) {
            vi -= tl * Gi[4][a] / Wi[0];
            vj -= tr * Gj[4][a] / Wj[0];
        }
        vf[a] = 0.5 * (vi + vj);
    }
    double vl[3], vr[3];
    for (int a = 0; a < 3; a++) { vl[a] = L_[1 + a] - vf[a]; vr[a] = R_[1 + a] - vf[a]; }
    double ul = vl[0] * nh[0] + vl[1] * nh[1] + vl[2] * nh[2];
    double ur = vr[0] * nh[0] + vr[1] * nh[1] + vr[2] * nh[2];
    double wl[3], wr[3];
    for (int a = 0; a < 3; a++) { wl[a] = vl[a] - ul * nh[a]; wr[a] = vr[a] - ur * nh[a]; }
    double rl = L_[0], pl = L_[4], rr = R_[0], pr = R_[4];
    if (face_out) {
        face_out[0] = rl; face_out[1] = ul; face_out[2] = pl;
        face_out[3] = rr; face_out[4] = ur; face_out[5] = pr;
    }

    double F[5];
    if (c->riemann == 1) {
        double ps, ss;
        orc_hllc(rl, ul, pl, wl, rr, ur, pr, wr, nh, g, F, &ps, &ss);
        if (c->scheme == 1) {
            F[0] = 0.0;
            for (int a = 0; a < 3; a++) F[1 + a] = ps * nh[a];
            F[4] = ps * ss;
        }
        st->faces++;
    } else {
        double ps, us;
        int it, bis;
        double p0 = pguess ? *pguess : -1.0;
        int vac = orc_riemann_star(rl, ul, pl, rr, ur, pr, g, p0, c->p_tol, c->max_newton,
                                   &ps, &us, &it, &bis);
        st->faces++;
        st->newton_iters += it;
        st->bisect_fallback += bis;
        if (face_out) { face_out[6] = ps; face_out[7] = us; face_out[8] = it; }
        if (vac) {
            st->vacuum++;
            return;  /* zero flux */
        }
        if (c->scheme == 1) {
            /* MFM: the face moves with the contact: no mass flux */
            F[0] = 0.0;
            for (int a = 0; a < 3; a++) F[1 + a] = ps * nh[a];
            F[4] = ps * us;
        } else {
            double rs, uu, pp;
            int side;
            orc_riemann_sample(rl, ul, pl, rr, ur, pr, g, ps, us, &rs, &uu, &pp, &side);
            const double *wt = side < 0 ? wl : wr;
            double v2 = uu * uu + wt[0] * wt[0] + wt[1] * wt[1] + wt[2] * wt[2];
            double etot = 0.5 * rs * v2 + pp / (g - 1.0);
            F[0] = rs * uu;
            for (int a = 0; a < 3; a++) F[1 + a] = rs * uu * (uu * nh[a] + wt[a]) + pp * nh[a];
            F[4] = uu * (etot + pp);
        }
    }
    /* de-boost to the lab frame */
    double vf2 = vf[0] * vf[0] + vf[1] * vf[1] + vf[2] * vf[2];
    double Fe = F[4] + (F[1] * vf[0] + F[2] * vf[1] + F[3] * vf[2]) + 0.5 * F[0] * vf2;
    double Fp[3];
    for (int a = 0; a < 3; a++) Fp[a] = F[1 + a] + F[0] * vf[a];
    double s = dt * Amag;
    cflux[0] = s * F[0];
    cflux[1] = s * Fp[0];
    cflux[2] = s * Fp[1];
    cflux[3] = s * Fp[2];
    cflux[4] = s * Fe;
}

/* All unordered pairs {i, j} with r_ij < max(h_i, h_j), i < j, in ascending
 * (i, j) order; returns the pair count (nothing is written past cap).
 * pairs[2k] = i, pairs[2k+1] = j. */
int64_t orc_flux_pairs(int64_t n, const double *x, const double *y, const double *z,
                       const double *L, const double *h, int64_t cap, int64_t *pairs)
{
    double hmax = 0.0;
    for (int64_t i = 0; i < n; i++) if (h[i] > hmax) hmax = h[i];
    orc_grid g;
    orc_grid_build(&g, n, x, y, z, L, hmax);
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; pass++) {
        #pragma omp parallel
        {
            int64_t *buf = NULL, bcap = 0;
            #pragma omp for schedule(dynamic, 256)
            for (int64_t i = 0; i < n; i++) {
                int64_t nc = orc_gather(&g, x, y, z, i, hmax, &buf, &bcap);
                int64_t c = 0;
                for (int64_t k = 0; k < nc; k++) {
                    int64_t j = buf[k];
                    if (j <= i) continue;
                    double d[3];
                    double r2 = orc_sep(x, y, z, L, i, j, d);
                    double hm = h[i] > h[j] ? h[i] : h[j];
                    if (r2 < hm * hm) {
                        if (pass == 1) { pairs[2 * (cnt[i] + c)] = i; pairs[2 * (cnt[i] + c) + 1] = j; }
                        c++;
                    }
                }
                if (pass == 0) cnt[i + 1] = c;
            }
            free(buf);
        }
        if (pass == 0) {
            for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
            if (cnt[n] > cap) break;
        }
    }
    int64_t np = cnt[n];
    free(cnt);
    orc_grid_free(&g);
    return np;
}

/* dQ_i = -dt sum_j F_ij . A_ij  (Eq. 16) for (mass, momentum, total energy),
 * accumulated per particle with Neumaier compensation over the pair list in
 * ascending (i, j) order, and dU_i from Eq. 24 with the start-of-step
 * velocity.  dQ[6 i + (0..5)] = (dm, dpx, dpy, dpz, dE, dU).
 * pair_guess (optional, one per pair) overrides the Riemann initial guess.
 * face_out (optional, 9 per pair): rho_L, u_L, p_L, rho_R, u_R, p_R, p*, u*,
 * Newton iterations. */
static void orc_fluxes_impl(const orc_config *c, int64_t n, const double *x, const double *y,
                            const double *z, const double *L, const double *h,
                            const double *omega, const double *B6, const double *rho,
                            const double *vx, const double *vy, const double *vz,
                            const double *p, const double *grad, const double *alpha, double dt,
                            const double *dtp, const double *toff, int64_t npairs,
                            const int64_t *pairs, const double *pair_guess, double *dQ,
                            orc_flux_stats *st, double *face_out, double *dQabs, double *dM,
                            const double *A, double *dS);

void orc_fluxes(const orc_config *c, int64_t n, const double *x, const double *y,
                const double *z, const double *L, const double *h, const double *omega,
                const double *B6, const double *rho, const double *vx, const double *vy,
                const double *vz, const double *p, const double *grad, const double *alpha,
                double dt, int64_t npairs, const int64_t *pairs, const double *pair_guess,
                double *dQ, orc_flux_stats *st, double *face_out, double *dQabs, double *dM,
                const double *A, double *dS)
{
    orc_fluxes_impl(c, n, x, y, z, L, h, omega, B6, rho, vx, vy, vz, p, grad, alpha, dt, NULL,
                    NULL, npairs, pairs, pair_guess, dQ, st, face_out, dQabs, dM, A, dS);
}

/* The face arithmetic of a rung sub-step on its own, for the tests: dtp[i]
 * the particle's step and toff[i] the time since its state was taken (the
 * impl's individual-timestep form below; dQ, stats and face states as in
 * orc_fluxes). */
void orc_fluxes_rung(const orc_config *c, int64_t n, const double *x, const double *y,
                     const double *z, const double *L, const double *h, const double *omega,
                     const double *B6, const double *rho, const double *vx, const double *vy,
                     const double *vz, const double *p, const double *grad, const double *alpha,
                     const double *dtp, const double *toff, int64_t npairs,
                     const int64_t *pairs, double *dQ, orc_flux_stats *st, double *face_out)
{
    orc_fluxes_impl(c, n, x, y, z, L, h, omega, B6, rho, vx, vy, vz, p, grad, alpha, 0.0, dtp,
                    toff, npairs, pairs, NULL, dQ, st, face_out, NULL, NULL, NULL, NULL);
}

/* orc_fluxes with individual timesteps (dtp non-NULL): the face (i, j)
 * takes dt_ij = min(dtp_i, dtp_j) (§2.3.4, the rule of Springel 2010 §7.2),
 * and its predictor advances each side over toff + dt_ij / 2, toff the time
 * since that particle's state was taken.  dt is unused then. */
static void orc_fluxes_impl(const orc_config *c, int64_t n, const double *x, const double *y,
                            const double *z, const double *L, const double *h,
                            const double *omega, const double *B6, const double *rho,
                            const double *vx, const double *vy, const double *vz,
                            const double *p, const double *grad, const double *alpha, double dt,
                            const double *dtp, const double *toff, int64_t npairs,
                            const int64_t *pairs, const double *pair_guess, double *dQ,
                            orc_flux_stats *st, double *face_out, double *dQabs, double *dM,
                            const double *A, double *dS)
{
    const double *Wp[5] = {rho, vx, vy, vz, p};
    double *cf = (double *)malloc((size_t)(npairs > 0 ? npairs : 1) * 5 * sizeof(double));
    orc_flux_stats tot;
    memset(&tot, 0, sizeof tot);
    #pragma omp parallel
    {
        orc_flux_stats loc;
        memset(&loc, 0, sizeof loc);
        #pragma omp for schedule(dynamic, 1024)
        for (int64_t k = 0; k < npairs; k++) {
            int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
            double d[3];
            double r = sqrt(orc_sep(x, y, z, L, i, j, d));
            double dtf = dt, tl = 0.5 * dt, tr = 0.5 * dt;
            if (dtp) {
                dtf = dtp[i] < dtp[j] ? dtp[i] : dtp[j];
                tl = toff[i] + 0.5 * dtf;
                tr = toff[j] + 0.5 * dtf;
            }
            orc_face(c, i, j, d, r, h, omega, B6, Wp, grad, alpha, dtf, tl, tr,
                     pair_guess ? pair_guess + k : NULL, cf + 5 * k, &loc,
                     face_out ? face_out + 9 * k : NULL);
        }
        #pragma omp critical
        {
            tot.newton_iters += loc.newton_iters;
            tot.faces += loc.faces;
            tot.vacuum += loc.vacuum;
            tot.bisect_fallback += loc.bisect_fallback;
            tot.first_order += loc.first_order;
        }
    }
    tot.pairs = npairs;
    if (st) *st = tot;
    /* sequential, compensated scatter: i loses c, j gains c */
    orc_ksum *acc = (orc_ksum *)calloc((size_t)n * 5, sizeof(orc_ksum));
    for (int64_t k = 0; k < npairs; k++) {
        int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        for (int q = 0; q < 5; q++) {
            ks_add(&acc[5 * i + q], -cf[5 * k + q]);
            ks_add(&acc[5 * j + q], cf[5 * k + q]);
        }
    }
    for (int64_t i = 0; i < n; i++) {
        double dm = acc[5 * i + 0].s + acc[5 * i + 0].c;
        double dpx = acc[5 * i + 1].s + acc[5 * i + 1].c;
        double dpy = acc[5 * i + 2].s + acc[5 * i + 2].c;
        double dpz = acc[5 * i + 3].s + acc[5 * i + 3].c;
        double dE = acc[5 * i + 4].s + acc[5 * i + 4].c;
        double v2 = vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
        double dU = dE - (vx[i] * dpx + vy[i] * dpy + vz[i] * dpz) + 0.5 * v2 * dm;
        dQ[6 * i + 0] = dm;
        dQ[6 * i + 1] = dpx;
        dQ[6 * i + 2] = dpy;
        dQ[6 * i + 3] = dpz;
        dQ[6 * i + 4] = dE;
        dQ[6 * i + 5] = dU;
    }
    free(acc);
    /* the mass exchanged through the faces times the separation, for the
     * gravitational work of §2.3.8: sum_j dm_ij r_ij with dm_ij the mass i
     * gains from j and r_ij = x_i - x_j.  A face gives c_m from i to j, so
     * both particles add c_m (x_j - x_i) (compensated sums) */
    if (dM) {
        orc_ksum *am = (orc_ksum *)calloc((size_t)n * 3, sizeof(orc_ksum));
        for (int64_t k = 0; k < npairs; k++) {
            int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
            double d[3];
            orc_sep(x, y, z, L, i, j, d);
            for (int q = 0; q < 3; q++) {
                ks_add(&am[3 * i + q], cf[5 * k] * d[q]);
                ks_add(&am[3 * j + q], cf[5 * k] * d[q]);
            }
        }
        for (int64_t i = 0; i < 3 * n; i++) dM[i] = am[i].s + am[i].c;
        free(am);
    }
    /* the extensive entropy m A carried by the mass fluxes (§2.3.7, the MFV
     * entropy advection): a face giving c_m > 0 from i to j carries
     * c_m A_i, one with c_m < 0 carries c_m A_j (the upwind entropic function) */
    if (dS && A) {
        orc_ksum *as = (orc_ksum *)calloc((size_t)n, sizeof(orc_ksum));
        for (int64_t k = 0; k < npairs; k++) {
            int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
            const double cm = cf[5 * k];
            const double sflux = cm * (cm > 0.0 ? A[i] : A[j]);
            ks_add(&as[i], -sflux);
            ks_add(&as[j], sflux);
        }
        for (int64_t i = 0; i < n; i++) dS[i] = as[i].s + as[i].c;
        free(as);
    }
    /* scale of the per-particle flux error (sum over the particle's faces of
     * |c| per component), used to normalise comparisons of dQ whose net
     * value may cancel */
    if (dQabs) {
        memset(dQabs, 0, (size_t)n * 5 * sizeof(double));
        for (int64_t k = 0; k < npairs; k++) {
            int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
            for (int q = 0; q < 5; q++) {
                dQabs[5 * i + q] += fabs(cf[5 * k + q]);
                dQabs[5 * j + q] += fabs(cf[5 * k + q]);
            }
        }
    }
    free(cf);
}

/* ------------------------------------------------------------------------ */
/* one full step (§2.3.4 with a global dt, Eqs. 15-16, 23-24, 31-32)          */
/* ------------------------------------------------------------------------ */

typedef struct {
    double dt;            /* timestep used */
    double dt_next;       /* CFL estimate after... (from the start-of-step state) */
    int ngb_rounds;       /* N_cond growth rounds taken */
    int64_t ncond_fail;   /* particles still above the threshold at the end */
    int64_t grad_pairs;   /* directed pairs j != i with r < h_i */
    orc_flux_stats flux;
} orc_step_info;

/* State (caller order): x, y, z, m, px, py, pz, E, U, h (in: guess; out:
 * solved), omega (out).  dt <= 0 selects the CFL timestep
 * min_i C_CFL h_i / v_sig,i (Eqs. 31-32).  Steps: density (Eq. 18), N_cond
 * guard (§2.3.5), primitives, gradients + limiter, fluxes (Eq. 16),
 * conserved update, internal energy (Eq. 24), drift with the mean of the
 * old and new velocity.  acc (3 per particle, may be NULL): an external
 * (gravitational) acceleration held fixed over the step; its sources are
 * added to the updated state by the trapezoidal rule of §2.3.4 between the
 * start-of-step state and the state the fluxes updated: momentum
 * dt/2 (m^n + m~) a, energy dt/2 (P^n + P~).a plus the work of the
 * exchanged mass, (1/2) a . sum_j dm_ij r_ij (§2.3.8); it also enters the
 * pressure switch through E_grav = m |a| h (§2.3.7).  The internal energy
 * takes no gravitational source.  Optional outputs (NULL to skip): B6,
 * grad, alpha, ncond, dQ (the hydrodynamic change only). */
int orc_step(const orc_config *c, int64_t n, double *x, double *y, double *z,
             const double *L, double *m, double *px, double *py, double *pz, double *E,
             double *U, double *h, double *omega, const double *acc, double *A, double dt,
             double *B6_out, double *grad_out, double *alpha_out, double *ncond_out,
             double *dQ_out, orc_step_info *info)
{
    int status = ORC_OK;
    double *nngb = (double *)malloc((size_t)n * sizeof(double));
    int32_t *act = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    double *B6 = (double *)malloc((size_t)n * 6 * sizeof(double));
    double *nc = (double *)malloc((size_t)n * sizeof(double));
    double *rho = (double *)malloc((size_t)n * sizeof(double));
    double *vx = (double *)malloc((size_t)n * sizeof(double));
    double *vy = (double *)malloc((size_t)n * sizeof(double));
    double *vz = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *grad = (double *)malloc((size_t)n * 15 * sizeof(double));
    double *alpha = (double *)malloc((size_t)n * 5 * sizeof(double));
    double *vsig = (double *)malloc((size_t)n * sizeof(double));
    double *dQ = (double *)malloc((size_t)n * 6 * sizeof(double));
    for (int64_t i = 0; i < n; i++) { nngb[i] = c->n_ngb; act[i] = 1; }
    int rounds = 0;
    int64_t fail = 0;
    for (;;) {
        int s = orc_density(c, n, x, y, z, L, nngb, act, h, omega, NULL);
        if (s != ORC_OK) status = s;
        orc_matrices(c, n, x, y, z, L, h, omega, B6, NULL, nc);
        fail = 0;
        for (int64_t i = 0; i < n; i++) {
            act[i] = nc[i] > c->ncond_crit;
            fail += act[i];
        }
        if (fail == 0 || rounds == c->max_ngb_grow) break;
        for (int64_t i = 0; i < n; i++) if (act[i]) nngb[i] *= c->ngb_grow;
        rounds++;
    }
    if (fail && status == ORC_OK) status = ORC_ENCOND;
    /* entropy switch (§2.3.7): E_kin^max at the solved h; the entropic
     * function A follows the pressure actually used (resynchronised where it
     * came from the energies; entries <= 0 are unset and resynchronised) */
    const int ent = c->entropy && A;
    double *ekm = ent ? (double *)malloc((size_t)n * sizeof(double)) : NULL;
    int32_t *src = ent ? (int32_t *)malloc((size_t)n * sizeof(int32_t)) : NULL;
    if (ent) orc_ekin_max(n, x, y, z, L, h, m, px, py, pz, ekm);
    orc_primitives(c, n, m, px, py, pz, E, U, omega, h, acc, ent ? A : NULL, ekm, src, rho, vx,
                   vy, vz, p);
    if (ent)
        for (int64_t i = 0; i < n; i++)
            if (src[i] != 1) A[i] = p[i] / pow(rho[i], c->gamma);
    orc_gradients(c, n, x, y, z, L, h, omega, rho, vx, vy, vz, p, B6, nc, grad, alpha, vsig);
    double dtc = INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double t = c->c_cfl * h[i] / vsig[i];
        if (t < dtc) dtc = t;
    }
    if (!(dt > 0.0)) dt = dtc;
    /* pairs */
    int64_t cap = n * 64;
    int64_t *pairs = (int64_t *)malloc((size_t)cap * 2 * sizeof(int64_t));
    int64_t np = orc_flux_pairs(n, x, y, z, L, h, cap, pairs);
    if (np > cap) {
        free(pairs);
        cap = np;
        pairs = (int64_t *)malloc((size_t)cap * 2 * sizeof(int64_t));
        np = orc_flux_pairs(n, x, y, z, L, h, cap, pairs);
    }
    orc_flux_stats fst;
    double *dM = acc ? (double *)malloc((size_t)n * 3 * sizeof(double)) : NULL;
    double *dS = ent ? (double *)malloc((size_t)n * sizeof(double)) : NULL;
    orc_fluxes(c, n, x, y, z, L, h, omega, B6, rho, vx, vy, vz, p, grad, alpha, dt, np, pairs,
               NULL, dQ, &fst, NULL, NULL, dM, ent ? A : NULL, dS);
    free(pairs);
    /* directed gradient pairs */
    if (info) {
        int64_t *off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
        int64_t tot = orc_neighbours(n, x, y, z, L, h, 1, 0, off, NULL);
        info->grad_pairs = tot - n;
        free(off);
    }
    /* update */
    for (int64_t i = 0; i < n; i++) {
        double vox = vx[i], voy = vy[i], voz = vz[i];
        const double m0 = m[i], p0[3] = {px[i], py[i], pz[i]};
        m[i] += dQ[6 * i + 0];
        /* entropy: constant along MFM particles (no mass flux); MFV carries
         * m A with the mass fluxes */
        if (ent && c->scheme == 0) A[i] = (m0 * A[i] + dS[i]) / m[i];
        px[i] += dQ[6 * i + 1];
        py[i] += dQ[6 * i + 2];
        pz[i] += dQ[6 * i + 3];
        E[i] += dQ[6 * i + 4];
        U[i] += dQ[6 * i + 5];
        if (acc) {
            const double *a = acc + 3 * i;
            const double ph[3] = {px[i], py[i], pz[i]};   /* hydro-updated */
            const double w = 0.5 * dt * (m0 + m[i]);
            double eg = 0.0, ex = 0.0;
            for (int q = 0; q < 3; q++) {
                eg += (p0[q] + ph[q]) * a[q];
                ex += a[q] * dM[3 * i + q];
            }
            px[i] += w * a[0];
            py[i] += w * a[1];
            pz[i] += w * a[2];
            E[i] += 0.5 * dt * eg + 0.5 * ex;
        }
        double nx = px[i] / m[i], ny = py[i] / m[i], nz = pz[i] / m[i];
        double xs[3] = {x[i] + dt * 0.5 * (vox + nx), y[i] + dt * 0.5 * (voy + ny),
                        z[i] + dt * 0.5 * (voz + nz)};
        for (int a = 0; a < 3; a++) {
            if (xs[a] >= L[a]) xs[a] -= L[a];
            if (xs[a] < 0.0) xs[a] += L[a];
        }
        x[i] = xs[0]; y[i] = xs[1]; z[i] = xs[2];
    }
    if (B6_out) memcpy(B6_out, B6, (size_t)n * 6 * sizeof(double));
    if (grad_out) memcpy(grad_out, grad, (size_t)n * 15 * sizeof(double));
    if (alpha_out) memcpy(alpha_out, alpha, (size_t)n * 5 * sizeof(double));
    if (ncond_out) memcpy(ncond_out, nc, (size_t)n * sizeof(double));
    free(dM);
    free(dS);
    free(ekm);
    free(src);
    if (dQ_out) memcpy(dQ_out, dQ, (size_t)n * 6 * sizeof(double));
    if (info) {
        info->dt = dt;
        info->dt_next = dtc;
        info->ngb_rounds = rounds;
        info->ncond_fail = fail;
        info->flux = fst;
    }
    free(nngb); free(act); free(B6); free(nc); free(rho); free(vx); free(vy); free(vz);
    free(p); free(grad); free(alpha); free(vsig); free(dQ);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Individual timesteps (§2.3.4 power-of-two hierarchy, §2.3.10 criteria)    */
/* ------------------------------------------------------------------------ */

/* The rung of one particle (§2.3.10): the smallest integer r >= 0 with
 * min(dt_cfl, dt_acc) > 2^-r dt0, at most max_rung (*capped set when even
 * max_rung does not satisfy the criterion). */
int orc_rung_select(double dt_cfl, double dt_acc, double dt0, int max_rung, int *capped)
{
    const double t = dt_cfl < dt_acc ? dt_cfl : dt_acc;
    int r = 0;
    while (r < max_rung && !(t > ldexp(dt0, -r))) r++;
    if (capped) *capped = !(t > ldexp(dt0, -r));
    return r;
}

/* The neighbour limiter of §2.3.10 (Saitoh & Makino 2009): interacting
 * particles (the unordered flux pairs) differ by at most two rungs.  Rungs
 * only rise: r_i <- max(r_i, r_j - 2) over the pairs, swept until nothing
 * changes (the least such assignment above the input).  Returns the sweeps. */
int orc_rung_limit(int64_t npairs, const int64_t *pairs, int32_t *rung)
{
    int sweeps = 0, changed = 1;
    while (changed) {
        changed = 0;
        sweeps++;
        for (int64_t k = 0; k < npairs; k++) {
            const int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
            if (rung[i] < rung[j] - 2) { rung[i] = rung[j] - 2; changed = 1; }
            if (rung[j] < rung[i] - 2) { rung[j] = rung[i] - 2; changed = 1; }
        }
    }
    return sweeps;
}

typedef struct {
    int status;
    int rung_max;            /* deepest rung of the base step */
    int64_t substeps;        /* 2^rung_max */
    int64_t active_steps;    /* particle steps taken over the base step */
    int64_t faces;           /* faces solved over the base step */
    int64_t capped;          /* particles the criteria wanted beyond max_rung */
    int limiter_sweeps;
} orc_rung_info;

/* density + N_cond guard (§2.3.5) for the particles with ract set (all when
 * ract is NULL): N_NGB restarts from n_ngb; h and omega of the others stay.
 * B6 and nc receive the matrices of every particle (the caller keeps the
 * rows it needs). */
static int orc_density_guard(const orc_config *c, int64_t n, const double *x, const double *y,
                             const double *z, const double *L, const int32_t *ract, double *h,
                             double *omega, double *B6, double *nc, int *rounds_out,
                             int64_t *fail_out)
{
    int status = ORC_OK;
    double *nngb = (double *)malloc((size_t)n * sizeof(double));
    int32_t *act = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; i++) { nngb[i] = c->n_ngb; act[i] = ract ? ract[i] : 1; }
    int rounds = 0;
    int64_t fail = 0;
    for (;;) {
        int s = orc_density(c, n, x, y, z, L, nngb, act, h, omega, NULL);
        if (s != ORC_OK) status = s;
        orc_matrices(c, n, x, y, z, L, h, omega, B6, NULL, nc);
        fail = 0;
        for (int64_t i = 0; i < n; i++) {
            act[i] = (ract ? ract[i] : 1) && nc[i] > c->ncond_crit;
            fail += act[i];
        }
        if (fail == 0 || rounds == c->max_ngb_grow) break;
        for (int64_t i = 0; i < n; i++) if (act[i]) nngb[i] *= c->ngb_grow;
        rounds++;
    }
    if (fail && status == ORC_OK) status = ORC_ENCOND;
    free(nngb);
    free(act);
    if (rounds_out) *rounds_out = rounds;
    if (fail_out) *fail_out = fail;
    return status;
}

/* unordered flux pairs r_ij < max(h_i, h_j) at the current positions;
 * *np receives the count; the caller frees the array */
static int64_t *orc_pairs_alloc(int64_t n, const double *x, const double *y, const double *z,
                                const double *L, const double *h, int64_t *np)
{
    int64_t cap = n * 64 + 64;
    int64_t *pairs = (int64_t *)malloc((size_t)cap * 2 * sizeof(int64_t));
    int64_t k = orc_flux_pairs(n, x, y, z, L, h, cap, pairs);
    if (k > cap) {
        free(pairs);
        cap = k;
        pairs = (int64_t *)malloc((size_t)cap * 2 * sizeof(int64_t));
        k = orc_flux_pairs(n, x, y, z, L, h, cap, pairs);
    }
    *np = k;
    return pairs;
}

/* One base step dt0 > 0 with individual timesteps (§2.3.4, §2.3.10).
 * Sub-step 0 synchronises every particle: density, guard, primitives and
 * gradients as in orc_step; then each particle's rung from the CFL
 * timestep (Eq. 31) and the acceleration criterion
 * dt_acc = c_acc sqrt(h / |a|), a = -grad p / rho (the limited pressure
 * gradient of the face reconstruction; no external acceleration), the
 * rung selection and the neighbour limiter above.  The base step then
 * runs 2^rmax sub-steps of dt0 2^-rmax; at sub-step k the particles with
 * k divisible by 2^(rmax - r_i) start a step of dt0 2^-r_i: their density,
 * guard, primitives and gradients are recomputed at the current positions
 * (the others keep those of their last start, used as they are).  Every
 * unordered flux pair with an active particle exchanges, with
 * dt_ij = min(dt_i, dt_j), c = dt_ij |A_ij| F, subtracted from i and added
 * to j (so the exchange is symmetric), each side predicted over the time
 * since its start plus dt_ij / 2.  Every particle then takes its received
 * change (U by Eq. 24 with its current velocity) and drifts by the
 * sub-step with the mean of its velocities before and after.  Rungs are
 * fixed over the base step.  rung (out): the rungs used; dt_cfl, dt_acc
 * (optional outputs): the two criteria at sub-step 0. */
int orc_step_rungs(const orc_config *c, int64_t n, double *x, double *y, double *z,
                   const double *L, double *m, double *px, double *py, double *pz, double *E,
                   double *U, double *h, double *omega, double dt0, double c_acc, int max_rung,
                   int32_t *rung, double *dt_cfl, double *dt_acc, orc_rung_info *info)
{
    int status = ORC_OK;
    double *B6 = (double *)malloc((size_t)n * 6 * sizeof(double));
    double *B6t = (double *)malloc((size_t)n * 6 * sizeof(double));
    double *nc = (double *)malloc((size_t)n * sizeof(double));
    double *prim[5], *primt[5];
    for (int f = 0; f < 5; f++) {
        prim[f] = (double *)malloc((size_t)n * sizeof(double));
        primt[f] = (double *)malloc((size_t)n * sizeof(double));
    }
    double *grad = (double *)malloc((size_t)n * 15 * sizeof(double));
    double *alpha = (double *)malloc((size_t)n * 5 * sizeof(double));
    double *gradt = (double *)malloc((size_t)n * 15 * sizeof(double));
    double *alphat = (double *)malloc((size_t)n * 5 * sizeof(double));
    double *vsig = (double *)malloc((size_t)n * sizeof(double));
    double *dQ = (double *)malloc((size_t)n * 6 * sizeof(double));
    double *dtp = (double *)malloc((size_t)n * sizeof(double));
    double *toff = (double *)malloc((size_t)n * sizeof(double));
    int32_t *ract = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *kstart = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    orc_rung_info inf;
    memset(&inf, 0, sizeof inf);

    /* sub-step 0: everything, as in orc_step */
    int s = orc_density_guard(c, n, x, y, z, L, NULL, h, omega, B6, nc, NULL, NULL);
    if (s != ORC_OK) status = s;
    orc_primitives(c, n, m, px, py, pz, E, U, omega, NULL, NULL, NULL, NULL, NULL, prim[0],
                   prim[1], prim[2], prim[3], prim[4]);
    orc_gradients(c, n, x, y, z, L, h, omega, prim[0], prim[1], prim[2], prim[3], prim[4], B6,
                  nc, grad, alpha, vsig);
    /* rungs (§2.3.10) */
    for (int64_t i = 0; i < n; i++) {
        const double dtc = c->c_cfl * h[i] / vsig[i];
        const double gx = alpha[5 * i + 4] * grad[15 * i + 12];
        const double gy = alpha[5 * i + 4] * grad[15 * i + 13];
        const double gz = alpha[5 * i + 4] * grad[15 * i + 14];
        const double acc = sqrt(gx * gx + gy * gy + gz * gz) / prim[0][i];
        const double dta = acc > 0.0 ? c_acc * sqrt(h[i] / acc) : INFINITY;
        if (dt_cfl) dt_cfl[i] = dtc;
        if (dt_acc) dt_acc[i] = dta;
        int cap = 0;
        rung[i] = orc_rung_select(dtc, dta, dt0, max_rung, &cap);
        inf.capped += cap;
    }
    {
        int64_t np;
        int64_t *pairs = orc_pairs_alloc(n, x, y, z, L, h, &np);
        inf.limiter_sweeps = orc_rung_limit(np, pairs, rung);
        free(pairs);
    }
    int rmax = 0;
    for (int64_t i = 0; i < n; i++) if (rung[i] > rmax) rmax = rung[i];
    const int64_t K = (int64_t)1 << rmax;
    const double dtmin = ldexp(dt0, -rmax);
    for (int64_t i = 0; i < n; i++) {
        dtp[i] = ldexp(dt0, -rung[i]);
        kstart[i] = 0;
    }
    for (int64_t k = 0; k < K; k++) {
        for (int64_t i = 0; i < n; i++) {
            ract[i] = k % ((int64_t)1 << (rmax - rung[i])) == 0;
            inf.active_steps += ract[i];
        }
        if (k > 0) {
            s = orc_density_guard(c, n, x, y, z, L, ract, h, omega, B6t, nc, NULL, NULL);
            if (s != ORC_OK && status == ORC_OK) status = s;
            for (int64_t i = 0; i < n; i++)
                if (ract[i]) memcpy(B6 + 6 * i, B6t + 6 * i, 6 * sizeof(double));
            orc_primitives(c, n, m, px, py, pz, E, U, omega, NULL, NULL, NULL, NULL, NULL,
                           primt[0], primt[1], primt[2], primt[3], primt[4]);
            for (int f = 0; f < 5; f++)
                for (int64_t i = 0; i < n; i++)
                    if (ract[i]) prim[f][i] = primt[f][i];
            orc_gradients(c, n, x, y, z, L, h, omega, prim[0], prim[1], prim[2], prim[3],
                          prim[4], B6, nc, gradt, alphat, vsig);
            for (int64_t i = 0; i < n; i++)
                if (ract[i]) {
                    memcpy(grad + 15 * i, gradt + 15 * i, 15 * sizeof(double));
                    memcpy(alpha + 5 * i, alphat + 5 * i, 5 * sizeof(double));
                }
        }
        for (int64_t i = 0; i < n; i++) {
            if (ract[i]) kstart[i] = k;
            toff[i] = (double)(k - kstart[i]) * dtmin;
        }
        /* the faces with an active particle */
        int64_t np;
        int64_t *pairs = orc_pairs_alloc(n, x, y, z, L, h, &np);
        int64_t w = 0;
        for (int64_t q = 0; q < np; q++) {
            const int64_t i = pairs[2 * q], j = pairs[2 * q + 1];
            if (ract[i] || ract[j]) { pairs[2 * w] = i; pairs[2 * w + 1] = j; w++; }
        }
        orc_flux_stats fst;
        orc_fluxes_impl(c, n, x, y, z, L, h, omega, B6, prim[0], prim[1], prim[2], prim[3],
                        prim[4], grad, alpha, dtmin, dtp, toff, w, pairs, NULL, dQ, &fst, NULL,
                        NULL, NULL, NULL, NULL);
        free(pairs);
        inf.faces += w;
        /* every particle takes what it received and drifts */
        for (int64_t i = 0; i < n; i++) {
            const double vox = px[i] / m[i], voy = py[i] / m[i], voz = pz[i] / m[i];
            const double dm = dQ[6 * i + 0], dpx = dQ[6 * i + 1], dpy = dQ[6 * i + 2];
            const double dpz = dQ[6 * i + 3], dE = dQ[6 * i + 4];
            const double v2 = vox * vox + voy * voy + voz * voz;
            const double dU = dE - (vox * dpx + voy * dpy + voz * dpz) + 0.5 * v2 * dm;
            m[i] += dm;
            px[i] += dpx;
            py[i] += dpy;
            pz[i] += dpz;
            E[i] += dE;
            U[i] += dU;
            const double nx = px[i] / m[i], ny = py[i] / m[i], nz = pz[i] / m[i];
            double xs[3] = {x[i] + dtmin * 0.5 * (vox + nx), y[i] + dtmin * 0.5 * (voy + ny),
                            z[i] + dtmin * 0.5 * (voz + nz)};
            for (int a = 0; a < 3; a++) {
                if (xs[a] >= L[a]) xs[a] -= L[a];
                if (xs[a] < 0.0) xs[a] += L[a];
            }
            x[i] = xs[0]; y[i] = xs[1]; z[i] = xs[2];
        }
    }
    inf.status = status;
    inf.rung_max = rmax;
    inf.substeps = K;
    if (info) *info = inf;
    free(B6); free(B6t); free(nc);
    for (int f = 0; f < 5; f++) { free(prim[f]); free(primt[f]); }
    free(grad); free(alpha); free(gradt); free(alphat); free(vsig); free(dQ); free(dtp);
    free(toff); free(ract); free(kstart);
    return status;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
