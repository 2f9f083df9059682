/*
 * Operation counts of the oracle's per-face arithmetic (TEST AND MEASUREMENT
 * INFRASTRUCTURE ONLY, like the rest of oracle/).
 *
 * The algorithmic work of one face -- what the method itself computes, as
 * the oracle states it -- is counted by compiling hydro_oracle.c unchanged
 * with its scalar type replaced by `cdouble`, a double that counts every
 * arithmetic operation applied to it.  orc_count_faces() runs the oracle's
 * per-face routine (the separation and orc_face: face vector, extrapolation,
 * limiters, predictor, boost, Riemann solver, flux, de-boost) over a list of
 * pairs and returns the totals; the per-particle scatter and its compensated
 * sums (accumulation, not face arithmetic) are not run.  Counts:
 *   [0] add/sub   [1] mul   [2] div   [3] sqrt   [4] pow   [5] compare
 *   [6] fabs      [7] faces solved    [8] Newton iterations
 * A fused multiply-add does not exist in this build (each product and sum is
 * its own operation, as in the oracle compiled with -ffp-contract=off).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {
long long g_ops[7];
}

struct cdouble {
    double v;
    cdouble() = default;
    cdouble(double x) : v(x) {}
    template <class T>
    explicit operator T() const { return (T)v; }
    cdouble &operator+=(cdouble b) { g_ops[0]++; v += b.v; return *this; }
    cdouble &operator-=(cdouble b) { g_ops[0]++; v -= b.v; return *this; }
    cdouble &operator*=(cdouble b) { g_ops[1]++; v *= b.v; return *this; }
    cdouble &operator/=(cdouble b) { g_ops[2]++; v /= b.v; return *this; }
    cdouble operator-() const { return cdouble(-v); }
    cdouble operator+() const { return *this; }
    friend cdouble operator+(cdouble a, cdouble b) { g_ops[0]++; return cdouble(a.v + b.v); }
    friend cdouble operator-(cdouble a, cdouble b) { g_ops[0]++; return cdouble(a.v - b.v); }
    friend cdouble operator*(cdouble a, cdouble b) { g_ops[1]++; return cdouble(a.v * b.v); }
    friend cdouble operator/(cdouble a, cdouble b) { g_ops[2]++; return cdouble(a.v / b.v); }
    friend bool operator<(cdouble a, cdouble b) { g_ops[5]++; return a.v < b.v; }
    friend bool operator>(cdouble a, cdouble b) { g_ops[5]++; return a.v > b.v; }
    friend bool operator<=(cdouble a, cdouble b) { g_ops[5]++; return a.v <= b.v; }
    friend bool operator>=(cdouble a, cdouble b) { g_ops[5]++; return a.v >= b.v; }
    friend bool operator==(cdouble a, cdouble b) { g_ops[5]++; return a.v == b.v; }
    friend bool operator!=(cdouble a, cdouble b) { g_ops[5]++; return a.v != b.v; }
};
static_assert(sizeof(cdouble) == sizeof(double), "cdouble must lay out as a double");

static inline cdouble sqrt(cdouble a) { g_ops[3]++; return cdouble(::sqrt(a.v)); }
static inline cdouble pow(cdouble a, cdouble b) { g_ops[4]++; return cdouble(::pow(a.v, b.v)); }
static inline cdouble fabs(cdouble a) { g_ops[6]++; return cdouble(::fabs(a.v)); }
static inline cdouble floor(cdouble a) { return cdouble(::floor(a.v)); }
static inline cdouble ldexp(cdouble a, int e) { return cdouble(::ldexp(a.v, e)); }
static inline bool isfinite(cdouble a) { return std::isfinite(a.v); }

#define double cdouble
#include "hydro_oracle.c"
#undef double

extern "C" void orc_count_faces(const orc_config *c, int64_t n, const double *x, const double *y,
                                const double *z, const double *L, const double *h,
                                const double *omega, const double *B6, const double *rho,
                                const double *vx, const double *vy, const double *vz,
                                const double *p, const double *grad, const double *alpha,
                                double dt, int64_t npairs, const int64_t *pairs,
                                long long counts[9])
{
    typedef const cdouble *P;
    P Wp[5] = {(P)rho, (P)vx, (P)vy, (P)vz, (P)p};
    memset(g_ops, 0, sizeof g_ops);
    orc_flux_stats st;
    memset(&st, 0, sizeof st);
    for (int64_t k = 0; k < npairs; k++) {
        const int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        cdouble d[3], cf[5];
        cdouble r = sqrt(orc_sep((P)x, (P)y, (P)z, (P)L, i, j, d));
        orc_face(c, i, j, d, r, (P)h, (P)omega, (P)B6, Wp, (P)grad, (P)alpha, cdouble(dt),
                 cdouble(0.5 * dt), cdouble(0.5 * dt), NULL, cf, &st, NULL);
    }
    for (int q = 0; q < 7; q++) counts[q] = g_ops[q];
    counts[7] = st.faces;
    counts[8] = st.newton_iters;
}
