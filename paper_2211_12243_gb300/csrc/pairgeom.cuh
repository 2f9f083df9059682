// Pair geometry shared by the pair kernels: separation of two particles
// from their records, and exact membership r_ij < h.
#pragma once

#include "hydro_internal.cuh"

namespace hyd {

// positions from the first three record slots
__device__ __forceinline__ void rec_sep(const double *ri, const double *rj, const Box &bx,
                                        double d[3], double &r2) {
    d[0] = fold64(__dsub_rn(rj[0], ri[0]), bx.L[0]);
    d[1] = fold64(__dsub_rn(rj[1], ri[1]), bx.L[1]);
    d[2] = fold64(__dsub_rn(rj[2], ri[2]), bx.L[2]);
    r2 = r2_exact(d[0], d[1], d[2]);
}

__device__ __forceinline__ void rec_sep(const float *ri, const float *rj, const Box &bx,
                                        float d[3], float &r2) {
    d[0] = qdiff(__float_as_uint(ri[0]), __float_as_uint(rj[0]), bx.s[0]);
    d[1] = qdiff(__float_as_uint(ri[1]), __float_as_uint(rj[1]), bx.s[1]);
    d[2] = qdiff(__float_as_uint(ri[2]), __float_as_uint(rj[2]), bx.s[2]);
    r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

// Exact decision of r_ij^2 < h^2 as the definition states it in double
// (minimum image folded once, (dx^2 + dy^2) + dz^2, each step rounded).
struct Member {
    const double *xs, *ys, *zs;
    int64_t i;
    double xi, yi, zi;
    double h2;          // h * h in double
    float lo2, hi2;     // float band around h^2 (empty when h is tiny vs L)
    Box bx;
    __device__ __forceinline__ void init(const double *xs_, const double *ys_, const double *zs_,
                                         int64_t i_, double h, const Box &b) {
        xs = xs_; ys = ys_; zs = zs_; i = i_;
        xi = xs[i]; yi = ys[i]; zi = zs[i];
        h2 = __dmul_rn(h, h);
        float hf = (float)h;
        lo2 = hf * hf * (1.0f - 1e-4f);
        hi2 = hf * hf * (1.0f + 1e-4f);
        // fixed-point separations are exact to L/2^32; below h = L/4096 the
        // float band would no longer be conservative, so decide every pair
        // in double there
        double Lmin = fmin(b.L[0], fmin(b.L[1], b.L[2]));
        if (h < Lmin * (1.0 / 4096.0)) { lo2 = -1.0f; hi2 = 3.0e38f; }
        bx = b;
    }
    __device__ __forceinline__ bool exact(int64_t j) const {
        double ex = fold64(__dsub_rn(xs[j], xi), bx.L[0]);
        double ey = fold64(__dsub_rn(ys[j], yi), bx.L[1]);
        double ez = fold64(__dsub_rn(zs[j], zi), bx.L[2]);
        return r2_exact(ex, ey, ez) < h2;
    }
    // float path: r2 from the fixed-point separation
    __device__ __forceinline__ bool operator()(float r2, int64_t j) const {
        if (r2 < lo2) return true;
        if (r2 > hi2) return false;
        return exact(j);
    }
    // double path: r2 is already the exact value
    __device__ __forceinline__ bool operator()(double r2, int64_t) const { return r2 < h2; }
};

}  // namespace hyd
