// Device Riemann solvers for the per-face problem of §2.3.3: the exact
// iterative solver (Toro 2009, ch. 4; the paper's choice) and HLLC
// (Toro 2009, ch. 10).  Templated on the arithmetic type: double for the
// FP64 path, float for the mixed path.
#pragma once

#include "hydro_internal.cuh"

namespace hyd {

template <typename R> __device__ __forceinline__ R rsqrt_(R v);
template <> __device__ __forceinline__ float rsqrt_<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_<double>(double v) { return rsqrt(v); }

template <typename R> __device__ __forceinline__ R pow_(R a, R b);
template <> __device__ __forceinline__ float pow_<float>(float a, float b) { return __powf(a, b); }
template <> __device__ __forceinline__ double pow_<double>(double a, double b) { return pow(a, b); }

// division and square root: IEEE in double; in float the hardware
// approximations (a few ulp), well inside the mixed path's 1e-5 budget
__device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_(double a, double b) { return a / b; }
__device__ __forceinline__ float sqrt_(float a) { return a > 0.f ? a * rsqrtf(a) : 0.f; }
__device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }

// gamma-dependent constants of Toro's formulae
template <typename R>
struct GasK {
    R g, gm1, gp1;
    R z;      // (g-1)/(2g)
    R zi;     // 2g/(g-1)
    R g4;     // 2/(g-1)
    R g5;     // 2/(g+1)
    R g6;     // (g-1)/(g+1)
    R g2;     // (g+1)/(2g)
    R inv_g;  // 1/g
    R mzr;    // -(g+1)/(2g)
    GasK() = default;
    __host__ __device__ explicit GasK(double gamma) {
        g = (R)gamma;
        gm1 = (R)(gamma - 1.0);
        gp1 = (R)(gamma + 1.0);
        z = (R)((gamma - 1.0) / (2.0 * gamma));
        zi = (R)(2.0 * gamma / (gamma - 1.0));
        g4 = (R)(2.0 / (gamma - 1.0));
        g5 = (R)(2.0 / (gamma + 1.0));
        g6 = (R)((gamma - 1.0) / (gamma + 1.0));
        g2 = (R)((gamma + 1.0) / (2.0 * gamma));
        inv_g = (R)(1.0 / gamma);
        mzr = (R)(-(gamma + 1.0) / (2.0 * gamma));
    }
};

// one side's pressure function and derivative
template <typename R>
__device__ __forceinline__ void side_f(const GasK<R> &k, R p, R rk, R pk, R ck, R &f, R &df);

// float: both branches evaluated and selected, so that the lanes of a warp
// (faces with shock and rarefaction sides mixed) do not diverge
template <>
__device__ __forceinline__ void side_f<float>(const GasK<float> &k, float p, float rk, float pk,
                                              float ck, float &f, float &df) {
    float A = __fdividef(k.g5, rk);
    float Bk = k.g6 * pk;
    float ia = __fdividef(1.f, p + Bk);
    float q = sqrt_(A * ia);
    float fs = (p - pk) * q;
    float dfs = q * (1.f - 0.5f * (p - pk) * ia);
    float pr = __fdividef(p, pk);
    float t = __powf(pr, k.z);
    float fr = k.g4 * ck * (t - 1.f);
    float dfr = __fdividef(t * ck, pr * k.g * pk);
    bool shock = p > pk;
    f = shock ? fs : fr;
    df = shock ? dfs : dfr;
}

// float path inside the Newton loop: the per-face constants of one side
// (the shock branch's A_K = 2/((g+1) rho_K) and B_K = (g-1)/(g+1) p_K, 1/p_K,
// c_K/g) are formed once per face, and 1/p once per iteration for both
// sides, which leaves two reciprocals, a square root and a power per side
// and step on the special-function unit
struct SideF {
    float A, sA, B, ipk, cg, pk, ck;   // (sA = sqrt(A))
};

__device__ __forceinline__ SideF side_prep(const GasK<float> &k, float rk, float pk, float ck) {
    SideF s;
    s.A = __fdividef(k.g5, rk);
    s.sA = sqrt_(s.A);
    s.B = k.g6 * pk;
    s.ipk = __fdividef(1.f, pk);
    s.cg = ck * k.inv_g;
    s.pk = pk;
    s.ck = ck;
    return s;
}

// f_K(p) and f_K'(p) with ip = 1/p: both branches evaluated and selected
// (no divergence between shock and rarefaction sides); the rarefaction
// derivative (1/(rho_K c_K)) (p/p_K)^(-(g+1)/(2g)) is written as
// (p/p_K)^((g-1)/(2g)) c_K / (g p); the shock branch's sqrt(A / (p + B)) and
// 1 / (p + B) come from one reciprocal square root
__device__ __forceinline__ void side_eval(const GasK<float> &k, const SideF &s, float p, float ip,
                                          float &f, float &df) {
    const float rq = rsqrtf(p + s.B);
    const float ia = rq * rq;
    const float q = s.sA * rq;
    const float fs = (p - s.pk) * q;
    const float dfs = q * (1.f - 0.5f * (p - s.pk) * ia);
    const float t = __powf(p * s.ipk, k.z);
    const float fr = k.g4 * s.ck * (t - 1.f);
    const float dfr = t * s.cg * ip;
    const bool shock = p > s.pk;
    f = shock ? fs : fr;
    df = shock ? dfs : dfr;
}

template <typename R>
__device__ __forceinline__ void side_f(const GasK<R> &k, R p, R rk, R pk, R ck, R &f, R &df) {
    if (p > pk) {
        R A = div_(k.g5, rk);
        R Bk = k.g6 * pk;
        R q = sqrt_(div_(A, p + Bk));
        f = (p - pk) * q;
        df = q * (R(1) - R(0.5) * div_(p - pk, Bk + p));
    } else {
        R pr = div_(p, pk);
        R t = pow_(pr, k.z);
        f = k.g4 * ck * (t - R(1));
        df = div_(t, pr * k.g * pk) * ck;   // = (1/(rk ck)) (p/pk)^(-(g+1)/(2g))
    }
}

// Toro's adaptive initial guess
template <typename R>
__device__ __forceinline__ R star_guess(const GasK<R> &k, R rl, R ul, R pl, R cl, R rr, R ur,
                                        R pr, R cr) {
    R ppv = R(0.5) * (pl + pr) - R(0.125) * (ur - ul) * (rl + rr) * (cl + cr);
    ppv = ppv > R(0) ? ppv : R(0);
    R pmin = pl < pr ? pl : pr, pmax = pl > pr ? pl : pr;
    if (pmax <= R(2) * pmin && ppv >= pmin && ppv <= pmax) return ppv;
    if (ppv < pmin) {
        const R icl = div_(R(1), cl), icr = div_(R(1), cr);
        R pq = pow_(div_(pl, pr), k.z);
        R um = div_(pq * ul * icl + ur * icr + k.g4 * (pq - R(1)), pq * icl + icr);
        R tl = R(1) + R(0.5) * k.gm1 * (ul - um) * icl;
        R tr = R(1) + R(0.5) * k.gm1 * (um - ur) * icr;
        return R(0.5) * (pl * pow_(tl, k.zi) + pr * pow_(tr, k.zi));
    }
    R gl = sqrt_(div_(k.g5, rl * (k.g6 * pl + ppv)));
    R gr = sqrt_(div_(k.g5, rr * (k.g6 * pr + ppv)));
    return div_(gl * pl + gr * pr - (ur - ul), gl + gr);
}

struct StarOut {
    int iters;
    int bisect;
    int vacuum;
};

// Newton iteration for p* from p0 (> 0, else the adaptive guess); stop when
// the relative change falls below tol, then one more Newton step; bisection
// on the bracket after max_newton iterations.  kd (float path only, else
// NULL): after the float iteration converged, one more Newton step with the
// pressure function evaluated in FP64, and u* from it.
// (cl, cr: the two sides' sound speeds, which the caller's sampling of
// the solution needs as well)
template <typename R>
__device__ __forceinline__ StarOut star_solve(const GasK<R> &k, R rl, R ul, R pl, R cl, R rr, R ur,
                                              R pr, R cr, R p0, R tol, int max_newton, R &ps,
                                              R &us, const GasK<double> *kd = nullptr) {
    StarOut o{0, 0, 0};
    R du = ur - ul;
    if (k.g4 * (cl + cr) <= du) {
        o.vacuum = 1;
        ps = R(0);
        us = R(0);
        return o;
    }
    R p = p0 > R(0) ? p0 : star_guess(k, rl, ul, pl, cl, rr, ur, pr, cr);
    const R pfloor = sizeof(R) == 8 ? R(1e-300) : R(1e-37);
    if (!(p > pfloor)) p = pfloor;
    bool conv = false;
    R fl, dfl, fr, dfr;
    R dp_last = R(0);
    if constexpr (sizeof(R) == 4) {
        const SideF sl = side_prep(k, rl, pl, cl), sr = side_prep(k, rr, pr, cr);
        const float htol = 0.5f * tol;
        for (int it = 1; it <= max_newton; it++) {
            const float ip = __fdividef(1.f, p);
            side_eval(k, sl, p, ip, fl, dfl);
            side_eval(k, sr, p, ip, fr, dfr);
            float pn = p - __fdividef(fl + fr + du, dfl + dfr);
            if (!(pn > pfloor)) pn = pfloor;
            // relative change 2 |pn - p| / (pn + p) < tol, without a division
            const bool done = fabsf(pn - p) < htol * (pn + p);
            dp_last = pn - p;
            p = pn;
            o.iters = it;
            if (done) { conv = true; break; }
        }
    } else {
        for (int it = 1; it <= max_newton; it++) {
            side_f(k, p, rl, pl, cl, fl, dfl);
            side_f(k, p, rr, pr, cr, fr, dfr);
            R pn = p - div_(fl + fr + du, dfl + dfr);
            if (!(pn > pfloor)) pn = pfloor;
            R ch = R(2) * div_(fabs(pn - p), pn + p);
            dp_last = pn - p;
            p = pn;
            o.iters = it;
            if (ch < tol) { conv = true; break; }
        }
    }
    if (conv && sizeof(R) == 4 && kd) {
        // the root of the float face states to double precision: one Newton
        // step of f(p) = f_L(p) + f_R(p) + u_R - u_L evaluated in FP64 from
        // the converged float root, then u* from the same evaluation
        // corrected to first order for that step
        const double pd = (double)p;
        const double rld = rl, uld = ul, pld = pl, rrd = rr, urd = ur, prd = pr;
        const double cld = sqrt(kd->g * pld / rld), crd = sqrt(kd->g * prd / rrd);
        double fld, dfld, frd, dfrd;
        side_f<double>(*kd, pd, rld, pld, cld, fld, dfld);
        side_f<double>(*kd, pd, rrd, prd, crd, frd, dfrd);
        const double dpd = -(fld + frd + (urd - uld)) / (dfld + dfrd);
        if (pd + dpd > 0.0) {
            ps = (R)(pd + dpd);
            us = (R)(0.5 * (uld + urd) + 0.5 * (frd - fld) + 0.5 * (dfrd - dfld) * dpd);
            return o;
        }
    }
    if (conv && sizeof(R) == 4) {
        // float: the iteration has converged to rounding; u* from the last
        // evaluation, corrected to first order for the last Newton step
        // (p held p_old at that evaluation, p_new - p_old = pn - p_old)
        ps = p;
        us = R(0.5) * (ul + ur) + R(0.5) * (fr - fl) + R(0.5) * (dfr - dfl) * dp_last;
        return o;
    }
    if (conv) {
        side_f(k, p, rl, pl, cl, fl, dfl);
        side_f(k, p, rr, pr, cr, fr, dfr);
        R pn = p - div_(fl + fr + du, dfl + dfr);
        if (pn > pfloor) p = pn;
    } else {
        R lo = R(0), hi = pl > pr ? pl : pr;
        for (int guard = 0; guard < 2100; guard++) {
            side_f(k, hi, rl, pl, cl, fl, dfl);
            side_f(k, hi, rr, pr, cr, fr, dfr);
            if (fl + fr + du > R(0)) break;
            lo = hi;
            hi = hi * R(2);
        }
        for (int it = 0; it < 200; it++) {
            R mid = R(0.5) * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            side_f(k, mid, rl, pl, cl, fl, dfl);
            side_f(k, mid, rr, pr, cr, fr, dfr);
            if (fl + fr + du > R(0)) hi = mid; else lo = mid;
        }
        p = R(0.5) * (lo + hi);
        o.bisect = 1;
    }
    side_f(k, p, rl, pl, cl, fl, dfl);
    side_f(k, p, rr, pr, cr, fr, dfr);
    ps = p;
    us = R(0.5) * (ul + ur) + R(0.5) * (fr - fl);
    return o;
}

// state at x/t = 0 of the exact solution; side = -1 left of the contact.
// The side the contact leaves at x/t = 0 is sampled as a left side: a right
// side enters with its velocities negated (u -> -u, which maps the right
// waves onto left ones exactly, since rounding to nearest is symmetric) and
// the sampled velocity is negated back, so the lanes of a warp follow one
// branch tree whichever side each face samples.
template <typename R>
__device__ __forceinline__ void star_sample(const GasK<R> &k, R rl, R ul, R pl, R cl, R rr, R ur,
                                            R pr, R cr, R ps, R us, R &rho, R &u, R &p, int &side) {
    const bool left = R(0) <= us;
    side = left ? -1 : 1;
    const R rK = left ? rl : rr, pK = left ? pl : pr, cK = left ? cl : cr;
    const R uK = left ? ul : -ur, uS = left ? us : -us;
    R rs, vs, qs;
    if (ps > pK) {
        // shock: the pre-shock state beyond it, else the star state
        const R sK = uK - cK * sqrt_(k.g2 * div_(ps, pK) + k.z);
        if (R(0) <= sK) { rs = rK; vs = uK; qs = pK; }
        else {
            const R t = div_(ps, pK);
            rs = rK * div_(t + k.g6, k.g6 * t + R(1));
            vs = uS;
            qs = ps;
        }
    } else if (R(0) <= uK - cK) {
        rs = rK; vs = uK; qs = pK;   // beyond the rarefaction's head
    } else {
        const R t = div_(ps, pK);
        const R cm = cK * pow_(t, k.z);
        // (a right side keeps its tail point in the star region)
        const bool star = left ? R(0) > uS - cm : R(0) >= uS - cm;
        if (star) { rs = rK * pow_(t, k.inv_g); vs = uS; qs = ps; }
        else {
            // inside the fan
            const R cc = k.g5 + div_(k.g6, cK) * uK;
            rs = rK * pow_(cc, k.g4);
            vs = k.g5 * (cK + R(0.5) * k.gm1 * uK);
            qs = pK * pow_(cc, k.zi);
        }
    }
    rho = rs;
    u = left ? vs : -vs;
    p = qs;
}

// HLLC flux along n (face frame) with the pressure-based wave speeds.
// F[0] mass, F[1..3] momentum, F[4] energy; ps/ss: star pressure, contact.
template <typename R>
__device__ __forceinline__ void hllc_flux(const GasK<R> &k, R rl, R ul, R pl, const R *wl, R rr,
                                          R ur, R pr, const R *wr, const R *n, R *F, R &ps,
                                          R &ss) {
    R cl = sqrt_(div_(k.g * pl, rl)), cr = sqrt_(div_(k.g * pr, rr));
    R ppv = R(0.5) * (pl + pr) - R(0.125) * (ur - ul) * (rl + rr) * (cl + cr);
    ppv = ppv > R(0) ? ppv : R(0);
    R ql = ppv <= pl ? R(1) : sqrt_(R(1) + k.g2 * (div_(ppv, pl) - R(1)));
    R qr = ppv <= pr ? R(1) : sqrt_(R(1) + k.g2 * (div_(ppv, pr) - R(1)));
    R sl = ul - cl * ql, sr = ur + cr * qr;
    ss = div_(pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur), rl * (sl - ul) - rr * (sr - ur));
    ps = pl + rl * (sl - ul) * (ss - ul);
    R w2l = wl[0] * wl[0] + wl[1] * wl[1] + wl[2] * wl[2];
    R w2r = wr[0] * wr[0] + wr[1] * wr[1] + wr[2] * wr[2];
    R El = div_(pl, k.gm1) + R(0.5) * rl * (ul * ul + w2l);
    R Er = div_(pr, k.gm1) + R(0.5) * rr * (ur * ur + w2r);
    R fm, fn, fe;
    const R *wt;
    if (R(0) <= sl) {
        fm = rl * ul; fn = rl * ul * ul + pl; fe = ul * (El + pl); wt = wl;
    } else if (R(0) <= ss) {
        R kk = div_(rl * (sl - ul), sl - ss);
        R e2 = kk * (div_(El, rl) + (ss - ul) * (ss + div_(pl, rl * (sl - ul))));
        fm = rl * ul + sl * (kk - rl);
        fn = rl * ul * ul + pl + sl * (kk * ss - rl * ul);
        fe = ul * (El + pl) + sl * (e2 - El);
        wt = wl;
    } else if (R(0) <= sr) {
        R kk = div_(rr * (sr - ur), sr - ss);
        R e2 = kk * (div_(Er, rr) + (ss - ur) * (ss + div_(pr, rr * (sr - ur))));
        fm = rr * ur + sr * (kk - rr);
        fn = rr * ur * ur + pr + sr * (kk * ss - rr * ur);
        fe = ur * (Er + pr) + sr * (e2 - Er);
        wt = wr;
    } else {
        fm = rr * ur; fn = rr * ur * ur + pr; fe = ur * (Er + pr); wt = wr;
    }
    F[0] = fm;
    F[1] = fn * n[0] + fm * wt[0];
    F[2] = fn * n[1] + fm * wt[1];
    F[3] = fn * n[2] + fm * wt[2];
    F[4] = fe;
}

}  // namespace hyd
