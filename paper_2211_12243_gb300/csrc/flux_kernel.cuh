// Pair fluxes (§2.3.3 and §2.3.4): for every unordered pair with
// r_ij < max(h_i, h_j), the effective face
//   A_ij = V_i omega_j B_i mu(x_i, x_j) - V_j omega_i B_j mu(x_j, x_i)
//        = omega_i omega_j [B_i dx W(r, h_i) + B_j dx W(r, h_j)],  dx = x_j - x_i,
// face states extrapolated to the midpoint (Eqs. 20-21) with the limited
// gradients, the pairwise limiter, the half-step predictor, a Riemann
// problem along A_ij in the frame moving with (v_i + v_j)/2, and the flux
// c = dt |A_ij| F applied antisymmetrically: Q_i -= c, Q_j += c (Eq. 16).
//
// Ownership: particle i computes the pair {i, j} found in its own list
// (r < h_i) when i < j or when r >= h_j (then j's list does not see i), so
// each unordered pair is computed exactly once.
//
// Work layout: one warp per bucket of 32 owners.  The warp walks the 32
// neighbour lists in lock-step, tests membership and ownership (cheap), and
// compacts the owned faces into a shared-memory queue; every 32 queued
// faces are solved one per lane, so the expensive face arithmetic runs with
// full lanes regardless of how the faces are spread over the owners.  The
// owner's -c is gathered back from shared memory into its own register
// accumulator (float-float in the mixed path, double in FP64); the
// partner's +c goes to memory through double-precision atomics.
#pragma once

#include <algorithm>

#include "hydro_internal.cuh"
#include "pairgeom.cuh"
#include "riemann.cuh"
#include "mlp.cuh"

namespace hyd {

struct FluxArgs {
    int64_t n;
    const int64_t *nbr_off;
    const int32_t *nbr_cnt;
    const int32_t *nbr_idx;
    const double *xs, *ys, *zs, *h;
    const int32_t *pbox;
    const Box *boxes;
    int kernel, scheme, riemann, limiter, time_extrap;
    double gamma, psi1, psi2, p_tol;
    int max_newton;
    double dt;
    const double *dt_dev;
    double *dQ;              // 5 n, sorted SoA
    DevCounters *cnt;
    const unsigned char *mlp_blob;   // packed network (hard-face kernel)
    int mlp_stall;                   // error-path test hook (hydro_test_mlp_stall)
    int riemann_polish;              // float path: FP64 Newton step after convergence
    float *hard;             // deferred hard faces: FaceState fields [HF_N][hard_cap]
    int32_t *hard_idx;       // their owner and partner (sorted indices) [2][hard_cap]
    unsigned long long *hard_cursor;   // faces taken in each of the HARD_SUB sub-buffers
    int64_t hard_cap;        // HARD_SUB sub-buffers of hard_cap / HARD_SUB slots
    float *rec_faces;        // face recording [7][rec_cap] (NULL: off)
    unsigned long long *rec_cursor;
    int64_t rec_cap;
    uint32_t rec_keep;
    int rec_hard_only;
    GasK<float> Kf;          // gas constants, precomputed on the host
    GasK<double> Kd;
    float psi1f, psi2f, ptolf, lmin_tiny;   // float copies (no per-face conversions)
    int64_t nbucket;
    const int32_t *node_first, *node_cnt;
    // gravity (§2.3.8): sum_j dm_ij r_ij, 3 n sorted SoA (NULL: no gravity);
    // both particles of a face add c_m (x_j - x_i).  recf: the float
    // records, for the hard-face kernel's separations
    double *dM;
    const float *recf;
    // entropy switch (§2.3.7), MFV: sum_j c_m,ij A_upwind, n sorted (NULL:
    // off); A is the records' R_PAD slot.  A face whose mass flux c_m
    // leaves the owner carries c_m A_owner, else c_m A_partner
    double *dS;
    // individual timesteps (§2.3.4; NULL: one global dt): per sorted
    // particle its rung, the time since its state was taken and whether it
    // starts a step now.  A face with an active particle exchanges over
    // dt_ij = dt0 2^-max(r_i, r_j) = min(dt_i, dt_j), each side predicted
    // over toff + dt_ij / 2; faces of two inactive particles are skipped
    const int32_t *rung;
    const double *toff;
    const uint8_t *ract;
    double dt0;
    // the buckets to walk (NULL: all nbucket; else nbucket of these ids):
    // the sub-steps of individual timesteps walk only the buckets whose
    // particles can reach a particle starting a step
    const int32_t *bucket_ids;
    // persistent launch: the warps draw bucket indices from this cursor
    // (zeroed before the launch); NULL: one bucket per warp
    unsigned long long *queue;
};

template <typename R> __device__ __forceinline__ const GasK<R> &gas(const FluxArgs &a);
template <> __device__ __forceinline__ const GasK<float> &gas<float>(const FluxArgs &a) { return a.Kf; }
template <> __device__ __forceinline__ const GasK<double> &gas<double>(const FluxArgs &a) { return a.Kd; }

namespace {

template <typename R>
__device__ __forceinline__ int sgn_(R v) { return (v > R(0)) - (v < R(0)); }

// pairwise limiter of the face value e seen from the side with cell value a
template <typename R>
__device__ __forceinline__ R pair_limit(R e, R a, R b, R psi1, R psi2, bool positive) {
    if (a == b) return a;
    R d = fabs(a - b);
    R mean = R(0.5) * (a + b);
    R d1 = psi1 * d, d2 = psi2 * d;
    R lo = a < b ? a : b, hi = a > b ? a : b;
    R lox = lo - d1, hix = hi + d1;
    if (positive) {
        if (sgn_(lox) != sgn_(lo)) lox = lo == R(0) ? R(0) : div_(lo, R(1) + div_(d1, fabs(lo)));
        if (sgn_(hix) != sgn_(hi)) hix = hi == R(0) ? R(0) : div_(hi, R(1) + div_(d1, fabs(hi)));
    }
    if (a < b) {
        R t = e < mean + d2 ? e : mean + d2;
        return t > lox ? t : lox;
    }
    R t = e > mean - d2 ? e : mean - d2;
    return t < hix ? t : hix;
}

template <typename R>
__device__ __forceinline__ void load_full(const R *p, R v[REC]) {
    if (sizeof(R) == 4) {
#pragma unroll
        for (int k = 0; k < REC / 4; k++) {
            float4 t = reinterpret_cast<const float4 *>(p)[k];
            v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < REC / 2; k++) {
            double2 t = reinterpret_cast<const double2 *>(p)[k];
            v[2 * k] = t.x; v[2 * k + 1] = t.y;
        }
    }
}

template <typename R>
__device__ __forceinline__ void load4(const R *p, R v[4]) {
    if (sizeof(R) == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        double2 t0 = reinterpret_cast<const double2 *>(p)[0];
        double2 t1 = reinterpret_cast<const double2 *>(p)[1];
        v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
    }
}

// r < h_j decided exactly (float path: band + double fallback)
__device__ __forceinline__ bool member_j(float r2, float hjf, const FluxArgs &a, int64_t i,
                                         int64_t j, const Box &bx) {
    float lo = hjf * hjf * (1.0f - 1e-4f), hi = hjf * hjf * (1.0f + 1e-4f);
    if (hjf >= a.lmin_tiny) {
        if (r2 < lo) return true;
        if (r2 > hi) return false;
    }
    double hj = a.h[j];
    double ex = fold64(__dsub_rn(a.xs[j], a.xs[i]), bx.L[0]);
    double ey = fold64(__dsub_rn(a.ys[j], a.ys[i]), bx.L[1]);
    double ez = fold64(__dsub_rn(a.zs[j], a.zs[i]), bx.L[2]);
    return r2_exact(ex, ey, ez) < __dmul_rn(hj, hj);
}
__device__ __forceinline__ bool member_j(double r2, double hj, const FluxArgs &, int64_t,
                                         int64_t, const Box &) {
    return r2 < __dmul_rn(hj, hj);
}

struct FaceStats {
    unsigned long long pairs, iters, vacuum, first_order;
};

// Riemann problem of one face in the frame moving with (v_i + v_j)/2:
// normal n, left/right normal velocities and densities/pressures,
// tangential velocities, the frame velocity and dt |A_ij|
template <typename R>
struct FaceState {
    R rl, ul, pl, rr, ur, pr;
    R wl[3], wr[3], nh[3], vf[3];
    R sA;
};

// face vector, extrapolated and limited states; false when A_ij = 0 (no flux)
// hl, hr: the times the predictor advances the owner and partner states
// over (dt / 2 for one global dt)
template <typename R>
__device__ __forceinline__ bool face_state(const FluxArgs &a, const GasK<R> &K, const R *ri,
                                           const R *rj, const R d[3], R r, R dt, R hl, R hr,
                                           FaceState<R> &st, FaceStats &fs) {
    const R pi = R(3.14159265358979323846);
    const R hi_ = ri[R_H], hj = rj[R_H];
    const R kn = a.kernel == 0 ? R(21) / (R(2) * pi) : R(8) / pi;
    const R ihi = div_(R(1), hi_), ihj = div_(R(1), hj);
    const R wi = kn * ihi * ihi * ihi * kernel_shape<R>(a.kernel, r * ihi);
    const R wj = kn * ihj * ihj * ihj * kernel_shape<R>(a.kernel, r * ihj);
    const R *Bi = ri + R_B, *Bj = rj + R_B;
    R A[3];
    {
        R ti0 = Bi[0] * d[0] + Bi[1] * d[1] + Bi[2] * d[2];
        R ti1 = Bi[1] * d[0] + Bi[3] * d[1] + Bi[4] * d[2];
        R ti2 = Bi[2] * d[0] + Bi[4] * d[1] + Bi[5] * d[2];
        R tj0 = Bj[0] * d[0] + Bj[1] * d[1] + Bj[2] * d[2];
        R tj1 = Bj[1] * d[0] + Bj[3] * d[1] + Bj[4] * d[2];
        R tj2 = Bj[2] * d[0] + Bj[4] * d[1] + Bj[5] * d[2];
        R oo = ri[R_OM] * rj[R_OM];
        A[0] = oo * (ti0 * wi + tj0 * wj);
        A[1] = oo * (ti1 * wi + tj1 * wj);
        A[2] = oo * (ti2 * wi + tj2 * wj);
    }
    R Amag = sqrt_(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    if (!(Amag > R(0))) return false;
    const R inA = div_(R(1), Amag);
    st.nh[0] = A[0] * inA; st.nh[1] = A[1] * inA; st.nh[2] = A[2] * inA;

    R Lf[5], Rf[5];
    const R *Gi = ri + R_G, *Gj = rj + R_G;
#pragma unroll
    for (int f = 0; f < 5; f++) {
        Lf[f] = ri[R_RHO + f] + R(0.5) * (d[0] * Gi[3 * f] + d[1] * Gi[3 * f + 1] + d[2] * Gi[3 * f + 2]);
        Rf[f] = rj[R_RHO + f] - R(0.5) * (d[0] * Gj[3 * f] + d[1] * Gj[3 * f + 1] + d[2] * Gj[3 * f + 2]);
    }
    if (a.limiter) {
        const R p1 = sizeof(R) == 4 ? (R)a.psi1f : (R)a.psi1;
        const R p2 = sizeof(R) == 4 ? (R)a.psi2f : (R)a.psi2;
#pragma unroll
        for (int f = 0; f < 5; f++) {
            bool pos = (f == 0 || f == 4);
            Lf[f] = pair_limit<R>(Lf[f], ri[R_RHO + f], rj[R_RHO + f], p1, p2, pos);
            Rf[f] = pair_limit<R>(Rf[f], rj[R_RHO + f], ri[R_RHO + f], p1, p2, pos);
        }
    }
    const R g = K.g;
    // the face moves with the mean of the particles' velocities at the half
    // step (the predictor's acceleration over hl, hr; Eq. 16's fluxes are
    // those of the half step)
    R av[3] = {R(0), R(0), R(0)};
    if (a.time_extrap) {
        R divi = Gi[3] + Gi[7] + Gi[11];
        R divj = Gj[3] + Gj[7] + Gj[11];
        Lf[0] -= hl * ri[R_RHO] * divi;
        Rf[0] -= hr * rj[R_RHO] * divj;
        const R iri = div_(hl, ri[R_RHO]), irj = div_(hr, rj[R_RHO]);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const R ai = Gi[12 + q] * iri, aj = Gj[12 + q] * irj;
            Lf[1 + q] -= ai;
            Rf[1 + q] -= aj;
            av[q] = ai + aj;
        }
        Lf[4] -= hl * g * ri[R_P] * divi;
        Rf[4] -= hr * g * rj[R_P] * divj;
    }
    if (!(Lf[0] > R(0) && Lf[4] > R(0) && Rf[0] > R(0) && Rf[4] > R(0))) {
#pragma unroll
        for (int f = 0; f < 5; f++) { Lf[f] = ri[R_RHO + f]; Rf[f] = rj[R_RHO + f]; }
        fs.first_order++;
    }
    st.vf[0] = R(0.5) * ((ri[R_VX] + rj[R_VX]) - av[0]);
    st.vf[1] = R(0.5) * ((ri[R_VY] + rj[R_VY]) - av[1]);
    st.vf[2] = R(0.5) * ((ri[R_VZ] + rj[R_VZ]) - av[2]);
    R vl[3], vr[3];
#pragma unroll
    for (int q = 0; q < 3; q++) { vl[q] = Lf[1 + q] - st.vf[q]; vr[q] = Rf[1 + q] - st.vf[q]; }
    st.ul = vl[0] * st.nh[0] + vl[1] * st.nh[1] + vl[2] * st.nh[2];
    st.ur = vr[0] * st.nh[0] + vr[1] * st.nh[1] + vr[2] * st.nh[2];
#pragma unroll
    for (int q = 0; q < 3; q++) { st.wl[q] = vl[q] - st.ul * st.nh[q]; st.wr[q] = vr[q] - st.ur * st.nh[q]; }
    st.rl = Lf[0]; st.pl = Lf[4]; st.rr = Rf[0]; st.pr = Rf[4];
    st.sA = dt * Amag;
    return true;
}

// Toro's adaptive guess falls back to the two-shock value on this face (the
// same tests as star_guess: not the PVRS value, and p_PVRS >= p_min so not
// the two-rarefaction value, which is exact for two rarefactions).  These
// "hard" faces are the ones where the guess is only approximate.
template <typename R>
__device__ __forceinline__ bool two_shock_guess(const GasK<R> &k, const FaceState<R> &st) {
    R cl = sqrt_(div_(k.g * st.pl, st.rl)), cr = sqrt_(div_(k.g * st.pr, st.rr));
    R ppv = R(0.5) * (st.pl + st.pr) - R(0.125) * (st.ur - st.ul) * (st.rl + st.rr) * (cl + cr);
    ppv = ppv > R(0) ? ppv : R(0);
    R pmin = st.pl < st.pr ? st.pl : st.pr, pmax = st.pl > st.pr ? st.pl : st.pr;
    const bool pvrs = pmax <= R(2) * pmin && ppv >= pmin && ppv <= pmax;
    return !pvrs && !(ppv < pmin);
}

// the flux c (mass, momentum, energy) that particle i gives to particle j,
// from the face's Riemann problem; p0 > 0 is the exact solver's starting
// pressure (else its adaptive guess).  ps: the star pressure (exact solver,
// 0 on vacuum or HLLC).
template <typename R, int RIEM, int SCHEME>
__device__ __forceinline__ void face_finish(const FluxArgs &a, const GasK<R> &K,
                                            const FaceState<R> &st, R p0, R c[5], FaceStats &fs,
                                            R &ps_out) {
    c[0] = c[1] = c[2] = c[3] = c[4] = R(0);
    ps_out = R(0);
    const R rl = st.rl, ul = st.ul, pl = st.pl, rr = st.rr, ur = st.ur, pr = st.pr;
    const R *nh = st.nh, *wl = st.wl, *wr = st.wr, *vf = st.vf;
    R F[5];
    if (RIEM == HYDRO_RIEMANN_HLLC) {
        R ps, ss;
        hllc_flux<R>(K, rl, ul, pl, wl, rr, ur, pr, wr, nh, F, ps, ss);
        if (SCHEME == HYDRO_MFM) {
            F[0] = R(0);
            F[1] = ps * nh[0]; F[2] = ps * nh[1]; F[3] = ps * nh[2];
            F[4] = ps * ss;
        }
    } else {
        R ps, us;
        R tol = sizeof(R) == 8 ? (R)a.p_tol : (R)a.ptolf;
        const GasK<double> *kd = sizeof(R) == 4 && a.riemann_polish ? &a.Kd : nullptr;
        const R cl = sqrt_(div_(K.g * pl, rl)), cr = sqrt_(div_(K.g * pr, rr));
        StarOut so = star_solve<R>(K, rl, ul, pl, cl, rr, ur, pr, cr, p0, tol, a.max_newton, ps, us,
                                   kd);
        fs.iters += so.iters;
        if (so.vacuum) { fs.vacuum++; return; }
        ps_out = ps;
        if (SCHEME == HYDRO_MFM) {
            F[0] = R(0);
            F[1] = ps * nh[0]; F[2] = ps * nh[1]; F[3] = ps * nh[2];
            F[4] = ps * us;
        } else {
            R rs, uu, pp;
            int side;
            star_sample<R>(K, rl, ul, pl, cl, rr, ur, pr, cr, ps, us, rs, uu, pp, side);
            R w0 = side < 0 ? wl[0] : wr[0];
            R w1 = side < 0 ? wl[1] : wr[1];
            R w2 = side < 0 ? wl[2] : wr[2];
            R v2 = uu * uu + w0 * w0 + w1 * w1 + w2 * w2;
            R et = R(0.5) * (rs * v2 + K.g4 * pp);   // (g4 = 2 / (gamma - 1))
            R m = rs * uu;
            F[0] = m;
            F[1] = m * (uu * nh[0] + w0) + pp * nh[0];
            F[2] = m * (uu * nh[1] + w1) + pp * nh[1];
            F[3] = m * (uu * nh[2] + w2) + pp * nh[2];
            F[4] = uu * (et + pp);
        }
    }
    // back to the lab frame
    const R vf2 = vf[0] * vf[0] + vf[1] * vf[1] + vf[2] * vf[2];
    const R Fe = F[4] + (F[1] * vf[0] + F[2] * vf[1] + F[3] * vf[2]) + R(0.5) * F[0] * vf2;
    const R sA = st.sA;
    c[0] = sA * F[0];
    c[1] = sA * (F[1] + F[0] * vf[0]);
    c[2] = sA * (F[2] + F[0] * vf[1]);
    c[3] = sA * (F[3] + F[0] * vf[2]);
    c[4] = sA * Fe;
}

// append a solved face problem (rho_L, u_L, p_L, rho_R, u_R, p_R, p*) to the
// recording buffer when the pair's hash falls under the keep threshold
template <typename R>
__device__ __forceinline__ void record_face(const FluxArgs &a, const GasK<R> &K,
                                            const FaceState<R> &st, R ps, int64_t s, int64_t j) {
    // only physical problems (a cell with negative pressure can reach here)
    if (!(ps > R(0) && st.rl > R(0) && st.pl > R(0) && st.rr > R(0) && st.pr > R(0))) return;
    uint64_t z = (uint64_t)s * 0x9E3779B97F4A7C15ull ^ ((uint64_t)j + 0x632BE59BD9B4E019ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    if ((uint32_t)(z >> 32) >= a.rec_keep) return;
    if (a.rec_hard_only && !two_shock_guess<R>(K, st)) return;
    const unsigned long long k = atomicAdd(a.rec_cursor, 1ull);
    if ((int64_t)k >= a.rec_cap) return;
    float *o = a.rec_faces + k;
    const int64_t c = a.rec_cap;
    o[0] = (float)st.rl; o[c] = (float)st.ul; o[2 * c] = (float)st.pl;
    o[3 * c] = (float)st.rr; o[4 * c] = (float)st.ur; o[5 * c] = (float)st.pr;
    o[6 * c] = (float)ps;
}

// deferred hard faces: the FaceState fields, structure of arrays, in
// HARD_SUB sub-buffers with a cursor each (CTA b writes sub-buffer b mod HARD_SUB)
constexpr int HF_N = 19;
constexpr int HARD_SUB = 256;
// free slots a sub-buffer must keep before a warp defers more hard faces:
// at most 16 warps (4 resident CTAs of 4 warps, 152 SMs x 6 CTAs / 256
// sub-buffers rounded up) can fill one at once, each with up to HQ queued
constexpr int64_t HARD_MARGIN = 2048;

template <typename R>
__device__ __forceinline__ void store_hard(const FluxArgs &a, const FaceState<R> &st, int64_t k,
                                           int32_t s, int32_t j) {
    float *o = a.hard + k;
    const int64_t c = a.hard_cap;
    const float v[HF_N] = {(float)st.rl, (float)st.ul, (float)st.pl, (float)st.rr, (float)st.ur,
                           (float)st.pr, (float)st.wl[0], (float)st.wl[1], (float)st.wl[2],
                           (float)st.wr[0], (float)st.wr[1], (float)st.wr[2], (float)st.nh[0],
                           (float)st.nh[1], (float)st.nh[2], (float)st.vf[0], (float)st.vf[1],
                           (float)st.vf[2], (float)st.sA};
#pragma unroll
    for (int q = 0; q < HF_N; q++) o[q * c] = v[q];
    a.hard_idx[k] = s;
    a.hard_idx[c + k] = j;
}

__device__ __forceinline__ void load_hard(const FluxArgs &a, int64_t k, FaceState<float> &st,
                                          int32_t &s, int32_t &j) {
    const float *o = a.hard + k;
    const int64_t c = a.hard_cap;
    st.rl = o[0]; st.ul = o[c]; st.pl = o[2 * c]; st.rr = o[3 * c]; st.ur = o[4 * c];
    st.pr = o[5 * c];
#pragma unroll
    for (int q = 0; q < 3; q++) {
        st.wl[q] = o[(6 + q) * c];
        st.wr[q] = o[(9 + q) * c];
        st.nh[q] = o[(12 + q) * c];
        st.vf[q] = o[(15 + q) * c];
    }
    st.sA = o[18 * c];
    s = a.hard_idx[k];
    j = a.hard_idx[c + k];
}


// owner accumulators: float-float (value = hi + lo) in the mixed path
struct AccF {
    float hi[5], lo[5];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < 5; q++) hi[q] = lo[q] = 0.f;
    }
    __device__ __forceinline__ void sub(int q, float v) {
        float a = hi[q], b = -v;
        float s = a + b;
        float bb = s - a;
        float e = (a - (s - bb)) + (b - bb);
        hi[q] = s;
        lo[q] += e;
    }
    __device__ __forceinline__ double get(int q) const { return (double)hi[q] + (double)lo[q]; }
};
struct AccD {
    double v[5];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < 5; q++) v[q] = 0.0;
    }
    __device__ __forceinline__ void sub(int q, double x) { v[q] -= x; }
    __device__ __forceinline__ double get(int q) const { return v[q]; }
};
template <typename R> struct AccOf;
template <> struct AccOf<float> { using T = AccF; };
template <> struct AccOf<double> { using T = AccD; };

__device__ __forceinline__ unsigned long long wsum(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int FLUX_WARPS = 4;
constexpr int QCAP = 64;

template <typename R>
struct FluxSmem {
    R cb[32][5];               // solved faces' c, read back by the owners
    unsigned peers[32];        // per owner lane: the batch lanes holding its faces
    int32_t qj[QCAP];          // queued faces: partner j
    uint8_t qo[QCAP];          // queued faces: owner lane
};

// per-warp queue of hard faces waiting to be written to the deferred-face
// buffer (32 at a time, one cursor atomic per 32)
constexpr int HQ = 64;
struct HardQ {
    float v[HF_N][HQ];
    int32_t s[HQ], j[HQ];
    int cnt;   // faces queued (slots taken with shared-memory atomics)
};

// MINB: resident CTAs per SM the register allocation must allow (the
// launch-bounds variants the autotuner chooses from; 4 by default in float)
// LEAN: compiled without the optional per-face work (individual timesteps,
// face recording, the gravity and entropy sums); the launchers take it
// when none is on, which keeps the kernel's code small
template <typename R, int RIEM, int SCHEME, bool DEFER, int MINB = (sizeof(R) == 4 ? 4 : 2),
          bool LEAN = false>
__global__ void __launch_bounds__(FLUX_WARPS * 32, MINB)
k_fluxes(FluxArgs a, const R *__restrict__ rec) {
    __shared__ FluxSmem<R> sm_all[FLUX_WARPS];
    __shared__ HardQ hq_all[DEFER ? FLUX_WARPS : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FluxSmem<R> &sm = sm_all[warp];
    HardQ &hq = hq_all[DEFER ? warp : 0];
    int hh = 0;   // the oldest entry of the warp's hard queue (a ring of HQ)
    if (DEFER && lane == 0) hq.cnt = 0;
    __syncwarp();
    FaceStats fs{0, 0, 0, 0};
    unsigned long long n_hard = 0, n_noroom = 0;
    // buckets: one per warp by its index, or (queue non-NULL) drawn by each
    // warp from a global cursor until none is left -- a warp that finishes
    // a light bucket takes the next one at once instead of idling until the
    // heaviest bucket of its CTA is done
    int64_t bi = blockIdx.x * (int64_t)FLUX_WARPS + warp;
    for (;;) {
        if (a.queue) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(a.queue, 1ull);
            bi = (int64_t)__shfl_sync(0xffffffffu, t, 0);
        }
        if (bi >= a.nbucket) break;
        const int64_t b = a.bucket_ids ? (int64_t)a.bucket_ids[bi] : bi;
        const int f = a.node_first[b], nown = a.node_cnt[b];
        const bool own = lane < nown;
        const int s = f + (own ? lane : 0);
        const Box bx = a.boxes[a.pbox[s]];
        const GasK<R> &K = gas<R>(a);
        const R dt = (R)(a.dt_dev ? *a.dt_dev : a.dt);
        R own4[4];   // the lane's own position and h (enumeration)
        load4<R>(rec + (int64_t)s * REC, own4);
        Member mem;
        mem.init(a.xs, a.ys, a.zs, s, a.h[s], bx);
        typename AccOf<R>::T acc;
        acc.zero();
        const int64_t o = a.nbr_off[s];
        const int cnt = own ? a.nbr_cnt[s] : 0;
        int maxc = cnt;
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, m));
        const unsigned lt = (1u << lane) - 1u;
        int qn = 0;
        __syncwarp();

        // write the k oldest queued hard faces (a ring of HQ entries from hh)
        // to the deferred-face buffer: the CTA's sub-buffer; a full
        // sub-buffer sets hard_ovf and the host redoes the flux stage with a
        // larger buffer
        auto flush_hard = [&](int k) {
            __syncwarp();
            const int sub = blockIdx.x & (HARD_SUB - 1);
            const int64_t subcap = a.hard_cap / HARD_SUB;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&a.hard_cursor[sub], (unsigned long long)k);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (lane < k) {
                const int e = (hh + lane) & (HQ - 1);
                const int64_t slot = (int64_t)base + lane;
                if (slot < subcap) {
                    const int64_t g = sub * subcap + slot, c = a.hard_cap;
#pragma unroll
                    for (int q = 0; q < HF_N; q++) a.hard[q * c + g] = hq.v[q][e];
                    a.hard_idx[g] = hq.s[e];
                    a.hard_idx[c + g] = hq.j[e];
                } else {
                    atomicOr(&a.cnt->hard_ovf, 1ull);
                }
            }
            hh = (hh + k) & (HQ - 1);
            __syncwarp();
            if (lane == 0) hq.cnt -= k;
            __syncwarp();
        };

        // solve the first nb queued faces, one per lane, and hand -c back
        auto solve = [&](int nb) {
            R c[5] = {R(0), R(0), R(0), R(0), R(0)};
            int ol = 32 + lane;   // idle lanes: a key no owner has
            // room left in the CTA's deferred-face sub-buffer (read once per
            // batch): with less than HARD_MARGIN slots -- more than the warps
            // that can share a sub-buffer at once hold in their rings -- the
            // hard faces are solved here from the plain guess instead
            bool room = true;
            if constexpr (DEFER) {
                unsigned long long used = 0;
                if (lane == 0)
                    used = *(volatile const unsigned long long *)&a.hard_cursor[blockIdx.x &
                                                                               (HARD_SUB - 1)];
                used = __shfl_sync(0xffffffffu, used, 0);
                room = (int64_t)used + HARD_MARGIN < a.hard_cap / HARD_SUB;
            }
            if (lane < nb) {
                ol = sm.qo[lane];
                const int j = sm.qj[lane];
                R ri[REC], rj[REC];
                load_full<R>(rec + (int64_t)(f + ol) * REC, ri);   // owner (L1-resident)
                load_full<R>(rec + (int64_t)j * REC, rj);
                R d[3], r2;
                rec_sep(ri, rj, bx, d, r2);
                FaceState<R> st;
                R dtf = dt, hl = R(0.5) * dt, hr = hl;
                if (!LEAN && a.rung) {
                    const int64_t so = f + ol;
                    const double dtd = ldexp(a.dt0, -max(a.rung[so], a.rung[j]));
                    dtf = (R)dtd;
                    hl = (R)(a.toff[so] + 0.5 * dtd);
                    hr = (R)(a.toff[j] + 0.5 * dtd);
                }
                if (face_state<R>(a, K, ri, rj, d, sqrt_(r2), dtf, hl, hr, st, fs)) {
                    bool deferred = false;
                    if constexpr (DEFER) {
                        // hard faces are queued for the learned-guess pass,
                        // which applies both sides of their flux
                        const bool hard = two_shock_guess<R>(K, st);
                        n_hard += hard;
                        n_noroom += hard && !room;
                        if (hard && room) {
                            const int e = (hh + atomicAdd(&hq.cnt, 1)) & (HQ - 1);
                            const float v[HF_N] = {st.rl, st.ul, st.pl, st.rr, st.ur, st.pr,
                                                   st.wl[0], st.wl[1], st.wl[2], st.wr[0],
                                                   st.wr[1], st.wr[2], st.nh[0], st.nh[1],
                                                   st.nh[2], st.vf[0], st.vf[1], st.vf[2], st.sA};
#pragma unroll
                            for (int q = 0; q < HF_N; q++) hq.v[q][e] = v[q];
                            hq.s[e] = f + ol;
                            hq.j[e] = j;
                            deferred = true;
                        }
                    }
                    if (!deferred) {
                        R ps;
                        face_finish<R, RIEM, SCHEME>(a, K, st, R(-1), c, fs, ps);
                        if (!LEAN && RIEM == HYDRO_RIEMANN_EXACT && a.rec_faces)
                            record_face<R>(a, K, st, ps, f + ol, j);
#pragma unroll
                        for (int q = 0; q < 5; q++) atomicAdd(&a.dQ[q * a.n + j], widen(c[q]));
                        if (!LEAN && a.dM && c[0] != R(0)) {
                            const double cm = widen(c[0]);
                            for (int q = 0; q < 3; q++) {
                                atomicAdd(&a.dM[q * a.n + f + ol], cm * (double)d[q]);
                                atomicAdd(&a.dM[q * a.n + j], cm * (double)d[q]);
                            }
                        }
                        if (!LEAN && a.dS && c[0] != R(0)) {
                            const double cm = widen(c[0]);
                            const double sf = cm * widen(c[0] > R(0) ? ri[R_PAD] : rj[R_PAD]);
                            atomicAdd(&a.dS[f + ol], -sf);
                            atomicAdd(&a.dS[j], sf);
                        }
                    }
                }
                fs.pairs++;
            }
#pragma unroll
            for (int q = 0; q < 5; q++) sm.cb[lane][q] = c[q];
            // hand each owner the set of batch lanes that solved its faces
            sm.peers[lane] = 0u;
            unsigned grp = __match_any_sync(0xffffffffu, ol);
            __syncwarp();
            if (lane < nb) sm.peers[ol] = grp;   // equal values from all members
            __syncwarp();
            unsigned mine = sm.peers[lane];
            while (mine) {
                const int t = __ffs(mine) - 1;
                mine &= mine - 1;
#pragma unroll
                for (int q = 0; q < 5; q++) acc.sub(q, sm.cb[t][q]);
            }
            __syncwarp();
            if constexpr (DEFER) {
                if (hq.cnt >= 32) flush_hard(32);   // read after the warp sync above
            }
        };

        // software pipeline over the list: the index two entries ahead and
        // the record of the next entry are in flight while an entry is tested
        int jc = 0 < cnt ? a.nbr_idx[o] : 0;
        int jn = 1 < cnt ? a.nbr_idx[o + 1] : 0;
        R rc4[4] = {R(0), R(0), R(0), R(0)};
        if (0 < cnt) load4<R>(rec + (int64_t)jc * REC, rc4);
        // (one call site of solve: the face code is instantiated once, which
        // keeps the kernel's instruction footprint small; the last pass
        // drains the queue)
        for (int k = 0; k < maxc || qn > 0; k++) {
            if (k < maxc) {
                R rn4[4] = {R(0), R(0), R(0), R(0)};
                if (k + 1 < cnt) load4<R>(rec + (int64_t)jn * REC, rn4);
                const int jnn = k + 2 < cnt ? a.nbr_idx[o + k + 2] : 0;
                bool has = false;
                const int j = jc;
                if (k < cnt && j != s) {
                    R d[3], r2;
                    rec_sep(own4, rc4, bx, d, r2);
                    if (mem(r2, j)) has = (j > s) || !member_j(r2, rc4[R_H], a, s, j, bx);
                    if (!LEAN && has && a.ract && !a.ract[s] && !a.ract[j]) has = false;
                }
                jc = jn;
                jn = jnn;
#pragma unroll
                for (int q = 0; q < 4; q++) rc4[q] = rn4[q];
                unsigned m = __ballot_sync(0xffffffffu, has);
                if (has) {
                    int pos = qn + __popc(m & lt);
                    sm.qj[pos] = j;
                    sm.qo[pos] = (uint8_t)lane;
                }
                qn += __popc(m);
                __syncwarp();
            }
            if (qn >= 32 || (k >= maxc && qn > 0)) {
                const int nb = qn < 32 ? qn : 32;
                solve(nb);
                // move the remainder to the front
                int rest = qn - nb;
                int tj = 0;
                uint8_t to = 0;
                if (lane < rest) { tj = sm.qj[32 + lane]; to = sm.qo[32 + lane]; }
                __syncwarp();
                if (lane < rest) { sm.qj[lane] = tj; sm.qo[lane] = to; }
                qn = rest;
                __syncwarp();
            }
        }
        if constexpr (DEFER) {
            const int rest = hq.cnt;
            if (rest > 0) flush_hard(rest);
        }
        if (own) {
#pragma unroll
            for (int q = 0; q < 5; q++) atomicAdd(&a.dQ[q * a.n + s], acc.get(q));
        }
        if (!a.queue) break;
        __syncwarp();
    }
    unsigned long long p = wsum(fs.pairs), it = wsum(fs.iters), va = wsum(fs.vacuum),
                       fo = wsum(fs.first_order), ha = DEFER ? wsum(n_hard) : 0ull,
                       nr = DEFER ? wsum(n_noroom) : 0ull;
    if (lane == 0) {
        if (p) atomicAdd(&a.cnt->flux_pairs, p);
        if (ha) atomicAdd(&a.cnt->hard_faces, ha);
        if (nr) atomicAdd(&a.cnt->guess_fallbacks, nr);
        if (it) atomicAdd(&a.cnt->newton_iters, it);
        if (va) atomicAdd(&a.cnt->vacuum, va);
        if (fo) atomicAdd(&a.cnt->first_order, fo);
    }
}

// Hard faces deferred by the flux kernel, solved from the learned starting
// pressure.  Each CTA evaluates the network on tiles of 128 faces with
// tcgen05.mma (mlp.cuh), one face per thread (row = thread), then runs the
// exact solver from p_TS exp(y) -- or from Toro's guess when the prediction
// is out of range -- and applies c to both sides (dQ_i -= c, dQ_j += c).
// The iteration always runs to the same tolerance, so the guess changes the
// iteration count, not the flux beyond rounding.
template <int SCHEME>
__global__ void __launch_bounds__(128) k_hard_faces(FluxArgs a) {
    extern __shared__ unsigned char dyn_raw[];
    MlpTile &T = *reinterpret_cast<MlpTile *>(
        (reinterpret_cast<uintptr_t>(dyn_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, lane = tid & 31;
    bool ok = mlp_tile_setup(T, a.mlp_blob, a.mlp_stall != 0);
    uint32_t phase = 0;
    const GasK<float> &K = a.Kf;
    // tiles of 128 slots never straddle sub-buffers (their size is a
    // multiple of 128); tiles past a sub-buffer's count are skipped whole
    const int64_t subcap = a.hard_cap / HARD_SUB;
    const int64_t ntile = a.hard_cap / 128;
    FaceStats fs{0, 0, 0, 0};
    unsigned long long n_learned = 0, n_fallback = 0;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t i = tile * 128 + tid;
        const int64_t sub = (tile * 128) / subcap;
        const int64_t cnt = min((int64_t)a.hard_cursor[sub], subcap);
        const int64_t first = tile * 128 - sub * subcap;
        if (first >= cnt) continue;   // uniform over the CTA
        const bool active = i - sub * subcap < cnt;
        FaceState<float> st;
        int32_t s = 0, j = 0;
        if (active) load_hard(a, i, st, s, j);
        float p0 = -1.f;
        if (ok) {
            float x[MLP_NF], pa = 1.f, lts = 0.f;
            bool in = false;
            if (active) {
                mlp_features(K, st.rl, st.ul, st.pl, st.rr, st.ur, st.pr, x, pa);
                lts = x[9];
                in = mlp_standardise(T, x);
            } else {
#pragma unroll
                for (int q = 0; q < MLP_NF; q++) x[q] = 0.f;
            }
            mlp_put_row(T, tid, x);
            const float y = mlp_tile_eval(T, phase, &ok);
            const float pg = mlp_guess(in, pa, lts, y);
            // a correction below 1e-3 is kept at the two-shock value: a
            // start within 1e-3 converges in as few iterations either way,
            // and the two-shock value may be nearly exact (weak shocks)
            if (active && ok && pg > 0.f && fabsf(y) >= 1e-3f) p0 = pg;
        }
        if (active) {
            if (p0 > 0.f) n_learned++; else n_fallback++;
            float c[5], ps;
            face_finish<float, HYDRO_RIEMANN_EXACT, SCHEME>(a, K, st, p0, c, fs, ps);
            if (a.rec_faces) record_face<float>(a, K, st, ps, s, j);
#pragma unroll
            for (int q = 0; q < 5; q++) {
                const double v = widen(c[q]);
                atomicAdd(&a.dQ[q * a.n + s], -v);
                atomicAdd(&a.dQ[q * a.n + j], v);
            }
            if (a.dM && c[0] != 0.f) {
                float ri4[4], rj4[4], d[3], r2;
                load4<float>(a.recf + (int64_t)s * REC, ri4);
                load4<float>(a.recf + (int64_t)j * REC, rj4);
                rec_sep(ri4, rj4, a.boxes[a.pbox[s]], d, r2);
                const double cm = widen(c[0]);
                for (int q = 0; q < 3; q++) {
                    atomicAdd(&a.dM[q * a.n + s], cm * (double)d[q]);
                    atomicAdd(&a.dM[q * a.n + j], cm * (double)d[q]);
                }
            }
            if (a.dS && c[0] != 0.f) {
                const double cm = widen(c[0]);
                const double sf =
                    cm * (double)a.recf[(int64_t)(c[0] > 0.f ? s : j) * REC + R_PAD];
                atomicAdd(&a.dS[s], -sf);
                atomicAdd(&a.dS[j], sf);
            }
        }
    }
    const unsigned long long it = wsum(fs.iters), va = wsum(fs.vacuum), le = wsum(n_learned),
                             fb = wsum(n_fallback);
    if (lane == 0) {
        if (it) atomicAdd(&a.cnt->newton_iters, it);
        if (va) atomicAdd(&a.cnt->vacuum, va);
        if (le) atomicAdd(&a.cnt->learned_faces, le);
        if (fb) atomicAdd(&a.cnt->guess_fallbacks, fb);
    }
    if (!ok && tid == 0) atomicOr(&a.cnt->flags, ST_MLP);
    mlp_tile_teardown(T);
}

// one flux launch, in the lean variant when no optional per-face work is on
template <typename R, int RIEM, int SCHEME, bool DEFER, int MINB>
cudaError_t launch_k_fluxes(const FluxArgs &a, const R *rec, stream_t st) {
    // persistent: as many CTAs as the register bound lets every SM hold
    unsigned grid = (unsigned)((a.nbucket + FLUX_WARPS - 1) / FLUX_WARPS);
    if (a.queue) grid = std::min<unsigned>(grid, 152u * MINB);
    if (!a.rung && !a.rec_faces && !a.dM && !a.dS && !a.ract) {
        k_fluxes<R, RIEM, SCHEME, DEFER, MINB, true><<<grid, FLUX_WARPS * 32, 0, st>>>(a, rec);
        return launch_check();
    }
    k_fluxes<R, RIEM, SCHEME, DEFER, MINB, false><<<grid, FLUX_WARPS * 32, 0, st>>>(a, rec);
    return launch_check();
}

}  // namespace
}  // namespace hyd
