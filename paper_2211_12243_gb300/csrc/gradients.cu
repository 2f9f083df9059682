// Primitive variables, the E matrix and its inverse, the condition number,
// the Lanson-Vila gradients and the conditioned Barth-Jespersen limiter
// (§2.3.3 Eqs. 10-11, §2.3.5 Eq. 19, §2.3.6, §2.3.7 Eq. 23).
//
// One thread per particle walks its neighbour list twice: pass 1
// accumulates E_i = sum_j omega_j W(r_ij, h_i) dx dx^T (6 unique entries),
// S_f = sum_j omega_j W (f_j - f_i) dx for f = (rho, vx, vy, vz, p), the
// neighbour extremes of f and the signal velocity of Eq. 32; B_i = E_i^-1 is
// formed in double by cofactors (the one place the mixed path pays for
// FP64 per particle), grad f = B S_f; pass 2 collects the largest midpoint
// extrapolations (1/2) dx . grad f that the limiter compares with the
// extremes.  Neighbour records are read as whole vectors from the sorted
// record array (the first 40 B of the line in float).
#include "hydro_internal.cuh"
#include "pairgeom.cuh"
#include "riemann.cuh"
#include "tile_rank.cuh"

namespace hyd {

namespace {

struct GradArgs {
    int64_t n;
    const int64_t *nbr_off;
    const int32_t *nbr_cnt;
    const int32_t *nbr_idx;
    const double *xs, *ys, *zs, *h;
    const int32_t *pbox;
    const Box *boxes;
    int kernel;
    double gamma;
    double ncond_crit, beta_min, beta_max, c_cfl;
    int limiter;
    double *outB, *outG, *outA, *outN;   // sorted staging (may be NULL)
    uint8_t *active;                     // ACT_NCOND set when N_cond fails
    bool only_redo;                      // only the particles flagged ACT_REDO
    double *dt_part;                     // per-particle CFL dt (+inf: no signal)
    int32_t *npair;                      // per-particle gradient pairs
    DevCounters *cnt;
    const uint8_t *ract;                 // individual timesteps: only these (NULL: all)
    const int32_t *list;                 // only these particles (NULL: all n) ...
    const int *nlist;                    // ... their count (device) ...
    int *cursor;                         // ... taken by the warps 32 at a time
    int rank_rounds;                     // dense pass: rank tiles of 128 x this many particles
                                         // by list length (0: no ranking)
};

template <typename R>
__device__ __forceinline__ void load10(const R *p, R v[10]);

template <>
__device__ __forceinline__ void load10<float>(const float *p, float v[10]) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    float4 b = *reinterpret_cast<const float4 *>(p + 4);
    float2 c = *reinterpret_cast<const float2 *>(p + 8);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    v[8] = c.x; v[9] = c.y;
}

template <>
__device__ __forceinline__ void load10<double>(const double *p, double v[10]) {
#pragma unroll
    for (int k = 0; k < 5; k++) {
        double2 a = *reinterpret_cast<const double2 *>(p + 2 * k);
        v[2 * k] = a.x;
        v[2 * k + 1] = a.y;
    }
}

// MINB: resident CTAs per SM the register allocation must allow (1: no
// bound; 5, 6: the variants hydro_autotune times)
// LEAN: compiled without the staged outputs (outB, outG, outA, outN) and
// the individual-timestep mask, which hydro_step does not use
template <typename R, bool LEAN>
__device__ __forceinline__ void grad_one(const GradArgs &a, R *__restrict__ rec, int64_t s) {
    int mypairs = 0;
    if (s < a.n && (!a.only_redo || (a.active[s] & ACT_REDO)) && (LEAN || !a.ract || a.ract[s])) {
        const Box bx = a.boxes[a.pbox[s]];
        R ri[10];
        load10<R>(rec + s * REC, ri);
        const double hd = a.h[s];
        const R h = (R)hd;
        Member mem;
        mem.init(a.xs, a.ys, a.zs, s, hd, bx);
        const R ih = R(1) / h;
        const R norm = kernel_norm<R>(a.kernel, h);
        const R fi[5] = {ri[R_RHO], ri[R_VX], ri[R_VY], ri[R_VZ], ri[R_P]};
        const R g = (R)a.gamma;
        const R ci = sqrt_(div_(g * ri[R_P], ri[R_RHO]));
        R E[6] = {0, 0, 0, 0, 0, 0};
        R S[5][3];
        R fmx[5], fmn[5];
#pragma unroll
        for (int f = 0; f < 5; f++) {
            S[f][0] = S[f][1] = S[f][2] = R(0);
            fmx[f] = fmn[f] = fi[f];
        }
        R vs = R(0);
        const int64_t o = a.nbr_off[s];
        const int c = a.nbr_cnt[s];
        // software pipeline: the index two entries ahead and the record of
        // the next entry are in flight while an entry is summed
        int jc = 0 < c ? a.nbr_idx[o] : 0;
        int jn = 1 < c ? a.nbr_idx[o + 1] : 0;
        R rn[10];
        if (0 < c) load10<R>(rec + (int64_t)jc * REC, rn);
        for (int k = 0; k < c; k++) {
            const int j = jc;
            R rj[10];
#pragma unroll
            for (int q = 0; q < 10; q++) rj[q] = rn[q];
            if (k + 1 < c) load10<R>(rec + (int64_t)jn * REC, rn);
            jc = jn;
            jn = k + 2 < c ? a.nbr_idx[o + k + 2] : 0;
            if (j == s) continue;
            R d[3], r2;
            rec_sep(ri, rj, bx, d, r2);
            if (!mem(r2, j)) continue;
            mypairs++;
            R r = sqrt_(r2);
            R w = rj[R_OM] * norm * kernel_shape<R>(a.kernel, r * ih);
            E[0] += w * d[0] * d[0];
            E[1] += w * d[0] * d[1];
            E[2] += w * d[0] * d[2];
            E[3] += w * d[1] * d[1];
            E[4] += w * d[1] * d[2];
            E[5] += w * d[2] * d[2];
            const R fj[5] = {rj[R_RHO], rj[R_VX], rj[R_VY], rj[R_VZ], rj[R_P]};
#pragma unroll
            for (int f = 0; f < 5; f++) {
                R wd = w * (fj[f] - fi[f]);
                S[f][0] += wd * d[0];
                S[f][1] += wd * d[1];
                S[f][2] += wd * d[2];
                fmx[f] = fj[f] > fmx[f] ? fj[f] : fmx[f];
                fmn[f] = fj[f] < fmn[f] ? fj[f] : fmn[f];
            }
            R cj = sqrt_(div_(g * rj[R_P], rj[R_RHO]));
            R wdot = div_(d[0] * (rj[R_VX] - ri[R_VX]) + d[1] * (rj[R_VY] - ri[R_VY]) +
                          d[2] * (rj[R_VZ] - ri[R_VZ]), r);
            R sig = ci + cj - (wdot < R(0) ? wdot : R(0));
            vs = sig > vs ? sig : vs;
        }
        // B = E^-1 in double, N_cond (Eq. 19)
        double e00 = E[0], e01 = E[1], e02 = E[2], e11 = E[3], e12 = E[4], e22 = E[5];
        double c00 = e11 * e22 - e12 * e12;
        double c01 = e12 * e02 - e01 * e22;
        double c02 = e01 * e12 - e11 * e02;
        double det = e00 * c00 + e01 * c01 + e02 * c02;
        double Bd[6];
        double ncond;
        if (det != 0.0 && isfinite(det)) {
            double id = 1.0 / det;
            Bd[0] = c00 * id;
            Bd[1] = c01 * id;
            Bd[2] = c02 * id;
            Bd[3] = (e00 * e22 - e02 * e02) * id;
            Bd[4] = (e02 * e01 - e00 * e12) * id;
            Bd[5] = (e00 * e11 - e01 * e01) * id;
            if (sizeof(R) == 8) {
                double nE = e00 * e00 + e11 * e11 + e22 * e22 + 2.0 * (e01 * e01 + e02 * e02 + e12 * e12);
                double nB = Bd[0] * Bd[0] + Bd[3] * Bd[3] + Bd[5] * Bd[5] +
                            2.0 * (Bd[1] * Bd[1] + Bd[2] * Bd[2] + Bd[4] * Bd[4]);
                ncond = sqrt(nB * nE) / 3.0;
            } else {
                // N_cond only feeds the threshold test and the limiter's beta
                float b0 = (float)Bd[0], b1 = (float)Bd[1], b2 = (float)Bd[2], b3 = (float)Bd[3],
                      b4 = (float)Bd[4], b5 = (float)Bd[5];
                float nE = E[0] * E[0] + E[3] * E[3] + E[5] * E[5] + 2.f * (E[1] * E[1] + E[2] * E[2] + E[4] * E[4]);
                float nB = b0 * b0 + b3 * b3 + b5 * b5 + 2.f * (b1 * b1 + b2 * b2 + b4 * b4);
                ncond = (double)(sqrtf(nB * nE) * (1.f / 3.f));
            }
        } else {
            for (int k = 0; k < 6; k++) Bd[k] = 0.0;
            ncond = INFINITY;
        }
        const R B[6] = {(R)Bd[0], (R)Bd[1], (R)Bd[2], (R)Bd[3], (R)Bd[4], (R)Bd[5]};
        R G[5][3];
#pragma unroll
        for (int f = 0; f < 5; f++) {
            G[f][0] = B[0] * S[f][0] + B[1] * S[f][1] + B[2] * S[f][2];
            G[f][1] = B[1] * S[f][0] + B[3] * S[f][1] + B[4] * S[f][2];
            G[f][2] = B[2] * S[f][0] + B[4] * S[f][1] + B[5] * S[f][2];
        }
        R alpha[5] = {R(1), R(1), R(1), R(1), R(1)};
        if (a.limiter) {
            R dp[5] = {0, 0, 0, 0, 0}, dm[5] = {0, 0, 0, 0, 0};
            auto pos4 = [&](int j, R v[4]) {
                const R *pj = rec + (int64_t)j * REC;
                if (sizeof(R) == 4) {
                    float4 t = *reinterpret_cast<const float4 *>(pj);
                    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
                } else {
                    v[0] = pj[0]; v[1] = pj[1]; v[2] = pj[2]; v[3] = pj[3];
                }
            };
            // (same pipeline as pass 1)
            int jc2 = 0 < c ? a.nbr_idx[o] : 0;
            int jn2 = 1 < c ? a.nbr_idx[o + 1] : 0;
            R rn4[4];
            if (0 < c) pos4(jc2, rn4);
            for (int k = 0; k < c; k++) {
                const int j = jc2;
                R rj[4] = {rn4[0], rn4[1], rn4[2], rn4[3]};
                if (k + 1 < c) pos4(jn2, rn4);
                jc2 = jn2;
                jn2 = k + 2 < c ? a.nbr_idx[o + k + 2] : 0;
                if (j == s) continue;
                R d[3], r2;
                rec_sep(ri, rj, bx, d, r2);
                if (!mem(r2, j)) continue;
#pragma unroll
                for (int f = 0; f < 5; f++) {
                    R e = R(0.5) * (d[0] * G[f][0] + d[1] * G[f][1] + d[2] * G[f][2]);
                    dp[f] = e > dp[f] ? e : dp[f];
                    dm[f] = e < dm[f] ? e : dm[f];
                }
            }
            R ratio = (R)a.ncond_crit / (R)ncond;
            R beta = (R)a.beta_max * (ratio * ratio < R(1) ? ratio * ratio : R(1));
            beta = beta > (R)a.beta_min ? beta : (R)a.beta_min;
#pragma unroll
            for (int f = 0; f < 5; f++) {
                R rp = dp[f] > R(0) ? (fmx[f] - fi[f]) / dp[f] : R(INFINITY);
                R rm = dm[f] < R(0) ? (fmn[f] - fi[f]) / dm[f] : R(INFINITY);
                R al = (R)beta * (rp < rm ? rp : rm);
                alpha[f] = al < R(1) ? al : R(1);
            }
        }
        R *rs = rec + s * REC;
#pragma unroll
        for (int k = 0; k < 6; k++) rs[R_B + k] = B[k];
#pragma unroll
        for (int f = 0; f < 5; f++)
#pragma unroll
            for (int q = 0; q < 3; q++) rs[R_G + 3 * f + q] = alpha[f] * G[f][q];
        if (!LEAN && a.outB) {
            for (int k = 0; k < 6; k++) a.outB[k * a.n + s] = Bd[k];
        }
        if (!LEAN && a.outG) {
            for (int f = 0; f < 5; f++)
                for (int q = 0; q < 3; q++) a.outG[(3 * f + q) * a.n + s] = (double)G[f][q];
        }
        if (!LEAN && a.outA) {
            for (int f = 0; f < 5; f++) a.outA[f * a.n + s] = (double)alpha[f];
        }
        if (!LEAN && a.outN) a.outN[s] = ncond;
        // CFL timestep of Eq. 31 with the signal velocity of Eq. 32 (the
        // minimum over particles is taken by k_grad_reduce)
        double dti = INFINITY;
        if (vs > R(0))
            dti = sizeof(R) == 8 ? a.c_cfl * hd / (double)vs
                                 : (double)((float)a.c_cfl * (float)hd / (float)vs);
        a.dt_part[s] = dti;
        a.npair[s] = mypairs;
        // N_cond guard (§2.3.5)
        if (!(ncond <= a.ncond_crit)) {
            a.active[s] |= ACT_NCOND;
            atomicAdd(&a.cnt->ncond_fail, 1);
        }
    } else if (!LEAN && s < a.n && a.ract && !a.ract[s]) {
        // not starting a step: no pairs, no CFL limit in this sub-step
        a.dt_part[s] = INFINITY;
        a.npair[s] = 0;
    }
}

// one thread per particle: every particle (list NULL), or the *nlist
// particles of list (a guard round's recomputed particles; the count is
// read on the device, the warps take them 32 at a time)
template <typename R, int MINB, bool LEAN = false>
__global__ void __launch_bounds__(128, MINB) k_gradients(GradArgs a, R *__restrict__ rec) {
    if (a.list) {
        const int nl = *a.nlist;
        for (int base = warp_chunk(a.cursor); base < nl; base = warp_chunk(a.cursor)) {
            const int t = base + (threadIdx.x & 31);
            if (t < nl) grad_one<R, LEAN>(a, rec, a.list[t]);
        }
        return;
    }
    // tiles of 128 R consecutive particles ranked by list length (R rounds
    // of 128 threads; one thread per particle, so a warp runs until its
    // longest list is done), or the CTA's 128 in their order
    const int rounds = a.rank_rounds > 0 ? a.rank_rounds : 1;
    const int64_t tile = blockIdx.x * (int64_t)RANK_THREADS * rounds;
    extern __shared__ unsigned rank_key[];
    if (a.rank_rounds) rank_tile(rank_key, rounds, a.nbr_cnt, tile, a.n);
    for (int r = 0; r < rounds; r++) {
        const int t = r * RANK_THREADS + threadIdx.x;
        grad_one<R, LEAN>(a, rec, tile + (a.rank_rounds ? rank_index(rank_key[t], rounds) : t));
    }
}

// the particles with one of `bits` set, appended to idx (count in *nidx;
// the order of the warps' appends is not fixed); warps stride over the
// particles 32 at a time
__global__ void k_compact_flags(int64_t n, const uint8_t *__restrict__ active, uint8_t bits,
                                int32_t *__restrict__ idx, int *__restrict__ nidx) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s - lane < n; s += stride) {
        const bool on = s < n && (active[s] & bits);
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (!m) continue;
        int base = 0;
        if (lane == 0) base = atomicAdd(nidx, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (on) idx[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)s;
    }
}

// global CFL dt (minimum of the per-particle values, Eq. 31) and the count
// of gradient pairs; dt_min_bits and grad_pairs were reset by the launcher
__global__ void __launch_bounds__(256) k_grad_reduce(int64_t n, const double *__restrict__ dt_part,
                                                     const int32_t *__restrict__ npair,
                                                     DevCounters *cnt) {
    __shared__ double smin[8];
    __shared__ unsigned long long ssum[8];
    double m = INFINITY;
    unsigned long long t = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        m = fmin(m, dt_part[s]);
        t += (unsigned long long)npair[s];
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
        t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { smin[w] = m; ssum[w] = t; }
    __syncthreads();
    if (threadIdx.x == 0) {
        m = smin[0];
        t = ssum[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) { m = fmin(m, smin[k]); t += ssum[k]; }
        // positive doubles order like their bit patterns
        atomicMin(&cnt->dt_min_bits, (unsigned long long)__double_as_longlong(m));
        if (t) atomicAdd(&cnt->grad_pairs, t);
    }
}

// entropy switch inputs (§2.3.7); A0 NULL: switch off
struct EntArgs {
    const double *A0;      // entropic function at the start of the step (sorted)
    double *A1;            // the value the step uses (sorted out)
    uint8_t *cand;         // 1: the energies did not give the pressure (sorted)
    double gamma, alpha2, alpha3;
};

// primitives from the sorted conserved state and omega (§2.3.2, Eq. 23),
// the pressure by the switch of §2.3.7
template <typename R>
__global__ void k_primitives(int64_t n, const double *__restrict__ Q,
                             const double *__restrict__ om, const double *__restrict__ h,
                             double gm1, double alpha1, const uint8_t *__restrict__ active,
                             bool only_guard, const double *__restrict__ agrav, EntArgs ent,
                             const uint8_t *__restrict__ ract, R *__restrict__ rec,
                             const int32_t *__restrict__ list, const int *__restrict__ nlist) {
    // (list non-NULL: a guard round's pass over its guard list, on a small
    // grid, instead of one thread per particle)
    const int64_t cnt = list ? (int64_t)*nlist : n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt;
         t += (int64_t)gridDim.x * blockDim.x) [&] {
        const int64_t s = list ? list[t] : t;
        if (only_guard && !(active[s] & ACT_GUARD)) return;
        if (ract && !ract[s]) return;   // (individual timesteps: its record is kept)
        double m = Q[s], px = Q[n + s], py = Q[2 * n + s], pz = Q[3 * n + s];
        double E = Q[4 * n + s], U = Q[5 * n + s];
        double w = om[s];
        // E_grav = m |a| h enters the total-energy switch (§2.3.7)
        double egrav = 0.0;
        if (agrav) {
            const double ax = agrav[s], ay = agrav[n + s], az = agrav[2 * n + s];
            egrav = m * sqrt(ax * ax + ay * ay + az * az) * h[s];
        }
        R *r = rec + s * REC;
        // the pressure route of §2.3.7: 0 total energy, 2 internal energy; the
        // entropy route (1) is taken over by k_entropy_route, which needs the
        // neighbours' velocities this kernel writes
        auto route = [&](double ekin) -> int {
            if (U > alpha1 * (egrav + ekin) && E - ekin > 0.0) return 0;
            return 2;
        };
        double pd = 0.0;   // the pressure in double (entropy switch only)
        int from;
        if (sizeof(R) == 8) {
            double ekin = (px * px + py * py + pz * pz) / (2.0 * m);
            from = route(ekin);
            const double therm = from == 0 ? E - ekin : U;
            const double rho = m / w;
            pd = therm * gm1 / w;
            r[R_H] = (R)h[s];
            r[R_RHO] = (R)rho;
            r[R_VX] = (R)(px / m);
            r[R_VY] = (R)(py / m);
            r[R_VZ] = (R)(pz / m);
            r[R_P] = (R)pd;
            r[R_OM] = (R)w;
        } else {
            // float record: only E - E_kin needs double (cancellation); 1/m
            // from a float reciprocal and one Newton step in double (relative
            // error ~1e-13) and the conversions to float by integer
            // operations keep the work off the narrow FP64 pipe
            const float mf = narrow(m);
            double im = widen(__fdividef(1.f, mf));
            im = fma(im, fma(-m, im, 1.0), im);
            double ekin = 0.5 * (px * px + py * py + pz * pz) * im;
            from = route(ekin);
            const double therm = from == 0 ? E - ekin : U;
            const float wf = narrow(w), imf = narrow(im);
            r[R_H] = (R)narrow(h[s]);
            r[R_RHO] = (R)(mf / wf);
            r[R_VX] = (R)(narrow(px) * imf);
            r[R_VY] = (R)(narrow(py) * imf);
            r[R_VZ] = (R)(narrow(pz) * imf);
            r[R_OM] = (R)wf;
            r[R_P] = (R)(narrow(therm) * narrow(gm1) / wf);
            if (ent.A1) pd = therm * gm1 / w;
        }
        if (ent.A1) {
            // A follows the pressure the energies gave (k_entropy_route keeps A
            // where it takes the entropy route instead)
            const double A = pd / pow(m / w, ent.gamma);
            ent.A1[s] = A;
            r[R_PAD] = (R)A;
            ent.cand[s] = from != 0;
        }
    }();
}

// The entropy route of §2.3.7 for the particles the energies did not
// claim (U <= alpha1 (E_grav + E_kin) or E - E_kin <= 0) and whose A is
// set: p = A rho^gamma when U < alpha3 E_grav or U < alpha2 (E_kin^max + U),
// E_kin^max = max_j (1/2) m_i |v_j - v_i|^2 over j != i with r_ij < h_i.
// alpha2 (e + U) grows with e, so the walk of the particle's list stops at
// the first neighbour whose e satisfies the test (then E_kin^max does);
// velocities are the records' (written by k_primitives for every particle).
template <typename R>
__global__ void k_entropy_route(int64_t n, const int64_t *__restrict__ nbr_off,
                                const int32_t *__restrict__ nbr_cnt,
                                const int32_t *__restrict__ nbr_idx, const double *__restrict__ xs,
                                const double *__restrict__ ys, const double *__restrict__ zs,
                                const double *__restrict__ h, const int32_t *__restrict__ pbox,
                                const Box *__restrict__ boxes, const double *__restrict__ Q,
                                const double *__restrict__ om, const double *__restrict__ agrav,
                                const uint8_t *__restrict__ active, bool only_guard, EntArgs ent,
                                R *__restrict__ rec) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    if (only_guard && !(active[s] & ACT_GUARD)) return;
    if (!ent.cand[s]) return;   // (k_primitives: the energies gave the pressure)
    const double A = ent.A0[s];
    if (!(A > 0.0)) return;
    const double m = Q[s], U = Q[5 * n + s];
    double egrav = 0.0;
    if (agrav) {
        const double ax = agrav[s], ay = agrav[n + s], az = agrav[2 * n + s];
        egrav = m * sqrt(ax * ax + ay * ay + az * az) * h[s];
    }
    R *ri = rec + s * REC;
    bool cold = U < ent.alpha3 * egrav;
    if (!cold) {
        const Box bx = boxes[pbox[s]];
        Member mem;
        mem.init(xs, ys, zs, s, h[s], bx);
        const double vx = (double)ri[R_VX], vy = (double)ri[R_VY], vz = (double)ri[R_VZ];
        const int64_t o = nbr_off[s];
        const int c = nbr_cnt[s];
        for (int k = 0; k < c && !cold; k++) {
            const int j = nbr_idx[o + k];
            if (j == s) continue;
            const R *rj = rec + (int64_t)j * REC;
            R d[3], r2;
            rec_sep(ri, rj, bx, d, r2);
            if (!mem(r2, j)) continue;
            const double dx = (double)rj[R_VX] - vx, dy = (double)rj[R_VY] - vy,
                         dz = (double)rj[R_VZ] - vz;
            const double e = 0.5 * m * ((dx * dx + dy * dy) + dz * dz);
            cold = U < ent.alpha2 * (e + U);
        }
    }
    if (cold) {
        ri[R_P] = (R)(A * pow(m / om[s], ent.gamma));
        ent.A1[s] = A;
        ri[R_PAD] = (R)A;
    }
}

constexpr double GUARD_SEARCH = 2.0;

__device__ __forceinline__ void grow_one(int64_t s, uint8_t *__restrict__ active,
                                         double *__restrict__ nngb, double grow,
                                         int32_t *__restrict__ guard_idx, int *__restrict__ nguard,
                                         double *__restrict__ hs, const double *__restrict__ h,
                                         const int32_t *__restrict__ pbox,
                                         const Box *__restrict__ boxes) {
    uint8_t a = active[s];
    if (a & ACT_NCOND) {
        nngb[s] *= grow;
        // the root moves out with N_NGB, and further than the cube root of
        // the growth where the particle's surroundings are sparse: its list
        // is rebuilt at GUARD_SEARCH h (at most half the shortest box side)
        // before the re-solve, rather than after a failed one
        const Box bx = boxes[pbox[s]];
        const double half = 0.5 * fmin(bx.L[0], fmin(bx.L[1], bx.L[2]));
        hs[s] = fmin(fmax(hs[s], h[s] * GUARD_SEARCH), half);
        active[s] = ACT_SOLVE | ACT_GUARD;
        guard_idx[atomicAdd(nguard, 1)] = (int32_t)s;
    } else {
        active[s] = 0;
    }
}

// N_NGB *= grow for particles that failed the N_cond check; they (only)
// get their density solved again.  After a guard round's gradient pass the
// flags can be set only on the particles it recomputed (its redo list,
// which holds the round's guard particles): then only those are visited;
// after the full pass, every particle.
__global__ void k_guard_grow(int64_t n, uint8_t *__restrict__ active, double *__restrict__ nngb,
                             double grow, int32_t *__restrict__ guard_idx, int *__restrict__ nguard,
                             double *__restrict__ hs, const double *__restrict__ h,
                             const int32_t *__restrict__ pbox, const Box *__restrict__ boxes,
                             const int32_t *__restrict__ redo_idx, const DevCounters *cnt) {
    const bool redo = cnt->redo_pass;
    const int64_t m = redo ? (int64_t)cnt->nredo : n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x)
        grow_one(redo ? (int64_t)redo_idx[t] : t, active, nngb, grow, guard_idx, nguard, hs, h,
                 pbox, boxes);
}

// caller's B, grad, alpha (already gathered to sorted SoA staging) into
// the records: B and the limited gradients alpha * grad
template <typename R>
__global__ void k_load_grads(int64_t n, const double *__restrict__ st, R *__restrict__ rec) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    R *r = rec + s * REC;
    for (int k = 0; k < 6; k++) r[R_B + k] = (R)st[k * n + s];
    for (int f = 0; f < 5; f++) {
        double al = st[(21 + f) * n + s];
        for (int q = 0; q < 3; q++) r[R_G + 3 * f + q] = (R)(al * st[(6 + 3 * f + q) * n + s]);
    }
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t compact_flags(int64_t n, const uint8_t *active, uint8_t bits, int32_t *idx, int *nidx,
                          stream_t st) {
    HYD_CUDA(cudaMemsetAsync(nidx, 0, sizeof(int), st));
    k_compact_flags<<<std::min(grid_for(n, 256), SWEEP_GRID), 256, 0, st>>>(n, active, bits, idx,
                                                                           nidx);
    return launch_check();
}

cudaError_t run_primitives(hydro_ctx *c, stream_t st, bool only_guard) {
    const int64_t n = c->plan.n;
    double gm1 = c->cfg.gamma - 1.0;
    const uint8_t *act = c->d_active.get();
    const double *ag = c->grav_live ? c->d_agrav.get() : nullptr;
    const bool mixed = c->cfg.precision == HYDRO_MIXED;
    const uint8_t *ract = c->rung_live ? c->d_ract.get() : nullptr;
    EntArgs ent = {};
    if (c->ent_live) {
        ent.A0 = c->d_A0.get();
        ent.A1 = c->d_A1.get();
        ent.cand = c->d_ecand.get();
        ent.gamma = c->cfg.gamma;
        ent.alpha2 = c->cfg.alpha2;
        ent.alpha3 = c->cfg.alpha3;
    }
    const unsigned pgrid = only_guard ? 152 * 4 : grid_for(n, 256);
    const int32_t *glist = only_guard ? c->d_guard_idx.get() : nullptr;
    if (mixed)
        k_primitives<float><<<pgrid, 256, 0, st>>>(n, c->d_Q.get(), c->d_omsorted.get(),
                                                              c->d_hsorted.get(), gm1,
                                                              c->cfg.alpha1, act, only_guard, ag,
                                                              ent, ract, c->d_recf.get(), glist,
                                                              &c->d_cnt->nguard);
    else
        k_primitives<double><<<pgrid, 256, 0, st>>>(n, c->d_Q.get(), c->d_omsorted.get(),
                                                               c->d_hsorted.get(), gm1,
                                                               c->cfg.alpha1, act, only_guard, ag,
                                                               ent, ract, c->d_recd.get(), glist,
                                                               &c->d_cnt->nguard);
    HYD_CUDA(launch_check());
    if (c->ent_live) {
        // the entropy route for the particles the energies did not claim
        // (in a guard round, of the re-solved particles: only their h moved)
        if (mixed)
            k_entropy_route<float><<<grid_for(n, 128), 128, 0, st>>>(
                n, c->d_nbr_off.get(), c->d_nbr_cnt.get(), c->d_nbr_idx.get(), c->d_xs.get(),
                c->d_ys.get(), c->d_zs.get(), c->d_hsorted.get(), c->d_pbox.get(), c->d_boxes.get(),
                c->d_Q.get(), c->d_omsorted.get(), ag, act, only_guard, ent, c->d_recf.get());
        else
            k_entropy_route<double><<<grid_for(n, 128), 128, 0, st>>>(
                n, c->d_nbr_off.get(), c->d_nbr_cnt.get(), c->d_nbr_idx.get(), c->d_xs.get(),
                c->d_ys.get(), c->d_zs.get(), c->d_hsorted.get(), c->d_pbox.get(), c->d_boxes.get(),
                c->d_Q.get(), c->d_omsorted.get(), ag, act, only_guard, ent, c->d_recd.get());
        HYD_CUDA(launch_check());
    }
    return cudaSuccess;
}

cudaError_t gather_entropy(hydro_ctx *c, stream_t st) {
    c->ent_live = c->cfg.entropy_switch && c->entA != nullptr;
    if (!c->ent_live) return cudaSuccess;
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_A0.ensure(n));
    HYD_CUDA(c->d_A1.ensure(n));
    HYD_CUDA(c->d_ecand.ensure(n));
    HYD_CUDA(c->d_dS.ensure(n));
    return gather_from_caller(c->d_perm.get(), c->entA, n, 1, c->d_A0.get(), n, st);
}

cudaError_t gather_gravity(hydro_ctx *c, stream_t st) {
    c->grav_live = c->grav != nullptr;
    if (!c->grav) return cudaSuccess;
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_agrav.ensure((size_t)3 * n));
    HYD_CUDA(c->d_dM.ensure((size_t)3 * n));
    return gather_from_caller(c->d_perm.get(), c->grav, n, 3, c->d_agrav.get(), n, st);
}

// the global CFL dt and the gradient pair count over every particle's
// latest values (after the guard rounds, which only need N_cond)
cudaError_t grad_reduce(hydro_ctx *c, stream_t st) {
    const int64_t n = c->plan.n;
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->grad_pairs, 0, sizeof(unsigned long long), st));
    HYD_CUDA(set_u64(&c->d_cnt->dt_min_bits, 0x7FF0000000000000ull, st));   // +inf
    k_grad_reduce<<<152 * 8, 256, 0, st>>>(n, c->d_vsig_dt.get(), c->d_gpairs.get(), c->d_cnt);
    return launch_check();
}

cudaError_t run_gradients(hydro_ctx *c, double *B_out, double *grad_out, double *alpha_out,
                          double *ncond_out, bool only_redo, stream_t st, bool reduce) {
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_vsig_dt.ensure(n));
    HYD_CUDA(c->d_gpairs.ensure(n));
    GradArgs a;
    a.n = n;
    a.nbr_off = c->d_nbr_off.get();
    a.nbr_cnt = c->d_nbr_cnt.get();
    a.nbr_idx = c->d_nbr_idx.get();
    a.xs = c->d_xs.get(); a.ys = c->d_ys.get(); a.zs = c->d_zs.get();
    a.h = c->d_hsorted.get();
    a.pbox = c->d_pbox.get();
    a.boxes = c->d_boxes.get();
    a.kernel = c->cfg.kernel;
    a.gamma = c->cfg.gamma;
    a.ncond_crit = c->cfg.ncond_crit;
    a.beta_min = c->cfg.beta_min;
    a.beta_max = c->cfg.beta_max;
    a.c_cfl = c->cfg.c_cfl;
    a.limiter = c->cfg.limiter;
    a.outB = B_out; a.outG = grad_out; a.outA = alpha_out; a.outN = ncond_out;
    a.active = c->d_active.get();
    a.only_redo = only_redo;
    a.dt_part = c->d_vsig_dt.get();
    a.npair = c->d_gpairs.get();
    a.cnt = c->d_cnt;
    a.ract = c->rung_live ? c->d_ract.get() : nullptr;
    a.list = nullptr;
    a.nlist = nullptr;
    a.cursor = nullptr;
    a.rank_rounds = c->grad_rank == 2 ? rank_rounds(n) : c->grad_rank;
    unsigned grid = a.rank_rounds ? grid_for(n, RANK_THREADS * a.rank_rounds) : grid_for(n, 128);
    size_t smem = a.rank_rounds ? sizeof(unsigned) * RANK_THREADS * a.rank_rounds : 0;
    if (only_redo) {
        // the particles whose lists hold a re-solved one, compacted: a
        // guard round recomputes few particles, spread over the whole set
        // (the re-solved particles' radii into the tree first: the next
        // round's reverse walk bounds by them)
        HYD_CUDA(raise_tree(c, st));
        HYD_CUDA(mark_guard_reverse(c, st));
        HYD_CUDA(c->d_redo_idx.ensure(n));
        HYD_CUDA(compact_flags(n, c->d_active.get(), ACT_REDO, c->d_redo_idx.get(),
                               &c->d_cnt->nredo, st));
        HYD_CUDA(cudaMemsetAsync(&c->d_cnt->redo_cursor, 0, sizeof(int), st));
        a.list = c->d_redo_idx.get();
        a.nlist = &c->d_cnt->nredo;
        a.cursor = &c->d_cnt->redo_cursor;
        a.rank_rounds = 0;
        grid = 152 * 8;
        smem = 0;
    }
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->ncond_fail, 0, sizeof(int), st));
    // (non-zero bytes for a redo pass: the next guard growth reads the flag)
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->redo_pass, only_redo ? 1 : 0, sizeof(int), st));
    const bool lean = !a.outB && !a.outG && !a.outA && !a.outN && !a.ract;
    if (c->cfg.precision == HYDRO_MIXED) {
        float *r = c->d_recf.get();
        if (lean) {
            if (c->grad_minb == 4) k_gradients<float, 4, true><<<grid, 128, smem, st>>>(a, r);
            else if (c->grad_minb == 5) k_gradients<float, 5, true><<<grid, 128, smem, st>>>(a, r);
            else if (c->grad_minb == 6) k_gradients<float, 6, true><<<grid, 128, smem, st>>>(a, r);
            else k_gradients<float, 1, true><<<grid, 128, smem, st>>>(a, r);
        } else {
            if (c->grad_minb == 4) k_gradients<float, 4><<<grid, 128, smem, st>>>(a, r);
            else if (c->grad_minb == 5) k_gradients<float, 5><<<grid, 128, smem, st>>>(a, r);
            else if (c->grad_minb == 6) k_gradients<float, 6><<<grid, 128, smem, st>>>(a, r);
            else k_gradients<float, 1><<<grid, 128, smem, st>>>(a, r);
        }
    } else {
        double *r = c->d_recd.get();
        if (lean) {
            if (c->grad_minb == 4) k_gradients<double, 4, true><<<grid, 128, smem, st>>>(a, r);
            else if (c->grad_minb == 5) k_gradients<double, 5, true><<<grid, 128, smem, st>>>(a, r);
            else if (c->grad_minb == 6) k_gradients<double, 6, true><<<grid, 128, smem, st>>>(a, r);
            else k_gradients<double, 1, true><<<grid, 128, smem, st>>>(a, r);
        } else {
            if (c->grad_minb == 4) k_gradients<double, 4><<<grid, 128, smem, st>>>(a, r);
            else if (c->grad_minb == 5) k_gradients<double, 5><<<grid, 128, smem, st>>>(a, r);
            else if (c->grad_minb == 6) k_gradients<double, 6><<<grid, 128, smem, st>>>(a, r);
            else k_gradients<double, 1><<<grid, 128, smem, st>>>(a, r);
        }
    }
    HYD_CUDA(launch_check());
    return reduce ? grad_reduce(c, st) : cudaSuccess;
}

cudaError_t guard_grow(hydro_ctx *c, stream_t st) {
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_guard_idx.ensure(n));
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->nguard, 0, sizeof(int), st));
    HYD_CUDA(c->d_redo_idx.ensure(n));
    k_guard_grow<<<std::min(grid_for(n, 256), SWEEP_GRID), 256, 0, st>>>(
        n, c->d_active.get(), c->d_nngb.get(), c->cfg.ngb_grow, c->d_guard_idx.get(),
        &c->d_cnt->nguard, c->d_hs.get(), c->d_hsorted.get(), c->d_pbox.get(), c->d_boxes.get(),
        c->d_redo_idx.get(), c->d_cnt);
    return launch_check();
}

cudaError_t load_gradients(hydro_ctx *c, const double *B, const double *grad,
                           const double *alpha, stream_t st) {
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_out.ensure((size_t)27 * n));
    double *stg = c->d_out.get();
    HYD_CUDA(gather_from_caller(c->d_perm.get(), B, n, 6, stg, n, st));
    HYD_CUDA(gather_from_caller(c->d_perm.get(), grad, n, 15, stg + 6 * n, n, st));
    HYD_CUDA(gather_from_caller(c->d_perm.get(), alpha, n, 5, stg + 21 * n, n, st));
    if (c->cfg.precision == HYDRO_MIXED)
        k_load_grads<float><<<grid_for(n, 256), 256, 0, st>>>(n, stg, c->d_recf.get());
    else
        k_load_grads<double><<<grid_for(n, 256), 256, 0, st>>>(n, stg, c->d_recd.get());
    return launch_check();
}

}  // namespace hyd
