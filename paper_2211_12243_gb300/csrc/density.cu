// Smoothing length and particle volume (§2.3.2 Eqs. 5-6, §2.3.5 Eq. 18):
// per particle, solve g(h) = (4 pi/3) h^3 sum_j W(r_ij, h) - N_NGB = 0 by
// safeguarded Newton over the particle's neighbour list, then
// omega = 1 / sum_j W(r_ij, h) (self term included).
//
// g is non-decreasing in h (h^3 W(r, h) is a function of r/h that grows as
// r/h falls), so [lo, hi] brackets the root; a Newton proposal outside the
// bracket (or beyond the list's search radius) is replaced by bisection or
// clamped.  The list covers every j with r < h_search, so g is exact for
// any h <= h_search; a root beyond h_search is reported for a re-search.
//
// FP64 path: everything in double.  Mixed path: the Newton iteration runs in
// float on the fixed-point separations, then one Newton step evaluated in
// double-float (pairs of floats, Dekker/Knuth error-free transformations)
// on the exact 64-bit separations refines h to double-class accuracy
// without the GPU's scarce FP64 pipe; omega is taken from that evaluation.
//
// Tight lists (hydro_step only): once an upper bracket hi of the root is
// known, no later iterate exceeds it, so the particle's list is compacted in
// place to the entries within hi (plus a relative slack that covers the
// float separation's error) and the last pass compacts it to the final h.
// The search radius hs is lowered to the radius the compacted list is
// complete for; the gradient and flux kernels, which test r_ij < h_i
// exactly on every entry, then walk only the members.  Compaction keeps the
// order of the entries, so the members are summed in the same order as in
// the full list.
#include "hydro_internal.cuh"
#include "tile_rank.cuh"

namespace hyd {

namespace {

struct DensArgs {
    int64_t n;
    const int64_t *nbr_off;
    int32_t *nbr_cnt;         // rewritten when lists are compacted
    int32_t *nbr_idx;
    double *hs;               // lowered to the compacted lists' radius
    const double *xs, *ys, *zs;
    const int32_t *pbox;
    const Box *boxes;
    uint8_t *active;          // bit0: solve this particle; bit1: search failed
    const double *nngb;       // per particle N_NGB (NULL: n_ngb)
    double n_ngb;
    int kernel;
    double tol;
    int max_iter;
    bool only_active;
    bool compact;             // compact the lists to the root (see above)
    double *h;                // sorted, in: guess, out: solution
    double *om;               // sorted out
    DevCounters *cnt;
    bool rank;                // full solve: rank the CTA's 128 particles by list length
    const int32_t *list;      // a guard round: only these particles (the round's guard
    const int *nlist;         // list, count on the device), taken by the warps 32 at a
    int *cursor;              // time from a global cursor
};

// Growth of the search radius hs after a failed solve.  First failure
// (hs within 1.3 of the particle's h guess): the weighted count at the
// radius, kf = N_enc(hs), grows about as hs^3 in a locally uniform
// distribution, so the root lies near hs (N / kf)^(1/3): take 10% beyond
// that, at least 5% and at most a doubling.  A radius grown before: double.
__device__ __forceinline__ double search_growth(double N, double kf, double hs, double h) {
    if (!(hs <= 1.3 * h)) return 2.0;
    double g = kf > 0.0 ? 1.1 * cbrt(N / kf) : 2.0;
    return fmin(fmax(g, 1.05), 2.0);
}

// ---------------------------------------------------------------- FP64 path
__global__ void k_density_f64(DensArgs a, double *__restrict__ rec) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= a.n) return;
    if (a.only_active && !(a.active[s] & 1)) return;
    const Box bx = a.boxes[a.pbox[s]];
    const double xi = a.xs[s], yi = a.ys[s], zi = a.zs[s];
    double hsi = a.hs[s];
    const double N = a.nngb ? a.nngb[s] : a.n_ngb;
    const int64_t o = a.nbr_off[s];
    int32_t *idx = a.nbr_idx + o;
    int c = a.nbr_cnt[s];
    const double Kn = kernel_Kn<double>(a.kernel);
    double h = a.h[s];
    if (!(h > 0.0) || h > hsi) h = hsi;
    double lo = 0.0, hi = -1.0;
    bool conv = false, fail = false;
    double kf_fail = 0.0;   // N_enc(hsi) = Kn sum f at a failure
    auto sep = [&](int j) {
        double dx = fold64(a.xs[j] - xi, bx.L[0]);
        double dy = fold64(a.ys[j] - yi, bx.L[1]);
        double dz = fold64(a.zs[j] - zi, bx.L[2]);
        return sqrt(dx * dx + dy * dy + dz * dz);
    };
    for (int it = 1; it <= a.max_iter; it++) {
        double f = 0.0, mq = 0.0, ih = 1.0 / h;
        // an upper bracket well inside the list radius: drop the entries
        // beyond it (relative slack 1e-9 >> the rounding of r)
        const bool shrink = a.compact && hi > 0.0 && hi < 0.8 * hsi;
        const double keep = hi * (1.0 + 1e-9);
        int w = 0;
        for (int k = 0; k < c; k++) {
            const int j = idx[k];
            const double r = sep(j);
            if (shrink && r < keep) idx[w++] = j;
            double fv, mv;
            kernel_f<double>(a.kernel, r * ih, fv, mv);
            f += fv;
            mq += mv;
        }
        if (shrink) { c = w; hsi = hi * (1.0 + 5e-10); }   // complete below this
        double g = Kn * f - N;
        double dg = Kn * mq * ih;
        if (g == 0.0) { conv = true; break; }
        if (g < 0.0) {
            if (h >= hsi) { fail = true; kf_fail = Kn * f; break; }
            lo = fmax(lo, h);
        } else {
            hi = (hi < 0.0 || h < hi) ? h : hi;
        }
        double hn = dg > 0.0 ? h - g / dg : -1.0;
        if (hn > 0.0 && fabs(hn - h) <= a.tol * h && hn <= hsi) { h = hn; conv = true; break; }
        if (hi < 0.0) {
            if (!(hn > lo) || hn > 2.0 * h) hn = 2.0 * h;
            if (hn > hsi) hn = hsi;
        } else if (!(hn > lo && hn < hi)) {
            hn = 0.5 * (lo + hi);
        }
        h = hn;
    }
    if (fail) {   // (no compaction happened: failing needs h >= hsi, below any bracket)
        a.hs[s] = hsi * search_growth(N, kf_fail, hsi, a.h[s]);
        a.active[s] = (a.active[s] & ACT_GUARD) | 3;
        atomicAdd(&a.cnt->search_fail, 1);
        set_flag(a.cnt, ST_SEARCH);
        return;
    }
    if (!conv) set_flag(a.cnt, ST_NOCONV_H);
    double sw = 0.0, ih = 1.0 / h;
    const double keep = h * (1.0 + 1e-9);
    int w = 0;
    for (int k = 0; k < c; k++) {
        const int j = idx[k];
        const double r = sep(j);
        if (a.compact && r < keep) idx[w++] = j;
        sw += kernel_shape<double>(a.kernel, r * ih);
    }
    if (a.compact) {
        // complete for every r < h (1 + 5e-10)
        a.nbr_cnt[s] = w;
        a.hs[s] = h * (1.0 + 5e-10);
    }
    sw *= kernel_norm<double>(a.kernel, h);
    double om = 1.0 / sw;
    a.h[s] = h;
    a.om[s] = om;
    rec[s * REC + R_H] = h;
    rec[s * REC + R_OM] = om;
}

// ------------------------------------------------------- double-float tools
// value = hi + lo, |lo| <= ulp(hi)/2
struct df {
    float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = a * b;
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }
// square root by one Newton correction of the float root
__device__ __forceinline__ df df_sqrt(df a) {
    if (a.hi <= 0.f) return {0.f, 0.f};
    float x = sqrtf(a.hi);
    df xx = two_prod(x, x);
    df r = df_sub(a, xx);
    float corr = __fdividef(r.hi, 2.f * x);
    return quick_two_sum(x, corr);
}
__device__ __forceinline__ df df_div(df a, df b) {
    float q1 = a.hi / b.hi;
    df r = df_sub(a, df_mulf(b, q1));
    float q2 = r.hi / b.hi;
    return quick_two_sum(q1, q2);
}
// float-float of a 64-bit integer |v| < 2^62 from three 21-bit pieces,
// each converted exactly without a conversion instruction
__device__ __forceinline__ df from_i64(long long v) {
    int32_t hi = (int32_t)(v >> 42);                                   // |hi| < 2^20
    int32_t mid = (int32_t)(((unsigned long long)v >> 21) & 0x1FFFFFull);
    int32_t lo = (int32_t)((unsigned long long)v & 0x1FFFFFull);
    float fh = i2f_small(hi) * 4398046511104.0f;                       // 2^42
    float fm = i2f_small(mid) * 2097152.0f;                            // 2^21
    df s = two_sum(fh, fm);
    return df_add(s, {i2f_small(lo), 0.f});
}

// ---------------------------------------------------------------- mixed path
constexpr int DENS_THREADS = 128;
static_assert(DENS_THREADS == RANK_THREADS, "the ranked tiles take 128 threads a round");

// one particle's float Newton solve, then the double-float refinement
__device__ __forceinline__ void dens_one(const DensArgs &a, const uint64_t *__restrict__ q64x,
                                         const uint64_t *__restrict__ q64y,
                                         const uint64_t *__restrict__ q64z,
                                         float *__restrict__ rec, int64_t s) {
    if (s >= a.n) return;
    if (a.only_active && !(a.active[s] & 1)) return;
    const Box bx = a.boxes[a.pbox[s]];
    const float *ri = rec + s * REC;
    const uint32_t qxi = __float_as_uint(ri[R_X]), qyi = __float_as_uint(ri[R_Y]),
                   qzi = __float_as_uint(ri[R_Z]);
    const double hsi_d = a.hs[s];
    float hsi = (float)hsi_d;
    const float N = (float)(a.nngb ? a.nngb[s] : a.n_ngb);
    const int64_t o = a.nbr_off[s];
    int32_t *idx = a.nbr_idx + o;
    int c = a.nbr_cnt[s];
    const float Kn = kernel_Kn<float>(a.kernel);
    float h = (float)a.h[s];
    if (!(h > 0.f) || h > hsi) h = hsi;
    float lo = 0.f, hi = -1.f;
    bool conv = false, fail = false;
    float comp = -1.f;   // radius the compacted list is complete for (none yet)
    float kf_fail = 0.f;  // N_enc(hsi) = Kn sum f at a failure
    const float ftol = 2e-6f;
    // The float separation from the fixed-point positions is within
    // 4e-7 r + 4e-10 L of the exact one, so keeping the entries with float
    // r < X (1 + 1e-4) leaves the list complete for every r < X (1 + 5e-5)
    // when X > L / 65536 (compaction is skipped below that).
    const float xmin = (float)(fmin(bx.L[0], fmin(bx.L[1], bx.L[2])) * (1.0 / 65536.0));
    auto sep_r = [&](int j) {
        const float *rj = rec + (int64_t)j * REC;
        float4 pj = *reinterpret_cast<const float4 *>(rj);
        float dx = qdiff(qxi, __float_as_uint(pj.x), bx.s[0]);
        float dy = qdiff(qyi, __float_as_uint(pj.y), bx.s[1]);
        float dz = qdiff(qzi, __float_as_uint(pj.z), bx.s[2]);
        float r2 = dx * dx + dy * dy + dz * dz;
        return r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
    };
    for (int it = 1; it <= a.max_iter; it++) {
        float f = 0.f, mq = 0.f, ih = 1.f / h;
        // an upper bracket well inside the list radius: drop the entries
        // beyond it (no later iterate exceeds hi)
        const bool shrink = a.compact && hi > xmin && hi < 0.8f * hsi;
        const float keep = hi * 1.0001f;
        int w = 0;
        for (int k = 0; k < c; k++) {
            const int j = idx[k];
            const float r = sep_r(j);
            if (shrink && r < keep) idx[w++] = j;
            float fv, mv;
            kernel_f<float>(a.kernel, r * ih, fv, mv);
            f += fv;
            mq += mv;
        }
        if (shrink) { c = w; comp = hi * 1.00005f; hsi = comp; }
        float g = Kn * f - N;
        float dg = Kn * mq * ih;
        if (g == 0.f) { conv = true; break; }
        if (g < 0.f) {
            if (h >= hsi) { fail = true; kf_fail = Kn * f; break; }
            lo = fmaxf(lo, h);
        } else {
            hi = (hi < 0.f || h < hi) ? h : hi;
        }
        float hn = dg > 0.f ? h - g / dg : -1.f;
        if (hn > 0.f && fabsf(hn - h) <= ftol * h && hn <= hsi) { h = hn; conv = true; break; }
        if (hi < 0.f) {
            if (!(hn > lo) || hn > 2.f * h) hn = 2.f * h;
            if (hn > hsi) hn = hsi;
        } else if (!(hn > lo && hn < hi)) {
            hn = 0.5f * (lo + hi);
        }
        h = hn;
    }
    if (fail) {   // (no compaction happened: failing needs h >= hsi, below any bracket)
        a.hs[s] = hsi_d * search_growth((double)N, (double)kf_fail, hsi_d, a.h[s]);
        a.active[s] = (a.active[s] & ACT_GUARD) | 3;
        atomicAdd(&a.cnt->search_fail, 1);
        set_flag(a.cnt, ST_SEARCH);
        return;
    }
    if (!conv) set_flag(a.cnt, ST_NOCONV_H);
    // one Newton step in double-float on exact 64-bit fixed-point separations
    const uint64_t xi64 = q64x[s], yi64 = q64y[s], zi64 = q64z[s];
    const float sx = (float)(bx.L[0] * 5.421010862427522e-20);  // L / 2^64
    const float sy = (float)(bx.L[1] * 5.421010862427522e-20);
    const float sz = (float)(bx.L[2] * 5.421010862427522e-20);
    df hd = {h, 0.f};
    df ih = df_div({1.f, 0.f}, hd);
    df F = {0.f, 0.f}, MQ = {0.f, 0.f};
    const float hcut = h * (1.f + 1e-5f);   // W = 0 beyond h: skip those (float r is good to 1e-7)
    const bool fin = a.compact && h > xmin;
    const float keep = h * 1.0001f;
    int w = 0;
    for (int k = 0; k < c; k++) {
        const int j = idx[k];
        const float rf = sep_r(j);
        if (fin && rf < keep) idx[w++] = j;
        if (rf >= hcut) continue;
        long long ix = (long long)(q64x[j] - xi64);
        long long iy = (long long)(q64y[j] - yi64);
        long long iz = (long long)(q64z[j] - zi64);
        df dx = df_mulf(from_i64(ix), sx);
        df dy = df_mulf(from_i64(iy), sy);
        df dz = df_mulf(from_i64(iz), sz);
        df r2 = df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz));
        df q = df_mul(df_sqrt(r2), ih);
        if (q.hi >= 1.f) continue;
        df one = {1.f, 0.f};
        df t = df_sub(one, q);
        df t2 = df_mul(t, t);
        if (a.kernel == 0) {
            df t3 = df_mul(t2, t);
            df fv = df_mul(df_mul(t3, t), df_add(one, df_mulf(q, 4.f)));
            df mv = df_mulf(df_mul(df_mul(q, q), t3), 20.f);
            F = df_add(F, fv);
            MQ = df_add(MQ, mv);
        } else {
            df q2 = df_mul(q, q);
            df fv, mv;
            if (q.hi <= 0.5f) {
                fv = df_add(df_sub(one, df_mulf(q2, 6.f)), df_mulf(df_mul(q2, q), 6.f));
                mv = df_sub(df_mulf(q2, 12.f), df_mulf(df_mul(q2, q), 18.f));
            } else {
                fv = df_mulf(df_mul(t2, t), 2.f);
                mv = df_mulf(df_mul(q, t2), 6.f);
            }
            F = df_add(F, fv);
            MQ = df_add(MQ, mv);
        }
    }
    // g = Kn F - N, dg = Kn MQ / h  ->  h_new = h - (F - N/Kn) h / MQ
    double Fd = (double)F.hi + (double)F.lo;
    double MQd = (double)MQ.hi + (double)MQ.lo;
    double hN = (double)h;
    double Kd = a.kernel == 0 ? 14.0 : 32.0 / 3.0;
    // (N_NGB in double: a guard round's grown 32 * 1.2^k is not a float)
    const double Nd = a.nngb ? a.nngb[s] : a.n_ngb;
    double hnew = MQd > 0.0 ? hN - (Fd - Nd / Kd) * hN / MQd : hN;
    if (fin || comp > 0.f) {
        // the compacted list is complete for r < crad
        const double crad = fin ? hN * (1.0 + 5e-5) : (double)comp;
        a.nbr_cnt[s] = fin ? w : c;
        a.hs[s] = crad;
        if (!(hnew < crad)) {
            // the refinement left the compacted radius (an unconverged float
            // root): search again from a rebuilt list
            a.active[s] = (a.active[s] & ACT_GUARD) | 3;
            atomicAdd(&a.cnt->search_fail, 1);
            set_flag(a.cnt, ST_SEARCH);
            return;
        }
    }
    // omega from the sum at h (first order in the small correction)
    // sum_j W(r, hnew) = norm(hnew) sum f(q_new); d/dh [h^3 sum W] = Kn MQ / h * 3/(4 pi)
    double normh = kernel_norm<double>(a.kernel, hnew);
    double fsum = Fd + (hnew - hN) * MQd / hN;   // first-order update of sum f(q)
    double om = 1.0 / (normh * fsum);
    a.h[s] = hnew;
    a.om[s] = om;
    float *rr = rec + s * REC;
    rr[R_H] = (float)hnew;
    rr[R_OM] = (float)om;
}

// one thread per particle, in the sorted order (a partial solve too: its
// particles are often many and clustered, and a compacted list would scatter
// each warp's gathers over the box); the full solve ranks the CTA's 128
// particles by list length.  (Larger ranked tiles spread the repeated
// gathers of the Newton iterations over more of the Morton curve: slower.)
__global__ void k_density_mixed(DensArgs a, const uint64_t *__restrict__ q64x,
                                const uint64_t *__restrict__ q64y,
                                const uint64_t *__restrict__ q64z, float *__restrict__ rec) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a.rank) {
        __shared__ unsigned rank_key[RANK_THREADS];
        const int64_t base = blockIdx.x * (int64_t)RANK_THREADS;
        rank_tile(rank_key, 1, a.nbr_cnt, base, a.n);
        s = base + rank_index(rank_key[threadIdx.x], 1);
    }
    dens_one(a, q64x, q64y, q64z, rec, s);
}

// a guard round's re-solve: the warps take the particles of the round's
// guard list 32 at a time (its own kernel: the branch would cost the full
// solve's kernel ten registers)
__global__ void k_density_mixed_list(DensArgs a, const uint64_t *__restrict__ q64x,
                                     const uint64_t *__restrict__ q64y,
                                     const uint64_t *__restrict__ q64z, float *__restrict__ rec) {
    const int nl = *a.nlist;
    for (int b0 = warp_chunk(a.cursor); b0 < nl; b0 = warp_chunk(a.cursor)) {
        const int t = b0 + (threadIdx.x & 31);
        if (t < nl) dens_one(a, q64x, q64y, q64z, rec, a.list[t]);
    }
}

// the search radius of particles whose root lay beyond it, as the density
// kernel grew it (not below margin h); never beyond half the shortest box
// side (one periodic image)
// (list non-NULL: only its *nlist particles -- a guard round's, the only
// ones it solves; every other particle's flags are clear then)
__global__ void k_grow_search(int64_t n, uint8_t *__restrict__ active, double *__restrict__ hs,
                              const double *__restrict__ h, double margin,
                              const int32_t *__restrict__ pbox, const Box *__restrict__ boxes,
                              const int32_t *__restrict__ list, const int *__restrict__ nlist) {
    const int64_t cnt = list ? (int64_t)*nlist : n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = list ? list[t] : t;
        const uint8_t a = active[s];
        if (a & 2) {
            const Box bx = boxes[pbox[s]];
            double half = 0.5 * fmin(bx.L[0], fmin(bx.L[1], bx.L[2]));
            hs[s] = fmin(fmax(hs[s], h[s] * margin), half);   // (grown by the density kernel)
            active[s] = (a & ACT_GUARD) | 1;
        } else {
            active[s] = a & ACT_GUARD;
        }
    }
}

__global__ void k_fixed64(int64_t n, const double *__restrict__ xs, const double *__restrict__ ys,
                          const double *__restrict__ zs, const int32_t *__restrict__ pbox,
                          const Box *__restrict__ boxes, uint64_t *__restrict__ qx,
                          uint64_t *__restrict__ qy, uint64_t *__restrict__ qz) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const Box bx = boxes[pbox[s]];
    const double two64 = 18446744073709551616.0;
    double t;
    t = xs[s] / bx.L[0] * two64; qx[s] = t >= two64 ? 0ull : (uint64_t)t;
    t = ys[s] / bx.L[1] * two64; qy[s] = t >= two64 ? 0ull : (uint64_t)t;
    t = zs[s] / bx.L[2] * two64; qz[s] = t >= two64 ? 0ull : (uint64_t)t;
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t run_density(hydro_ctx *c, bool only_active, bool compact, stream_t st, bool guard) {
    const int64_t n = c->plan.n;
    DensArgs a;
    a.n = n;
    a.nbr_off = c->d_nbr_off.get();
    a.nbr_cnt = c->d_nbr_cnt.get();
    a.nbr_idx = c->d_nbr_idx.get();
    a.hs = c->d_hs.get();
    a.xs = c->d_xs.get(); a.ys = c->d_ys.get(); a.zs = c->d_zs.get();
    a.pbox = c->d_pbox.get();
    a.boxes = c->d_boxes.get();
    a.active = c->d_active.get();
    a.nngb = c->d_nngb.get();
    a.n_ngb = c->cfg.n_ngb;
    a.kernel = c->cfg.kernel;
    a.tol = c->cfg.h_tol;
    a.max_iter = c->cfg.max_h_iter;
    a.only_active = only_active;
    a.compact = compact;
    a.h = c->d_hsorted.get();
    a.om = c->d_omsorted.get();
    a.cnt = c->d_cnt;
    // ranked when the gradient kernel ranks (the same divergence)
    a.rank = c->grad_rank && !only_active;
    a.list = nullptr;
    a.nlist = nullptr;
    a.cursor = nullptr;
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->search_fail, 0, sizeof(int), st));
    if (c->cfg.precision == HYDRO_MIXED) {
        // 64-bit fixed-point copies for the refinement step (xs.. are sorted)
        // (positions are fixed within a step: the solves of selected
        // particles reuse the copies of the step's first, full solve; the
        // sub-steps of individual timesteps move every particle)
        HYD_CUDA(c->d_q64.ensure((size_t)3 * n));
        uint64_t *q64 = c->d_q64.get();
        if (!only_active || c->rung_live) {
            k_fixed64<<<grid_for(n, 256), 256, 0, st>>>(n, c->d_xs.get(), c->d_ys.get(),
                                                         c->d_zs.get(), c->d_pbox.get(),
                                                         c->d_boxes.get(), q64, q64 + n, q64 + 2 * n);
            HYD_CUDA(launch_check());
        }
        if (guard && only_active) {
            // the round's guard particles, few and scattered, each with a
            // long list at its grown radius: one thread each, the warps
            // drawing them from the guard list
            HYD_CUDA(cudaMemsetAsync(&c->d_cnt->solve_cursor, 0, sizeof(int), st));
            a.list = c->d_guard_idx.get();
            a.nlist = &c->d_cnt->nguard;
            a.cursor = &c->d_cnt->solve_cursor;
            k_density_mixed_list<<<152 * 8, DENS_THREADS, 0, st>>>(a, q64, q64 + n, q64 + 2 * n,
                                                                   c->d_recf.get());
        } else {
            k_density_mixed<<<grid_for(n, DENS_THREADS), DENS_THREADS, 0, st>>>(
                a, q64, q64 + n, q64 + 2 * n, c->d_recf.get());
        }
    } else {
        k_density_f64<<<grid_for(n, 128), 128, 0, st>>>(a, c->d_recd.get());
    }
    return launch_check();
}

cudaError_t grow_search_radius(hydro_ctx *c, stream_t st, bool guard) {
    const int64_t n = c->plan.n;
    k_grow_search<<<guard ? 152 * 4 : grid_for(n, 256), 256, 0, st>>>(
        n, c->d_active.get(), c->d_hs.get(), c->d_hsorted.get(), c->cfg.search_margin,
        c->d_pbox.get(), c->d_boxes.get(), guard ? c->d_guard_idx.get() : nullptr,
        &c->d_cnt->nguard);
    return launch_check();
}

}  // namespace hyd
