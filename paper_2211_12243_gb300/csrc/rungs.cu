// Individual timesteps (§2.3.4 power-of-two hierarchy, §2.3.10 criteria):
// the per-particle bookkeeping of hydro_step_rungs.  The base step dt0 runs
// 2^rmax sub-steps; at sub-step k a particle of rung r starts a step when k
// is a multiple of 2^(rmax - r).  The master copies of the rungs and of the
// sub-step at which each particle's step started are kept in caller order;
// each sub-step gathers them into sorted order (the order of sub-step 0)
// with the flag "starts now" and the time since the particle's state was
// taken, and lists the starting particles for the reverse tree walk that
// finds the buckets whose lists the sub-step needs (rung_lists in api.cu).
// A particle that does not start keeps the
// record (h, rho, v, p, omega, B, limited gradients) of its last start: the
// records of the starting particles are saved in caller order after their
// gradients, and the others' are loaded back over the freshly gathered
// positions.
#include "hydro_internal.cuh"
#include "pairgeom.cuh"

namespace hyd {

namespace {

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__global__ void k_rung_prep(int64_t n, const int32_t *__restrict__ perm,
                            const int32_t *__restrict__ rung_c, int32_t *__restrict__ kstart_c,
                            int64_t k, int rmax, double dtmin, int32_t *__restrict__ rung_s,
                            uint8_t *__restrict__ ract, double *__restrict__ toff,
                            int32_t *__restrict__ act_idx, DevCounters *cnt) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool act = false;
    if (s < n) {
        const int64_t o = perm[s];
        const int r = rung_c[o];
        const int64_t period = (int64_t)1 << (rmax - r);
        act = k % period == 0;
        int64_t ks = kstart_c[o];
        if (act) {
            ks = k;
            kstart_c[o] = (int32_t)k;
        }
        rung_s[s] = r;
        ract[s] = act ? 1 : 0;
        toff[s] = (double)(k - ks) * dtmin;
    }
    const unsigned m = __ballot_sync(0xffffffffu, act);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && m) {
        atomicAdd(&cnt->rung_active, (unsigned long long)__popc(m));
        base = atomicAdd(&cnt->nguard, __popc(m));
    }
    // the starting particles also form the list the reverse walk reads
    base = __shfl_sync(0xffffffffu, base, 0);
    if (act) act_idx[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)s;
}

// the particles starting a step solve their density with N_NGB restarted
__global__ void k_rung_fill(int64_t n, const uint8_t *__restrict__ ract, double *__restrict__ nngb,
                            double n_ngb, uint8_t *__restrict__ active) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    nngb[s] = n_ngb;
    active[s] = ract[s] ? ACT_SOLVE : 0;
}

// the records of the particles that do not start: everything but the
// (current) positions from their last start
template <typename R>
__global__ void k_rec_load(int64_t n, const int32_t *__restrict__ perm,
                           const uint8_t *__restrict__ ract, const R *__restrict__ store,
                           R *__restrict__ rec) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n || ract[s]) return;
    const R *src = store + (int64_t)perm[s] * REC;
    R *dst = rec + s * REC;
#pragma unroll
    for (int q = R_H; q < REC; q++) dst[q] = src[q];
}

template <typename R>
__global__ void k_rec_save(int64_t n, const int32_t *__restrict__ perm,
                           const uint8_t *__restrict__ ract, const R *__restrict__ rec,
                           R *__restrict__ store) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n || !ract[s]) return;
    const R *src = rec + s * REC;
    R *dst = store + (int64_t)perm[s] * REC;
#pragma unroll
    for (int q = 0; q < REC; q++) dst[q] = src[q];
}

// rung from the two criteria (§2.3.10): dt_cfl (the gradient stage's
// per-particle Eq. 31 value) and dt_acc = c_acc sqrt(h / |a|) with
// |a| = |grad p| / rho from the record's limited pressure gradient; the
// smallest r >= 0 with min(dt_cfl, dt_acc) > 2^-r dt0, at most max_rung.
// The products are rounded one by one (no contraction) as the definition
// states them.
template <typename R>
__global__ void k_rung_assign(int64_t n, const double *__restrict__ dt_cfl,
                              const R *__restrict__ rec, const double *__restrict__ h,
                              double c_acc, double dt0, int max_rung, int32_t *__restrict__ rung_s,
                              DevCounters *cnt) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const R *r = rec + s * REC;
    const double gx = (double)r[R_G + 12], gy = (double)r[R_G + 13], gz = (double)r[R_G + 14];
    const double g2 = __dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz));
    const double acc = __ddiv_rn(sqrt(g2), (double)r[R_RHO]);
    const double dta = acc > 0.0 ? __dmul_rn(c_acc, sqrt(__ddiv_rn(h[s], acc))) : INFINITY;
    const double dtc = dt_cfl[s];
    const double t = dtc < dta ? dtc : dta;
    int q = 0;
    while (q < max_rung && !(t > ldexp(dt0, -q))) q++;
    if (!(t > ldexp(dt0, -q))) atomicAdd(&cnt->rung_capped, 1);
    rung_s[s] = q;
}

// one sweep of the neighbour limiter |r_i - r_j| <= 2 over the flux pairs
// (r_ij < max(h_i, h_j)): each such pair lies within the h of one of its
// particles, so every particle walks its own list (r_ij < h_i) and raises
// whichever side is more than two rungs coarser.  Rungs only rise; a sweep
// in which nothing rose leaves every pair satisfied (the host repeats until
// then).
template <typename R>
__global__ void k_rung_limit(int64_t n, const int64_t *__restrict__ nbr_off,
                             const int32_t *__restrict__ nbr_cnt,
                             const int32_t *__restrict__ nbr_idx, const double *__restrict__ xs,
                             const double *__restrict__ ys, const double *__restrict__ zs,
                             const double *__restrict__ h, const int32_t *__restrict__ pbox,
                             const Box *__restrict__ boxes, const R *__restrict__ rec,
                             int32_t *rung_s, DevCounters *cnt) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const Box bx = boxes[pbox[s]];
    Member mem;
    mem.init(xs, ys, zs, s, h[s], bx);
    volatile const int32_t *rg = rung_s;
    int mine = rg[s];
    bool raised = false;
    const int64_t o = nbr_off[s];
    const int c = nbr_cnt[s];
    for (int k = 0; k < c; k++) {
        const int j = nbr_idx[o + k];
        if (j == s) continue;
        R d[3], r2;
        rec_sep(rec + s * REC, rec + (int64_t)j * REC, bx, d, r2);
        if (!mem(r2, j)) continue;
        const int rj = rg[j];
        if (rj - 2 > mine) {
            mine = rj - 2;
            atomicMax(&rung_s[s], mine);
            raised = true;
        } else if (mine - 2 > rj) {
            atomicMax(&rung_s[j], mine - 2);
            raised = true;
        }
    }
    if (raised) atomicOr(&cnt->rung_changed, 1);
}

__global__ void k_rung_scatter(int64_t n, const int32_t *__restrict__ perm,
                               const int32_t *__restrict__ rung_s, int32_t *__restrict__ rung_c,
                               DevCounters *cnt) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int r = rung_s[s];
    rung_c[perm[s]] = r;
    atomicMax(&cnt->rung_max, r);
}

}  // namespace

cudaError_t rung_prep(hydro_ctx *c, int64_t k, int rmax, double dtmin, stream_t st) {
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_guard_idx.ensure(n));
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->nguard, 0, sizeof(int), st));
    k_rung_prep<<<grid_for(n, 256), 256, 0, st>>>(n, c->d_perm.get(), c->d_rung_c.get(),
                                                   c->d_kstart_c.get(), k, rmax, dtmin,
                                                   c->d_rung_s.get(), c->d_ract.get(),
                                                   c->d_toff.get(), c->d_guard_idx.get(), c->d_cnt);
    return launch_check();
}

cudaError_t rung_fill(hydro_ctx *c, stream_t st) {
    const int64_t n = c->plan.n;
    k_rung_fill<<<grid_for(n, 256), 256, 0, st>>>(n, c->d_ract.get(), c->d_nngb.get(),
                                                   c->cfg.n_ngb, c->d_active.get());
    return launch_check();
}

cudaError_t rung_records(hydro_ctx *c, bool save, stream_t st) {
    const int64_t n = c->plan.n;
    const unsigned g = grid_for(n, 128);
    if (c->cfg.precision == HYDRO_MIXED) {
        float *store = reinterpret_cast<float *>(c->d_rec_store.get());
        if (save) k_rec_save<float><<<g, 128, 0, st>>>(n, c->d_perm.get(), c->d_ract.get(),
                                                       c->d_recf.get(), store);
        else k_rec_load<float><<<g, 128, 0, st>>>(n, c->d_perm.get(), c->d_ract.get(), store,
                                                  c->d_recf.get());
    } else {
        double *store = c->d_rec_store.get();
        if (save) k_rec_save<double><<<g, 128, 0, st>>>(n, c->d_perm.get(), c->d_ract.get(),
                                                        c->d_recd.get(), store);
        else k_rec_load<double><<<g, 128, 0, st>>>(n, c->d_perm.get(), c->d_ract.get(), store,
                                                   c->d_recd.get());
    }
    return launch_check();
}

cudaError_t rung_assign(hydro_ctx *c, double dt0, stream_t st) {
    const int64_t n = c->plan.n;
    const unsigned g = grid_for(n, 256);
    if (c->cfg.precision == HYDRO_MIXED)
        k_rung_assign<float><<<g, 256, 0, st>>>(n, c->d_vsig_dt.get(), c->d_recf.get(),
                                                c->d_hsorted.get(), c->cfg.c_acc, dt0,
                                                c->cfg.max_rung, c->d_rung_s.get(), c->d_cnt);
    else
        k_rung_assign<double><<<g, 256, 0, st>>>(n, c->d_vsig_dt.get(), c->d_recd.get(),
                                                 c->d_hsorted.get(), c->cfg.c_acc, dt0,
                                                 c->cfg.max_rung, c->d_rung_s.get(), c->d_cnt);
    return launch_check();
}

cudaError_t rung_limit_sweep(hydro_ctx *c, stream_t st) {
    const int64_t n = c->plan.n;
    const unsigned g = grid_for(n, 128);
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->rung_changed, 0, sizeof(int), st));
    if (c->cfg.precision == HYDRO_MIXED)
        k_rung_limit<float><<<g, 128, 0, st>>>(
            n, c->d_nbr_off.get(), c->d_nbr_cnt.get(), c->d_nbr_idx.get(), c->d_xs.get(),
            c->d_ys.get(), c->d_zs.get(), c->d_hsorted.get(), c->d_pbox.get(), c->d_boxes.get(),
            c->d_recf.get(), c->d_rung_s.get(), c->d_cnt);
    else
        k_rung_limit<double><<<g, 128, 0, st>>>(
            n, c->d_nbr_off.get(), c->d_nbr_cnt.get(), c->d_nbr_idx.get(), c->d_xs.get(),
            c->d_ys.get(), c->d_zs.get(), c->d_hsorted.get(), c->d_pbox.get(), c->d_boxes.get(),
            c->d_recd.get(), c->d_rung_s.get(), c->d_cnt);
    return launch_check();
}

cudaError_t rung_scatter(hydro_ctx *c, stream_t st) {
    const int64_t n = c->plan.n;
    k_rung_scatter<<<grid_for(n, 256), 256, 0, st>>>(n, c->d_perm.get(), c->d_rung_s.get(),
                                                      c->d_rung_c.get(), c->d_cnt);
    return launch_check();
}

}  // namespace hyd
