// End of the step (§2.3.4 Eq. 16, §2.3.7 Eq. 24): conserved update, the
// separately integrated internal energy, the drift, and fixed-order totals
// of mass, momentum and energy for the conservation diagnostics (taken
// before the update and after it, so external sources count).
#include <algorithm>

#include "hydro_internal.cuh"

namespace hyd {

namespace {

constexpr int SUM_THREADS = 256;
constexpr int SUM_BLOCKS = 608;   // 4 per SM on 152 SMs

struct UpdArgs {
    int64_t n;
    const int32_t *perm;
    const int32_t *pbox;
    const Box *boxes;
    double *Q;             // 6 n sorted (updated in place)
    const double *dQ;      // 5 n sorted
    const double *xs, *ys, *zs, *h, *om;
    double dt;
    const double *dt_dev;
    hydro_particles p;
    DevCounters *cnt;
    bool abort_check;
    int skip_flags;        // status bits that leave the caller's state untouched
    bool sorted_out;       // write the state back in the sorted order
    const double *agrav;   // sorted SoA 3 n (NULL: no gravity)
    const double *dM;      // sum_j dm_ij r_ij, sorted SoA 3 n
    // entropy switch (§2.3.7): the value of A the step used (sorted; NULL:
    // off), MFV's sum_j c_m,ij A_upwind (NULL for MFM) and the caller's array
    const double *A1;
    const double *dS;
    double *A_out;
};

__global__ void k_update(UpdArgs a) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= a.n) return;
    if (a.abort_check) {
        // the graph step found a condition it cannot resolve on the device:
        // leave the caller's state as it was (the host redoes the step)
        const DevCounters &k = *a.cnt;
        if (k.abort || k.hard_ovf || (k.flags & (ST_LIST_CAPACITY | ST_STACK))) return;
    }
    // an error the step reports (h not converged, the network's wait gave
    // up): the caller's state stays as it was
    if (a.skip_flags && (a.cnt->flags & a.skip_flags)) return;
    const int64_t n = a.n;
    const double dt = a.dt_dev ? *a.dt_dev : a.dt;
    double m0 = a.Q[s], px0 = a.Q[n + s], py0 = a.Q[2 * n + s], pz0 = a.Q[3 * n + s];
    double E0 = a.Q[4 * n + s], U0 = a.Q[5 * n + s];
    double dm = a.dQ[s], dpx = a.dQ[n + s], dpy = a.dQ[2 * n + s], dpz = a.dQ[3 * n + s];
    double dE = a.dQ[4 * n + s];
    double vx0 = px0 / m0, vy0 = py0 / m0, vz0 = pz0 / m0;
    double dU = dE - (vx0 * dpx + vy0 * dpy + vz0 * dpz) + 0.5 * (vx0 * vx0 + vy0 * vy0 + vz0 * vz0) * dm;
    double m1 = m0 + dm, px1 = px0 + dpx, py1 = py0 + dpy, pz1 = pz0 + dpz;
    double E1 = E0 + dE, U1 = U0 + dU;
    if (a.agrav) {
        // gravity (§2.3.8), trapezoidal between the start-of-step state and
        // the state the fluxes updated (§2.3.4): momentum dt/2 (m^n + m~) a,
        // energy dt/2 (P^n + P~).a + (1/2) a . sum_j dm_ij r_ij; the internal
        // energy takes no source
        const double ax = a.agrav[s], ay = a.agrav[n + s], az = a.agrav[2 * n + s];
        const double w = 0.5 * dt * (m0 + m1);
        const double eg = (px0 + px1) * ax + (py0 + py1) * ay + (pz0 + pz1) * az;
        const double ex = ax * a.dM[s] + ay * a.dM[n + s] + az * a.dM[2 * n + s];
        E1 += 0.5 * dt * eg + 0.5 * ex;
        px1 += w * ax;
        py1 += w * ay;
        pz1 += w * az;
    }
    double vx1 = px1 / m1, vy1 = py1 / m1, vz1 = pz1 / m1;
    const Box bx = a.boxes[a.pbox[s]];
    double x = a.xs[s] + dt * 0.5 * (vx0 + vx1);
    double y = a.ys[s] + dt * 0.5 * (vy0 + vy1);
    double z = a.zs[s] + dt * 0.5 * (vz0 + vz1);
    if (x >= bx.L[0]) x -= bx.L[0];
    if (x < 0.0) x += bx.L[0];
    if (y >= bx.L[1]) y -= bx.L[1];
    if (y < 0.0) y += bx.L[1];
    if (z >= bx.L[2]) z -= bx.L[2];
    if (z < 0.0) z += bx.L[2];
    if (!(isfinite(m1) && isfinite(px1) && isfinite(py1) && isfinite(pz1) && isfinite(E1) &&
          isfinite(U1) && isfinite(x) && isfinite(y) && isfinite(z)))
        atomicOr(&a.cnt->flags, ST_NONFINITE);
    a.Q[s] = m1; a.Q[n + s] = px1; a.Q[2 * n + s] = py1; a.Q[3 * n + s] = pz1;
    a.Q[4 * n + s] = E1; a.Q[5 * n + s] = U1;
    const int64_t o = a.sorted_out ? s : a.perm[s];
    a.p.x[o] = x; a.p.y[o] = y; a.p.z[o] = z;
    a.p.mass[o] = m1; a.p.px[o] = px1; a.p.py[o] = py1; a.p.pz[o] = pz1;
    a.p.etot[o] = E1; a.p.eint[o] = U1;
    a.p.h[o] = a.h[s];
    a.p.omega[o] = a.om[s];
    // the entropic function: constant along an MFM particle; MFV carries
    // m A with the mass fluxes
    if (a.A1) a.A_out[o] = a.dS ? (m0 * a.A1[s] + a.dS[s]) / m1 : a.A1[s];
}

// every value of the caller's state finite (positions, conserved
// quantities, smoothing lengths); a bad one sets *bad (a flag in mapped
// host memory, cleared by the host before the launch: a plain store, the
// same value from every block that finds one)
__global__ void k_check_inputs(int64_t n, hydro_particles p, int *bad) {
    const double *arr[10] = {p.x, p.y, p.z, p.mass, p.px, p.py, p.pz, p.etot, p.eint, p.h};
    bool ok = true;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < 10; q++) ok = ok && isfinite(arr[q][i]);
    }
    if (__syncthreads_or(!ok) && threadIdx.x == 0) *(volatile int *)bad = 1;
}

// totals in plain double with a fixed order (no atomics): each thread sums
// its strided share (n / 155,648 values), a block folds its 256 partials as
// a binary tree, the final kernel folds the 608 block partials the same
// way.  The rounding error is at most about (n / 155,648 + 18) ulp of
// sum |x| (1e-13 relative at 2^27 particles), far inside the 1e-12
// conservation budget, and the result does not depend on scheduling.  One
// double add per value: the FP64 pipe is narrow on this GPU, so a
// compensated sum (six FP64 operations per value) would cost several times
// more.
__device__ __forceinline__ void tree_fold(double (*sh)[5], int t, int width) {
    for (int w = width / 2; w > 0; w >>= 1) {
        __syncthreads();
        if (t < w)
#pragma unroll
            for (int q = 0; q < 5; q++) sh[t][q] += sh[t + w][q];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(SUM_THREADS) k_sums(int64_t n, const double *__restrict__ Q,
                                                      double *__restrict__ partials) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; q++) acc[q] += Q[q * n + s];
    __shared__ double sh[SUM_THREADS][5];
#pragma unroll
    for (int q = 0; q < 5; q++) sh[threadIdx.x][q] = acc[q];
    tree_fold(sh, threadIdx.x, SUM_THREADS);
    if (threadIdx.x < 5) partials[blockIdx.x * 5 + threadIdx.x] = sh[0][threadIdx.x];
}

// the block partials (nb <= 1024) folded as a binary tree
__global__ void __launch_bounds__(1024) k_sums_final(const double *__restrict__ partials, int nb,
                                                     double *__restrict__ out) {
    __shared__ double sh[1024][5];
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 5; q++) sh[t][q] = t < nb ? partials[t * 5 + q] : 0.0;
    tree_fold(sh, t, 1024);
    if (t < 5) out[t] = sh[0][t];
}

__global__ void k_export_dQ(int64_t n, const int32_t *__restrict__ perm,
                            const double *__restrict__ Q, const double *__restrict__ dQ,
                            double *__restrict__ out) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    double m0 = Q[s];
    double vx = Q[n + s] / m0, vy = Q[2 * n + s] / m0, vz = Q[3 * n + s] / m0;
    double dm = dQ[s], dpx = dQ[n + s], dpy = dQ[2 * n + s], dpz = dQ[3 * n + s];
    double dE = dQ[4 * n + s];
    double dU = dE - (vx * dpx + vy * dpy + vz * dpz) + 0.5 * (vx * vx + vy * vy + vz * vz) * dm;
    int64_t o = perm[s];
    out[6 * o + 0] = dm;
    out[6 * o + 1] = dpx;
    out[6 * o + 2] = dpy;
    out[6 * o + 3] = dpz;
    out[6 * o + 4] = dE;
    out[6 * o + 5] = dU;
}

__global__ void k_set_u64(unsigned long long *p, unsigned long long v) { *p = v; }

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t set_u64(unsigned long long *p, unsigned long long v, stream_t st) {
    k_set_u64<<<1, 1, 0, st>>>(p, v);
    return launch_check();
}

cudaError_t run_update(hydro_ctx *c, hydro_particles *p, double dt, const double *dt_dev,
                       bool abort_check, int skip_flags, stream_t st) {
    UpdArgs a;
    a.n = c->plan.n;
    a.perm = c->d_perm.get();
    a.pbox = c->d_pbox.get();
    a.boxes = c->d_boxes.get();
    a.Q = c->d_Q.get();
    a.dQ = c->d_dQ.get();
    a.xs = c->d_xs.get(); a.ys = c->d_ys.get(); a.zs = c->d_zs.get();
    a.h = c->d_hsorted.get();
    a.om = c->d_omsorted.get();
    a.dt = dt;
    a.dt_dev = dt_dev;
    a.p = *p;
    a.cnt = c->d_cnt;
    a.abort_check = abort_check;
    a.skip_flags = skip_flags;
    a.sorted_out = c->cfg.sorted_output != 0 && !c->rung_live;
    a.agrav = c->grav_live ? c->d_agrav.get() : nullptr;
    a.dM = c->grav_live ? c->d_dM.get() : nullptr;
    a.A1 = c->ent_live ? c->d_A1.get() : nullptr;
    a.dS = c->ent_live && c->cfg.scheme == HYDRO_MFV ? c->d_dS.get() : nullptr;
    a.A_out = c->entA;
    k_update<<<grid_for(a.n, 256), 256, 0, st>>>(a);
    return launch_check();
}

// totals of m, px, py, pz, E over the sorted conserved state, into
// sums[which] of the counters (k_sums: fixed order, independent of
// scheduling).  The partials buffer is allocated with the context
// (ensure_sum_partials), never here, so the step can be captured.
cudaError_t ensure_sum_partials(hydro_ctx *c) {
    return c->d_partials.ensure((size_t)SUM_BLOCKS * 5);
}

cudaError_t run_sums(hydro_ctx *c, int which, stream_t st) {
    const int64_t n = c->plan.n;
    k_sums<<<SUM_BLOCKS, SUM_THREADS, 0, st>>>(n, c->d_Q.get(), c->d_partials.get());
    HYD_CUDA(launch_check());
    static_assert(SUM_BLOCKS <= 1024, "the final fold takes one thread per block partial");
    k_sums_final<<<1, 1024, 0, st>>>(c->d_partials.get(), SUM_BLOCKS, c->d_cnt->sums[which]);
    return launch_check();
}

cudaError_t run_check_inputs(hydro_ctx *c, const hydro_particles *p, stream_t st) {
    const unsigned grid = (unsigned)std::min<int64_t>(std::max<int64_t>((p->n + 255) / 256, 1), SUM_BLOCKS);
    k_check_inputs<<<grid, 256, 0, st>>>(p->n, *p, c->d_bad);
    return launch_check();
}

cudaError_t export_dQ(hydro_ctx *c, double *dQ, stream_t st) {
    const int64_t n = c->plan.n;
    k_export_dQ<<<grid_for(n, 256), 256, 0, st>>>(n, c->d_perm.get(), c->d_Q.get(), c->d_dQ.get(),
                                                   dQ);
    return launch_check();
}

}  // namespace hyd
