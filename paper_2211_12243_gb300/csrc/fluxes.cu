// Host side of the pair-flux stage (§2.3.3-2.3.4): the launchers of the
// flux kernels (flux_kernel.cuh), the adaptive learned-path choice, and
// run_fluxes, which clears the accumulators and runs the plain or the
// learned (deferred hard faces) path.
#include <algorithm>

#include "flux_kernel.cuh"

namespace hyd {

// the float flux kernel with 5 or 6 resident CTAs per SM (fluxes_occ.cu)
cudaError_t launch_fluxes_occ(int minb, const FluxArgs &a, const float *rec, int riem, int scheme,
                              bool defer, stream_t st);

namespace {

template <typename R>
cudaError_t launch_fluxes(const FluxArgs &a, const R *rec, int riem, int scheme, int minb,
                          stream_t st, cudaEvent_t *ev) {
    constexpr int MB = sizeof(R) == 4 ? 4 : 2;
    constexpr int E = HYDRO_RIEMANN_EXACT, H = HYDRO_RIEMANN_HLLC;
    if (a.queue) HYD_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), st));
    if (ev) HYD_CUDA(record_event(ev[0], st));
    bool done = false;
    if constexpr (sizeof(R) == 4) {
        if (minb == 5 || minb == 6) {
            HYD_CUDA(launch_fluxes_occ(minb, a, rec, riem, scheme, false, st));
            done = true;
        }
    }
    if (!done) {
        if (riem == H) {
            if (scheme == HYDRO_MFM) HYD_CUDA((launch_k_fluxes<R, H, HYDRO_MFM, false, MB>(a, rec, st)));
            else HYD_CUDA((launch_k_fluxes<R, H, HYDRO_MFV, false, MB>(a, rec, st)));
        } else {
            if (scheme == HYDRO_MFM) HYD_CUDA((launch_k_fluxes<R, E, HYDRO_MFM, false, MB>(a, rec, st)));
            else HYD_CUDA((launch_k_fluxes<R, E, HYDRO_MFV, false, MB>(a, rec, st)));
        }
    }
    if (ev) HYD_CUDA(record_event(ev[1], st));
    return cudaSuccess;
}

// mixed precision, exact solver, learned guess: the flux kernel defers the
// hard faces (pass 1) ...
cudaError_t launch_fluxes_defer(const FluxArgs &a, const float *rec, int scheme, int minb,
                                stream_t st) {
    if (minb == 5 || minb == 6)
        return launch_fluxes_occ(minb, a, rec, HYDRO_RIEMANN_EXACT, scheme, true, st);
    if (scheme == HYDRO_MFM) return launch_k_fluxes<float, HYDRO_RIEMANN_EXACT, HYDRO_MFM, true, 4>(a, rec, st);
    return launch_k_fluxes<float, HYDRO_RIEMANN_EXACT, HYDRO_MFV, true, 4>(a, rec, st);
}

// ... then the hard-face kernel solves them from the network (pass 2)
cudaError_t launch_hard_faces(const FluxArgs &a, int scheme, stream_t st) {
    const size_t smem = sizeof(MlpTile) + 1024;
    static bool configured = false;
    if (!configured) {
        HYD_CUDA(cudaFuncSetAttribute(k_hard_faces<HYDRO_MFM>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HYD_CUDA(cudaFuncSetAttribute(k_hard_faces<HYDRO_MFV>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    // persistent: the count of hard faces is known on the device only
    const unsigned hgrid = 152 * 4;
    if (scheme == HYDRO_MFM) k_hard_faces<HYDRO_MFM><<<hgrid, 128, smem, st>>>(a);
    else k_hard_faces<HYDRO_MFV><<<hgrid, 128, smem, st>>>(a);
    return launch_check();
}

}  // namespace

void read_learn_probe(hydro_ctx *c) {
    if (!c->learn_probe) return;
    const bool lp = c->learn_probe == 1;
    float ms = 0.f;
    if (cudaEventSynchronize(c->ev[lp ? 8 : 7]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, c->ev[6], c->ev[lp ? 8 : 7]) == cudaSuccess && ms > 0.f) {
        c->learn_t[lp ? 1 : 0] = ms;
    } else {
        (void)cudaGetLastError();
        c->learn_t[lp ? 1 : 0] = lp ? 1e30f : 0.f;   // unknown: prefer the plain path
    }
    if (lp) {
        c->learn_used = false;
        if (cudaEventSynchronize(c->ev[9]) == cudaSuccess)
            c->learn_used = c->h_learn[0] * 10 > c->h_learn[1];
    }
    c->learn_probe = 0;
}

bool decide_learned(hydro_ctx *c) {
    const bool want = c->cfg.precision == HYDRO_MIXED && c->cfg.riemann == HYDRO_RIEMANN_EXACT &&
                      c->cfg.learned_guess && c->have_mlp;
    if (!want) return false;
    if (c->cfg.learned_guess == 2) return true;
    // adaptive: the previous call was a probe -> collect its time (and, for
    // the learned probe, how many hard faces started from the network)
    read_learn_probe(c);
    if (c->learn_phase == 0) {
        c->learn_phase = 1;
        c->learn_probe = 1;
        return true;
    }
    if (c->learn_phase == 1) {
        c->learn_phase = 2;
        c->learn_probe = 2;
        c->learn_skip = 0;
        return false;
    }
    if (c->learn_skip == 0) {
        // the network must start more than 10% of the hard faces and the
        // learned path must be the faster of the two probes
        c->learn_winner = c->learn_used && c->learn_t[1] < c->learn_t[0];
        c->learn_skip = 15;
    }
    if (--c->learn_skip == 0) c->learn_phase = 0;
    return c->learn_winner;
}

cudaError_t run_fluxes(hydro_ctx *c, double dt, const double *dt_dev, stream_t st) {
    const int64_t n = c->plan.n;
    HYD_CUDA(c->d_dQ.ensure((size_t)5 * n));
    if (c->grav_live) HYD_CUDA(c->d_dM.ensure((size_t)3 * n));
    // the entropy flux only matters where mass moves (MFV)
    const bool ent_flux = c->ent_live && c->cfg.scheme == HYDRO_MFV;
    auto clear = [&]() -> cudaError_t {
        HYD_CUDA(cudaMemsetAsync(c->d_dQ.get(), 0, sizeof(double) * 5 * n, st));
        if (c->grav_live) HYD_CUDA(cudaMemsetAsync(c->d_dM.get(), 0, sizeof(double) * 3 * n, st));
        if (ent_flux) HYD_CUDA(cudaMemsetAsync(c->d_dS.get(), 0, sizeof(double) * n, st));
        // flux_pairs, newton_iters, guess_fallbacks, vacuum, first_order,
        // learned_faces, hard_faces, hard_ovf
        return cudaMemsetAsync(&c->d_cnt->flux_pairs, 0, 8 * sizeof(unsigned long long), st);
    };
    HYD_CUDA(clear());
    FluxArgs a;
    a.n = n;
    a.nbr_off = c->d_nbr_off.get();
    a.nbr_cnt = c->d_nbr_cnt.get();
    a.nbr_idx = c->d_nbr_idx.get();
    a.xs = c->d_xs.get(); a.ys = c->d_ys.get(); a.zs = c->d_zs.get();
    a.h = c->d_hsorted.get();
    a.pbox = c->d_pbox.get();
    a.boxes = c->d_boxes.get();
    a.kernel = c->cfg.kernel;
    a.scheme = c->cfg.scheme;
    a.riemann = c->cfg.riemann;
    a.limiter = c->cfg.limiter;
    a.time_extrap = c->cfg.time_extrap;
    a.gamma = c->cfg.gamma;
    a.psi1 = c->cfg.psi1;
    a.psi2 = c->cfg.psi2;
    a.p_tol = c->cfg.p_tol;
    a.max_newton = c->cfg.max_newton;
    a.dt = dt;
    a.dt_dev = dt_dev;
    a.dQ = c->d_dQ.get();
    a.cnt = c->d_cnt;
    a.mlp_blob = c->d_mlp_blob.get();
    a.mlp_stall = c->mlp_stall;
    a.riemann_polish = c->cfg.riemann_polish;
    a.hard = nullptr;
    a.hard_idx = nullptr;
    a.hard_cursor = nullptr;
    a.hard_cap = 0;
    const bool learned = c->learned_decision >= 0 ? c->learned_decision != 0 : decide_learned(c);
    c->learned_active = learned;
    // room for 2 hard faces per particle, at least 4096 per sub-buffer (twice
    // the margin the kernel keeps) and at most 2^26 faces in all (sub-buffer
    // sizes a multiple of 128): a sub-buffer near full makes the flux kernel
    // solve further hard faces itself from the plain guess, so the buffer
    // does not grow with the problem; a pass that still fills one (a backstop)
    // is redone with twice the room
    const int64_t unit = (int64_t)HARD_SUB * 128;
    auto reserve_hard = [&](int64_t want) -> cudaError_t {
        const int64_t cap = (want + unit - 1) / unit * unit;
        if (c->hard_cap < cap) {
            c->hard_cap = 0;
            HYD_CUDA(c->d_hard.ensure((size_t)HF_N * cap));
            HYD_CUDA(c->d_hard_idx.ensure((size_t)2 * cap));
            c->hard_cap = cap;
        }
        HYD_CUDA(c->d_hard_cursor.ensure(HARD_SUB));
        a.hard = c->d_hard.get();
        a.hard_idx = c->d_hard_idx.get();
        a.hard_cursor = c->d_hard_cursor.get();
        a.hard_cap = c->hard_cap;
        return cudaSuccess;
    };
    if (learned)
        HYD_CUDA(reserve_hard(std::min<int64_t>(std::max<int64_t>(2 * n + 65536, (int64_t)HARD_SUB * 4096),
                                                (int64_t)1 << 26)));
    a.rec_faces = c->rec_faces;
    a.rec_cursor = c->d_rec_cursor.get();
    a.rec_cap = c->rec_cap;
    a.rec_keep = c->rec_keep;
    a.rec_hard_only = c->rec_hard_only;
    a.psi1f = (float)c->cfg.psi1;
    a.psi2f = (float)c->cfg.psi2;
    a.ptolf = (float)std::max(c->cfg.p_tol, 2e-6);
    {
        // below h = Lmin / 4096 every membership is decided in double
        double lmin = 1e300;
        for (size_t k = 0; k < c->plan.box_len.size(); k++) lmin = std::min(lmin, c->plan.box_len[k]);
        a.lmin_tiny = (float)(lmin / 4096.0);
    }
    a.Kf = GasK<float>(c->cfg.gamma);
    a.Kd = GasK<double>(c->cfg.gamma);
    a.nbucket = c->plan.nbucket;
    a.node_first = c->d_node_first.get();
    a.node_cnt = c->d_node_cnt.get();
    a.recf = c->d_recf.get();
    a.dM = c->grav_live ? c->d_dM.get() : nullptr;
    a.dS = ent_flux ? c->d_dS.get() : nullptr;
    a.rung = c->rung_live ? c->d_rung_s.get() : nullptr;
    a.toff = c->rung_live ? c->d_toff.get() : nullptr;
    a.ract = c->rung_live ? c->d_ract.get() : nullptr;
    a.dt0 = c->rung_dt0;
    a.bucket_ids = nullptr;
    a.queue = c->flux_queue ? &c->d_cnt->flux_cursor : nullptr;
    if (c->rung_live && c->rung_touch_n >= 0) {
        a.bucket_ids = c->d_touch.get();
        a.nbucket = c->rung_touch_n;
    }
    // the adaptive learned path times its probes with the same events
    const bool adapt = c->cfg.learned_guess == 1 && c->cfg.precision == HYDRO_MIXED &&
                       c->cfg.riemann == HYDRO_RIEMANN_EXACT && c->have_mlp;
    cudaEvent_t *ev = (c->timing || adapt) ? c->ev + 6 : nullptr;
    if (learned) {
        for (int attempt = 0;; attempt++) {
            HYD_CUDA(cudaMemsetAsync(a.hard_cursor, 0, HARD_SUB * sizeof(unsigned long long), st));
            if (a.queue) HYD_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), st));
            if (ev) HYD_CUDA(record_event(ev[0], st));
            HYD_CUDA(launch_fluxes_defer(a, c->d_recf.get(), c->cfg.scheme, c->flux_minb, st));
            if (ev) HYD_CUDA(record_event(ev[1], st));
            // a graph step cannot wait here: a full sub-buffer (hard_ovf)
            // stops its update and the host redoes the step
            if (c->capturing) break;
            unsigned long long ovf = 0;
            HYD_CUDA(cudaMemcpyAsync(&ovf, &c->d_cnt->hard_ovf, sizeof(ovf), cudaMemcpyDeviceToHost, st));
            HYD_CUDA(cudaStreamSynchronize(st));
            if (!ovf) break;
            if (attempt >= 6) return cudaErrorMemoryAllocation;
            HYD_CUDA(reserve_hard(2 * a.hard_cap));
            HYD_CUDA(clear());
        }
        HYD_CUDA(launch_hard_faces(a, c->cfg.scheme, st));
        if (ev) HYD_CUDA(record_event(ev[2], st));
        // learned_faces and hard_faces (adjacent) for the adaptive decision
        HYD_CUDA(cudaMemcpyAsync(c->h_learn, &c->d_cnt->learned_faces, 2 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, st));
        HYD_CUDA(record_event(c->ev[9], st));
        return cudaSuccess;
    }
    if (c->cfg.precision == HYDRO_MIXED)
        return launch_fluxes<float>(a, c->d_recf.get(), c->cfg.riemann, c->cfg.scheme,
                                    c->flux_minb, st, ev);
    return launch_fluxes<double>(a, c->d_recd.get(), c->cfg.riemann, c->cfg.scheme, 0, st, ev);
}

}  // namespace hyd
