// hydro_step as one captured CUDA graph.
//
// The host-driven step (api.cu) waits on the device at every decision: the
// count of overflowing neighbour lists, the particles whose h root left the
// list radius (§2.3.5: rebuild and solve again), and the particles above the
// N_cond threshold (§2.3.5: grow N_NGB, solve their density again, recompute
// the gradients).  Here those decisions run on the device: the overflow pass
// reads its bucket count itself, and the two loops are graph WHILE nodes
// whose condition a one-thread kernel sets from the step's counters:
//
//   counters = 0; sort; gather; tree; lists; overflow lists
//   density (compacting)
//   WHILE (search failures and round < 8):                       [search loop]
//       grow radii; rebuild the failed particles' buckets; density of those
//   primitives; gradients
//   WHILE (N_cond failures and round < max_ngb_grow):             [guard loop]
//       grow N_NGB; density of the grown particles
//       WHILE (search failures and round < 8): ...                [search loop]
//       primitives; gradients of the particles the new densities change
//   fluxes (plain or learned path); update; totals
//
// Both loops are bounded by counters the condition kernel increments, so
// the graph always ends.  A step the device cannot finish (a re-search that
// exhausts its rounds, an overflow region or deferred-face buffer too small
// to grow on the device) sets `abort` or a flag that makes the update kernel
// leave the caller's state untouched; the host then reports the error or
// runs the host-driven step, which grows the buffers.
//
// One executable graph is kept per learned-path choice, with the launch
// parameters it was captured with (caller pointers, dt, sizes, every scratch
// pointer); a change recaptures.
#include <string.h>

#include "hydro_internal.cuh"

namespace hyd {

namespace {

constexpr int MAX_SEARCH_ROUNDS = 8;   // as the host-driven density solve


__global__ void k_cond_search(cudaGraphConditionalHandle h, DevCounters *c) {
    const bool fail = c->search_fail > 0;
    const bool go = fail && c->search_round < MAX_SEARCH_ROUNDS;
    if (go) {
        c->search_round++;
        c->rebuilds++;
    } else if (fail) {
        c->abort = 1;   // h beyond the radius after every round: HYDRO_ESEARCH
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_cond_guard(cudaGraphConditionalHandle h, DevCounters *c, int max_rounds) {
    const bool go = !c->abort && c->ncond_fail > 0 && c->guard_round < max_rounds;
    if (go) c->guard_round++;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_note_ovf(DevCounters *c) { c->ovf_first = c->ovf_buckets; }

// Append to the graph captured on `st`: the condition kernel `cond` (which
// sets the handle), then a WHILE node whose body `body(bs, h)` is captured
// on capture stream `level` (the body must end with the condition kernel).
template <class Cond, class Body>
cudaError_t capture_while(hydro_ctx *c, int level, cudaStream_t st, Cond &&cond, Body &&body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t ndeps = 0;
    HYD_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edata, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphConditionalHandle h;
    HYD_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0u, 0u));
    HYD_CUDA(cond(st, h));
    HYD_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edata, &ndeps));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};   // (aggregate: all else zero)
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    HYD_CUDA(cudaGraphAddNode(&node, g, deps, edata, ndeps, &np));
    HYD_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies));
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    cudaStream_t bs = c->cap_stream[level];
    HYD_CUDA(cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed));
    cudaError_t e = body(bs, h);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(bs, &out);
    return e != cudaSuccess ? e : e2;
}

cudaError_t cond_search(hydro_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h) {
    k_cond_search<<<1, 1, 0, s>>>(h, c->d_cnt);
    return launch_check();
}

// one re-search round: radii of the failed particles grow, their buckets get
// new lists, their density is solved again
cudaError_t search_body(hydro_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h, bool guard) {
    const long long k0 = launch_count();
    HYD_CUDA(grow_search_radius(c, s, guard));
    HYD_CUDA(rebuild_active_lists_dev(c, s, guard));
    HYD_CUDA(run_density(c, true, true, s, guard));
    HYD_CUDA(cond_search(c, s, h));
    c->cap_k_search = launch_count() - k0;
    return cudaSuccess;
}

cudaError_t search_loop(hydro_ctx *c, int level, cudaStream_t st) {
    HYD_CUDA(cudaMemsetAsync(&c->d_cnt->search_round, 0, sizeof(int), st));
    return capture_while(
        c, level, st, [&](cudaStream_t s, cudaGraphConditionalHandle h) { return cond_search(c, s, h); },
        [&](cudaStream_t s, cudaGraphConditionalHandle h) { return search_body(c, s, h, level == 2); });
}

cudaError_t cond_guard(hydro_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h) {
    k_cond_guard<<<1, 1, 0, s>>>(h, c->d_cnt, c->cfg.max_ngb_grow);
    return launch_check();
}

// one N_cond guard round (§2.3.5)
cudaError_t guard_body(hydro_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h) {
    const long long k0 = launch_count();
    HYD_CUDA(guard_grow(c, s));
    HYD_CUDA(guard_particle_lists(c, s));       // (the tree's radius bounds are not used)
    HYD_CUDA(run_density(c, true, true, s, true));
    HYD_CUDA(search_loop(c, 2, s));
    HYD_CUDA(run_primitives(c, s, true));
    HYD_CUDA(run_gradients(c, nullptr, nullptr, nullptr, nullptr, true, s, false));
    HYD_CUDA(cond_guard(c, s, h));
    c->cap_k_guard = launch_count() - k0 - c->cap_k_search;   // its re-search body runs per round
    return cudaSuccess;
}

cudaError_t enqueue_step(hydro_ctx *c, hydro_particles *p, double dt, bool sums, bool timing,
                         cudaStream_t st) {
    HYD_CUDA(cudaMemsetAsync(c->d_cnt, 0, sizeof(DevCounters), st));
    if (timing) HYD_CUDA(record_event(c->ev[0], st));
    HYD_CUDA(sort_particles(c, p, st));
    HYD_CUDA(gather_state(c, p, p->h, nullptr, c->cfg.search_margin, true, st));
    HYD_CUDA(gather_gravity(c, st));
    HYD_CUDA(gather_entropy(c, st));
    HYD_CUDA(build_tree(c, st));
    HYD_CUDA(build_lists(c, c->nbr_per_particle, st));
    k_note_ovf<<<1, 1, 0, st>>>(c->d_cnt);
    HYD_CUDA(launch_check());
    HYD_CUDA(build_lists_queued_dev(c, st));
    if (timing) HYD_CUDA(record_event(c->ev[1], st));
    HYD_CUDA(reset_guard(c, st));
    HYD_CUDA(run_density(c, false, true, st));
    HYD_CUDA(search_loop(c, 1, st));
    if (timing) HYD_CUDA(record_event(c->ev[2], st));
    HYD_CUDA(run_primitives(c, st));
    HYD_CUDA(run_gradients(c, nullptr, nullptr, nullptr, nullptr, false, st, false));
    // the tree with the solved h and search radii: the guard rounds only
    // raise its radius bounds for their particles
    HYD_CUDA(build_tree(c, st));
    HYD_CUDA(capture_while(
        c, 1, st, [&](cudaStream_t s, cudaGraphConditionalHandle h) { return cond_guard(c, s, h); },
        [&](cudaStream_t s, cudaGraphConditionalHandle h) { return guard_body(c, s, h); }));
    HYD_CUDA(grad_reduce(c, st));
    if (timing) HYD_CUDA(record_event(c->ev[3], st));
    const double *dt_dev =
        dt > 0.0 ? nullptr : reinterpret_cast<const double *>(&c->d_cnt->dt_min_bits);
    c->timing = timing;
    cudaError_t e = run_fluxes(c, dt, dt_dev, st);
    c->timing = false;
    HYD_CUDA(e);
    if (timing) HYD_CUDA(record_event(c->ev[4], st));
    if (sums) HYD_CUDA(run_sums(c, 0, st));
    HYD_CUDA(run_update(c, p, dt, dt_dev, true, STEP_SKIP_FLAGS, st));
    if (sums) HYD_CUDA(run_sums(c, 1, st));
    if (timing) HYD_CUDA(record_event(c->ev[5], st));
    return cudaSuccess;
}

// everything a captured graph depends on
std::vector<unsigned long long> graph_key(const hydro_ctx *c, const hydro_particles *p, double dt,
                                          bool sums, bool timing, bool learned) {
    std::vector<unsigned long long> k;
    auto put = [&](const void *ptr) { k.push_back((unsigned long long)(uintptr_t)ptr); };
    k.push_back((unsigned long long)p->n);
    for (const void *q : {(const void *)p->x, (const void *)p->y, (const void *)p->z,
                          (const void *)p->mass, (const void *)p->px, (const void *)p->py,
                          (const void *)p->pz, (const void *)p->etot, (const void *)p->eint,
                          (const void *)p->h, (const void *)p->omega})
        put(q);
    unsigned long long dtb;
    memcpy(&dtb, &dt, sizeof(dtb));
    k.push_back(dtb);
    k.push_back((sums ? 1 : 0) | (timing ? 2 : 0) | (learned ? 4 : 0) | (c->have_mlp ? 8 : 0));
    {
        unsigned char raw[sizeof(hydro_config)];
        memcpy(raw, &c->cfg, sizeof(raw));
        for (size_t o = 0; o < sizeof(raw); o += 8) {
            unsigned long long w = 0;
            memcpy(&w, raw + o, sizeof(raw) - o < 8 ? sizeof(raw) - o : 8);
            k.push_back(w);
        }
    }
    k.push_back((unsigned long long)c->nbr_per_particle);
    k.push_back((unsigned long long)c->flux_minb | ((unsigned long long)c->grad_minb << 8) |
                ((unsigned long long)c->flux_queue << 16) | ((unsigned long long)c->grad_rank << 24));
    k.push_back((unsigned long long)c->ovf_reserve);
    k.push_back((unsigned long long)c->hard_cap);
    k.push_back((unsigned long long)c->plan.n);
    k.push_back((unsigned long long)c->plan.nbucket);
    k.push_back((unsigned long long)c->plan.nlevels);
    put(c->rec_faces);
    put(c->grav);
    put(c->d_agrav.get());
    put(c->d_dM.get());
    put(c->entA);
    for (const void *q : {(const void *)c->d_A0.get(), (const void *)c->d_A1.get(),
                          (const void *)c->d_ecand.get(), (const void *)c->d_dS.get()})
        put(q);
    k.push_back((unsigned long long)c->rec_cap);
    k.push_back((unsigned long long)c->mlp_stall);
    k.push_back((unsigned long long)c->rec_keep | ((unsigned long long)c->rec_hard_only << 32));
    for (const void *q :
         {(const void *)c->d_node_first.get(), (const void *)c->d_node_cnt.get(),
          (const void *)c->d_node_box.get(), (const void *)c->d_box_root.get(),
          (const void *)c->d_box_off.get(), (const void *)c->d_boxes.get(),
          (const void *)c->d_node_aabb.get(), (const void *)c->d_node_aabb_hi.get(),
          (const void *)c->d_keys.get(), (const void *)c->d_keys_alt.get(),
          (const void *)c->d_perm.get(), (const void *)c->d_perm_alt.get(),
          (const void *)c->d_scan_tmp.get(), (const void *)c->d_hist.get(),
          (const void *)c->d_xs.get(), (const void *)c->d_ys.get(), (const void *)c->d_zs.get(),
          (const void *)c->d_hs.get(), (const void *)c->d_hsorted.get(),
          (const void *)c->d_omsorted.get(), (const void *)c->d_qx.get(),
          (const void *)c->d_qy.get(), (const void *)c->d_qz.get(), (const void *)c->d_q64.get(),
          (const void *)c->d_pbox.get(), (const void *)c->d_Q.get(), (const void *)c->d_dQ.get(),
          (const void *)c->d_recf.get(), (const void *)c->d_recd.get(),
          (const void *)c->d_out.get(), (const void *)c->d_nngb.get(),
          (const void *)c->d_active.get(), (const void *)c->d_vsig_dt.get(),
          (const void *)c->d_gpairs.get(), (const void *)c->d_nbr_idx.get(),
          (const void *)c->d_nbr_off.get(), (const void *)c->d_nbr_cnt.get(),
          (const void *)c->d_ovf.get(), (const void *)c->d_partials.get(),
          (const void *)c->d_mlp_blob.get(), (const void *)c->d_hard.get(),
          (const void *)c->d_hard_idx.get(), (const void *)c->d_hard_cursor.get(),
          (const void *)c->d_rec_cursor.get(), (const void *)c->d_guard_idx.get(),
          (const void *)c->d_redo_idx.get(), (const void *)c->d_guard_bits.get()})
        put(q);
    k.push_back((unsigned long long)c->d_nbr_idx.cap);
    return k;
}

}  // namespace

void graph_release(hydro_ctx *c) {
    for (auto &g : c->graph_slot) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        g.key.clear();
    }
    for (auto &s : c->cap_stream) {
        if (s) cudaStreamDestroy(s);
        s = nullptr;
    }
}

int graph_step(hydro_ctx *c, hydro_particles *p, double dt, hydro_stats *stats, stream_t st) {
    if (!c->cap_stream[0]) {
        for (auto &s : c->cap_stream)
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return 1;
    }
    const bool learned = decide_learned(c);
    const bool timing = stats != nullptr && c->have_events;
    const bool sums = stats != nullptr;
    hydro_ctx::GraphSlot &slot = c->graph_slot[learned ? 1 : 0];
    std::vector<unsigned long long> key = graph_key(c, p, dt, sums, timing, learned);
    if (!slot.exec || slot.key != key) {
        // size the list storage now: no allocation inside the capture
        const size_t need = (size_t)p->n * c->nbr_per_particle + (size_t)c->ovf_reserve;
        if (c->d_nbr_idx.cap < need && c->d_nbr_idx.ensure(need + need / 8) != cudaSuccess)
            return HYDRO_ENOMEM;
        key = graph_key(c, p, dt, sums, timing, learned);
        if (slot.exec) cudaGraphExecDestroy(slot.exec);
        slot.exec = nullptr;
        slot.key.clear();
        c->learned_decision = learned ? 1 : 0;
        c->capturing = true;
        cudaGraph_t g = nullptr;
        const long long k0 = launch_count();
        cudaError_t e = cudaStreamBeginCapture(c->cap_stream[0], cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            e = enqueue_step(c, p, dt, sums, timing, c->cap_stream[0]);
            cudaError_t e2 = cudaStreamEndCapture(c->cap_stream[0], &g);
            if (e == cudaSuccess) e = e2;
        }
        // nothing ran yet: count the kernels when the graph runs
        const long long captured = launch_count() - k0;
        add_launches(-captured);
        slot.k_search = c->cap_k_search;
        slot.k_guard = c->cap_k_guard;
        // captured: the top level, two re-search bodies (top level and inside
        // the guard body) and one guard body
        slot.k_top = captured - 2 * c->cap_k_search - c->cap_k_guard;
        c->capturing = false;
        c->learned_decision = -1;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&slot.exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            slot.exec = nullptr;
            c->graph_off = true;   // this context runs host-driven from now on
            return 1;
        }
        slot.key = graph_key(c, p, dt, sums, timing, learned);
    }
    cudaError_t e = cudaGraphLaunch(slot.exec, st);
    if (e != cudaSuccess) return HYDRO_ECUDA;
    c->learned_active = learned;
    e = cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return HYDRO_ECUDA;
    const DevCounters &H = *c->h_cnt;
    add_launches(slot.k_top + (long long)H.rebuilds * slot.k_search +
                 (long long)H.guard_round * slot.k_guard);
    if (H.flags & ST_LIST_CAPACITY) {
        // the re-search lists did not fit the overflow region: make it hold
        // what this step asked for (the host-driven step redoes it now)
        grow_overflow(c, H.list_cursor);
        return 1;
    }
    if (H.hard_ovf || (H.flags & ST_STACK)) return 1;   // grown by the host-driven step
    if (H.abort) return HYDRO_ESEARCH;
    // long lists in more than 1/256 of the buckets: more fixed slots next time
    if (H.ovf_first > c->plan.nbucket / 256 && c->nbr_per_particle < 256) c->nbr_per_particle += 32;
    c->have_lists = true;
    hydro_stats &S = c->last_stats;
    S.ngb_rounds = H.guard_round;
    S.list_rebuilds = H.rebuilds;
    S.ncond_fail = H.ncond_fail;
    S.graph = 1;
    int status = flags_to_status(H.flags);
    if (H.ncond_fail && status == HYDRO_OK) status = HYDRO_ENCOND;
    S.status = status;
    if (stats) {
        fill_stats(c, dt, timing);
        *stats = S;
    }
    return status;
}

}  // namespace hyd
