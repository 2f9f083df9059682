// C ABI of the hydro library (declared in include/hydro.h).
#include <math.h>
#include <cmath>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "hydro_internal.cuh"

using namespace hyd;

namespace hyd {
static std::atomic<long long> g_launches{0};
cudaError_t launch_check() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace hyd

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? HYDRO_OK : (e == cudaErrorMemoryAllocation ? HYDRO_ENOMEM : HYDRO_ECUDA); }

#define API_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e__ = (call);                        \
        if (e__ != cudaSuccess) return cuda_status(e__); \
    } while (0)

bool valid_config(const hydro_config *c) {
    if (!c) return false;
    if (!(c->gamma > 1.0)) return false;
    if (c->kernel != HYDRO_KERNEL_WENDLAND_C2 && c->kernel != HYDRO_KERNEL_CUBIC) return false;
    double kn = c->kernel == HYDRO_KERNEL_WENDLAND_C2 ? 14.0 : 32.0 / 3.0;
    if (!(c->n_ngb > kn)) return false;   // the self term alone must not reach N_NGB
    if (c->scheme != HYDRO_MFV && c->scheme != HYDRO_MFM) return false;
    if (c->riemann != HYDRO_RIEMANN_EXACT && c->riemann != HYDRO_RIEMANN_HLLC) return false;
    if (c->precision != HYDRO_FP64 && c->precision != HYDRO_MIXED) return false;
    if (c->learned_guess < 0 || c->learned_guess > 2) return false;
    if (!(c->search_margin >= 1.0)) return false;
    if (c->graph != 0 && c->graph != 1) return false;
    if (c->max_h_iter < 1 || c->max_newton < 1 || c->max_ngb_grow < 0) return false;
    if (c->entropy_switch != 0 && c->entropy_switch != 1) return false;
    if (!(c->alpha2 >= 0.0) || !(c->alpha3 >= 0.0) || !isfinite(c->alpha2) || !isfinite(c->alpha3))
        return false;
    if (!(c->c_acc > 0.0) || c->max_rung < 0 || c->max_rung > 20) return false;
    if (c->riemann_polish != 0 && c->riemann_polish != 1) return false;
    if (c->sorted_output != 0 && c->sorted_output != 1) return false;
    return true;
}

bool valid_particles(const hydro_ctx *c, const hydro_particles *p, bool need_state) {
    if (!p || p->n != c->plan.n || p->n <= 0) return false;
    if (!p->x || !p->y || !p->z || !p->h) return false;
    if (need_state && (!p->mass || !p->px || !p->py || !p->pz || !p->etot || !p->eint || !p->omega))
        return false;
    return true;
}

// rows of the plan: buckets per box, then groups of 32 children per level
void make_plan(Plan &P) {
    P.nbucket = 0;
    for (int64_t k = 0; k < P.nbox; k++) P.nbucket += (P.box_off[k + 1] - P.box_off[k] + 31) / 32;
    P.node_first.clear(); P.node_cnt.clear(); P.node_box.clear(); P.level_off.clear();
    std::vector<int64_t> lvl_first(P.nbox), lvl_count(P.nbox);
    P.level_off.push_back(0);
    for (int64_t k = 0; k < P.nbox; k++) {
        int64_t o = P.box_off[k], e = P.box_off[k + 1];
        lvl_first[k] = (int64_t)P.node_first.size();
        for (int64_t s = o; s < e; s += 32) {
            P.node_first.push_back((int32_t)s);
            P.node_cnt.push_back((int32_t)std::min<int64_t>(32, e - s));
            P.node_box.push_back((int32_t)k);
        }
        lvl_count[k] = (int64_t)P.node_first.size() - lvl_first[k];
    }
    P.level_off.push_back((int64_t)P.node_first.size());
    P.nlevels = 1;
    for (;;) {
        bool all_one = true;
        for (int64_t k = 0; k < P.nbox; k++) all_one &= (lvl_count[k] == 1);
        if (all_one) break;
        for (int64_t k = 0; k < P.nbox; k++) {
            int64_t f = lvl_first[k], c = lvl_count[k];
            lvl_first[k] = (int64_t)P.node_first.size();
            for (int64_t t = 0; t < c; t += 32) {
                P.node_first.push_back((int32_t)(f + t));
                P.node_cnt.push_back((int32_t)std::min<int64_t>(32, c - t));
                P.node_box.push_back((int32_t)k);
            }
            lvl_count[k] = (int64_t)P.node_first.size() - lvl_first[k];
        }
        P.level_off.push_back((int64_t)P.node_first.size());
        P.nlevels++;
    }
    P.nnode = (int64_t)P.node_first.size();
    P.box_root.assign(P.nbox, 0);
    for (int64_t k = 0; k < P.nbox; k++) P.box_root[k] = (int32_t)lvl_first[k];
}

template <typename T>
cudaError_t upload(DevBuf<T> &b, const std::vector<T> &v) {
    HYD_CUDA(b.ensure(v.size()));
    return cudaMemcpy(b.get(), v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

cudaError_t ensure_state(hydro_ctx *c, int64_t n) {
    HYD_CUDA(c->d_nngb.ensure(n));
    HYD_CUDA(c->d_active.ensure(n));
    return cudaSuccess;
}

// tree boxes and lists for the current search radii: one pass into the
// fixed slots, then the count-reserve-fill passes for buckets with a list
// longer than the slots (with a larger overflow region if it did not fit)
int lists_all(hydro_ctx *c, cudaStream_t st) {
    API_CUDA(build_tree(c, st));
    API_CUDA(cudaMemsetAsync(&c->d_cnt->flags, 0, sizeof(int), st));
    API_CUDA(build_lists(c, c->nbr_per_particle, st));
    API_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    API_CUDA(cudaStreamSynchronize(st));
    if (c->h_cnt->flags & ST_STACK) return HYDRO_ECAPACITY;
    int nq = c->h_cnt->ovf_buckets;
    const int64_t n = c->plan.n;
    for (int attempt = 0; nq > 0; attempt++) {
        API_CUDA(build_lists_queued(c, nq, st));
        API_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
        int f = c->h_cnt->flags;
        if (f & ST_STACK) return HYDRO_ECAPACITY;
        if (!(f & ST_LIST_CAPACITY)) break;
        if (attempt >= 2) return HYDRO_ECAPACITY;
        // the overflow region was too small: grow it and redo the queued buckets
        grow_overflow(c, c->h_cnt->list_cursor);
        size_t need = (size_t)n * c->list_cap + (size_t)c->ovf_reserve;
        API_CUDA(c->d_nbr_idx.ensure(need));
        API_CUDA(set_u64(&c->d_cnt->list_cursor, (unsigned long long)n * c->list_cap, st));
        API_CUDA(cudaMemsetAsync(&c->d_cnt->flags, 0, sizeof(int), st));
        // the fixed slots survive a reallocation only if nothing moved; rebuild them
        API_CUDA(build_lists(c, c->list_cap, st));
        API_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
        nq = c->h_cnt->ovf_buckets;
    }
    // long lists in more than 1/256 of the buckets: more fixed slots next time
    if (nq > c->plan.nbucket / 256 && c->nbr_per_particle < 256) c->nbr_per_particle += 32;
    c->have_lists = true;
    return HYDRO_OK;
}

// sort, gather, tree, lists
int build_all(hydro_ctx *c, const hydro_particles *p, const double *h_in, const double *h_search,
              double margin, bool want_Q, cudaStream_t st) {
    API_CUDA(sort_particles(c, p, st));
    API_CUDA(gather_state(c, p, h_in, h_search, margin, want_Q, st));
    return lists_all(c, st);
}

// density with re-searches when a root leaves the list radius: the failed
// particles' radii grow and only their buckets get new lists (a full
// rebuild when the overflow region is too small)
int density_all(hydro_ctx *c, const hydro_particles *p, bool only_active, int &rebuilds,
                cudaStream_t st, bool guard = false) {
    API_CUDA(run_density(c, only_active, true, st, guard));
    for (int round = 0;; round++) {
        int sf = 0;
        API_CUDA(cudaMemcpyAsync(&sf, &c->d_cnt->search_fail, sizeof(int), cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
        if (sf == 0) return HYDRO_OK;
        if (round >= 8) return HYDRO_ESEARCH;
        rebuilds++;
        API_CUDA(grow_search_radius(c, st, guard));
        int nq = 0;
        API_CUDA(rebuild_active_lists(c, &nq, st, guard));
        API_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
        const int fl = c->h_cnt->flags;
        if (fl & (ST_LIST_CAPACITY | ST_STACK)) {
            if (fl & ST_LIST_CAPACITY) grow_overflow(c, c->h_cnt->list_cursor);
            int rc = lists_all(c, st);
            if (rc) return rc;
        }
        API_CUDA(run_density(c, true, true, st, guard));
    }
}

}  // namespace

namespace hyd {

int flags_to_status(int f) {
    if (f & ST_NONFINITE) return HYDRO_ENONFINITE;
    if (f & ST_LIST_CAPACITY) return HYDRO_ECAPACITY;
    if (f & ST_LIST_OVERFLOW) return HYDRO_ECAPACITY;
    if (f & ST_STACK) return HYDRO_ECAPACITY;
    if (f & ST_SEARCH) return HYDRO_ESEARCH;
    if (f & ST_NOCONV_H) return HYDRO_ENOCONV_H;
    if (f & ST_RIEMANN) return HYDRO_ERIEMANN;
    if (f & ST_NCOND) return HYDRO_ENCOND;
    if (f & ST_MLP) return HYDRO_EMLP;
    return HYDRO_OK;
}

__global__ void k_fill(int64_t n, double *a, double v, uint8_t *act) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < n) { a[s] = v; act[s] = 1; }
}

cudaError_t reset_guard(hydro_ctx *c, cudaStream_t st) {
    int64_t n = c->plan.n;
    k_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, c->d_nngb.get(), c->cfg.n_ngb,
                                                         c->d_active.get());
    return launch_check();
}

void grow_overflow(hydro_ctx *c, unsigned long long cursor) {
    const unsigned long long base = (unsigned long long)c->plan.n * c->list_cap;
    const unsigned long long used = cursor > base ? cursor - base : 0ull;
    const int64_t want = (int64_t)(used + used / 4 + 4096);
    if (want > c->ovf_reserve) c->ovf_reserve = want;
}

// last_stats from the counters already copied to h_cnt (the stream is idle)
void fill_stats(hydro_ctx *c, double dt, bool timing) {
    hydro_stats &S = c->last_stats;
    const DevCounters &H = *c->h_cnt;
    double dtmin;
    memcpy(&dtmin, &H.dt_min_bits, sizeof(double));
    S.dt_next = dtmin;
    S.dt = dt > 0.0 ? dt : dtmin;
    S.grad_pairs = (int64_t)H.grad_pairs;
    S.flux_pairs = (int64_t)H.flux_pairs;
    S.newton_iters = (int64_t)H.newton_iters;
    S.guess_fallbacks = (int64_t)H.guess_fallbacks;
    S.learned_faces = (int64_t)H.learned_faces;
    S.hard_faces = (int64_t)H.hard_faces;
    S.learned_active = c->learned_active ? 1 : 0;
    S.learned_probe_ms[0] = c->learn_t[0];
    S.learned_probe_ms[1] = c->learn_t[1];
    S.vacuum_faces = (int64_t)H.vacuum;
    S.first_order_faces = (int64_t)H.first_order;
    for (int w = 0; w < 2; w++) {
        S.mass[w] = H.sums[w][0];
        for (int a = 0; a < 3; a++) S.mom[w][a] = H.sums[w][1 + a];
        S.energy[w] = H.sums[w][4];
    }
    if (timing) {
        auto el = [&](float &out, int e0, int e1) {
            if (cudaEventElapsedTime(&out, c->ev[e0], c->ev[e1]) != cudaSuccess) {
                out = 0.f;
                (void)cudaGetLastError();
            }
        };
        el(S.ms_neighbours, 0, 1);
        el(S.ms_density, 1, 2);
        el(S.ms_gradients, 2, 3);
        el(S.ms_fluxes, 3, 4);
        el(S.ms_update, 4, 5);
        el(S.ms_flux_kernel, 6, 7);
        S.ms_hard_faces = 0.f;
        if (c->learned_active) el(S.ms_hard_faces, 7, 8);
        S.ms_sort = 0.f;
    }
}

}  // namespace hyd

extern "C" {

void hydro_config_default(hydro_config *c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->gamma = 5.0 / 3.0;
    c->kernel = HYDRO_KERNEL_WENDLAND_C2;
    c->n_ngb = 32.0;
    c->scheme = HYDRO_MFV;
    c->riemann = HYDRO_RIEMANN_EXACT;
    c->precision = HYDRO_FP64;
    c->learned_guess = 0;
    c->limiter = 1;
    c->time_extrap = 1;
    c->ncond_crit = 100.0;
    c->ngb_grow = 1.2;
    c->max_ngb_grow = 5;
    c->psi1 = 0.5;
    c->psi2 = 0.25;
    c->beta_min = 1.0;
    c->beta_max = 2.0;
    c->c_cfl = 0.2;
    c->alpha1 = 0.01;
    c->h_tol = 1e-10;
    c->p_tol = 1e-12;
    c->max_h_iter = 60;
    c->max_newton = 100;
    c->search_margin = 1.15;
    c->graph = 1;
    c->entropy_switch = 0;
    c->alpha2 = 1e-3;
    c->alpha3 = 1e-3;
    c->c_acc = 0.2;
    c->max_rung = 12;
    c->riemann_polish = 0;
    c->sorted_output = 0;
}

int hydro_create(hydro_ctx **out, const hydro_config *cfg) {
    if (!out) return HYDRO_EINVAL;
    *out = nullptr;
    if (!valid_config(cfg)) return HYDRO_EINVAL;
    hydro_ctx *c = new (std::nothrow) hydro_ctx();
    if (!c) return HYDRO_ENOMEM;
    c->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_cnt, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_cnt, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_learn, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c->h_bad, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&c->d_bad, c->h_bad, 0);
    if (e == cudaSuccess) e = cudaMemset(c->d_cnt, 0, sizeof(DevCounters));
    if (e == cudaSuccess) e = ensure_sum_partials(c);
    if (e == cudaSuccess) {
        for (int k = 0; k < 10 && e == cudaSuccess; k++) e = cudaEventCreate(&c->ev[k]);
        c->have_events = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        hydro_destroy(c);
        return cuda_status(e);
    }
    memset(&c->last_stats, 0, sizeof(c->last_stats));
    *out = c;
    return HYDRO_OK;
}

void hydro_destroy(hydro_ctx *c) {
    if (!c) return;
    graph_release(c);
    if (c->d_cnt) cudaFree(c->d_cnt);
    if (c->h_cnt) cudaFreeHost(c->h_cnt);
    if (c->h_learn) cudaFreeHost(c->h_learn);
    if (c->h_bad) cudaFreeHost(c->h_bad);
    if (c->have_events)
        for (int k = 0; k < 10; k++) cudaEventDestroy(c->ev[k]);
    delete c;
}

int hydro_set_config(hydro_ctx *c, const hydro_config *cfg) {
    if (!c || !valid_config(cfg)) return HYDRO_EINVAL;
    bool prec_changed = cfg->precision != c->cfg.precision;
    c->cfg = *cfg;
    if (prec_changed) c->have_lists = false;
    return HYDRO_OK;
}

int hydro_set_boxes(hydro_ctx *c, int64_t nbox, const int64_t *box_off, const double *box_len) {
    if (!c || nbox < 1 || !box_off || !box_len) return HYDRO_EINVAL;
    if (box_off[0] != 0) return HYDRO_EINVAL;
    for (int64_t k = 0; k < nbox; k++) {
        if (box_off[k + 1] <= box_off[k]) return HYDRO_EINVAL;
        for (int a = 0; a < 3; a++)
            if (!(box_len[3 * k + a] > 0.0) || !isfinite(box_len[3 * k + a])) return HYDRO_EINVAL;
    }
    if (box_off[nbox] > INT32_MAX) return HYDRO_EINVAL;
    Plan &P = c->plan;
    P.nbox = nbox;
    P.n = box_off[nbox];
    P.box_off.assign(box_off, box_off + nbox + 1);
    P.box_len.assign(box_len, box_len + 3 * nbox);
    make_plan(P);
    std::vector<Box> boxes(nbox);
    for (int64_t k = 0; k < nbox; k++) {
        for (int a = 0; a < 3; a++) {
            boxes[k].L[a] = box_len[3 * k + a];
            boxes[k].s[a] = (float)(box_len[3 * k + a] / 4294967296.0);
        }
        boxes[k].pad = 0.f;
    }
    API_CUDA(upload(c->d_boxes, boxes));
    API_CUDA(upload(c->d_box_off, P.box_off));
    API_CUDA(upload(c->d_node_first, P.node_first));
    API_CUDA(upload(c->d_node_cnt, P.node_cnt));
    API_CUDA(upload(c->d_node_box, P.node_box));
    API_CUDA(upload(c->d_box_root, P.box_root));
    API_CUDA(c->d_node_aabb.ensure(P.nnode));
    API_CUDA(c->d_node_aabb_hi.ensure(P.nnode));
    c->have_plan = true;
    c->have_lists = false;
    return HYDRO_OK;
}

int hydro_reserve(hydro_ctx *c, int64_t max_n, int nbr_per_particle) {
    if (!c || max_n <= 0 || nbr_per_particle < 0) return HYDRO_EINVAL;
    if (nbr_per_particle > 0) c->nbr_per_particle = nbr_per_particle;
    int64_t n = max_n;
    API_CUDA(c->d_keys.ensure(n)); API_CUDA(c->d_keys_alt.ensure(n));
    API_CUDA(c->d_perm.ensure(n)); API_CUDA(c->d_perm_alt.ensure(n));
    API_CUDA(c->d_xs.ensure(n)); API_CUDA(c->d_ys.ensure(n)); API_CUDA(c->d_zs.ensure(n));
    API_CUDA(c->d_qx.ensure(n)); API_CUDA(c->d_qy.ensure(n)); API_CUDA(c->d_qz.ensure(n));
    API_CUDA(c->d_hs.ensure(n)); API_CUDA(c->d_hsorted.ensure(n)); API_CUDA(c->d_omsorted.ensure(n));
    API_CUDA(c->d_pbox.ensure(n));
    API_CUDA(c->d_Q.ensure((size_t)6 * n));
    API_CUDA(c->d_dQ.ensure((size_t)5 * n));
    if (c->cfg.precision == HYDRO_MIXED) {
        API_CUDA(c->d_recf.ensure((size_t)REC * n));
        API_CUDA(c->d_q64.ensure((size_t)3 * n));
    } else {
        API_CUDA(c->d_recd.ensure((size_t)REC * n));
    }
    API_CUDA(c->d_nngb.ensure(n));
    API_CUDA(c->d_active.ensure(n));
    API_CUDA(c->d_nbr_off.ensure(n + 1));
    API_CUDA(c->d_nbr_cnt.ensure(n));
    API_CUDA(c->d_nbr_idx.ensure((size_t)n * c->nbr_per_particle));
    return HYDRO_OK;
}

int hydro_build_neighbours(hydro_ctx *c, const hydro_particles *p, const double *h_search,
                           hydro_nbrlist *out, hydro_stream stream) {
    if (!c || !c->have_plan || !h_search) return HYDRO_EINVAL;
    if (!valid_particles(c, p, false)) return HYDRO_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(ensure_state(c, p->n));
    int rc = build_all(c, p, p->h, h_search, 1.0, false, st);
    if (rc != HYDRO_OK) return rc;
    if (out) {
        if (!out->off) return HYDRO_EINVAL;
        API_CUDA(export_lists(c, out, st));
        API_CUDA(cudaStreamSynchronize(st));
        if (out->needed > out->capacity) return HYDRO_ECAPACITY;
    }
    return HYDRO_OK;
}

int hydro_density(hydro_ctx *c, hydro_particles *p, hydro_stream stream) {
    if (!c || !c->have_lists) return c ? HYDRO_ESTATE : HYDRO_EINVAL;
    if (!valid_particles(c, p, false) || !p->omega) return HYDRO_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // the guess h from the caller, in sorted order
    API_CUDA(gather_from_caller(c->d_perm.get(), p->h, p->n, 1, c->d_hsorted.get(), p->n, st));
    API_CUDA(reset_guard(c, st));
    API_CUDA(cudaMemsetAsync(&c->d_cnt->flags, 0, sizeof(int), st));
    API_CUDA(run_density(c, false, false, st));
    int sf = 0, fl = 0;
    API_CUDA(cudaMemcpyAsync(&sf, &c->d_cnt->search_fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    API_CUDA(cudaMemcpyAsync(&fl, &c->d_cnt->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    API_CUDA(scatter_to_caller(c->d_perm.get(), c->d_hsorted.get(), p->n, 1, p->n, p->h, st));
    API_CUDA(scatter_to_caller(c->d_perm.get(), c->d_omsorted.get(), p->n, 1, p->n, p->omega, st));
    API_CUDA(cudaStreamSynchronize(st));
    if (sf) return HYDRO_ESEARCH;
    return flags_to_status(fl);
}

// gather the caller's state (h, omega, conserved) into the sorted buffers
static int stage_state(hydro_ctx *c, const hydro_particles *p, cudaStream_t st) {
    const int64_t n = p->n;
    API_CUDA(c->d_Q.ensure((size_t)6 * n));
    API_CUDA(gather_from_caller(c->d_perm.get(), p->mass, n, 1, c->d_Q.get(), n, st));
    API_CUDA(gather_from_caller(c->d_perm.get(), p->px, n, 1, c->d_Q.get() + n, n, st));
    API_CUDA(gather_from_caller(c->d_perm.get(), p->py, n, 1, c->d_Q.get() + 2 * n, n, st));
    API_CUDA(gather_from_caller(c->d_perm.get(), p->pz, n, 1, c->d_Q.get() + 3 * n, n, st));
    API_CUDA(gather_from_caller(c->d_perm.get(), p->etot, n, 1, c->d_Q.get() + 4 * n, n, st));
    API_CUDA(gather_from_caller(c->d_perm.get(), p->eint, n, 1, c->d_Q.get() + 5 * n, n, st));
    API_CUDA(gather_from_caller(c->d_perm.get(), p->h, n, 1, c->d_hsorted.get(), n, st));
    API_CUDA(gather_from_caller(c->d_perm.get(), p->omega, n, 1, c->d_omsorted.get(), n, st));
    return HYDRO_OK;
}

int hydro_gradients(hydro_ctx *c, const hydro_particles *p, double *B, double *grad,
                    double *alpha, double *ncond, hydro_stream stream) {
    if (c) c->grav_live = c->ent_live = false;   // (gravity and entropy: hydro_step only)
    if (!c || !c->have_lists) return c ? HYDRO_ESTATE : HYDRO_EINVAL;
    if (!valid_particles(c, p, true)) return HYDRO_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = p->n;
    int rc = stage_state(c, p, st);
    if (rc) return rc;
    API_CUDA(reset_guard(c, st));
    API_CUDA(run_primitives(c, st));
    API_CUDA(c->d_out.ensure((size_t)27 * n));
    double *stg = c->d_out.get();
    API_CUDA(cudaMemsetAsync(&c->d_cnt->flags, 0, sizeof(int), st));
    API_CUDA(run_gradients(c, stg, stg + 6 * n, stg + 21 * n, stg + 26 * n, false, st));
    API_CUDA(scatter_to_caller(c->d_perm.get(), stg, n, 6, n, B, st));
    API_CUDA(scatter_to_caller(c->d_perm.get(), stg + 6 * n, n, 15, n, grad, st));
    API_CUDA(scatter_to_caller(c->d_perm.get(), stg + 21 * n, n, 5, n, alpha, st));
    API_CUDA(scatter_to_caller(c->d_perm.get(), stg + 26 * n, n, 1, n, ncond, st));
    return HYDRO_OK;
}

int hydro_fluxes(hydro_ctx *c, const hydro_particles *p, const double *B, const double *grad,
                 const double *alpha, double dt, double *dQ, hydro_stream stream) {
    if (c) c->grav_live = c->ent_live = false;   // (gravity and entropy: hydro_step only)
    if (!c || !c->have_lists) return c ? HYDRO_ESTATE : HYDRO_EINVAL;
    if (c->cfg.learned_guess && !c->have_mlp) return HYDRO_ESTATE;
    if (!valid_particles(c, p, true) || !B || !grad || !alpha || !dQ || !(dt > 0.0))
        return HYDRO_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = stage_state(c, p, st);
    if (rc) return rc;
    API_CUDA(run_primitives(c, st));
    API_CUDA(load_gradients(c, B, grad, alpha, st));
    API_CUDA(run_fluxes(c, dt, nullptr, st));
    API_CUDA(export_dQ(c, dQ, st));
    return HYDRO_OK;
}

static int step_impl(hydro_ctx *c, hydro_particles *p, double dt, hydro_stats *stats,
                     hydro_stream stream);

// every value of the caller's state finite, checked before anything runs
// (a non-finite input returns HYDRO_ENONFINITE and changes nothing)
static int check_inputs(hydro_ctx *c, const hydro_particles *p, cudaStream_t st) {
    *(volatile int *)c->h_bad = 0;   // (no earlier check is in flight: each one was waited for)
    API_CUDA(run_check_inputs(c, p, st));
    API_CUDA(cudaStreamSynchronize(st));
    return *(volatile int *)c->h_bad ? HYDRO_ENONFINITE : HYDRO_OK;
}

int hydro_step(hydro_ctx *c, hydro_particles *p, double dt, hydro_stats *stats,
               hydro_stream stream) {
    if (stats) memset(stats, 0, sizeof(*stats));
    const int rc = step_impl(c, p, dt, stats, stream);
    if (c && (rc == HYDRO_OK || rc == HYDRO_ENCOND)) c->have_order = true;
    // a step that stopped early reports its error in the statistics too
    if (stats && rc != HYDRO_OK && stats->status == HYDRO_OK) stats->status = rc;
    return rc;
}

// New lists for the particles of the guard round (their search radii grew
// in guard_grow), built one particle per warp before the re-solve; a full
// rebuild when the overflow region is too small.  first: the first round,
// which builds the tree with the solved h and search radii (the later rounds
// only raise its radius bounds for their particles).
static int guard_lists(hydro_ctx *c, bool first, cudaStream_t st) {
    if (first) API_CUDA(build_tree(c, st));
    API_CUDA(guard_particle_lists(c, st));
    API_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    API_CUDA(cudaStreamSynchronize(st));
    const int fl = c->h_cnt->flags;
    if (fl & (ST_LIST_CAPACITY | ST_STACK)) {
        if (fl & ST_LIST_CAPACITY) grow_overflow(c, c->h_cnt->list_cursor);
        return lists_all(c, st);
    }
    return HYDRO_OK;
}

// Lists for a sub-step of individual timesteps.  The faces with a particle
// a that starts a step are found from the lists of a and of the particles j
// with r_aj < h_j (the flux kernel's owner of a face is one of its two
// particles, seeing the other within its own h).  So only the buckets
// holding such particles need fresh lists and a flux walk: a reverse walk
// of the tree from every starting particle flags them (ACT_REDO), and when
// they are few their lists are rebuilt into the overflow region and the
// flux kernel walks only them; the other lists are stale and unused.  Too
// many, or no room: every list, every bucket.
static int rung_lists(hydro_ctx *c, cudaStream_t st) {
    const int64_t n = c->plan.n, nb = c->plan.nbucket;
    c->rung_touch_n = -1;
    API_CUDA(build_tree(c, st));
    API_CUDA(mark_reverse(c, st));
    API_CUDA(queue_flagged(c, ACT_REDO, st));
    int nq = 0;
    API_CUDA(cudaMemcpyAsync(&nq, &c->d_cnt->ovf_buckets, sizeof(int), cudaMemcpyDeviceToHost, st));
    API_CUDA(cudaStreamSynchronize(st));
    if (nq > 0 && nq <= nb / 4 && c->have_lists && c->list_cap > 0) {
        API_CUDA(c->d_touch.ensure(nb));
        API_CUDA(cudaMemcpyAsync(c->d_touch.get(), c->d_ovf.get(), (size_t)nq * sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, st));
        API_CUDA(set_u64(&c->d_cnt->list_cursor, (unsigned long long)n * c->list_cap, st));
        API_CUDA(build_lists_queued(c, nq, st));
        int fl = 0;
        unsigned long long cursor = 0;
        API_CUDA(cudaMemcpyAsync(&fl, &c->d_cnt->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaMemcpyAsync(&cursor, &c->d_cnt->list_cursor, sizeof(cursor),
                                 cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
        if (!(fl & (ST_LIST_CAPACITY | ST_STACK))) {
            c->rung_touch_n = nq;
            return HYDRO_OK;
        }
        if (fl & ST_LIST_CAPACITY) grow_overflow(c, cursor);
        API_CUDA(cudaMemsetAsync(&c->d_cnt->flags, 0, sizeof(int), st));
    }
    return lists_all(c, st);
}

// individual timesteps: the base step of 2^rmax sub-steps (see hydro.h)
static int rungs_impl(hydro_ctx *c, hydro_particles *p, double dt0, int32_t *rung,
                      hydro_stats *stats, cudaStream_t st) {
    if (!c || !c->have_plan) return HYDRO_EINVAL;
    if (!valid_particles(c, p, true) || !rung || !(dt0 > 0.0) || !isfinite(dt0))
        return HYDRO_EINVAL;
    if (c->grav || c->cfg.entropy_switch || c->cfg.sorted_output) return HYDRO_ESTATE;
    const int64_t n = p->n;
    if (int rc0 = check_inputs(c, p, st)) return rc0;
    API_CUDA(ensure_state(c, n));
    API_CUDA(c->d_rung_c.ensure(n));
    API_CUDA(c->d_kstart_c.ensure(n));
    API_CUDA(c->d_rung_s.ensure(n));
    API_CUDA(c->d_ract.ensure(n));
    API_CUDA(c->d_toff.ensure(n));
    API_CUDA(c->d_rec_store.ensure((size_t)n * REC));
    API_CUDA(cudaMemsetAsync(c->d_rung_c.get(), 0, n * sizeof(int32_t), st));
    API_CUDA(cudaMemsetAsync(c->d_kstart_c.get(), 0, n * sizeof(int32_t), st));
    c->rung_live = true;
    c->rung_dt0 = dt0;
    c->learned_decision = 0;   // plain Riemann guess
    c->grav_live = c->ent_live = false;
    hydro_stats S;
    memset(&S, 0, sizeof(S));
    S.dt = dt0;
    int rmax = 0, status = HYDRO_OK;
    int64_t K = 1;
    double dtmin = dt0;
    for (int64_t k = 0; k < K; k++) {
        API_CUDA(cudaMemsetAsync(c->d_cnt, 0, sizeof(DevCounters), st));
        // the order of sub-step 0 is kept: the sub-steps drift the particles
        // by a fraction of h, so only the boxes and lists are rebuilt
        int rc = HYDRO_OK;
        if (k == 0) {
            c->rung_touch_n = -1;
            rc = build_all(c, p, p->h, nullptr, c->cfg.search_margin, true, st);
        } else {
            API_CUDA(gather_state(c, p, p->h, nullptr, c->cfg.search_margin, true, st));
        }
        if (rc) return rc;
        // omega of the particles that do not start (the others' is solved)
        API_CUDA(gather_from_caller(c->d_perm.get(), p->omega, n, 1, c->d_omsorted.get(), n, st));
        API_CUDA(rung_prep(c, k, rmax, dtmin, st));
        if (k > 0) {
            API_CUDA(rung_records(c, false, st));
            API_CUDA(rung_fill(c, st));
            rc = rung_lists(c, st);
            if (rc) return rc;
            if (c->rung_touch_n >= 0) S.rung_sparse++;
        } else {
            API_CUDA(reset_guard(c, st));
        }
        int rebuilds = 0, rounds = 0, ncond_fail = 0;
        bool first = true;
        for (;;) {
            rc = density_all(c, p, !first || k > 0, rebuilds, st, !first);
            if (rc) return rc;
            API_CUDA(run_primitives(c, st, !first));
            API_CUDA(run_gradients(c, nullptr, nullptr, nullptr, nullptr, !first, st, false));
            API_CUDA(cudaMemcpyAsync(&ncond_fail, &c->d_cnt->ncond_fail, sizeof(int),
                                     cudaMemcpyDeviceToHost, st));
            API_CUDA(cudaStreamSynchronize(st));
            first = false;
            if (ncond_fail == 0 || rounds >= c->cfg.max_ngb_grow) break;
            API_CUDA(guard_grow(c, st));
            rc = guard_lists(c, rounds == 0, st);
            if (rc) return rc;
            rounds++;
        }
        API_CUDA(grad_reduce(c, st));
        if (k == 0) {
            // rungs (§2.3.10): criteria, then the limiter to its fixed point
            API_CUDA(rung_assign(c, dt0, st));
            for (int sweep = 0;; sweep++) {
                // each sweep carries a raise at least one hop further and a
                // raise travels at most max_rung / 2 + 1 hops
                if (sweep > 2 * c->cfg.max_rung + 8) return HYDRO_ESTATE;
                API_CUDA(rung_limit_sweep(c, st));
                int changed = 0;
                API_CUDA(cudaMemcpyAsync(&changed, &c->d_cnt->rung_changed, sizeof(int),
                                         cudaMemcpyDeviceToHost, st));
                API_CUDA(cudaStreamSynchronize(st));
                if (!changed) break;
            }
            API_CUDA(rung_scatter(c, st));
            int rinfo[2] = {0, 0};
            API_CUDA(cudaMemcpyAsync(rinfo, &c->d_cnt->rung_max, 2 * sizeof(int),
                                     cudaMemcpyDeviceToHost, st));
            API_CUDA(cudaStreamSynchronize(st));
            rmax = rinfo[0];
            S.rung_capped = rinfo[1];
            K = (int64_t)1 << rmax;
            dtmin = ldexp(dt0, -rmax);
            // every particle starts at sub-step 0 (counted once)
            API_CUDA(cudaMemsetAsync(&c->d_cnt->rung_active, 0, sizeof(unsigned long long), st));
            API_CUDA(rung_prep(c, 0, rmax, dtmin, st));
        }
        API_CUDA(rung_records(c, true, st));
        API_CUDA(run_fluxes(c, dtmin, nullptr, st));
        // totals before the first sub-step and after the last
        if (stats && k == 0) API_CUDA(run_sums(c, 0, st));
        API_CUDA(run_update(c, p, dtmin, nullptr, false, 0, st));
        if (stats && k == K - 1) API_CUDA(run_sums(c, 1, st));
        API_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
        const DevCounters &H = *c->h_cnt;
        if (k == 0) {
            double dtc;
            memcpy(&dtc, &H.dt_min_bits, sizeof(double));
            S.dt_next = dtc;
            for (int q = 0; q < 5; q++) (q == 0 ? S.mass[0] : q < 4 ? S.mom[0][q - 1] : S.energy[0]) = H.sums[0][q];
        }
        for (int q = 0; q < 5; q++) (q == 0 ? S.mass[1] : q < 4 ? S.mom[1][q - 1] : S.energy[1]) = H.sums[1][q];
        S.grad_pairs += (int64_t)H.grad_pairs;
        S.flux_pairs += (int64_t)H.flux_pairs;
        S.newton_iters += (int64_t)H.newton_iters;
        S.vacuum_faces += (int64_t)H.vacuum;
        S.first_order_faces += (int64_t)H.first_order;
        S.active_steps += (int64_t)H.rung_active;
        S.ngb_rounds = std::max(S.ngb_rounds, rounds);
        S.ncond_fail += ncond_fail;
        S.list_rebuilds += rebuilds;
        int sk = flags_to_status(H.flags);
        if (ncond_fail && sk == HYDRO_OK) sk = HYDRO_ENCOND;
        if (status == HYDRO_OK) status = sk;
        if (sk != HYDRO_OK && sk != HYDRO_ENCOND && sk != HYDRO_ENOCONV_H) break;
    }
    API_CUDA(cudaMemcpyAsync(rung, c->d_rung_c.get(), n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    API_CUDA(cudaStreamSynchronize(st));
    S.status = status;
    S.rung_max = rmax;
    S.substeps = K;
    if (stats) *stats = S;
    return status;
}

int hydro_step_rungs(hydro_ctx *c, hydro_particles *p, double dt0, int32_t *rung,
                     hydro_stats *stats, hydro_stream stream) {
    if (stats) memset(stats, 0, sizeof(*stats));
    const int rc = rungs_impl(c, p, dt0, rung, stats, (cudaStream_t)stream);
    if (c) {
        c->rung_live = false;
        c->learned_decision = -1;
    }
    if (stats && rc != HYDRO_OK && stats->status == HYDRO_OK) stats->status = rc;
    return rc;
}

static int step_impl(hydro_ctx *c, hydro_particles *p, double dt, hydro_stats *stats,
                     hydro_stream stream) {
    if (!c || !c->have_plan) return HYDRO_EINVAL;
    if (!valid_particles(c, p, true)) return HYDRO_EINVAL;
    if (c->cfg.learned_guess && !c->have_mlp) return HYDRO_ESTATE;
    if (c->cfg.entropy_switch && !c->entA) return HYDRO_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = p->n;
    const bool timing = stats != nullptr && c->have_events;
    if (int rc0 = check_inputs(c, p, st)) return rc0;
    API_CUDA(ensure_state(c, n));
    // the first step of a context runs host-driven (it sizes every buffer);
    // later ones replay the captured graph unless it asks for the host path
    int how = 0;   // hydro_stats.graph of a host-driven step
    if (c->cfg.graph && !c->graph_off && c->steps_done > 0) {
        int rg = graph_step(c, p, dt, stats, st);
        if (rg <= 0) {
            c->steps_done++;
            return rg;
        }
        how = c->graph_off ? 3 : 2;
    }
    c->last_stats.graph = how;
    API_CUDA(cudaMemsetAsync(c->d_cnt, 0, sizeof(DevCounters), st));
    if (timing) API_CUDA(record_event(c->ev[0], st));
    int rc = build_all(c, p, p->h, nullptr, c->cfg.search_margin, true, st);
    if (rc) return rc;
    API_CUDA(gather_gravity(c, st));
    API_CUDA(gather_entropy(c, st));
    if (timing) API_CUDA(record_event(c->ev[1], st));
    API_CUDA(reset_guard(c, st));
    int rebuilds = 0, rounds = 0, ncond_fail = 0;
    bool first = true;
    for (;;) {
        rc = density_all(c, p, !first, rebuilds, st, !first);
        if (rc) return rc;
        if (first && timing) API_CUDA(record_event(c->ev[2], st));
        // a guard round recomputes the primitives of its re-solved particles
        // and only the gradients their new densities change
        API_CUDA(run_primitives(c, st, !first));
        API_CUDA(run_gradients(c, nullptr, nullptr, nullptr, nullptr, !first, st, false));
        API_CUDA(cudaMemcpyAsync(&ncond_fail, &c->d_cnt->ncond_fail, sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
        first = false;
        if (ncond_fail == 0 || rounds >= c->cfg.max_ngb_grow) break;
        API_CUDA(guard_grow(c, st));
        rc = guard_lists(c, rounds == 0, st);
        if (rc) return rc;
        rounds++;
    }
    API_CUDA(grad_reduce(c, st));
    if (timing) API_CUDA(record_event(c->ev[3], st));
    const double *dt_dev = dt > 0.0 ? nullptr : reinterpret_cast<const double *>(&c->d_cnt->dt_min_bits);
    c->timing = timing;
    rc = run_fluxes(c, dt, dt_dev, st);
    c->timing = false;
    API_CUDA((cudaError_t)rc);
    if (timing) API_CUDA(record_event(c->ev[4], st));
    if (stats) API_CUDA(run_sums(c, 0, st));
    API_CUDA(run_update(c, p, dt, dt_dev, false, STEP_SKIP_FLAGS, st));
    if (stats) API_CUDA(run_sums(c, 1, st));
    if (timing) API_CUDA(record_event(c->ev[5], st));
    c->last_stats.ngb_rounds = rounds;
    c->last_stats.list_rebuilds = rebuilds;
    c->last_stats.ncond_fail = ncond_fail;
    c->steps_done++;
    if (stats) {
        API_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
        hydro_stats &S = c->last_stats;
        S.status = flags_to_status(c->h_cnt->flags);
        if (ncond_fail && S.status == HYDRO_OK) S.status = HYDRO_ENCOND;
        fill_stats(c, dt, timing);
        *stats = S;
        return S.status;
    }
    return HYDRO_OK;
}

int hydro_sync_status(hydro_ctx *c, hydro_stream stream) {
    if (!c) return HYDRO_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int f = 0;
    API_CUDA(cudaMemcpyAsync(&f, &c->d_cnt->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    API_CUDA(cudaStreamSynchronize(st));
    API_CUDA(cudaMemsetAsync(&c->d_cnt->flags, 0, sizeof(int), st));
    return flags_to_status(f);
}

int hydro_get_order(hydro_ctx *c, int32_t *perm, hydro_stream stream) {
    if (!c || !perm) return HYDRO_EINVAL;
    if (!c->have_order) return HYDRO_ESTATE;
    API_CUDA(cudaMemcpyAsync(perm, c->d_perm.get(), (size_t)c->plan.n * sizeof(int32_t),
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return HYDRO_OK;
}

int hydro_get_stats(hydro_ctx *c, hydro_stats *stats, hydro_stream stream) {
    if (!c || !stats) return HYDRO_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    API_CUDA(cudaStreamSynchronize(st));
    hydro_stats &S = c->last_stats;
    const DevCounters &H = *c->h_cnt;
    S.flux_pairs = (int64_t)H.flux_pairs;
    S.newton_iters = (int64_t)H.newton_iters;
    S.guess_fallbacks = (int64_t)H.guess_fallbacks;
    S.learned_faces = (int64_t)H.learned_faces;
    S.hard_faces = (int64_t)H.hard_faces;
    S.learned_active = c->learned_active ? 1 : 0;
    S.vacuum_faces = (int64_t)H.vacuum;
    S.first_order_faces = (int64_t)H.first_order;
    *stats = S;
    return HYDRO_OK;
}

static const size_t kMlpParams = 12 * 64 + 64 + 64 * 64 + 64 + 64 + 1 + 24 + 2 + 24;
static const size_t kMlpScale = 12 * 64 + 64 + 64 * 64 + 64 + 64 + 1 + 12;   // scale[12]
static const size_t kMlpTScale = kMlpScale + 13;
static const size_t kMlpXmin = kMlpTScale + 1;

int hydro_test_mlp_stall(hydro_ctx *c, int on) {
    if (!c || (on != 0 && on != 1)) return HYDRO_EINVAL;
    c->mlp_stall = on;
    return HYDRO_OK;
}

int hydro_mlp_load(hydro_ctx *c, const void *weights, size_t bytes) {
    if (!c || !weights) return HYDRO_EINVAL;
    if (bytes != kMlpParams * sizeof(float)) return HYDRO_EINVAL;
    const float *w = static_cast<const float *>(weights);
    for (size_t k = 0; k < kMlpParams; k++)
        if (!std::isfinite(w[k])) return HYDRO_EINVAL;
    for (size_t k = kMlpScale; k < kMlpScale + 12; k++)   // feature scales
        if (!(w[k] > 0.f)) return HYDRO_EINVAL;
    if (!(w[kMlpTScale] > 0.f)) return HYDRO_EINVAL;      // target scale
    for (size_t k = 0; k < 12; k++)                       // feature box
        if (!(w[kMlpXmin + k] <= w[kMlpXmin + 12 + k])) return HYDRO_EINVAL;
    API_CUDA(c->d_mlp.ensure(kMlpParams));
    API_CUDA(cudaMemcpy(c->d_mlp.get(), weights, bytes, cudaMemcpyHostToDevice));
    API_CUDA(mlp_pack(c, 0));
    API_CUDA(cudaStreamSynchronize(0));
    c->have_mlp = true;
    return HYDRO_OK;
}

int hydro_mlp_get(hydro_ctx *c, void *weights, size_t bytes) {
    if (!c || !weights || bytes != kMlpParams * sizeof(float)) return HYDRO_EINVAL;
    if (!c->have_mlp) return HYDRO_ESTATE;
    API_CUDA(cudaDeviceSynchronize());
    API_CUDA(cudaMemcpy(weights, c->d_mlp.get(), bytes, cudaMemcpyDeviceToHost));
    return HYDRO_OK;
}

int hydro_mlp_predict(hydro_ctx *c, const float *faces, int64_t n, float *p_guess,
                      hydro_stream stream) {
    if (!c || n < 0 || (n > 0 && (!faces || !p_guess))) return HYDRO_EINVAL;
    if (!c->have_mlp) return HYDRO_ESTATE;
    if (n == 0) return HYDRO_OK;
    API_CUDA(mlp_predict(c, faces, n, p_guess, (cudaStream_t)stream));
    return HYDRO_OK;
}

int hydro_mlp_features(hydro_ctx *c, const float *faces, int64_t n, float *x, float *t,
                       hydro_stream stream) {
    if (!c || n < 0 || (n > 0 && (!faces || !x || !t))) return HYDRO_EINVAL;
    if (n == 0) return HYDRO_OK;
    API_CUDA(mlp_features(c, faces, n, x, t, (cudaStream_t)stream));
    return HYDRO_OK;
}

int hydro_mlp_gradient(hydro_ctx *c, const float *x, const float *t, int64_t n, int quant,
                       float *grad, float *loss, hydro_stream stream) {
    if (!c || n <= 0 || !x || !t || !grad || !loss) return HYDRO_EINVAL;
    if (!c->have_mlp) return HYDRO_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), st));
    API_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st));
    API_CUDA(mlp_gradient(c, x, t, n, n, 0, 0, 0, quant ? 1 : 0, grad, loss, st));
    return HYDRO_OK;
}

// He-normal initial parameters from a counter-based generator (splitmix64
// of seed and index, Box-Muller); standardisation 0 / 1 until set from data
static std::vector<float> mlp_init(uint64_t seed) {
    auto mix = [](uint64_t z) {
        z += 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    uint64_t ctr = 0;
    auto normal = [&]() {
        const double u1 = ((mix(seed ^ mix(ctr++)) >> 11) + 1.0) * 0x1.0p-53;
        const double u2 = (mix(seed ^ mix(ctr++)) >> 11) * 0x1.0p-53;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    std::vector<float> w(kMlpParams, 0.f);
    size_t k = 0;
    for (int e = 0; e < 64 * 12; e++) w[k++] = (float)(normal() * std::sqrt(2.0 / 12.0));
    k += 64;   // b1
    for (int e = 0; e < 64 * 64; e++) w[k++] = (float)(normal() * std::sqrt(2.0 / 64.0));
    k += 64;   // b2
    for (int e = 0; e < 64; e++) w[k++] = (float)(normal() * std::sqrt(1.0 / 64.0));
    k += 1;    // b3
    k += 12;   // mean
    for (int e = 0; e < 12; e++) w[k++] = 1.f;
    k += 1;    // t_mean
    w[k++] = 1.f;   // t_scale
    for (int e = 0; e < 12; e++) w[k++] = -1e30f;   // feature box: set from data
    for (int e = 0; e < 12; e++) w[k++] = 1e30f;
    return w;
}

int hydro_mlp_train(hydro_ctx *c, const float *faces, int64_t n, int64_t steps, int64_t batch,
                    double lr, uint64_t seed, float *loss, hydro_stream stream) {
    if (!c || !faces || n <= 0 || steps < 0 || batch <= 0 || !(lr > 0.0)) return HYDRO_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(c->d_mlp_x.ensure((size_t)12 * n));
    API_CUDA(c->d_mlp_t.ensure((size_t)n));
    API_CUDA(c->d_mlp_grad.ensure(kMlpParams));
    API_CUDA(c->d_mlp_m.ensure(kMlpParams));
    API_CUDA(c->d_mlp_v.ensure(kMlpParams));
    API_CUDA(c->d_mlp_loss.ensure((size_t)std::max<int64_t>(steps, 1)));
    API_CUDA(c->d_mlp_acc.ensure(27));
    API_CUDA(mlp_features(c, faces, n, c->d_mlp_x.get(), c->d_mlp_t.get(), st));
    if (!c->have_mlp) {
        std::vector<float> w = mlp_init(seed);
        API_CUDA(c->d_mlp.ensure(kMlpParams));
        API_CUDA(cudaMemcpyAsync(c->d_mlp.get(), w.data(), w.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, st));
        API_CUDA(c->d_mlp_box.ensure(24));
        API_CUDA(mlp_normalise(c, c->d_mlp_x.get(), c->d_mlp_t.get(), n, c->d_mlp_acc.get(),
                               c->d_mlp_box.get(), st));
        API_CUDA(cudaStreamSynchronize(st));   // w is a host temporary
    }
    API_CUDA(cudaMemsetAsync(c->d_mlp_grad.get(), 0, kMlpParams * sizeof(float), st));
    API_CUDA(cudaMemsetAsync(c->d_mlp_m.get(), 0, kMlpParams * sizeof(float), st));
    API_CUDA(cudaMemsetAsync(c->d_mlp_v.get(), 0, kMlpParams * sizeof(float), st));
    API_CUDA(cudaMemsetAsync(c->d_mlp_loss.get(), 0, std::max<int64_t>(steps, 1) * sizeof(float), st));
    for (int64_t s = 1; s <= steps; s++) {
        API_CUDA(mlp_gradient(c, c->d_mlp_x.get(), c->d_mlp_t.get(), n, batch, 1, seed,
                              (uint64_t)s, 1, c->d_mlp_grad.get(), c->d_mlp_loss.get() + (s - 1),
                              st));
        // cosine decay of the learning rate to lr / 20 over the run
        const double frac = steps > 1 ? (double)(s - 1) / (double)(steps - 1) : 0.0;
        const double lr_s = lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.141592653589793 * frac)));
        API_CUDA(mlp_adam(c, c->d_mlp_grad.get(), c->d_mlp_m.get(), c->d_mlp_v.get(), (float)lr_s,
                          (int)std::min<int64_t>(s, 1 << 30), st));
    }
    if (loss && steps > 0)
        API_CUDA(cudaMemcpyAsync(loss, c->d_mlp_loss.get(), steps * sizeof(float),
                                 cudaMemcpyDeviceToDevice, st));
    API_CUDA(mlp_pack(c, st));
    c->have_mlp = true;
    return HYDRO_OK;
}

int hydro_record_faces(hydro_ctx *c, float *buf, int64_t capacity, double keep_fraction,
                       int hard_only) {
    if (!c) return HYDRO_EINVAL;
    if (buf && (capacity <= 0 || !(keep_fraction > 0.0 && keep_fraction <= 1.0)))
        return HYDRO_EINVAL;
    API_CUDA(c->d_rec_cursor.ensure(1));
    API_CUDA(cudaDeviceSynchronize());
    API_CUDA(cudaMemset(c->d_rec_cursor.get(), 0, sizeof(unsigned long long)));
    c->rec_faces = buf;
    c->rec_cap = buf ? capacity : 0;
    c->rec_keep = (uint32_t)std::min(4294967295.0, std::floor(keep_fraction * 4294967296.0));
    if (buf && c->rec_keep == 0) c->rec_keep = 1;
    c->rec_hard_only = hard_only ? 1 : 0;
    return HYDRO_OK;
}

int hydro_recorded_faces(hydro_ctx *c, int64_t *count, hydro_stream stream) {
    if (!c || !count) return HYDRO_EINVAL;
    unsigned long long v = 0;
    if (c->d_rec_cursor.get()) {
        cudaStream_t st = (cudaStream_t)stream;
        API_CUDA(cudaMemcpyAsync(&v, c->d_rec_cursor.get(), sizeof(v), cudaMemcpyDeviceToHost, st));
        API_CUDA(cudaStreamSynchronize(st));
    }
    *count = (int64_t)v;
    return HYDRO_OK;
}

int hydro_set_gravity(hydro_ctx *c, const double *acc) {
    if (!c) return HYDRO_EINVAL;
    c->grav = acc;
    return HYDRO_OK;
}

int hydro_set_entropy(hydro_ctx *c, double *A) {
    if (!c) return HYDRO_EINVAL;
    c->entA = A;
    return HYDRO_OK;
}

int hydro_set_tuning(hydro_ctx *c, const hydro_tuning *t) {
    if (!c || !t) return HYDRO_EINVAL;
    if (!(t->search_margin >= 1.0) || t->nbr_slots < 32 || t->nbr_slots > 256) return HYDRO_EINVAL;
    if (t->grad_min_ctas != 1 && (t->grad_min_ctas < 4 || t->grad_min_ctas > 6)) return HYDRO_EINVAL;
    if (t->flux_min_ctas < 4 || t->flux_min_ctas > 6) return HYDRO_EINVAL;
    if (t->flux_queue != 0 && t->flux_queue != 1) return HYDRO_EINVAL;
    if (t->grad_rank < 0 || t->grad_rank > 2) return HYDRO_EINVAL;
    c->cfg.search_margin = t->search_margin;
    c->flux_queue = t->flux_queue;
    c->grad_rank = t->grad_rank;
    c->nbr_per_particle = t->nbr_slots;
    c->grad_minb = t->grad_min_ctas;
    c->flux_minb = t->flux_min_ctas;
    return HYDRO_OK;
}

int hydro_autotune(hydro_ctx *c, hydro_particles *p, hydro_tuning *out, hydro_stream stream) {
    if (c) c->grav_live = c->ent_live = false;   // (gravity and entropy: hydro_step only)
    if (!c || !c->have_plan) return HYDRO_EINVAL;
    if (!valid_particles(c, p, true)) return HYDRO_EINVAL;
    if (c->cfg.learned_guess && !c->have_mlp) return HYDRO_ESTATE;
    cudaStream_t st = (cudaStream_t)stream;
    API_CUDA(ensure_state(c, p->n));
    static const double margins[4] = {1.05, 1.1, 1.15, 1.25};
    static const int slots[3] = {64, 96, 128};
    static const int gminb[4] = {1, 4, 5, 6};
    static const int fminb[3] = {4, 5, 6};
    hydro_tuning T;
    memset(&T, 0, sizeof(T));
    float ms = 0.f;
    // sort, lists and density (the part the radius and the slots change),
    // from the caller's particles each time
    auto front = [&](double margin, int nslots) -> int {
        c->cfg.search_margin = margin;
        c->nbr_per_particle = nslots;
        API_CUDA(record_event(c->ev[0], st));
        API_CUDA(cudaMemsetAsync(c->d_cnt, 0, sizeof(DevCounters), st));
        int rc = build_all(c, p, p->h, nullptr, margin, true, st);
        if (rc) return rc;
        API_CUDA(reset_guard(c, st));
        int rebuilds = 0;
        rc = density_all(c, p, false, rebuilds, st);
        if (rc) return rc;
        API_CUDA(record_event(c->ev[1], st));
        API_CUDA(cudaEventSynchronize(c->ev[1]));
        API_CUDA(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        c->nbr_per_particle = nslots;   // (lists_all may have grown it)
        return HYDRO_OK;
    };
    float best = 1e30f;
    double bm = c->cfg.search_margin;
    int bs = c->nbr_per_particle;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 3; j++) {
            float t = 1e30f;
            for (int rep = 0; rep < 2; rep++) {
                int rc = front(margins[i], slots[j]);
                if (rc) return rc;
                t = std::min(t, ms);
            }
            T.front_ms[i][j] = t;
            if (t < best) { best = t; bm = margins[i]; bs = slots[j]; }
        }
    int rc = front(bm, bs);
    if (rc) return rc;
    API_CUDA(run_primitives(c, st));
    // gradient stage
    best = 1e30f;
    int bg = 1;
    for (int k = 0; k < 4; k++) {
        c->grad_minb = gminb[k];
        float t = 1e30f;
        for (int rep = 0; rep < 2; rep++) {
            API_CUDA(record_event(c->ev[0], st));
            API_CUDA(run_gradients(c, nullptr, nullptr, nullptr, nullptr, false, st));
            API_CUDA(record_event(c->ev[1], st));
            API_CUDA(cudaEventSynchronize(c->ev[1]));
            API_CUDA(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
            t = std::min(t, ms);
        }
        T.grad_ms[k] = t;
        if (t < best) { best = t; bg = gminb[k]; }
    }
    c->grad_minb = bg;
    // lanes in particle order, ranked by list length in tiles of 128, or in
    // tiles of up to 1024, with that bound
    best = 1e30f;
    for (int r = 0; r < 3; r++) {
        c->grad_rank = r;
        float t = 1e30f;
        for (int rep = 0; rep < 2; rep++) {
            API_CUDA(record_event(c->ev[0], st));
            API_CUDA(run_gradients(c, nullptr, nullptr, nullptr, nullptr, false, st));
            API_CUDA(record_event(c->ev[1], st));
            API_CUDA(cudaEventSynchronize(c->ev[1]));
            API_CUDA(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
            t = std::min(t, ms);
        }
        T.grad_rank_ms[r] = t;
        if (t < best) { best = t; T.grad_rank = r; }
    }
    c->grad_rank = T.grad_rank;
    // flux stage, plain guess (the dt the gradients found)
    int bf = 4;
    if (c->cfg.precision == HYDRO_MIXED) {
        const double *dt_dev = reinterpret_cast<const double *>(&c->d_cnt->dt_min_bits);
        best = 1e30f;
        read_learn_probe(c);   // (the trials below reuse the probe events)
        c->learned_decision = 0;
        for (int k = 0; k < 3; k++) {
            c->flux_minb = fminb[k];
            float t = 1e30f;
            for (int rep = 0; rep < 2; rep++) {
                API_CUDA(record_event(c->ev[0], st));
                cudaError_t e = run_fluxes(c, -1.0, dt_dev, st);
                if (e != cudaSuccess) { c->learned_decision = -1; return cuda_status(e); }
                API_CUDA(record_event(c->ev[1], st));
                API_CUDA(cudaEventSynchronize(c->ev[1]));
                API_CUDA(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
                t = std::min(t, ms);
            }
            T.flux_ms[k] = t;
            if (t < best) { best = t; bf = fminb[k]; }
        }
        // buckets by index or drawn from the queue, with the chosen bound
        c->flux_minb = bf;
        best = 1e30f;
        for (int q = 0; q < 2; q++) {
            c->flux_queue = q;
            float t = 1e30f;
            for (int rep = 0; rep < 2; rep++) {
                API_CUDA(record_event(c->ev[0], st));
                cudaError_t e = run_fluxes(c, -1.0, dt_dev, st);
                if (e != cudaSuccess) { c->learned_decision = -1; return cuda_status(e); }
                API_CUDA(record_event(c->ev[1], st));
                API_CUDA(cudaEventSynchronize(c->ev[1]));
                API_CUDA(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
                t = std::min(t, ms);
            }
            T.flux_queue_ms[q] = t;
            if (t < best) { best = t; T.flux_queue = q; }
        }
        c->flux_queue = T.flux_queue;
        c->learned_decision = -1;
    }
    c->flux_minb = bf;
    c->cfg.search_margin = bm;
    c->nbr_per_particle = bs;
    T.search_margin = bm;
    T.nbr_slots = bs;
    T.grad_min_ctas = bg;
    T.flux_min_ctas = bf;
    T.flux_queue = c->flux_queue;
    if (out) *out = T;
    return HYDRO_OK;
}

int64_t hydro_kernel_launches(void) { return (int64_t)g_launches.load(); }

const char *hydro_strerror(int s) {
    switch (s) {
    case HYDRO_OK: return "ok";
    case HYDRO_EINVAL: return "invalid argument";
    case HYDRO_ENOMEM: return "device allocation failed";
    case HYDRO_ECAPACITY: return "neighbour-list capacity exceeded";
    case HYDRO_ENOCONV_H: return "smoothing-length iteration did not converge";
    case HYDRO_ENCOND: return "condition number above threshold after all N_NGB growths";
    case HYDRO_ERIEMANN: return "Riemann solver failed";
    case HYDRO_ENONFINITE: return "non-finite value";
    case HYDRO_ECUDA: return "CUDA runtime error";
    case HYDRO_ESTATE: return "call order violated";
    case HYDRO_ESEARCH: return "smoothing length beyond the neighbour search radius";
    case HYDRO_EMLP: return "tensor-core MLP wait gave up";
    default: return "unknown status";
    }
}

}  // extern "C"
