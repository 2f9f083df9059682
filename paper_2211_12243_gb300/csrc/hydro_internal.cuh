// Internal declarations of the GB300 hydro library (not part of the ABI).
//
// Data layout in HBM (all arrays in Morton-sorted order, index s):
//   xs, ys, zs        double   positions (master copy, exact geometry)
//   qx, qy, qz        uint32   fixed-point positions q = x/L * 2^32; an
//                              int32 difference is the minimum-image dx
//   hs                double   search radius of the neighbour lists
//   rec[s][32]        R        per-particle record, one 128 B (float) or
//                              256 B (double) line, read whole by the pair
//                              kernels when particle s is a neighbour:
//                              x y z h | rho vx vy vz | p omega B(6) |
//                              limited grad rho(3) v(9) p(3) | pad
//                              (in float records x y z hold the q bits)
//   Qs[6][n]          double   conserved m, px, py, pz, E, U (sorted copy)
//   nbr_off/nbr_cnt   int64/int32  per-particle slice of nbr_idx (sorted ids)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "hydro.h"

namespace hyd {

constexpr int BUCKET = 32;   // particles per bucket (one warp)
constexpr int REC = 32;      // scalars per particle record
constexpr int MAX_LEVELS = 8;

// record slots
enum : int {
    R_X = 0, R_Y = 1, R_Z = 2, R_H = 3,
    R_RHO = 4, R_VX = 5, R_VY = 6, R_VZ = 7,
    R_P = 8, R_OM = 9, R_B = 10,           // B: 10..15 (xx xy xz yy yz zz)
    R_G = 16,                              // 16..30: grad rho, vx, vy, vz, p (limited)
    R_PAD = 31
};

// device status bits (first error wins in the word; bits accumulate in flags)
enum : int {
    ST_LIST_OVERFLOW = 1,     // per-particle staging capacity exceeded
    ST_LIST_CAPACITY = 2,     // global list storage exceeded
    ST_SEARCH = 4,            // h root beyond the search radius
    ST_NOCONV_H = 8,
    ST_NCOND = 16,
    ST_RIEMANN = 32,
    ST_NONFINITE = 64,
    ST_STACK = 128,
    ST_MLP = 256,             // a tensor-core wait of the MLP gave up
};

// per-particle flag bits (d_active)
enum : uint8_t {
    ACT_SOLVE = 1,     // solve the density of this particle
    ACT_SEARCH = 2,    // its root lay beyond the list radius
    ACT_NCOND = 4,     // N_cond above the threshold (guard)
    ACT_REDO = 8,      // recompute its gradients (a neighbour's h changed)
    ACT_GUARD = 16,    // its N_NGB grew in the current guard round
};

struct Box {
    double L[3];      // lengths
    float s[3];       // L / 2^32 (metres per fixed-point unit)
    float pad;
};

// scalars the device reads every step
struct DevCounters {
    unsigned long long list_cursor;   // entries used in nbr_idx
    unsigned long long list_needed;   // entries the build wanted
    unsigned long long dt_min_bits;   // CFL dt, as ordered bits of a positive double
    int flags;                        // ST_* bits
    int search_fail;                  // particles whose h left the radius
    int ncond_fail;                   // particles above the N_cond threshold
    int ovf_buckets;                  // buckets queued for the long-list passes
    unsigned long long grad_pairs;
    unsigned long long flux_pairs;
    unsigned long long newton_iters;
    unsigned long long guess_fallbacks;
    unsigned long long vacuum;
    unsigned long long first_order;
    unsigned long long learned_faces;  // faces solved from the learned guess
    unsigned long long hard_faces;     // faces where Toro's guess is the two-shock value
    unsigned long long hard_ovf;       // a deferred-face sub-buffer was full (pass redone)
    double sums[2][5];                // totals before / after (m, px, py, pz, E)
    // device-driven loops of the graph step (graph.cu)
    int search_round;                 // re-search rounds of the current density solve
    int guard_round;                  // N_cond growth rounds taken
    int rebuilds;                     // re-search rounds in the step
    int abort;                        // the step cannot finish on the device: no update
    int ovf_first;                    // buckets of the first list pass with long lists
    int nguard;                       // particles whose N_NGB grew in this guard round
    // rung assignment (hydro_step_rungs)
    int rung_changed;                 // the limiter raised a rung in this sweep
    int rung_max;                     // the deepest rung
    int rung_capped;                  // particles the criteria wanted beyond max_rung
    unsigned long long rung_active;   // particles starting a step in this sub-step
    int nredo;                        // particles a guard round recomputes the gradients of
    int redo_cursor;                  // the guard round's gradient warps' place in theirs
    int solve_cursor;                 // the guard round's density warps' place in the guard list
    int redo_pass;                    // the last gradient pass took only the redo list (1) or
                                      // every particle (0): where flags can be set
    unsigned long long flux_cursor;   // the flux kernel's bucket queue
};

// bucket tree topology (host plan, mirrored on the device)
struct Plan {
    int64_t n = 0, nbox = 0;
    int64_t nbucket = 0, nnode = 0;
    int nlevels = 0;
    std::vector<int64_t> box_off;          // nbox+1
    std::vector<double> box_len;           // 3 nbox
    std::vector<int64_t> level_off;        // nlevels+1 (node ids, level-major)
    std::vector<int32_t> node_first, node_cnt, node_box;
    std::vector<int32_t> box_root;
};

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    // grow (contents not preserved); returns cudaSuccess or the error
    cudaError_t ensure(size_t n) {
        if (n <= cap && p) return cudaSuccess;
        release();
        size_t want = n > 0 ? n : 1;
        cudaError_t e = cudaMalloc((void **)&p, want * sizeof(T));
        if (e != cudaSuccess) { p = nullptr; cap = 0; return e; }
        cap = want;
        return cudaSuccess;
    }
    T *get() const { return p; }
};

}  // namespace hyd

struct hydro_ctx {
    hydro_config cfg;
    int device = 0;
    hyd::Plan plan;
    bool have_plan = false;
    bool have_lists = false;
    int64_t list_n = 0;
    int nbr_per_particle = 96;        // fixed slots per particle in nbr_idx
    int list_cap = 64;                // slots used by the current lists
    int64_t ovf_reserve = 0;          // entries kept for the overflow region

    // plan on device
    hyd::DevBuf<int32_t> d_node_first, d_node_cnt, d_node_box, d_box_root;
    hyd::DevBuf<int64_t> d_box_off;
    hyd::DevBuf<hyd::Box> d_boxes;
    hyd::DevBuf<uint4> d_node_aabb;          // lo.xyz, hmax bits | hi.xyz, pad
    hyd::DevBuf<uint4> d_node_aabb_hi;

    // sort scratch
    hyd::DevBuf<unsigned long long> d_keys, d_keys_alt;
    hyd::DevBuf<int32_t> d_perm, d_perm_alt;
    hyd::DevBuf<int64_t> d_scan_tmp;
    hyd::DevBuf<int32_t> d_hist;

    // sorted state
    hyd::DevBuf<double> d_xs, d_ys, d_zs, d_hs, d_hsorted, d_omsorted;
    hyd::DevBuf<uint32_t> d_qx, d_qy, d_qz;
    hyd::DevBuf<uint64_t> d_q64;      // 3 n, mixed-path refinement
    hyd::DevBuf<int32_t> d_pbox;
    hyd::DevBuf<double> d_Q;          // 6 n
    hyd::DevBuf<double> d_dQ;         // 5 n
    hyd::DevBuf<float> d_recf;        // 32 n (MIXED)
    hyd::DevBuf<double> d_recd;       // 32 n (FP64)
    hyd::DevBuf<double> d_out;        // staging of outputs (up to 27 n)
    hyd::DevBuf<double> d_nngb;       // per-particle N_NGB
    hyd::DevBuf<uint8_t> d_active;    // density / guard flags
    hyd::DevBuf<double> d_vsig_dt;    // per-particle CFL dt
    hyd::DevBuf<int32_t> d_gpairs;    // per-particle gradient pairs
    hyd::DevBuf<int32_t> d_guard_idx; // the guard round's grown particles (nguard of them)
    hyd::DevBuf<int32_t> d_redo_idx;  // the particles whose gradients it recomputes (nredo)
    hyd::DevBuf<uint32_t> d_guard_bits; // the round's guard particles as a bitmap

    // neighbour lists
    hyd::DevBuf<int32_t> d_nbr_idx;
    hyd::DevBuf<int64_t> d_nbr_off;
    hyd::DevBuf<int32_t> d_nbr_cnt;
    hyd::DevBuf<int32_t> d_ovf;       // bucket ids with long lists

    // external (gravitational) acceleration: the caller's array (3 per
    // particle, caller order) or NULL; sorted SoA copy; sum_j dm_ij r_ij
    const double *grav = nullptr;
    bool grav_live = false;           // d_agrav holds this step's sorted copy (hydro_step only)
    hyd::DevBuf<double> d_agrav;      // 3 n
    hyd::DevBuf<double> d_dM;         // 3 n

    // entropy switch (§2.3.7): the caller's entropic function A (caller
    // order, rewritten by each step) or NULL; its sorted copy at the start
    // of the step; the value the step uses (re-set where the energies gave
    // the pressure); sum_j c_m,ij A_upwind; the particles the energies did
    // not claim
    double *entA = nullptr;
    bool ent_live = false;            // d_A0 holds this step's sorted copy (hydro_step only)
    hyd::DevBuf<double> d_A0, d_A1, d_dS;   // n each
    hyd::DevBuf<uint8_t> d_ecand;

    // individual timesteps (hydro_step_rungs): rungs and the sub-step at
    // which each particle's current step started (caller order); per sorted
    // particle its rung, whether it starts a step at this sub-step and the
    // time since its state was taken; the records of every particle at its
    // last start (caller order, REC scalars of the precision's type)
    bool rung_live = false;
    double rung_dt0 = 0.0;
    hyd::DevBuf<int32_t> d_rung_c, d_kstart_c, d_rung_s;
    hyd::DevBuf<uint8_t> d_ract;
    hyd::DevBuf<double> d_toff;
    hyd::DevBuf<double> d_rec_store;  // n REC doubles (float records use half)
    // the buckets whose particles can reach a particle starting a step (the
    // only lists a sparse sub-step rebuilds and walks); -1: all buckets
    hyd::DevBuf<int32_t> d_touch;
    int64_t rung_touch_n = -1;

    // reductions
    hyd::DevBuf<double> d_partials;

    // MLP: float parameters, the packed bf16 tiles the kernels copy into
    // shared memory, and training scratch
    hyd::DevBuf<float> d_mlp;
    hyd::DevBuf<unsigned char> d_mlp_blob;
    hyd::DevBuf<float> d_mlp_x, d_mlp_t, d_mlp_grad, d_mlp_m, d_mlp_v, d_mlp_loss;
    hyd::DevBuf<double> d_mlp_acc;
    hyd::DevBuf<int> d_mlp_box;       // feature min / max as ordered integers
    bool have_mlp = false;
    int mlp_stall = 0;                // error-path test hook (hydro_test_mlp_stall)

    // hard faces deferred to the learned-guess pass (FaceState fields, owner/partner)
    hyd::DevBuf<float> d_hard;
    hyd::DevBuf<int32_t> d_hard_idx;
    hyd::DevBuf<unsigned long long> d_hard_cursor;
    // adaptive learned path (learned_guess = 1): a learned probe call, a
    // plain probe call, then the faster of the two for 15 calls.  The probe
    // times come from events 6-8 around the flux kernels, the learned probe's
    // counts from h_learn[0..1] (learned, hard faces; event 9)
    int learn_phase = 0;              // 0: probe learned next; 1: probe plain next; 2: run the winner
    int learn_skip = 0;               // winner calls left
    bool learn_winner = false;        // the learned path won the last comparison
    int learn_probe = 0;              // the last call was a probe: 1 learned, 2 plain
    float learn_t[2] = {0.f, 0.f};    // flux-stage time of the last probes: plain, learned
    bool learn_used = false;          // > 10% of the learned probe's hard faces used the network
    bool learned_active = false;
    unsigned long long *h_learn = nullptr;   // pinned
    int64_t hard_cap = 0;

    // face recording (training data for the MLP), mixed exact path
    float *rec_faces = nullptr;       // caller's device buffer [7][rec_cap]
    hyd::DevBuf<unsigned long long> d_rec_cursor;   // faces seen (may exceed rec_cap)
    int64_t rec_cap = 0;
    uint32_t rec_keep = 0;            // keep a face when its hash < rec_keep
    int rec_hard_only = 0;

    // device counters + pinned host mirror
    hyd::DevCounters *d_cnt = nullptr;
    hyd::DevCounters *h_cnt = nullptr;
    // the input check's flag in mapped host memory: the check kernel writes it
    // and the host reads it after the kernel, with no copy (a copy would queue
    // behind whatever the caller's copy streams are moving)
    int *h_bad = nullptr, *d_bad = nullptr;
    int pending_status = 0;

    hydro_stats last_stats;
    bool have_order = false;          // d_perm holds the order of a completed step
    cudaEvent_t ev[10];               // 0-5 stage boundaries, 6-8 around the flux kernels,
                                      // 9 after the learned-path counters' readback
    bool have_events = false;
    bool timing = false;              // record ev[6..9] in the flux launcher

    // graph step (graph.cu): one executable graph per learned-path choice,
    // with the launch parameters it was captured with
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        std::vector<unsigned long long> key;
        // kernels per run: top level, one re-search round, one guard round
        // (without its re-search rounds)
        long long k_top = 0, k_search = 0, k_guard = 0;
    } graph_slot[2];
    cudaStream_t cap_stream[3] = {nullptr, nullptr, nullptr};   // capture streams (top, bodies)
    long long cap_k_search = 0, cap_k_guard = 0;   // kernels in one captured loop body
    int learned_decision = -1;        // >= 0: run_fluxes takes this choice (graph capture)
    bool capturing = false;           // enqueue without host synchronisation
    bool graph_off = false;           // a capture failed: host-driven steps only
    // launch-bounds variants chosen by hydro_autotune (resident CTAs per SM
    // the register allocation allows): float flux kernel 4, 5 or 6;
    // gradient kernel 1 (no bound), 5 or 6
    int flux_minb = 4;
    int grad_minb = 1;
    int flux_queue = 1;               // flux kernel: buckets drawn from a cursor (0: by index)
    int grad_rank = 1;                // gradient kernel: lanes ranked by list length (0: not)
    int64_t steps_done = 0;           // hydro_step calls completed
};

namespace hyd {

// every kernel launch is followed by launch_check(): it returns the launch
// error and counts the launch (process-wide, see hydro_kernel_launches)
cudaError_t launch_check();
// an event record that a stream capture turns into a graph node (a plain
// record during capture only orders captured work and is never timed)
inline cudaError_t record_event(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t r = cudaStreamIsCapturing(st, &cs);
    if (r != cudaSuccess) return r;
    if (cs == cudaStreamCaptureStatusActive)
        return cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    return cudaEventRecord(e, st);
}
// the process-wide count behind hydro_kernel_launches: a kernel enqueued
// while a graph is captured is counted when the graph runs (graph.cu)
long long launch_count();
void add_launches(long long k);

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
using stream_t = cudaStream_t;

// sort.cu
cudaError_t sort_particles(hydro_ctx *c, const hydro_particles *p, stream_t st);
cudaError_t gather_state(hydro_ctx *c, const hydro_particles *p, const double *h_in,
                         const double *h_search, double search_margin, bool want_Q,
                         stream_t st);
cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp,
                               stream_t st);
cudaError_t scatter_to_caller(const int32_t *perm, const double *src, int64_t n, int ncomp,
                              int64_t src_stride, double *dst, stream_t st);
cudaError_t gather_from_caller(const int32_t *perm, const double *src, int64_t n, int ncomp,
                               double *dst, int64_t dst_stride, stream_t st);

// neighbours.cu
cudaError_t build_tree(hydro_ctx *c, stream_t st);
cudaError_t raise_tree(hydro_ctx *c, stream_t st);
cudaError_t build_lists(hydro_ctx *c, int cap, stream_t st);
cudaError_t build_lists_queued(hydro_ctx *c, int nq, stream_t st);
cudaError_t rebuild_active_lists(hydro_ctx *c, int *nq, stream_t st, bool guard = false);
// ACT_REDO on the guard round's particles and on every particle i with one
// of them in its list (r_ia < h_i), found by walks of the bucket tree
cudaError_t mark_reverse(hydro_ctx *c, stream_t st, bool use_h = false);
// the same marks for a guard round (bounded by the tree's largest h), by
// tree walks from the grown particles or, when they are many, by a scan of
// every particle's list (the choice made on the device)
cudaError_t mark_guard_reverse(hydro_ctx *c, stream_t st);
// gradients.cu: the particles with one of `bits` set in active, appended to
// idx (count in *nidx, reset first; their order is not fixed)
cudaError_t compact_flags(int64_t n, const uint8_t *active, uint8_t bits, int32_t *idx, int *nidx,
                          stream_t st);
// the same two passes with the bucket count read on the device (no host
// wait): the queued overflow buckets, and the re-search rebuild
cudaError_t build_lists_queued_dev(hydro_ctx *c, stream_t st);
cudaError_t rebuild_active_lists_dev(hydro_ctx *c, stream_t st, bool guard = false);
cudaError_t guard_particle_lists(hydro_ctx *c, stream_t st, bool only_search = false);
cudaError_t export_lists(hydro_ctx *c, hydro_nbrlist *out, stream_t st);

// density.cu
// compact: shrink each solved particle's list to its root (hydro_step only)
// guard: a guard round's solve, whose particles are all in the round's
// guard list (walked instead of every particle)
cudaError_t run_density(hydro_ctx *c, bool only_active, bool compact, stream_t st,
                        bool guard = false);
cudaError_t grow_search_radius(hydro_ctx *c, stream_t st, bool guard = false);

// gradients.cu
// only_guard: the particles of the current guard round (their omega changed)
cudaError_t run_primitives(hydro_ctx *c, stream_t st, bool only_guard = false);
// the caller's acceleration into sorted order (no-op without one)
cudaError_t gather_gravity(hydro_ctx *c, stream_t st);
// the caller's entropic function into sorted order (no-op with the switch off)
cudaError_t gather_entropy(hydro_ctx *c, stream_t st);

// rungs.cu (individual timesteps)
// sorted rung, "starts a step now" and time since the state was taken at
// sub-step k of 2^rmax (the starting particles' start moves to k)
cudaError_t rung_prep(hydro_ctx *c, int64_t k, int rmax, double dtmin, stream_t st);
// N_NGB restarted and the density solve flag for the starting particles
cudaError_t rung_fill(hydro_ctx *c, stream_t st);
// save: the starting particles' records to the caller-order store; load:
// the others' records (all but the positions) from it
cudaError_t rung_records(hydro_ctx *c, bool save, stream_t st);
// rung from the two criteria (gradient stage outputs), then limiter sweeps
cudaError_t rung_assign(hydro_ctx *c, double dt0, stream_t st);
cudaError_t rung_limit_sweep(hydro_ctx *c, stream_t st);
// sorted rungs to the caller-order master copy (and the deepest rung)
cudaError_t rung_scatter(hydro_ctx *c, stream_t st);
// the buckets holding a particle flagged ACT_REDO into d_ovf (count in
// ovf_buckets)
cudaError_t queue_flagged(hydro_ctx *c, uint8_t bits, stream_t st);
// only_redo: recompute only the particles whose list holds a particle that
// the guard re-solved (ACT_GUARD), keeping every other particle's results
// reduce: also the global dt and pair count (grad_reduce); the step's
// guard loops take them once, after their last round
cudaError_t run_gradients(hydro_ctx *c, double *B_out, double *grad_out, double *alpha_out,
                          double *ncond_out, bool only_redo, stream_t st, bool reduce = true);
cudaError_t grad_reduce(hydro_ctx *c, stream_t st);
cudaError_t guard_grow(hydro_ctx *c, stream_t st);
cudaError_t load_gradients(hydro_ctx *c, const double *B, const double *grad,
                           const double *alpha, stream_t st);

// fluxes.cu
cudaError_t run_fluxes(hydro_ctx *c, double dt, const double *dt_dev, stream_t st);
// the adaptive learned-path choice for the next flux call (host state)
bool decide_learned(hydro_ctx *c);
// collect the time of a pending probe call before other flux calls reuse
// its events (waits for the probe's events)
void read_learn_probe(hydro_ctx *c);

// api.cu: shared by the host-driven and the graph step
int flags_to_status(int flags);
cudaError_t reset_guard(hydro_ctx *c, stream_t st);   // N_NGB = n_ngb, every particle active
void fill_stats(hydro_ctx *c, double dt, bool timing); // last_stats from h_cnt and the events
// the overflow region of the lists asked for entries up to `cursor`: keep
// room for that (and a quarter more) from the next list build on
void grow_overflow(hydro_ctx *c, unsigned long long cursor);

// graph.cu: hydro_step as one captured graph; returns HYDRO_* (a positive
// value asks the caller to run the host-driven step instead)
int graph_step(hydro_ctx *c, hydro_particles *p, double dt, hydro_stats *stats, stream_t st);
void graph_release(hydro_ctx *c);

// mlp.cu (bytes of the packed weight tiles; faces are float [6 or 7][n])
constexpr size_t MLP_BLOB_BYTES = 11264;
cudaError_t mlp_pack(hydro_ctx *c, stream_t st);
cudaError_t mlp_predict(hydro_ctx *c, const float *faces, int64_t n, float *out, stream_t st);
cudaError_t mlp_features(hydro_ctx *c, const float *faces, int64_t n, float *x, float *t,
                         stream_t st);
cudaError_t mlp_gradient(hydro_ctx *c, const float *x, const float *t, int64_t n, int64_t nb,
                         int random, uint64_t seed, uint64_t step, int quant, float *grad,
                         float *loss, stream_t st);
cudaError_t mlp_adam(hydro_ctx *c, float *grad, float *m, float *v, float lr, int step,
                     stream_t st);
cudaError_t mlp_normalise(hydro_ctx *c, const float *x, const float *t, int64_t n, double *acc,
                          int *box, stream_t st);

// update.cu (abort_check: skip the update when the device step set an abort
// condition -- see graph.cu; skip_flags: status bits whose presence leaves
// the caller's state untouched)
cudaError_t run_update(hydro_ctx *c, hydro_particles *p, double dt, const double *dt_dev,
                       bool abort_check, int skip_flags, stream_t st);
// status bits after which hydro_step leaves the caller's state as it was
// A warp's next chunk of a device-sized list: 32 entries taken from a
// global cursor (reset by the launcher), so the warps of a persistent grid
// share the list as they come free -- the entries' costs vary (list lengths,
// Newton iterations) and a fixed share per thread would leave the grid
// waiting on its slowest threads.  Returns the chunk's first entry (>= nl:
// the list is done); every lane of the warp calls it.
__device__ __forceinline__ int warp_chunk(int *cursor) {
    int base = 0;
    if ((threadIdx.x & 31) == 0) base = atomicAdd(cursor, 32);
    return __shfl_sync(0xffffffffu, base, 0);
}

// grid of the sweeps that test a flag of every particle and act on few of
// them (the guard rounds' passes): 16 CTAs per SM of the 152, the threads
// striding over the particles, instead of a CTA per 128-256 particles.
// (Wider CTAs of 1024 threads were slower: a CTA holds its SM until its
// slowest warp is done.)
constexpr unsigned SWEEP_GRID = 152 * 16;
constexpr int STEP_SKIP_FLAGS = ST_NOCONV_H | ST_MLP;
// *p = v on the stream (a kernel: no host memory is referenced, so the call
// can be captured into a graph)
cudaError_t set_u64(unsigned long long *p, unsigned long long v, stream_t st);
cudaError_t run_sums(hydro_ctx *c, int which, stream_t st);
cudaError_t ensure_sum_partials(hydro_ctx *c);
cudaError_t run_check_inputs(hydro_ctx *c, const hydro_particles *p, stream_t st);
cudaError_t export_dQ(hydro_ctx *c, double *dQ, stream_t st);

}  // namespace hyd

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace hyd {

__device__ __forceinline__ void set_flag(DevCounters *c, int bit) { atomicOr(&c->flags, bit); }

// one fold of a separation into [-L/2, L/2]; exact IEEE operations only
__device__ __forceinline__ double fold64(double d, double L) {
    double half = __dmul_rn(0.5, L);
    if (d > half) return __dsub_rn(d, L);
    if (d < -half) return __dadd_rn(d, L);
    return d;
}

// r^2 = (dx^2 + dy^2) + dz^2 rounded step by step (no contraction)
__device__ __forceinline__ double r2_exact(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// int32 -> float for |k| < 2^22 by placing k in the mantissa of 1.5 * 2^23:
// an integer add and a float subtract instead of a conversion instruction
// (conversions share GB300's narrow FP64 pipe)
__device__ __forceinline__ float i2f_small(int32_t k) {
    return __int_as_float(0x4B400000 + k) - 12582912.0f;
}

// float -> double from the bit pattern with integer operations only (the
// conversion instruction runs on the FP64 pipe): exact for normal floats,
// infinities and NaNs; zeros and subnormals (below 1.2e-38) become signed 0
__device__ __forceinline__ double widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t ex = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned long long man = (unsigned long long)(u & 0x7fffffu) << 29;
    const unsigned long long e64 = ex == 0xffu ? 0x7ffull : (unsigned long long)(ex + 896u);
    const unsigned long long b = ex == 0u ? sign : (sign | (e64 << 52) | man);
    return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double widen(double f) { return f; }

// double -> float rounded to nearest even with integer operations only
// (the conversion instruction runs on the FP64 pipe); results outside the
// normal float exponents 1..253 (zeros, subnormals, the largest floats,
// infinities, NaNs) take the conversion instruction
__device__ __forceinline__ float narrow(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t ex = (hi >> 20) & 0x7ffu;
    if (ex - 897u >= 253u) return (float)d;
    const uint32_t keep = ((hi & 0xfffffu) << 3) | (lo >> 29);   // the top 23 of 52 bits
    const uint32_t rest = lo & 0x1fffffffu;                      // the 29 dropped
    uint32_t b = ((ex - 896u) << 23) + keep;   // (a carry out of keep moves the exponent)
    b += rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u));
    return __uint_as_float(b | (hi & 0x80000000u));
}

// minimum-image separation b - a of two fixed-point coordinates, times the
// unit s: the 32-bit difference split as hi * 2^11 + lo, each part exact
__device__ __forceinline__ float qdiff(uint32_t a, uint32_t b, float s) {
    int32_t d = (int32_t)(b - a);
    int32_t hi = d >> 11;
    int32_t lo = d & 0x7FF;
    return fmaf(i2f_small(hi), s * 2048.0f, i2f_small(lo) * s);
}

// Kernel normalised sums used by the density iteration:
//   (4 pi / 3) h^3 W(r, h) = Kn * f(q),  h dW/dh-term: d/dh [Kn f(q)] = Kn f'(q) (-q/h)
// Wendland C2: W = 21/(2 pi H^3) (1-q)^4 (1+4q)  -> Kn = 14
// cubic M4:    W = 8/(pi H^3) {1-6q^2+6q^3 ; 2(1-q)^3} -> Kn = 32/3
template <typename R>
__device__ __forceinline__ void kernel_f(int kernel, R q, R &f, R &mqfp) {
    // f(q) and -q f'(q)
    if (q >= R(1)) { f = R(0); mqfp = R(0); return; }
    if (kernel == 0) {
        R t = R(1) - q;
        R t3 = t * t * t;
        f = t3 * t * (R(1) + R(4) * q);
        mqfp = R(20) * q * q * t3;
    } else {
        if (q <= R(0.5)) {
            f = R(1) - R(6) * q * q + R(6) * q * q * q;
            mqfp = R(12) * q * q - R(18) * q * q * q;
        } else {
            R t = R(1) - q;
            f = R(2) * t * t * t;
            mqfp = R(6) * q * t * t;
        }
    }
}

template <typename R>
__device__ __forceinline__ R kernel_Kn(int kernel) {
    return kernel == 0 ? R(14) : R(32.0 / 3.0);
}

// W(r, H) / norm where norm = 21/(2 pi H^3) (Wendland) or 8/(pi H^3) (cubic)
template <typename R>
__device__ __forceinline__ R kernel_shape(int kernel, R q) {
    if (q >= R(1)) return R(0);
    if (kernel == 0) {
        R t = R(1) - q;
        R t2 = t * t;
        return t2 * t2 * (R(1) + R(4) * q);
    }
    if (q <= R(0.5)) return R(1) - R(6) * q * q + R(6) * q * q * q;
    R t = R(1) - q;
    return R(2) * t * t * t;
}

template <typename R>
__device__ __forceinline__ R kernel_norm(int kernel, R H) {
    const R pi = R(3.14159265358979323846);
    R H3 = H * H * H;
    return kernel == 0 ? R(21) / (R(2) * pi * H3) : R(8) / (pi * H3);
}

__device__ __forceinline__ double ordered_min_bits(double v) { return v; }

}  // namespace hyd
#endif

#define HYD_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e__ = (call);                                   \
        if (e__ != cudaSuccess) return e__;                         \
    } while (0)
