/*
 * hydro.h -- C ABI of the GB300 (sm_103a) MFV/MFM hydro step.
 *
 * The method is the mesh-less finite-volume / finite-mass scheme of
 * arXiv:2211.12243 ("Mesh-free hydrodynamics in pkdgrav3 for galaxy
 * formation simulations"), §2.2.3 and §2.3: a bucketed neighbour search,
 * kernel density and smoothing-length sums (Eqs. 5-7, 18), the
 * Lanson-Vila gradient with its E matrix and condition-number guard
 * (Eqs. 10-11, 19), slope limiters (§2.3.6), and per-pair Riemann fluxes
 * through the effective face A_ij (Eq. 13 and the definition after it),
 * scattered antisymmetrically (Eqs. 15-16) so that mass, momentum and energy
 * are conserved by construction.
 *
 * Conventions that hold for every entry point:
 *   - Every pointer argument documented as "device" is caller-owned device
 *     memory of the context's GPU; the library never frees it.  Host pointers
 *     are read before the call returns.
 *   - Particle arrays are structure-of-arrays in the CALLER's order; outputs
 *     are written in the caller's order too (the library sorts internally
 *     and un-permutes).
 *   - Calls are asynchronous on the given stream unless stated otherwise.
 *     They return a hydro_status; errors detected on the device are
 *     collected in a status word read by hydro_sync_status() (and by
 *     hydro_step when it is given a stats pointer).  No call aborts or
 *     throws across the ABI.
 *   - All particles must lie in [0, L) of their periodic box.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hydro_ctx hydro_ctx;       /* opaque: scratch, box plan, MLP */
typedef struct CUstream_st *hydro_stream; /* a cudaStream_t (NULL = legacy default) */

typedef enum {
    HYDRO_OK = 0,
    HYDRO_EINVAL = -1,      /* bad argument (NULL pointer, size mismatch, ...) */
    HYDRO_ENOMEM = -2,      /* device allocation failed */
    HYDRO_ECAPACITY = -3,   /* caller's neighbour-list buffer too small; needed set */
    HYDRO_ENOCONV_H = -4,   /* smoothing-length iteration did not converge */
    HYDRO_ENCOND = -5,      /* N_cond above threshold after all N_NGB growths */
    HYDRO_ERIEMANN = -6,    /* Riemann iteration failed (after bisection) */
    HYDRO_ENONFINITE = -7,  /* non-finite value produced or given */
    HYDRO_ECUDA = -8,       /* CUDA runtime error */
    HYDRO_ESTATE = -9,      /* call order violated (e.g. density before lists) */
    HYDRO_ESEARCH = -10,    /* a solved h exceeded the search radius of the lists */
    HYDRO_EMLP = -11        /* a tensor-core wait of the MLP gave up (result unusable) */
} hydro_status;

enum { HYDRO_KERNEL_WENDLAND_C2 = 0, HYDRO_KERNEL_CUBIC = 1 };
enum { HYDRO_MFV = 0, HYDRO_MFM = 1 };
enum { HYDRO_RIEMANN_EXACT = 0, HYDRO_RIEMANN_HLLC = 1 };
enum { HYDRO_FP64 = 0, HYDRO_MIXED = 1 };

/* Method parameters.  hydro_config_default() fills the values used by the
 * paper where it states them (N_cond threshold 100 and growth 1.2, §2.3.5;
 * pairwise limiter psi1 = 0.5, psi2 = 0.25, §2.3.6; alpha1 = 1/100 and
 * alpha2 = alpha3 = 1/1000, §2.3.7)
 * and this library's readings elsewhere. */
typedef struct {
    double gamma;        /* adiabatic index */
    int kernel;          /* HYDRO_KERNEL_*; compact support radius H = h */
    double n_ngb;        /* N_NGB of Eq. 18 */
    int scheme;          /* HYDRO_MFV or HYDRO_MFM (§2.3.3) */
    int riemann;         /* HYDRO_RIEMANN_EXACT (Toro 2009) or _HLLC */
    int precision;       /* HYDRO_FP64: every step in double.
                            HYDRO_MIXED: pair geometry, kernel sums and fluxes in
                            float; E^-1, h refinement and flux accumulation in
                            double-class precision. */
    int learned_guess;   /* MLP starting pressure for the exact solver on hard
                            faces (mixed precision; needs a network from
                            hydro_mlp_load / hydro_mlp_train, else the flux
                            calls return HYDRO_ESTATE; FP64 and HLLC ignore it):
                            0 off; 2 on in every flux call; 1 adaptive: one
                            flux call (hydro_fluxes or hydro_step) with the
                            learned path, one with the plain guess, both timed
                            with CUDA events, then 15 calls with the learned
                            path if more than 10% of its hard faces started
                            from the network and it was the faster, else with
                            the plain guess; then the two probes again */
    int limiter;         /* 1: conditioned BJ + pairwise limiters (§2.3.6) */
    int time_extrap;     /* 1: half-step predictor of the face states (Eq. 16) */
    double ncond_crit;   /* N_cond threshold (100) */
    double ngb_grow;     /* N_NGB growth factor on failure (1.2) */
    int max_ngb_grow;    /* growth rounds before HYDRO_ENCOND (5) */
    double psi1, psi2;   /* pairwise limiter (0.5, 0.25) */
    double beta_min, beta_max; /* conditioned BJ (1, 2) */
    double c_cfl;        /* CFL factor of Eq. 31 (0.2) */
    double alpha1;       /* total-energy pressure switch (1/100) */
    double h_tol;        /* relative Newton tolerance on h (1e-10) */
    double p_tol;        /* relative Newton tolerance on p* (1e-12 FP64) */
    int max_h_iter;      /* cap on the h iteration (60) */
    int max_newton;      /* cap on Riemann Newton iterations (100) */
    double search_margin;/* hydro_step: search radius = margin * h_in (1.15) */
    int graph;           /* hydro_step: 1 (default) runs the step as one captured
                            CUDA graph whose re-search and N_cond loops are
                            device-side WHILE nodes (no host waits inside the
                            step); the first step of a context, and a step that
                            must grow a buffer, run host-driven.  0: host-driven. */
    int entropy_switch;  /* hydro_step: 1 evolves the entropic function A of
                            §2.3.7 (held by hydro_set_entropy) and takes the
                            pressure from it where the flow is cold relative
                            to its kinetic or gravitational energy (0: off) */
    double alpha2;       /* entropy route when U < alpha2 (E_kin^max + U) (1/1000) */
    double alpha3;       /* ... or when U < alpha3 E_grav (1/1000) */
    double c_acc;        /* hydro_step_rungs: acceleration timestep factor,
                            dt_acc = c_acc sqrt(h / |a|) (§2.3.10; 0.2) */
    int max_rung;        /* hydro_step_rungs: deepest rung (12, at most 20) */
    int riemann_polish;  /* mixed precision, exact solver: 1 takes one more
                            Newton step of Toro's pressure function in FP64
                            once the float iteration has converged, so p* and
                            u* are the roots of the (float) face states to
                            double precision before they are rounded to float
                            for the flux; 0 (default): the float iteration
                            alone (its root is within a few float ulps) */
    int sorted_output;   /* hydro_step: 1 writes the particles back in the
                            step's own (Morton) order instead of the caller's:
                            after the step, index i of every array of
                            hydro_particles (and the entropy array of
                            hydro_set_entropy) holds the particle that was at
                            index perm[i] of the input, perm from hydro_get_order.
                            A state kept in that order is read and written
                            by the next step with coalesced accesses (the
                            caller's order is otherwise unrelated to the
                            sort, and the gathers and the write-back scatter).
                            The gravity array of hydro_set_gravity is input
                            only: the caller reorders it.  hydro_step_rungs
                            returns HYDRO_ESTATE while it is set.  A step
                            that returns an error leaves the arrays in their
                            input order.  0 (default): caller order. */
} hydro_config;

/* Caller-owned particle state, caller order, all device pointers, n each.
 * Conserved variables of Eq. 2 integrated over the particle volume:
 * mass, momentum (px, py, pz), total energy etot, internal energy eint
 * (Eq. 24).  h: compact-support radius (in: guess, out: solved);
 * omega: particle volume V_i = omega_i (out). */
typedef struct {
    int64_t n;
    double *x, *y, *z;
    double *mass, *px, *py, *pz, *etot, *eint;
    double *h, *omega;
} hydro_particles;

/* Neighbour lists in CSR form (device memory, caller order):
 * row i = { j : r_ij < h_search_i } including j = i, ascending j.
 * off has n+1 entries; idx has `capacity` entries.  `needed` receives the
 * total entry count (also when it exceeds capacity, in which case nothing
 * is written to idx and HYDRO_ECAPACITY is returned). */
typedef struct {
    int64_t *off;
    int32_t *idx;
    int64_t capacity;
    int64_t needed;
} hydro_nbrlist;

/* Per-step diagnostics (host struct filled by hydro_step / hydro_get_stats). */
typedef struct {
    int status;               /* device status word of the last step */
    double dt;                /* timestep used */
    double dt_next;           /* CFL estimate from the start-of-step state */
    int64_t grad_pairs;       /* directed pairs j != i, r_ij < h_i (gradient stage) */
    int64_t flux_pairs;       /* unordered pairs r_ij < max(h_i, h_j) (flux stage) */
    int64_t newton_iters;     /* Riemann Newton iterations summed over faces */
    int64_t guess_fallbacks;  /* hard faces that kept the plain guess: learned value
                                 out of range, a correction |y| < 1e-3 (kept at the
                                 two-shock value), or no room to defer the face */
    int64_t learned_faces;    /* faces whose Newton iteration started from the MLP */
    int64_t hard_faces;       /* faces where Toro's guess is the two-shock value
                                 (counted when the learned path ran) */
    int learned_active;       /* 1 if the step's fluxes ran the learned path */
    int64_t vacuum_faces;
    int64_t first_order_faces;
    int ngb_rounds;           /* N_cond growth rounds taken */
    int64_t ncond_fail;       /* particles above the threshold at the end */
    int list_rebuilds;        /* neighbour-list rebuilds for h beyond the radius */
    double mass[2], mom[2][3], energy[2];   /* totals of the state before / after the
                                 step: double sums in a fixed order over the
                                 particles (rounding below 1e-13 of sum |x| at
                                 2^27 particles), so any difference is the
                                 step's (fluxes and external sources) */
    float ms_sort;            /* 0: the sort is timed within ms_neighbours */
    float ms_neighbours, ms_density, ms_gradients, ms_fluxes, ms_update;
                              /* stage times (CUDA events on the stream; ms_neighbours:
                                 the sort, gathers, tree and lists; ms_gradients:
                                 primitives, gradients and the N_cond guard rounds) */
    float ms_flux_kernel;     /* the pair-flux kernel alone (CUDA events on the stream) */
    float ms_hard_faces;      /* the learned-guess hard-face kernel (0 when off) */
    int graph;                /* 1: the step ran as the captured graph; 0: host-driven
                                 (graph off, or the context's first step); 2: the
                                 graph step needed a larger buffer, the host-driven
                                 step redid it and grew the buffer; 3: a capture
                                 failed, this context runs host-driven from now on */
    float learned_probe_ms[2];/* learned_guess = 1: flux-stage times of the last plain
                                 and learned probe calls (CUDA events; 0 before) */
    /* hydro_step_rungs (0 after hydro_step): */
    int rung_max;             /* the deepest rung of the base step */
    int64_t substeps;         /* 2^rung_max */
    int64_t active_steps;     /* particle steps taken, sum_i 2^rung_i */
    int64_t rung_capped;      /* particles whose criteria asked for more than max_rung */
    int64_t rung_sparse;      /* sub-steps that rebuilt and walked only the lists of the
                                 buckets within reach of the starting particles */
} hydro_stats;

/* Defaults described above.  Always succeeds. */
void hydro_config_default(hydro_config *cfg);

/* Create a context on the current CUDA device.  HYDRO_EINVAL on bad config. */
int hydro_create(hydro_ctx **ctx, const hydro_config *cfg);
void hydro_destroy(hydro_ctx *ctx);

/* Replace the method parameters (the box plan and scratch are kept). */
int hydro_set_config(hydro_ctx *ctx, const hydro_config *cfg);

/* Define the independent periodic boxes the particles live in.
 * box_off: host, nbox+1 ascending offsets with box_off[0] = 0 -- particles
 * box_off[k] .. box_off[k+1]-1 (caller order) belong to box k (each box
 * holds at least one particle).  box_len: host, 3*nbox lengths Lx, Ly, Lz.
 * One box is the common case: nbox = 1, box_off = {0, n}.
 * Plans the bucket tree topology and allocates its storage (synchronous). */
int hydro_set_boxes(hydro_ctx *ctx, int64_t nbox, const int64_t *box_off,
                    const double *box_len);

/* Pre-allocate every per-particle scratch buffer for up to max_n particles
 * and `nbr_per_particle` candidate entries per particle, so that later calls
 * allocate nothing (synchronous).  Optional: calls grow scratch on demand. */
int hydro_reserve(hydro_ctx *ctx, int64_t max_n, int nbr_per_particle);

/* §2.2.3 bucketed neighbour search.  Sorts the particles along a Morton
 * curve, cuts buckets of 32, and lists for every particle all j with
 * r_ij < h_search_i (device, n doubles, caller order; minimum-image distance
 * r_ij^2 = (dx^2 + dy^2) + dz^2 in double, dx folded once into
 * [-L/2, L/2]).  The lists stay in the context for the next calls.
 * out (optional, may be NULL): the same lists exported in caller order,
 * rows ascending. */
int hydro_build_neighbours(hydro_ctx *ctx, const hydro_particles *p,
                           const double *h_search, hydro_nbrlist *out,
                           hydro_stream stream);

/* §2.3.2 / §2.3.5: solve (4 pi / 3) h_i^3 omega_i^-1 = N_NGB (Eq. 18) with
 * omega_i^-1 = sum_j W(r_ij, h_i) (Eq. 6, self term included), starting
 * from p->h, over the lists of the last hydro_build_neighbours.  Writes
 * p->h and p->omega.  A root beyond the list radius is HYDRO_ESEARCH
 * (reported through the status word). */
int hydro_density(hydro_ctx *ctx, hydro_particles *p, hydro_stream stream);

/* §2.3.3 / §2.3.6: primitives (rho = m/omega, v = P/m, p from Eq. 23 or the
 * internal energy), E_i (Eq. 11, weight omega_j, W(r, h_i)), B_i = E_i^-1,
 * N_cond,i (Eq. 19), the gradients of (rho, vx, vy, vz, p) (Eq. 10) and the
 * conditioned Barth-Jespersen factors.  Outputs, device, caller order:
 * B[6n] (xx, xy, xz, yy, yz, zz), grad[15n] (per particle: d rho/dx..dz,
 * d vx/dx..dz, d vy, d vz, d p), alpha[5n], ncond[n]; any may be NULL.
 * Requires p->h, p->omega (e.g. from hydro_density) and lists covering h. */
int hydro_gradients(hydro_ctx *ctx, const hydro_particles *p, double *B, double *grad,
                    double *alpha, double *ncond, hydro_stream stream);

/* §2.3.3 / §2.3.4 / §2.3.6: for every unordered pair with
 * r_ij < max(h_i, h_j): the face vector A_ij, extrapolated and limited face
 * states, the Riemann problem in the frame moving with (v_i + v_j)/2, the
 * MFV or MFM flux, and c = dt |A_ij| F scattered as dQ_i -= c, dQ_j += c.
 * Inputs B, grad, alpha as produced by hydro_gradients (device, caller
 * order).  dt > 0.  Output dQ[6n] (device, caller order): dm, dpx, dpy,
 * dpz, dE, dU (dU from Eq. 24 with the start-of-step velocity). */
int hydro_fluxes(hydro_ctx *ctx, const hydro_particles *p, const double *B,
                 const double *grad, const double *alpha, double dt, double *dQ,
                 hydro_stream stream);

/* One full step: neighbour search with radius search_margin * h, density
 * (re-searching when a root leaves the radius), the N_cond guard
 * (N_NGB,i *= ngb_grow, density redone, §2.3.5), gradients, fluxes with the
 * given dt (dt <= 0: CFL dt = min_i c_cfl h_i / v_sig,i, Eqs. 31-32),
 * conserved update (Eq. 16), internal energy (Eq. 24) and drift
 * x += dt (v^n + v^{n+1}) / 2 wrapped into the box.  Updates p in place.
 * stats (host, optional): filled after a stream synchronisation.
 * Errors that leave p exactly as it was: a non-finite value anywhere in
 * the caller's state (HYDRO_ENONFINITE, found by a check before any other
 * work), an h iteration that did not converge within max_h_iter
 * (HYDRO_ENOCONV_H), a tensor-core wait of the learned guess that gave up
 * (HYDRO_EMLP).  HYDRO_ENCOND (particles still ill-conditioned after all
 * N_NGB growths) completes the step and reports them. */
int hydro_step(hydro_ctx *ctx, hydro_particles *p, double dt, hydro_stats *stats,
               hydro_stream stream);

/* One base step dt0 > 0 with individual timesteps (§2.3.4 power-of-two
 * hierarchy, §2.3.10 criteria).  At its start every particle is
 * synchronised: neighbours, density, guard, primitives and gradients as in
 * hydro_step; then its rung r_i, the smallest r >= 0 (at most max_rung)
 * with min(dt_CFL,i, dt_acc,i) > 2^-r dt0, where dt_CFL is Eq. 31's
 * per-particle value and dt_acc = c_acc sqrt(h_i / |a_i|) with
 * a_i = -grad p_i / rho_i (the limited pressure gradient of the face
 * reconstruction); then the neighbour limiter |r_i - r_j| <= 2 over the
 * flux pairs (rungs only rise, to the least such assignment).  Rungs stay
 * fixed over the base step, which runs 2^rmax sub-steps of dt0 2^-rmax.
 * At sub-step k the particles with k divisible by 2^(rmax - r_i) start a
 * step of dt_i = dt0 2^-r_i: their neighbours, density, guard,
 * primitives and gradients are recomputed at the current positions; the
 * others keep those of their last start (h, omega, primitives, B and
 * gradients as they were).  Every flux pair with an active particle
 * exchanges c = dt_ij |A_ij| F with dt_ij = min(dt_i, dt_j), subtracted
 * from one particle and added to the other (Springel 2010 §7.2); each
 * side's state is predicted (Eq. 16's half step) over the time since its
 * start plus dt_ij / 2.  Every particle then takes what it received (U by
 * Eq. 24 with its current velocity) and drifts by the sub-step with the mean
 * of its velocities before and after.  rung (device, n int32, caller order,
 * out): the rungs used.  Host-driven (not a captured graph); plain Riemann
 * guess (learned_guess is not used); an external acceleration
 * (hydro_set_gravity) or the entropy switch give HYDRO_ESTATE.  On an error
 * the state holds the sub-steps completed before it.  stats (host,
 * optional): counters summed over the sub-steps, totals before the first
 * and after the last, dt = dt0, dt_next = the smallest CFL dt at the start,
 * rung_max, substeps, active_steps, rung_capped. */
int hydro_step_rungs(hydro_ctx *ctx, hydro_particles *p, double dt0, int32_t *rung,
                     hydro_stats *stats, hydro_stream stream);

/* Read (synchronising the stream) and clear the device status word:
 * returns the first error recorded by any kernel since the last read. */
int hydro_sync_status(hydro_ctx *ctx, hydro_stream stream);

/* Statistics of the last hydro_step (host copy, synchronising); the flux
 * counters (flux_pairs, newton_iters, guess_fallbacks, learned_faces,
 * hard_faces, vacuum_faces, first_order_faces) are re-read from the device,
 * so after hydro_fluxes they describe that call. */
int hydro_get_stats(hydro_ctx *ctx, hydro_stats *stats, hydro_stream stream);

/* Install the weights of the star-pressure MLP (12 -> 64 -> 64 -> 1) used
 * when cfg.learned_guess = 1.  `weights`: host, `bytes` = 4 * (12*64 + 64 +
 * 64*64 + 64 + 64 + 1 + 24 + 2 + 24) = 4 * 5115, float32 values in the order
 * W1, b1, W2, b2, w3, b3, feature mean[12], feature scale[12], t_mean,
 * t_scale, feature box xmin[12], xmax[12] (row-major, W[out][in]); output
 * y = t_mean + t_scale (w3 . h2 + b3).  HYDRO_EINVAL on a non-finite value,
 * a scale <= 0 or xmin > xmax.  Synchronous. */
int hydro_mlp_load(hydro_ctx *ctx, const void *weights, size_t bytes);

/* ---- Learned starting pressure of the exact Riemann solver -------------
 * Not part of the paper's method: the paper solves each face's Riemann
 * problem with the exact iterative solver of Toro (2009), whose Newton
 * iteration starts from Toro's adaptive guess (PVRS, two-rarefaction or
 * two-shock value).  These calls train and run a 12 -> 64 -> 64 -> 1 ReLU
 * network on 12 features of the face problem (log pressure and density
 * ratios to p_a = (p_L + p_R)/2 and rho_a, the velocity jump over the mean
 * sound speed, sound-speed ratios, and the PVRS, two-rarefaction and
 * two-shock values p_PVRS, p_TR, p_TS over p_a).  Its output y is a
 * correction of the two-shock value: target ln(p* / p_TS), starting
 * pressure p_TS exp(y).  With cfg.learned_guess = 1 (mixed precision,
 * exact solver), the faces where Toro's guess is the two-shock value
 * ("hard" faces: not the PVRS value, and p_PVRS >= min(p_L, p_R) so not
 * the two-rarefaction value, which is exact for two rarefactions) start
 * from the network's value unless it is out of range; the iteration
 * always runs to p_tol, so the flux is unchanged beyond rounding.
 *
 * Face problems are float arrays in rows of n (structure of arrays):
 * rho_L, u_L, p_L, rho_R, u_R, p_R [, p*], u along the face normal, in the
 * frame of the face.  Inference runs on the tensor cores (BF16 operands,
 * FP32 accumulation); training keeps FP32 master weights.
 * ----------------------------------------------------------------------- */

/* Copy the current float parameters (layout of hydro_mlp_load) to the host
 * buffer `weights` (bytes as in hydro_mlp_load).  HYDRO_ESTATE without a
 * network.  Synchronous. */
int hydro_mlp_get(hydro_ctx *ctx, void *weights, size_t bytes);

/* Predicted starting pressures: faces (device, 6 rows of n floats) ->
 * p_guess (device, n floats), -1 where the prediction is out of range (a
 * feature outside the box [xmin, xmax] of the training data, or a
 * correction |y| > 2, or not finite).  HYDRO_ESTATE without a network. */
int hydro_mlp_predict(hydro_ctx *ctx, const float *faces, int64_t n, float *p_guess,
                      hydro_stream stream);

/* Features x (device, n x 12 floats, row-major) and targets
 * t = ln(p_star / p_TS) (device, n floats) of recorded faces (device, 7 rows
 * of n floats). */
int hydro_mlp_features(hydro_ctx *ctx, const float *faces, int64_t n, float *x, float *t,
                       hydro_stream stream);

/* Gradient of the loss 0.5 mean_i (y_i - t_i)^2 over all n samples (x:
 * device n x 12, t: device n) with respect to the current parameters,
 * written to grad (device, 5115 floats in the hydro_mlp_load layout; the
 * entries of the fixed standardisations are 0) and the loss to *loss
 * (device, 1 float).
 * quant = 1 rounds the standardised inputs, W1, the hidden activations and
 * W2 to bf16 in the forward pass as the tensor-core inference does (the
 * backward pass differentiates through the rounded values as if the
 * rounding were the identity).  HYDRO_ESTATE without a network. */
int hydro_mlp_gradient(hydro_ctx *ctx, const float *x, const float *t, int64_t n, int quant,
                       float *grad, float *loss, hydro_stream stream);

/* Train on recorded faces (device, 7 rows of n floats): `steps` Adam steps
 * (beta 0.9 / 0.999) on minibatches of `batch` samples drawn with a
 * counter-based generator from `seed`, learning rate lr, bf16-rounded
 * forward pass.  Without a loaded network, first initialises one (He
 * normal from `seed`) and sets the feature and target standardisations and
 * the feature box from the data; with one, continues training it.  Samples
 * with a non-finite feature or target are skipped.  The learning rate decays
 * from lr to lr/20 along a cosine.  loss (device, `steps` floats, may be
 * NULL) receives the minibatch loss of each step. */
int hydro_mlp_train(hydro_ctx *ctx, const float *faces, int64_t n, int64_t steps,
                    int64_t batch, double lr, uint64_t seed, float *loss,
                    hydro_stream stream);

/* Record solved face problems of the following hydro_fluxes / hydro_step
 * calls (mixed precision, exact solver) into buf (device, 7 rows of
 * `capacity` floats: rho_L, u_L, p_L, rho_R, u_R, p_R, p*).  A face is kept
 * when a hash of its particle pair falls below keep_fraction (0..1], and,
 * with hard_only = 1, only when it is a hard face.  buf = NULL stops the
 * recording.  Only faces with positive densities and pressures on both
 * sides and p* > 0 are recorded.  Resets the recorded count (synchronous). */
int hydro_record_faces(hydro_ctx *ctx, float *buf, int64_t capacity, double keep_fraction,
                       int hard_only);

/* Number of faces that qualified since hydro_record_faces (those beyond
 * capacity were not stored).  Synchronising. */
int hydro_recorded_faces(hydro_ctx *ctx, int64_t *count, hydro_stream stream);

/* Test hook of the learned guess's error path (no counterpart in the
 * paper).  With on = 1 the network's kernels of this context (the
 * hard-face pass of hydro_step and hydro_mlp_predict) do not issue the copy
 * of the weights into shared memory, so the wait on its barrier can never
 * finish: it gives up after a short poll limit (about 0.3 ms), the kernel
 * records HYDRO_EMLP, releases its tensor memory (nothing is in flight) and
 * every face keeps the plain guess.  hydro_step then returns HYDRO_EMLP and
 * leaves the state untouched; hydro_sync_status reports it after
 * hydro_mlp_predict.  on = 0 restores the normal path.  EINVAL otherwise. */
int hydro_test_mlp_stall(hydro_ctx *ctx, int on);

/* Totals over the n particles of mass, px, py, pz and etot (compensated
 * sums), written to totals[0..4] (device), computed without allocating
 * anything and without a context.  For callers that cannot call cudaMalloc
 * -- a host application that owns every device allocation through its own
 * pool, or a plugin that must not change the device memory footprint once
 * it runs -- to check conservation around hydro_step.  No counterpart in
 * the paper: a utility of this library.
 * Inputs: device arrays of n doubles (caller order, any order works).
 * Limit: n <= 2^26 (67,108,864); larger n returns HYDRO_EINVAL.
 * Scratch: a fixed 640 KiB array in the library's static device memory,
 * held by every GPU that loads the library until the process exits.  The
 * first call on a device looks up that array's device address (once per
 * device, with the device current) and later calls reuse it, so make that
 * first call before capturing any stream, and do not call the entry point
 * again after cudaDeviceReset in the same process (the reset unloads the
 * array; the remembered address would be stale).  All calls share
 * the array: each overwrites the part it uses, so nothing needs clearing,
 * but calls that overlap on the GPU race on it.  Asynchronous on stream. */
int hydro_totals_noalloc(int64_t n, const double *mass, const double *px, const double *py,
                         const double *pz, const double *etot, double *totals,
                         hydro_stream stream);

/* An external (gravitational) acceleration for the following hydro_step
 * calls (§2.3.8): acc is a device array of 3 doubles per particle (ax, ay,
 * az; caller order), read at every step and held by pointer until replaced
 * (NULL: none; the caller keeps it alive).  The step, with a held fixed over
 * it, adds to the state the fluxes updated the sources integrated by the
 * trapezoidal rule of §2.3.4 between the start-of-step state U^n and that
 * state U~: momentum dt/2 (m^n + m~) a; total energy dt/2 (P^n + P~).a plus
 * the work on the exchanged mass, (1/2) a . sum_j dm_ij r_ij (dm_ij the mass
 * i gains from j through their face, r_ij = x_i - x_j; zero for MFM).  The
 * internal energy takes no source.  E_grav = m |a| h enters the
 * total-energy pressure switch (§2.3.7).  The totals in hydro_stats are
 * taken before and after the step, so their difference is the external
 * impulse and work (the fluxes conserve their part).  Always HYDRO_OK for a context. */
int hydro_set_gravity(hydro_ctx *ctx, const double *acc);

/* The entropic function A of the entropy switch (§2.3.7) for the following
 * hydro_step calls with cfg.entropy_switch = 1: A is a device array of n
 * doubles (caller order), read and rewritten by every step and held by
 * pointer until replaced (NULL: none; the caller keeps it alive).  Each
 * step takes the pressure of particle i from
 *   the total energy,     when U_i > alpha1 (E_grav,i + E_kin,i) and
 *                         E_i - E_kin,i > 0 (as without the switch);
 *   p = A_i rho_i^gamma,  else when A_i > 0 and U_i < alpha2 (E_kin^max,i +
 *                         U_i) or U_i < alpha3 E_grav,i;
 *   the internal energy,  otherwise;
 * with E_kin^max,i = max_j (1/2) m_i |v_j - v_i|^2 over the neighbours
 * j != i with r_ij < h_i at the step's h (0 without neighbours) and E_grav
 * as in hydro_set_gravity.  Where the energies gave the pressure, A_i is set
 * to p_i / rho_i^gamma (an entry <= 0 is unset and is set so).  A then stays
 * constant along MFM particles; in MFV the mass flux of each face carries
 * m A with the upwind value (the donor particle's A), so sum_i m_i A_i is
 * conserved and A_i^(n+1) = (m_i^n A_i + sum_j c_m,ij A_upwind) / m_i^(n+1).
 * The updated A is written back when the step completes.  hydro_step returns
 * HYDRO_ESTATE when the switch is on and no array is held.  Always HYDRO_OK
 * for a context. */
int hydro_set_entropy(hydro_ctx *ctx, double *A);

/* Launch parameters of the step that hydro_autotune chooses by timing the
 * candidates on the caller's own particles (no counterpart in the paper:
 * a property of this GPU implementation).  Candidates:
 *   search_margin x nbr_slots: the neighbour-list radius factor of
 *     hydro_step {1.05, 1.1, 1.15, 1.25} and the fixed list slots per
 *     particle {64, 96, 128} (longer lists take two extra passes into an
 *     overflow region), timed over sort + lists + density;
 *   grad_min_ctas: register bound of the gradient kernel (1: none; 4, 5, 6
 *     resident 128-thread CTAs per SM), timed over the gradient stage;
 *   flux_min_ctas: register bound of the float flux kernel (4, 5, 6),
 *     timed over the plain-guess flux stage (mixed precision only);
 *   flux_queue: the flux kernel's buckets one per warp by index (0) or
 *     drawn by persistent warps from a global cursor (1, the default: a
 *     warp done with a light bucket takes the next at once), timed over
 *     the same stage with the chosen bound (mixed precision only);
 *   grad_rank: the gradient kernel's particles taken in their order (0),
 *     or ranked by list length within tiles of 128 consecutive particles
 *     (1, the default: the lanes of a warp walk lists of similar length),
 *     or within tiles of 128 R (2: R = 8, or fewer while that leaves fewer
 *     than 8 CTAs per SM; the lengths even out further), timed over the
 *     gradient stage with the chosen bound; the full density solve ranks
 *     tiles of 128 when grad_rank is 1 or 2.
 * The times (ms, best of two) are returned beside the choices. */
typedef struct {
    double search_margin;
    int nbr_slots;
    int grad_min_ctas;
    int flux_min_ctas;
    float front_ms[4][3];     /* [margin][slots] */
    float grad_ms[4];         /* [1, 4, 5, 6] */
    float flux_ms[3];         /* [4, 5, 6]; 0 in FP64 */
    int flux_queue;
    float flux_queue_ms[2];   /* [by index, drawn]; 0 in FP64 */
    int grad_rank;
    float grad_rank_ms[3];    /* [in order, tiles of 128, larger tiles] */
} hydro_tuning;

/* Time the candidates above on the particles p (device, caller order; state
 * as for hydro_step) and keep the fastest in the context (search_margin
 * replaces the configured one).  The particles are read, never written.
 * `out` (host, may be NULL) receives the choices and times.  Synchronous.
 * Errors: HYDRO_EINVAL (no boxes / bad particles), HYDRO_ESTATE (learned
 * guess configured without a network), or any error a step would report. */
int hydro_autotune(hydro_ctx *ctx, hydro_particles *p, hydro_tuning *out, hydro_stream stream);

/* Apply choices saved from an earlier hydro_autotune (search_margin >= 1,
 * nbr_slots in [32, 256], grad_min_ctas in {1, 4, 5, 6}, flux_min_ctas in
 * {4, 5, 6}, flux_queue in {0, 1}, grad_rank in {0, 1, 2}; the time fields are
 * ignored).
 * HYDRO_EINVAL otherwise. */
int hydro_set_tuning(hydro_ctx *ctx, const hydro_tuning *t);

/* The order of the last hydro_step (no counterpart in the paper: a property
 * of the particle layout): perm[i] (device, n int32, caller-owned) receives
 * the input index of the particle the step placed at sorted position i --
 * with sorted_output, the index the particle had in the caller's arrays
 * before the step.  Enqueued on `stream`.  HYDRO_EINVAL (NULL), HYDRO_ESTATE
 * (no step taken yet). */
int hydro_get_order(hydro_ctx *ctx, int32_t *perm, hydro_stream stream);

/* Throughput of this GPU's arithmetic units, measured (no counterpart in the
 * paper: the denominators of the benchmark's roofline).  unit:
 * HYDRO_PROBE_FP32 float FMAs, HYDRO_PROBE_FP64 double FMAs (*value in
 * TFLOP/s, two flops per FMA), HYDRO_PROBE_MUFU reciprocal square roots on
 * the special-function unit (*value in T operations/s).  Independent FMA
 * (or rsqrt) chains on 8 blocks of 256 threads per SM, the best of three
 * timed launches (CUDA events on stream, synchronising).  Allocates and
 * frees a small device buffer.  EINVAL for another unit. */
enum { HYDRO_PROBE_FP32 = 0, HYDRO_PROBE_FP64 = 1, HYDRO_PROBE_MUFU = 2 };
int hydro_probe_peak(int unit, double *value, hydro_stream stream);

/* Number of kernels this library has launched in the process so far
 * (every entry point's launches, all contexts).  Diagnostics only. */
int64_t hydro_kernel_launches(void);

/* Human-readable message for a hydro_status. */
const char *hydro_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_H */
