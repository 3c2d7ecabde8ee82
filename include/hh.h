/*
 * libhh — list-driven 4th-order Hermite N-body force evaluation on GB300 (sm_103a).
 *
 * A C ABI around the data-parallel hot path of the tree + Hermite method of
 * Fukushige & Kawai, "Hierarchical Tree Algorithm for Collisional N-body
 * Simulations on GRAPE" (arXiv:1602.02832).  The calls follow the paper's
 * statement of the loop (Section 2, tree-loop steps 1-7):
 *   step 1   hh_set_j / hh_set_lists (or hh_rebuild): particles, tree nodes as
 *            pseudo-particles and one interaction list per particle group;
 *   step 2   block selection (inside hh_step / hh_advance);
 *   step 4   hh_predict: every j entry to the block time;
 *   4a + 5   hh_force: force, jerk and potential on the active particles,
 *            each from its group's list only;
 *   step 6   hh_correct: 4th-order Hermite corrector and new Aarseth step;
 *   step 7   advance (hh_step / hh_advance, device resident).
 *
 * Conventions
 *   - Arrays of 3-vectors are structure-of-arrays: double[3][n] (all x, then
 *     all y, then all z), unless stated otherwise.
 *   - "j array": entries [0, n) are particles, [n, n_j) tree nodes.  A node
 *     carries the total mass and the mass-weighted position, velocity,
 *     acceleration and jerk of its members at the tree time (Section 2, step 1)
 *     and is predicted like a particle.
 *   - Lists are CSR: off[n_groups + 1] (int64, off[0] = 0, non-decreasing),
 *     idx[off[n_groups]] (int32 indices into the j array).  group_of[p] gives
 *     the list of particle p.  Groups must be contiguous, ascending index
 *     ranges of particles (Barnes 1990 grouping of neighbouring particles).
 *   - Host pointers: the caller owns them; the library copies in or out
 *     before returning.  *_dev variants take device pointers that the caller
 *     owns (for instance torch tensors); they are used on the context's stream
 *     and must stay valid until that stream reaches the call.
 *   - Errors: every int-returning call returns HH_OK (0) or a negative code;
 *     hh_last_error(ctx) holds a one-line message.  Nothing throws across the
 *     ABI, no call aborts the process.  Inputs are validated on the host (and
 *     list indices on the device) before any kernel reads them.
 *   - Threading: a context may be used by one host thread at a time.
 */
#ifndef HH_H
#define HH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HH_OK 0
#define HH_EINVAL (-1)   /* bad argument, size, index or non-finite input */
#define HH_ENOMEM (-2)   /* device or host allocation failed, or capacity exceeded */
#define HH_ECUDA (-3)    /* a CUDA runtime call failed */
#define HH_ETIMEOUT (-4) /* a bounded device-side wait gave up */
#define HH_ESTATE (-5)   /* calls made in the wrong order (e.g. force before lists) */

#define HH_FP64 0  /* plain form: FP64 prediction, pairwise arithmetic and sums */
#define HH_MIXED 1 /* FP64 state and corrector; i-j difference from float pairs
                      (hi + lo), FP32 pairwise arithmetic, compensated FP32 sums */

typedef struct hh_ctx hh_ctx;

typedef struct hh_config {
    double eps2;    /* Plummer softening epsilon^2 (>= 0) */
    double eta;     /* Aarseth accuracy parameter (Section 3: eta = 0.01) */
    double eta_s;   /* initial step: dt = eta_s |a| / |jerk| */
    double dt_min;  /* smallest block step, a power of two */
    double dt_max;  /* largest block step, a power of two, <= dt_tree */
    double dt_tree; /* interval between tree/list rebuilds (Section 2; 1/64 in Section 3) */
    double theta;   /* opening angle for hh_rebuild */
    int32_t leaf;   /* max particles in a leaf cell for hh_rebuild (e.g. 8) */
    int32_t n_crit; /* max particles per group for hh_rebuild (Section 2) */
    int32_t precision; /* HH_FP64 or HH_MIXED */
    int32_t tile_i;    /* particles per static i tile, 1..32; 0 = 32 */
    int32_t tile_j;    /* shortest list part per work item: a multiple of 128 (HH_FP64) or 256
                          (HH_MIXED); 0 = 256 (HH_FP64), 512 (HH_MIXED) */
    int32_t work_item; /* 0 (default): every list part is tile_j entries long.  > 0: a tile with
                          n_a active particles takes parts of about work_item / n_a entries (at
                          least tile_j), so that work items cost about the same */
    int32_t order;     /* particle and node order of hh_rebuild's tree: HH_ORDER_MORTON (0,
                          default) or HH_ORDER_HILBERT (1, Peano-Hilbert, the paper's order,
                          Section 2).  The octree, groups and interaction sets are the same;
                          only the positions of particles, nodes and list entries differ */
    int32_t work_split; /* 0 (default): work_item applies to every block step.  > 0: the
                          batched loop (hh_batch_run, hh_batch_step) uses work_item only in
                          block steps with at least work_split active particles; in smaller
                          ones the mixed form takes parts of tile_j and the plain form
                          equal-cost parts of 2 x tile_j interactions (at least 32 entries):
                          short parts spread a small step over more SMs, equal-cost parts
                          balance a large one.  The other loops then use parts of tile_j.
                          The count is the simulation's own, so results still do not depend
                          on the rest of a batch */
    int32_t tile_j_small; /* 0 (default): off.  Otherwise a multiple of 32 in [32, tile_j]: the
                          batched loop splits the lists of block steps with at most 16 due
                          particles into parts of this length, so that such a step's few tiles
                          spread over more SMs (the item and partial-sum buffers are sized for
                          16 tiles of the longest list in such parts) */
} hh_config;

#define HH_ORDER_MORTON 0
#define HH_ORDER_HILBERT 1

typedef struct hh_counters {
    int64_t block_steps;    /* block steps executed (step 2-7 passes) */
    int64_t particle_steps; /* corrected particle steps */
    int64_t interactions;   /* pairwise terms evaluated, self excluded */
    int64_t rebuilds;       /* tree/list rebuilds */
    int64_t tile_steps;     /* static i tiles with active particles, summed over block steps:
                               particle_steps / tile_steps is the mean number of particles that
                               share one staged list chunk (the paper's n_i, Eq. 3) */
    int64_t list_steps;     /* block steps of the batched loop that predicted only the entries of their
                               list parts instead of every j entry (small steps of large simulations) */
} hh_counters;

/* Fills cfg with defaults: eps2 = 1e-8, eta = 0.02, eta_s = 0.01,
 * dt in [2^-30, 2^-6], dt_tree = 2^-6, theta = 0.5, leaf = 8, n_crit = 64,
 * HH_FP64, default tiles and work items.  A NULL cfg is ignored. */
void hh_config_default(hh_config *cfg);

/* Creates a context on CUDA device `device` with room for n_max particles,
 * nj_max j entries (particles + nodes), list_max list entries and groups_max
 * groups.  All device memory is allocated here.  Returns HH_ENOMEM if it does
 * not fit.  *out is NULL on failure; hh_last_error(NULL) then holds the reason. */
int hh_create(hh_ctx **out, int device, const hh_config *cfg, int64_t n_max, int64_t nj_max,
              int64_t list_max, int32_t groups_max);
/* Waits for the context's work, then frees everything it holds (a stream set
 * with hh_set_stream stays the caller's).  A NULL context is accepted; the
 * call returns HH_OK. */
int hh_destroy(hh_ctx *ctx);

/* Uses the given cudaStream_t (NULL = the context's own stream) for all
 * following work of this context, after synchronising the stream in use.
 * The caller owns the stream and keeps it alive while the context uses it.
 * Errors: HH_EINVAL for a NULL context; HH_ECUDA if the synchronisation
 * fails (the old stream stays in use). */
int hh_set_stream(hh_ctx *ctx, void *cuda_stream);

/* Step 1 (Section 2): writes j entries [first, first + n) — particles and/or
 * nodes — with their positions, velocities, accelerations, jerks, masses and
 * times t (the time at which x, v, a, jk hold; for nodes the tree time).
 * Host SoA arrays [3][n] (m, t: [n]).  Requires first + n <= nj_max; masses
 * must be > 0 and all values finite.  Errors: HH_EINVAL for a range outside
 * [0, nj_max), a NULL array (n > 0), a non-finite value or a mass that is not
 * positive (checked on the host before anything is copied); HH_ECUDA if a
 * copy fails.  hh_set_j_dev takes device arrays and checks the values on the
 * device after the copy, so a failed call (HH_EINVAL) has written the range,
 * which must be rewritten before use. */
int hh_set_j(hh_ctx *ctx, int64_t first, int64_t n, const double *x, const double *v,
             const double *a, const double *jk, const double *m, const double *t);
int hh_set_j_dev(hh_ctx *ctx, int64_t first, int64_t n, const double *x, const double *v,
                 const double *a, const double *jk, const double *m, const double *t);

/* Step 1: interaction lists (host arrays).  n_particles particles occupy j
 * entries [0, n_particles) and n_j entries are in use.  Every idx must be in
 * [0, n_j); group ranges must tile [0, n_particles) in ascending order.  The
 * static i tiles are built here.  Validated before any kernel reads them.
 * Errors: HH_EINVAL for n_particles outside [1, n_max], n_j outside
 * [n_particles, nj_max], n_groups outside [1, groups_max], a NULL array,
 * off[0] != 0, a decreasing off, an index outside [0, n_j) or groups that are
 * not ascending contiguous ranges; HH_ENOMEM for more than list_max entries
 * or more tiles and list parts than the work-item buffers hold. */
int hh_set_lists(hh_ctx *ctx, int64_t n_particles, int64_t n_j, int32_t n_groups,
                 const int64_t *off, const int32_t *idx, const int32_t *group_of);

/* Per-particle block steps dt[n_particles] (powers of two).  hh_init_dt
 * derives them from the stored a and jk instead (dt = eta_s |a| / |jk|,
 * quantised).  Both set nothing else.  Errors: HH_ESTATE before
 * hh_set_lists (which fixes n_particles); HH_EINVAL for a NULL dt or a step
 * that is not a positive power of two (hh_set_dt, nothing is copied then). */
int hh_set_dt(hh_ctx *ctx, const double *dt);
int hh_init_dt(hh_ctx *ctx);

/* Step 4 (GRAPE predictor): predicts every j entry to time t into the
 * context's predicted-record buffer: x + v D + a D^2/2 + jk D^3/6 and
 * v + a D + jk D^2/2, with D = t - t_entry.  Errors: HH_ESTATE before
 * hh_set_lists; HH_EINVAL for a non-finite t. */
int hh_predict(hh_ctx *ctx, double t);

/* Steps 4a + 5: acc, jerk and potential on the n_act particles i_idx (indices
 * < n_particles, no repeats) from the predicted records of the last
 * hh_predict, each particle summing over its group's list and skipping its
 * own entry.  Outputs host SoA acc[3][n_act], jerk[3][n_act], pot[n_act]
 * (any of them may be NULL).  The results also stay on the device for
 * hh_correct.  hh_force_dev takes device arrays (i_idx included) used on the
 * context's stream.  Errors: HH_ESTATE without lists, or when the j
 * entries, lists or particle state changed (hh_set_j, hh_set_lists,
 * hh_correct, hh_advance, hh_rebuild, a batch run) after the last
 * prediction (hh_predict; hh_init_forces and hh_step also leave every entry
 * predicted); HH_EINVAL for n_act outside [0, n_particles], a NULL i_idx
 * (n_act > 0), or an index outside [0, n_particles) (hh_force also rejects
 * repeats; hh_force_dev checks the range on the device); HH_ECUDA. */
int hh_force(hh_ctx *ctx, int32_t n_act, const int32_t *i_idx, double *acc, double *jerk,
             double *pot);
int hh_force_dev(hh_ctx *ctx, int32_t n_act, const int32_t *i_idx_dev, double *acc_dev,
                 double *jerk_dev, double *pot_dev);

/* Step 6: corrects the n_act particles i_idx at time t with the forces of the
 * last hh_force, then sets each one's new block step (Aarseth criterion,
 * power-of-two quantisation, at most doubling, doubling only on a boundary
 * of the doubled step, clamped to [dt_min, dt_max]) and its time to t.
 * Every particle of i_idx must have t_i + dt_i == t.  Errors: HH_ESTATE
 * without a hh_force and steps (hh_set_dt / hh_init_dt) before it; HH_EINVAL
 * for bad i_idx as in hh_force, or for a particle that is not due at t
 * (found on the device: that particle is left as it was, the others of the
 * call are corrected); HH_ECUDA. */
int hh_correct(hh_ctx *ctx, double t, int32_t n_act, const int32_t *i_idx);

/* Initial forces: evaluates acc and jerk of ALL particles at their (common)
 * time t from the current j entries and lists and stores them as the
 * particles' a and jk (nodes are left unchanged).  Errors: HH_ESTATE before
 * hh_set_lists; HH_EINVAL for an error found on the device; HH_ECUDA. */
int hh_init_forces(hh_ctx *ctx, double t);

/* One block step on the device: t_next = min(t_i + dt_i); active particles
 * {t_i + dt_i == t_next}; predict; force; correct.  Returns t_next and the
 * number of active particles (synchronises the stream).  Errors: HH_ESTATE
 * without lists and steps; HH_EINVAL for an error found on the device;
 * HH_ECUDA. */
int hh_step(hh_ctx *ctx, double *t_next_out, int32_t *n_act_out);

/* Block steps on the device until the next block time would exceed t_end,
 * without host round trips per step (CUDA graph of unrolled block steps,
 * replayed; each kernel becomes a no-op once done).  *n_steps_out (may be
 * NULL) receives the number of block steps taken.  Errors: HH_ESTATE
 * without lists and steps; HH_EINVAL for a NaN t_end or an error found on
 * the device; HH_ETIMEOUT if the replays stop making progress; HH_ECUDA. */
int hh_advance(hh_ctx *ctx, double t_end, int64_t *n_steps_out);

/* Step 1 done by the library: copies the (synchronised) particle state to
 * the host, rebuilds the Morton octree, groups (n_crit) and lists (theta,
 * leaf) with the library's own host builder, reorders particles into Morton
 * order, and uploads particles, nodes (tree time t) and lists (or does all of
 * this on the device, see hh_set_rebuild_device).  All particles must be at
 * time t (HH_ESTATE otherwise).  If it fails (HH_ENOMEM for a tree beyond
 * nj_max / groups_max, HH_ECUDA, ...), the lists are invalid until a later
 * hh_rebuild succeeds (calls that need them return HH_ESTATE); the particle
 * state is unchanged, or consistently reordered together with hh_get_ids. */
int hh_rebuild(hh_ctx *ctx, double t);

/* Selects where hh_rebuild does step 1 of the tree loop (Section 2: tree,
 * groups of up to n_crit particles, one interaction list per group):
 * on_device = 0 (the default) uses the host builder (hh_tree_build, with
 * host copies of the state); 1 builds them on the GPU with the same rules
 * (21-bit Morton keys, pre-order cells split above `leaf` particles, maximal
 * groups, the same opening walk and list order) without the state leaving
 * the device.  The device builder sums node moments bottom-up (children's
 * sums), so a node's centre of mass can differ from the host builder's in
 * the last bits; the lists are the same unless an opening test sits exactly
 * on that difference.  Its buffers (about 300 bytes per j entry plus 150 per
 * group) are allocated by the first device rebuild and counted in
 * hh_ctx_device_bytes; that rebuild returns HH_ENOMEM if they do not fit.
 * A device rebuild whose lists exceed list_max grows the list buffer (to the
 * need plus a quarter) instead of failing, so list_max may be a guess.
 * Errors: HH_EINVAL for a NULL context. */
int hh_set_rebuild_device(hh_ctx *ctx, int on_device);

/* Loads n particles (host SoA, any order) at time t with a = jk = 0 and
 * assigns them ids 0..n-1; hh_get_ids reports each slot's id after Morton
 * reordering.  Any lists, steps and forces of an earlier load are dropped
 * (calls that need lists return HH_ESTATE until hh_rebuild or hh_run).
 * Errors: HH_EINVAL for n < 2, n above n_max, a NULL array, a non-finite
 * position or velocity, a mass that is not finite and positive, or a
 * non-finite t (nothing is copied then); HH_ECUDA if the copy fails. */
int hh_load_particles(hh_ctx *ctx, int64_t n, const double *x, const double *v, const double *m,
                      double t);

/* Full run of the tree loop from the loaded state at time t0 to t_end
 * (a multiple of dt_tree): rebuild, initial forces, rebuild with node
 * derivatives, initial steps, then alternate hh_advance and hh_rebuild
 * every dt_tree.  Errors: HH_EINVAL unless t0 and t_end are multiples of
 * dt_tree with t_end >= t0; otherwise the first failing call's code (the
 * state is left where that call stopped). */
int hh_run(hh_ctx *ctx, double t0, double t_end);

/* Copies particle state [0, n_particles) to host SoA arrays (any may be
 * NULL).  Errors: HH_ESTATE before any particles are loaded; HH_ECUDA. */
int hh_get_state(hh_ctx *ctx, double *x, double *v, double *a, double *jk, double *t, double *dt);
/* ids[n_particles]: the id (input index at hh_load_particles) of each
 * particle slot.  Errors: HH_EINVAL for a NULL context or array; HH_ECUDA if
 * the ids kept on the device by a device rebuild cannot be copied. */
int hh_get_ids(hh_ctx *ctx, int64_t *ids);
/* The current lists (step 1 output): group count, list length, and host
 * copies of off[n_groups + 1], idx[list_len], group_of[n_particles] (any
 * array may be NULL; call with NULL arrays first to size them).  Errors:
 * HH_ESTATE when there are no valid lists (none set, or a failed rebuild);
 * HH_ECUDA. */
int hh_get_lists(hh_ctx *ctx, int32_t *n_groups, int64_t *list_len, int64_t *off, int32_t *idx, int32_t *group_of);
/* Host SoA copies of j entries [first, first + count): x, v, a, jk [3][count],
 * m, t [count] (any may be NULL), e.g. the node records after a rebuild.
 * Errors: HH_EINVAL for a range outside [0, n_j); HH_ECUDA. */
int hh_get_j(hh_ctx *ctx, int64_t first, int64_t count, double *x, double *v, double *a, double *jk, double *m,
             double *t);
/* Particles and j entries in use; -1 for a NULL context. */
int64_t hh_n_particles(const hh_ctx *ctx);
int64_t hh_n_j(const hh_ctx *ctx);
/* Work counters since the last hh_reset_counters (synchronises).  Errors:
 * HH_EINVAL for a NULL out, or for an error found on the device since the
 * last check (returned once, then cleared); HH_ECUDA. */
int hh_get_counters(hh_ctx *ctx, hh_counters *out);
int hh_reset_counters(hh_ctx *ctx);
/* Active i tiles by their number of active particles: counts[k] = tiles
 * evaluated with k + 1 active particles, summed over block steps since the
 * last reset (the distribution of the paper's n_i, Eq. 3, per staged list
 * chunk).  Errors: HH_EINVAL for NULL counts, or for an error found on the
 * device since the last check (returned once, then cleared); HH_ECUDA. */
int hh_get_tile_histogram(hh_ctx *ctx, int64_t counts[32]);

/* Kernel-time accounting: CUDA-event time (ms) of the list-force kernel
 * launches since the last reset, and their number (*ms_out and
 * *launches_out, each may be NULL).  enable >= 0 then switches the timing on
 * (1) or off (0) and resets both; enable < 0 only reads.  Events are recorded
 * on the stream the kernels run on.  Errors: HH_EINVAL for a NULL context. */
int hh_force_timing(hh_ctx *ctx, int enable, double *ms_out, int64_t *launches_out);

/* Total number of kernels this library launched in the process (all
 * contexts; graph replays count every kernel node).  Cannot fail. */
int64_t hh_kernel_launches(void);

const char *hh_last_error(const hh_ctx *ctx);

/* ---- Batched persistent block steps (many simulations, one launch) ------ */
/* The paper's Section 4 notes that a GPU needs far more parallel work than
 * one list evaluation offers.  A batch advances many independent
 * simulations (contexts) in one cooperative, persistent kernel: each global
 * step gives every live simulation one block step (steps 2-7 of Section 2),
 * with the predict, force and correct phases of all simulations separated by
 * grid barriers and the force work of all simulations drawn from one queue.
 * A simulation's results do not depend on the others in the batch (its
 * tiles, active sets and list parts are its own; sums run in fixed order),
 * so they equal what hh_advance computes for it alone (with work_split = 0;
 * with step-adaptive parts they equal the simulation alone in a batch).
 *
 * hh_batch_create: device, precision (every context of a run must match it),
 *   up to max_sims (1..32767) simulations per run and max_steps (1..2^20)
 *   global steps per run.  It captures a run once as a CUDA graph: one
 *   fixed-size copy from a pinned host block of the simulation descriptors,
 *   the cooperative launch, and one fixed-size copy back of the step count,
 *   next times and phase stamps; hh_batch_run fills the host block and
 *   replays the graph.  A batch is used by one thread at a time.
 * hh_batch_run: runs the n contexts (distinct, same device and precision,
 *   with lists and steps set) until each one's next block time exceeds its
 *   t_end[s] (normally its next rebuild time) or max_steps global steps have
 *   run.  Outputs (each may be NULL): the number of global steps; t_next_out[n],
 *   each simulation's next block time (> t_end[s] when it reached t_end[s]);
 *   step_us_out[max_steps], the duration of each global step in
 *   microseconds (device timer); phase_us_out[3 max_steps], per step the
 *   durations of the predict/select phase, the force phase (which includes
 *   the corrector: the worker that completes a tile corrects it) and a third,
 *   empty correct phase (0, kept for the layout).  Synchronises.
 *   A grid-barrier wait gives up after 2 s (HH_ETIMEOUT).
 *   Every particle must follow the block rule (dt a power of two in
 *   [2^-31, 1], t a multiple of dt, t + dt after the latest t), as states
 *   made by hh_init_dt, hh_step, hh_advance and hh_rebuild do; otherwise
 *   HH_EINVAL.  The loop keeps a per-simulation histogram of step levels
 *   and per-tile level masks, so a block step touches only the due tiles. */
typedef struct hh_batch hh_batch;
/* Errors of hh_batch_create (message in hh_last_error(NULL)): HH_EINVAL for a
 * NULL out, a bad precision, max_sims or max_steps; HH_ECUDA for a bad device,
 * one without cooperative launch, or a failed capture; HH_ENOMEM if its
 * buffers do not fit.  Errors of hh_batch_run (message in
 * hh_batch_last_error): HH_EINVAL for n outside [1, max_sims], a NULL array
 * or context, max_steps outside [1, the batch's max_steps], a context that
 * appears twice or differs in device or precision, a NaN t_end, or a state
 * that breaks the block rule; HH_ESTATE for a context without lists or
 * steps, or a batch whose launch could not be captured again
 * (hh_batch_set_ctas); HH_ENOMEM if the work queue cannot grow to the
 * contexts' tiles; HH_ETIMEOUT for a grid-barrier wait that gave up;
 * HH_ECUDA. */
int hh_batch_create(hh_batch **out, int device, int precision, int32_t max_sims, int32_t max_steps);
/* Number of persistent CTAs (one per SM) of the batch's launches: n_ctas > 0
 * uses that many SMs, n_ctas <= 0 all SMs but |n_ctas|, which stay free for
 * other streams' kernels (tree rebuilds of simulations outside the launch).
 * The default is every SM.  HH_EINVAL outside [1, SM count]. */
int hh_batch_set_ctas(hh_batch *b, int32_t n_ctas);
/* Waits for the batch's work and frees it; a NULL batch is accepted. */
int hh_batch_destroy(hh_batch *b);
int hh_batch_run(hh_batch *b, int32_t n, hh_ctx *const *ctxs, const double *t_end, int32_t max_steps,
                 int32_t *steps_out, double *t_next_out, double *step_us_out, double *phase_us_out);
const char *hh_batch_last_error(const hh_batch *b);

/* ---- Resident set: admission by device-memory budget, continuous batching -- */
/* The serving form of the batched loop.  Simulations are admitted to a
 * batch's resident set while their device memory fits a budget; each
 * hh_batch_step is one hh_batch_run over the running residents, followed by
 * the tree rebuild (Section 2, step 1) of every simulation that reached its
 * next rebuild time; a simulation that reached its end time is reported once
 * and stays resident (its state readable) until the caller retires it.
 * Contexts stay owned by the caller: the batch borrows them while resident,
 * and a resident context must not be destroyed or used elsewhere until
 * retired.  Calls on one batch come from one thread at a time.
 *
 * hh_batch_set_budget: budget_bytes of device memory for the resident
 *   contexts together (their hh_ctx_device_bytes at admission; 0 = no
 *   limit) and launch_particles, the most particles advanced by one launch
 *   (0 = no limit; at least one simulation runs per launch).  With a cap,
 *   launches take the running residents in round-robin order, so each global
 *   block step carries a bounded amount of work (its latency stays bounded)
 *   and every resident advances in turn.  HH_EINVAL for negative values.
 * hh_batch_admit: adds ctx (same device and precision as the batch, with
 *   lists and steps set, e.g. by hh_run(ctx, t0, t0)) to the resident set,
 *   to run from its last rebuild time to t_end, a multiple of dt_tree not
 *   before it.  HH_ENOMEM if every slot (max_sims) is taken or the context's
 *   device bytes do not fit the budget beside the residents (nothing
 *   changes; retry after a retirement); HH_EINVAL for a NULL or already
 *   resident context, another device or precision, or a bad t_end;
 *   HH_ESTATE for a context without lists or steps.
 * hh_batch_step: one launch (at most max_steps global steps) over the
 *   running residents, each to its next rebuild time, then the rebuilds of
 *   those that reached it (those that build on the device together, as by
 *   hh_batch_rebuild; the others concurrently, one host thread each).  Outputs (may
 *   be NULL): global steps run, simulations launched, the number and the
 *   contexts (done_out, room for max_sims) that reached their end time since
 *   the last call, and the per-step times of hh_batch_run.  With no running
 *   resident it launches nothing.  Errors: those of hh_batch_run; a failed
 *   rebuild returns its code, and that context stops running (retire it).
 * hh_batch_retire: removes ctx from the resident set and frees its share of
 *   the budget.  HH_EINVAL if it is not resident.
 * hh_batch_resident: resident count, running count and device bytes held
 *   against the budget (each output may be NULL). */
int hh_batch_set_budget(hh_batch *b, int64_t budget_bytes, int64_t launch_particles);
int hh_batch_admit(hh_batch *b, hh_ctx *ctx, double t_end);
int hh_batch_step(hh_batch *b, int32_t max_steps, int32_t *steps_out, int32_t *launched_out, int32_t *n_done_out,
                  hh_ctx **done_out, double *step_us_out, double *phase_us_out);
int hh_batch_retire(hh_batch *b, hh_ctx *ctx);
int hh_batch_resident(const hh_batch *b, int32_t *n_out, int32_t *running_out, int64_t *bytes_out);

/* hh_rebuild (Section 2, step 1: tree, groups, interaction lists, node
 * records) of n distinct contexts of the batch's device at times t[s].
 * Contexts set to build on the device (hh_set_rebuild_device) with at most
 * 32768 particles are rebuilt together when there are two or more of them:
 * each step of the device builder is one launch over all of them, its sorts
 * are segmented sorts and its scans one scan over all of them, so the launch
 * count does not grow with n.  Each context gets the tree, lists, node
 * records and particle order that hh_rebuild gives it alone.  The others are
 * rebuilt one after another by hh_rebuild (larger trees sort faster alone).
 * Returns HH_OK when every
 * rebuild succeeded, else the first failed context's code; rc_out[n] (may be
 * NULL) receives each context's code and hh_last_error(ctx) its message.  A
 * context whose rebuild failed has no lists (as after a failed hh_rebuild).
 * HH_EINVAL for n < 1, NULL arrays or contexts, or a context that appears
 * twice; HH_ECUDA if the batch's rebuild stream cannot be made. */
int hh_batch_rebuild(hh_batch *b, int32_t n, hh_ctx *const *ctxs, const double *t, int *rc_out);

/* Self-test of the bounded grid barrier of the batched kernel: a
 * cooperative launch of one CTA per SM runs 64 barriers; with skip_cta >= 0
 * that CTA never arrives, so every other CTA's wait must give up after its
 * limit (2 s) and the call returns HH_ETIMEOUT with the
 * GPU still usable; skip_cta < 0 must return HH_OK.  *elapsed_s (may be
 * NULL) receives the kernel's duration. */
int hh_barrier_selftest(int device, int skip_cta, double *elapsed_s);

/* Self-test of the corrector's timestep criterion (Aarseth's formula, used
 * at step 6 of Section 2): for i < n, out[i] = the device's value of the
 * criterion from the squared norms A = |a|^2, J = |j|^2, S = |a2|^2,
 * T = |a3|^2 (host arrays of n doubles, caller-owned) and eta.  Where the
 * device decides in FP32 the value is the exact power of two at or below
 * sqrt(eta (sqrt(A S) + J) / (sqrt(J T) + S)) evaluated in FP64; elsewhere it
 * is that FP64 value.  n <= 2^26; synchronises.  Errors: HH_EINVAL for
 * n < 0, n > 2^26 or a NULL array (n > 0); HH_ECUDA for a bad device or a
 * failed launch; HH_ENOMEM if the device buffers do not fit. */
int hh_selftest_aarseth(int device, int64_t n, const double *A, const double *J, const double *S, const double *T,
                        double eta, double *out);

/* Self-test of the corrector's block quantisation (Section 2, step 6: the
 * new step is the largest power of two below the criterion, at most double
 * the old one, doubled only where the new time is a multiple of the doubled
 * step, clamped to [dt_min, dt_max]): out[i] = the device's step for want[i],
 * dt_old[i], t_new[i] (host arrays of n doubles, caller-owned).  n <= 2^26;
 * synchronises.  Errors: as hh_selftest_aarseth. */
int hh_selftest_block_dt(int device, int64_t n, const double *want, const double *dt_old, const double *t_new,
                         double dt_min, double dt_max, double *out);

/* Device memory held by a context (bytes), for admission by memory budget;
 * -1 for a NULL context. */
int64_t hh_ctx_device_bytes(const hh_ctx *ctx);

/* ---- Allocation-free force call ---------------------------------------- */
/* The paper has no counterpart to this call.  It computes the same list
 * force as hh_force, with the same kernel, for callers that cannot allocate
 * device memory: code whose device memory all comes from another allocator
 * or pool, and loops that must not call cudaMalloc / cudaFree because those
 * calls synchronise the whole device.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.  Its scratch (packed j records, i tiles, work
 * items, per-part partial sums, counters) is one fixed array of about 25 MB
 * in libhh's own device memory (a file-scope __device__ array) that every
 * GPU which loads libhh holds until the process exits.
 *
 * Inputs, device pointers owned by the caller: j entries already predicted
 * to the force time, xj[3][n_j] and vj[3][n_j] (SoA) and mj[n_j]; CSR lists
 * off[n_groups + 1] and idx[off[n_groups]] (indices into the j entries);
 * the active particles as j indices i_idx[n_act] with their list numbers
 * gid[n_act].  Consecutive actives with the same gid share i tiles, so
 * ordering the actives by list is faster but not required.  Each active
 * particle skips the list entry equal to its own index.  Outputs, device,
 * caller-owned: acc[3][n_act], jerk[3][n_act], pot[n_act] by active position.
 * stream: a cudaStream_t (NULL = the legacy default stream).
 *
 * Limits: n_j <= 131072, n_act <= 65536, and at most 8192 work items of
 * (i tile, 2048-entry part of its list).  Sizes above the first two are
 * rejected with HH_EINVAL before any GPU work; too many work items return
 * HH_ENOMEM and device inputs with bad offsets or indices return HH_EINVAL,
 * both detected on the device before the force kernel reads anything, and
 * no output is written then.  The message is in hh_last_error(NULL).
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one scratch array, which
 * keeps the last call's contents; each call clears what must start at zero.
 * Calls whose kernels overlap on the GPU (other streams, other host threads)
 * race on the scratch and must be serialised by the caller.  The call
 * synchronises `stream` before it returns.  `stream` must belong to
 * `device`; the calling thread's current device is the same after the call
 * as before it. */
int hh_force_static(int device, int precision, double eps2, int64_t n_j, const double *xj, const double *vj,
                    const double *mj, int32_t n_groups, const int64_t *off, const int32_t *idx, int32_t n_act,
                    const int32_t *i_idx, const int32_t *gid, double *acc, double *jerk, double *pot,
                    void *stream);

/* ---- Host tree builder (Section 2, step 1; Barnes 1990 grouping) -------- */
/* Morton octree (21 bits per axis, root cube from the bounding box), groups =
 * maximal cells with <= n_crit particles, one list per group: ancestors of
 * the group are opened, the group's own particles enter directly, a cell with
 * one particle enters as that particle, any other cell enters as a node when
 * side < theta * (distance from its centre of mass to the group's bounding
 * box), otherwise it is opened (a leaf gives its particles).  Lists are
 * sorted ascending.  Node j index = n + cell number (cells in pre-order).
 * The tree is host memory owned by the caller until hh_tree_free.  Errors
 * (hh_tree_build*): HH_EINVAL for a NULL out or array, n outside
 * [1, 2^30), leaf or n_crit < 1, theta < 0 or NaN, a non-finite position,
 * velocity, acceleration or jerk, or a mass that is not positive and finite;
 * HH_ENOMEM if host memory runs out.  The other calls return HH_EINVAL for
 * a NULL tree; hh_tree_free accepts NULL. */
typedef struct hh_tree hh_tree;
int hh_tree_build(hh_tree **out, int64_t n, const double *x, const double *v, const double *a,
                  const double *jk, const double *m, int32_t leaf, int32_t n_crit, double theta);
/* The same with the order of the tree: HH_ORDER_MORTON or HH_ORDER_HILBERT
 * (HH_EINVAL otherwise). */
int hh_tree_build_ordered(hh_tree **out, int64_t n, const double *x, const double *v, const double *a,
                          const double *jk, const double *m, int32_t leaf, int32_t n_crit, double theta,
                          int32_t order);
int hh_tree_sizes(const hh_tree *t, int64_t *n_nodes, int32_t *n_groups, int64_t *list_len);
/* perm[k] = input index of slot k in the tree's order; node arrays SoA
 * [3][n_nodes], off[n_groups + 1], idx[list_len], group_of[n] (any may be
 * NULL; hh_tree_sizes gives the sizes). */
int hh_tree_export(const hh_tree *t, int32_t *perm, double *node_x, double *node_v,
                   double *node_a, double *node_jk, double *node_m, int64_t *off, int32_t *idx,
                   int32_t *group_of);
int hh_tree_free(hh_tree *t);

#ifdef __cplusplus
}
#endif
#endif
