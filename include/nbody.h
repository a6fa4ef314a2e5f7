/*
 * nbody.h - C ABI of libnbody.so, the GB300-native direct-summation Hermite
 * N-body core (CUDA kernels for sm_103a).
 *
 * Paper: S. Portegies Zwart & J. Bedorf, "Computational Gravitational Dynamics
 * with Modern Numerical Accelerators". The problem the calls follow is the
 * one stated in Sect. III.A: a j-set of particles exerts a softened
 * Newtonian force (Sect. II) on an i-set, which may be a subset of the j-set
 * (the particles that are due at the current block time, Sect. III) or a
 * disjoint set; a 4th-order Hermite predictor-corrector (Sect. II, VI: ph4)
 * with individual block time steps (Sect. III) drives the evaluations.
 *
 * Conventions
 *  - Every call returns an int status (NB_OK = 0 or an NB_ERR_* code). The
 *    message of the last failure on a handle is nb_last_error(h).
 *  - Handles are opaque. The library owns all device memory it allocates;
 *    the caller owns every host buffer it passes, which the library only
 *    reads or writes during the call.
 *  - Arrays are structure-of-arrays, binary64: a vector field over n
 *    particles (positions, velocities, accelerations, jerks) is ONE buffer
 *    of 3*n doubles laid out x[0..n), y[0..n), z[0..n). Masses, potentials,
 *    times and steps are n doubles. Indices are 0-based int32.
 *  - Host-pointer calls are synchronous: they return after the result is in
 *    the caller's buffer. *_dev calls take device pointers, run on the
 *    handle's stream (nb_set_stream) and return without waiting.
 *  - A handle is not thread-safe; use one handle per thread. The server
 *    calls (nb_submit / nb_poll / nb_cancel / nb_result_release) are
 *    thread-safe.
 *  - No call falls back to the CPU: without a usable CUDA device nb_create
 *    fails with NB_ERR_CUDA.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define NB_OK 0
#define NB_ERR_ARG 1        /* invalid argument (size, NULL, range, order) */
#define NB_ERR_OOM 2        /* device allocation failed */
#define NB_ERR_BUDGET 3     /* request exceeds the handle's memory budget */
#define NB_ERR_CUDA 4       /* a CUDA runtime call failed */
#define NB_ERR_TIMEOUT 5    /* a bounded device-side wait gave up */
#define NB_ERR_NONFINITE 6  /* non-finite input, or a force that overflowed
                               (e.g. coincident particles with eps = 0) */
#define NB_ERR_BUSY 7       /* server queue full */
#define NB_ERR_NOTFOUND 8   /* unknown ticket */
#define NB_ERR_STATE 9      /* call out of order (e.g. nb_correct with no force) */

/* ---- pair-arithmetic variants (Sect. III.A: emulated vs native FP64) ---- */
#define NB_F32 0   /* FP32 pair math, FP32 positions and sums (reported only) */
#define NB_F32DS 1 /* FP32 pair math; double-single (hi+lo FP32) relative
                      coordinates and double-single accumulation of acc, jerk
                      and pot (the paper's emulated double precision for the
                      inter-particle distance); FP64 state */
#define NB_F64 2   /* IEEE FP64 pair math (the paper's native double path for
                      extreme mass ratios) */

/* ---- configuration ------------------------------------------------------ */
#define NB_FLAG_TIMING 1 /* time every kernel launch with CUDA events (nb_stats) */
/* Block steps of NB_F32 / NB_F32DS handles normally run in the fused
 * persistent kernel: one cooperative launch takes block steps (scheduler +
 * predictor, force, reduction, corrector, with grid-wide barriers between
 * the stages) until a due set larger than nb_config.fused_max_na (default
 * NB_FUSED_DEFAULT_NA) or t_end, so small
 * steps need no host round trip; larger due sets go to the planned force
 * kernels. NB_FLAG_NO_FUSED takes every block step with separate launches. */
#define NB_FLAG_NO_FUSED 2
#define NB_FUSED_MAX_NA 4096      /* upper bound of nb_config.fused_max_na */
#define NB_FUSED_DEFAULT_NA 1024  /* fused_max_na = 0 */
#define NB_FUSED6_MAX_NA 64       /* largest due set of the order-6 fused kernel */

typedef struct nb_config {
    int n_max;           /* particle capacity of the handle, >= 1 */
    int variant;         /* NB_F32, NB_F32DS or NB_F64 */
    double eps;          /* Plummer softening length, >= 0 */
    double eta;          /* Aarseth step-criterion accuracy, > 0 */
    double eta_s;        /* initial-step parameter (dt0 = eta_s |a|/|jerk|); 0 means eta */
    double dt_max;       /* largest block step: a power of two */
    double dt_min;       /* smallest block step: a power of two, <= dt_max */
    double shared_dt;    /* > 0: shared-step mode with this step; 0: block steps */
    size_t budget_bytes; /* device-memory cap for the handle; 0 = none */
    int device;          /* CUDA device ordinal */
    int flags;           /* NB_FLAG_* */
    int fused_max_na;    /* largest due set the fused kernel takes itself (<= NB_FUSED_MAX_NA);
                          * 0 = NB_FUSED_DEFAULT_NA */
    int n_corr;          /* force evaluations + corrections per step in nb_step: 0 or 1 = PEC,
                          * n > 1 = the iterated corrector P(EC)^n (Hermite iteration: the
                          * corrected active particles are evaluated and corrected again);
                          * at most NB_MAX_CORR. Steps with n > 1 use separate launches. */
    int order;           /* integrator order: 4 (0 = 4), the Hermite scheme with acc and jerk,
                          * or 6, the 6th-order Hermite scheme that also evaluates the snap
                          * (the second time derivative of the acceleration) of every pair
                          * and predicts through the crackle (Sect. II: >= 4th-order
                          * integrators with individual steps; the cited 6th-order Hermite
                          * scheme of Nitadori & Makino). Order 6 needs NB_F32DS or NB_F64
                          * pairs and n_corr <= 1, and has no external i-sets or bridge
                          * calls; its fused kernel (NB_F32DS) takes due sets of
                          * up to min(fused_max_na, NB_FUSED6_MAX_NA) particles. Its
                          * steps follow Aarseth's criterion with the evaluated snap as a2
                          * and the end-of-step crackle as a3 (eta ~ 0.01-0.04). */
} nb_config;
#define NB_MAX_CORR 8

/* Fills cfg with: n_max 1024, NB_F32DS, eps 0, eta 0.01, eta_s 0 (= eta),
 * dt_max 1/16, dt_min 2^-30, shared_dt 0, budget 0, device 0, flags 0,
 * fused_max_na 0, n_corr 0, order 4. */
void nb_config_default(nb_config *cfg);

/* Counters of a handle since creation or nb_reset_stats. Kernel times are
 * filled only with NB_FLAG_TIMING. */
typedef struct nb_stats {
    long long block_steps;      /* block (or shared) steps taken */
    long long force_launches;   /* force evaluations launched */
    double interactions;        /* sum over evaluations of N_i * N_j */
    double force_ms;            /* pair-force kernel time (CUDA events) */
    double reduce_ms;           /* partial-sum reduction kernel time */
    double predict_ms;          /* j-prediction kernel time */
    double correct_ms;          /* corrector + step kernel time */
    double sched_ms;            /* block scheduler kernel time */
    long long dt_min_hits;      /* corrections whose step was clamped at dt_min */
    long long active_hist[32];  /* block steps by floor(log2(N_active)) */
    long long kernel_launches;  /* CUDA kernels this library launched */
    double force_ms_hist[32];   /* force kernel time by floor(log2(N_i)) (NB_FLAG_TIMING) */
    double inter_hist[32];      /* interactions by floor(log2(N_i)) */
    long long fused_steps;      /* block steps taken inside the fused kernel */
    long long fused_launches;   /* fused-kernel launches */
    double fused_ms;            /* fused-kernel time (NB_FLAG_TIMING) */
    double fused_stage_ms[4];   /* fused kernel: predict, force (small due sets: with their
                                 * reduction and corrector), reduce + correct, step barrier */
    double fused_step_ms_hist[32]; /* fused kernel: step time by floor(log2(N_active)) */
} nb_stats;

typedef struct nb_handle_s *nb_handle;

/* Human-readable name of a status code (static storage). */
const char *nb_status_string(int status);

/* Message of the last failure on h (static or handle-owned storage; valid
 * until the next call on h). With h == NULL: the last nb_create failure. */
const char *nb_last_error(nb_handle h);

/* Version string of the library. */
const char *nb_version(void);

/* ---- lifetime ------------------------------------------------------------
 * nb_create allocates the device state for cfg->n_max particles on
 * cfg->device. Rejects eps < 0, eta <= 0, dt_max or dt_min not a power of
 * two, dt_min > dt_max, shared_dt < 0, n_max < 1, an unknown variant
 * (NB_ERR_ARG), and a state larger than budget_bytes (NB_ERR_BUDGET).
 * nb_destroy frees everything; it is a no-op on NULL. */
int nb_create(const nb_config *cfg, nb_handle *out);
int nb_destroy(nb_handle h);

/* Stream for all later device work of h (a cudaStream_t; NULL selects the
 * CUDA default stream). A new handle works on a non-blocking stream of its
 * own. The caller keeps the stream alive. */
int nb_set_stream(nb_handle h, void *stream);

/* ---- state ----------------------------------------------------------------
 * nb_set_particles copies n particles (m[n], pos[3n], vel[3n]) and sets every
 * own time t_i = t0. acc, jerk and steps are left unset until nb_init (or the
 * first nb_step, which calls it). Rejects n < 1 or n > n_max (NB_ERR_ARG),
 * negative masses (NB_ERR_ARG) and non-finite values (NB_ERR_NONFINITE). */
int nb_set_particles(nb_handle h, int n, const double *m, const double *pos,
                     const double *vel, double t0);

/* Evaluate acc and jerk of every particle at its current (common) time and
 * assign the initial block steps dt0 = eta_s |a|/|jerk| (quantized), or the
 * shared step. One full N*N evaluation. */
int nb_init(nb_handle h);

/* Copy out masses and the current (corrected, not predicted) positions and
 * velocities. Any pointer may be NULL to skip it. */
int nb_get_particles(nb_handle h, double *m, double *pos, double *vel);

/* Full integrator state for checkpoint / resume: m[n], pos[3n], vel[3n],
 * acc[3n], jerk[3n], own time t[n], own step dt[n]. nb_set_state restores a
 * state taken by nb_get_state (same n <= n_max), after which nb_step resumes
 * bit-identically. Any output pointer of nb_get_state may be NULL. */
int nb_get_state(nb_handle h, int *n, double *m, double *pos, double *vel,
                 double *acc, double *jerk, double *t, double *dt);
int nb_set_state(nb_handle h, int n, const double *m, const double *pos,
                 const double *vel, const double *acc, const double *jerk,
                 const double *t, const double *dt);

/* ---- the hot path ----------------------------------------------------------
 * nb_predict (Sect. III.A, prediction of the j particles): every particle is
 * moved by its Taylor series from its own time t_i to time t,
 *   xp = x + v d + a d^2/2 + jerk d^3/6,  vp = v + a d + jerk d^2/2,  d = t - t_i.
 * Rejects t < t_i for any particle (NB_ERR_ARG). */
int nb_predict(nb_handle h, double t);

/* nb_force (Sect. III.A): acc, jerk and pot of the i-particles idx[0..n_i)
 * (members of the j-set; idx == NULL means all particles in order) from
 * every predicted j-particle, the pair i == j left out:
 *   r = x_j - x_i, v = v_j - v_i, s2 = |r|^2 + eps^2,
 *   acc_i  += m_j r / s2^(3/2)
 *   jerk_i += m_j (v - 3 (r.v) r / s2) / s2^(3/2)
 *   pot_i  -= m_j / s2^(1/2).
 * Outputs: acc[3 n_i], jerk[3 n_i], pot[n_i] (any may be NULL), indexed by
 * position k in idx. Duplicate indices are allowed. Requires a preceding
 * nb_predict (NB_ERR_STATE). Coincident particles with eps = 0 give
 * NB_ERR_NONFINITE. n_i = 0 is a no-op. */
int nb_force(nb_handle h, const int *idx, int n_i, double *acc, double *jerk,
             double *pot);

/* nb_force with device buffers (idx_dev: n_i int32 or NULL; outputs as
 * nb_force but device memory, any may be NULL), asynchronous on the handle's
 * stream. Errors found on the device (non-finite results) are reported by
 * the next synchronous call. */
int nb_force_dev(nb_handle h, const int *idx_dev, int n_i, double *acc_dev,
                 double *jerk_dev, double *pot_dev);

/* nb_force on a handle of order 6 (NB_ERR_ARG otherwise), with the snap:
 * acc, jerk, snap[3 n_i] (structure of arrays, any may be NULL) and pot of the members idx
 * from every other particle at the state predicted by nb_predict (positions,
 * velocities and accelerations through the crackle term). The pair snap is
 * the second time derivative of the pair acceleration along the motion:
 * with r, v, a the j-minus-i position, velocity and acceleration,
 * r2 = |r|^2 + eps^2, alpha = r.v / r2, beta = (|v|^2 + r.a) / r2 + alpha^2:
 * S = m a / r2^(3/2) - 6 alpha J - 3 beta A (A, J as in nb_force). nb_correct
 * may follow (the 6th-order corrector). Errors as nb_force. */
int nb_force_snap(nb_handle h, const int *idx, int n_i, double *acc, double *jerk,
                  double *snap, double *pot);

/* The 6th-order state beyond nb_get_state: snap and crackle (the 2nd and 3rd
 * time derivatives of the acceleration) of the n particles, [3 n] structure of
 * arrays each, either may be NULL. Order-6 handles only (NB_ERR_ARG otherwise). */
int nb_get_snap(nb_handle h, double *snap, double *crackle);

/* Completes a checkpoint restored by nb_set_state on an order-6 handle (both
 * arrays [3 n], required, finite: else NB_ERR_ARG / NB_ERR_NONFINITE). Until it
 * is called after nb_set_state, nb_step on that handle returns NB_ERR_STATE.
 * With it the run resumes bit-identically. */
int nb_set_snap(nb_handle h, const double *snap, const double *crackle);

/* nb_force_ext (Sect. III.A, disjoint i-set): the force of the predicted
 * j-set on n_i external particles (pos[3 n_i], vel[3 n_i]); no pair is left
 * out. Outputs as nb_force. */
int nb_force_ext(nb_handle h, int n_i, const double *pos, const double *vel,
                 double *acc, double *jerk, double *pot);

/* nb_correct (4th-order Hermite corrector, Sect. II/VI): advance the
 * particles of the last nb_force (idx, n_i must repeat that call's list,
 * without duplicates; NB_ERR_ARG otherwise) from their own times to t using
 * their predicted state and the new acc/jerk, then give each a new step:
 * Aarseth's criterion quantized to a power of two in [dt_min, dt_max] that
 * divides t (block mode), or the shared step. */
int nb_correct(nb_handle h, const int *idx, int n_i, double t);

/* nb_step: block-step Hermite loop (Sect. III, III.A) until every particle
 * reaches t_end (t_end must be a multiple of the current steps, e.g. of
 * dt_max). Each block step: t_next = min_i(t_i + dt_i); the due particles
 * (t_i + dt_i == t_next, ascending index) are the i-set; predict all j,
 * force on the i-set, correct. Calls nb_init first if needed. st (may be
 * NULL) receives the counters of this call only. */
int nb_step(nb_handle h, double t_end, nb_stats *st);

/* Kinetic and potential energy of the synchronised system (all t_i equal,
 * else NB_ERR_STATE): K = sum m v^2/2, W = sum m_i pot_i / 2 with pot from an
 * FP64 evaluation at the current positions. */
int nb_energy(nb_handle h, double *kin, double *pot);

/* Counters accumulated since creation or the last reset. */
int nb_get_stats(nb_handle h, nb_stats *st);
int nb_reset_stats(nb_handle h);

/* ---- launch plans and the autotuner ---------------------------------------
 * How a force evaluation of n_i i-particles is laid out on the GPU (the
 * paper's i-parallel and j-parallel mappings, Sect. III.A):
 *   kind 0: tiles - a CTA of 256 threads holds 2 i-particles per thread in
 *           256/nwj/32 warp columns; nwj warp rows share each j-tile;
 *           nsplit CTAs split the j-range (FP32 kinds: nwj in {1, 4, 8});
 *   kind 1: j-parallel warp groups - each warp holds up to 2 i-particles (FP64:
 *           all threads share up to 4) and its lanes stride over j; nsplit
 *           CTAs split the j-range;
 *   kind 2: tiny i-sets (FP32 kinds) - all threads share up to 4 i-particles
 *           and each holds up to 4 j-records; the split count follows from
 *           the j-set size (nsplit is ignored).
 * A plan changes only the order in which pair terms are summed, not which are
 * summed. Plans are looked up by bucket b = ceil(log2(n_i)) (0..31). An
 * order-6 handle's table holds kind 0 entries only (the 6th-order tile kernel:
 * nwj = 1, 2, 4 or 8 warp rows of 256 / nwj i-particles each; FP64 pairs use
 * one warp row). */
typedef struct nb_plan {
    int kind;   /* 0 tiles, 1 warp groups, 2 tiny sets, -1 = built-in heuristic */
    int nwj;    /* warp rows per CTA (kind 0) */
    int nsplit; /* j-range splits (>= 1; clamped to the j-set) */
} nb_plan;

/* The plan used for an evaluation of n_i i-particles on the current j-set
 * (for an entry nb_autotune wrote: with its split count scaled, see there). */
int nb_plan_for(nb_handle h, int n_i, nb_plan *out);

/* Set the plan table (n <= 32 entries, entry b for bucket b; kind -1 entries
 * and buckets >= n use the heuristic); table == NULL restores the heuristic.
 * Rejects malformed entries (NB_ERR_ARG). */
int nb_set_plan_table(nb_handle h, const nb_plan *table, int n);
int nb_get_plan_table(nb_handle h, nb_plan *table /* 32 entries */);

/* Autotuner: for every bucket up to the current N, times candidate plans
 * (kind, nwj, nsplit around the heuristic) on the handle's own particles with
 * CUDA events, reps repetitions each, and stores the fastest in the plan
 * table. Bucket b is timed at n_i = min(2^b, N); for the other sizes of the
 * bucket a tuned tile or warp-group entry keeps the number of CTAs it was
 * timed with (its split count scales with the count of i-blocks), so that it
 * fills the same waves of the GPU. Entries set by nb_set_plan_table are used
 * as given. The particle state is left unchanged; the prediction is not (the
 * j-set is predicted to the latest own time), so call nb_predict again before
 * a manual nb_force. Order-6 handles (NB_F32DS) time the 6th-order tile kernel
 * with 1, 2, 4 and 8 warp rows, each at the split counts that fill 1..8 whole
 * waves, and the built-in plan; an order-6 FP64 handle keeps the built-in plan
 * (NB_OK, table unchanged). */
int nb_autotune(nb_handle h, int reps);

/* ---- batched systems -------------------------------------------------------
 * Many independent systems (clusters of uneven N) advanced together with
 * shared-step 4th-order Hermite (Sect. II/VI), every system with its own
 * softening; one step of all systems is one CUDA-graph replay of three
 * kernels: predictor over all particles, one batched force launch (work
 * items = (system, i-block) pairs in decreasing work, persistent CTAs), and
 * corrector over all particles. FP32 kinds only (NB_F32DS or NB_F32).
 * Arrays are concatenated over the systems in order: m[Ntot], pos/vel as 3
 * rows of Ntot (Ntot = sum of sizes). */
typedef struct nb_batch_s *nb_batch;

/* cfg supplies variant, device, flags and budget_bytes (its n_max, eps, eta,
 * dt limits and shared_dt are not used); sizes[n_sys] >= 1; eps[n_sys] >= 0;
 * dt > 0 the shared step. */
int nb_batch_create(const nb_config *cfg, int n_sys, const int *sizes, const double *eps,
                    double dt, nb_batch *out);
int nb_batch_destroy(nb_batch b);

/* Set every system's particles (concatenated) at time t0; the first step
 * evaluates the initial acc/jerk. Non-finite values: NB_ERR_NONFINITE. */
int nb_batch_set(nb_batch b, const double *m, const double *pos, const double *vel, double t0);

/* Advance all systems by n_steps shared steps of dt. st (may be NULL)
 * receives this call's counters (interactions = sum over systems of N^2 per
 * step). */
int nb_batch_step(nb_batch b, int n_steps, nb_stats *st);

/* Current positions and velocities (concatenated; NULL skips) and time. */
int nb_batch_get(nb_batch b, double *pos, double *vel, double *t);

/* Kinetic and potential energy of every system (kin[n_sys], pot[n_sys]),
 * with the potential from the batch's pair arithmetic. */
int nb_batch_energy(nb_batch b, double *kin, double *pot);

/* Autotune the batched kernel's CTA size (64, 128 or 256 threads, i.e.
 * i-blocks of 128, 256 or 512) on the current particles; returns the choice
 * in *threads (may be NULL). */
int nb_batch_autotune(nb_batch b, int *threads);

/* Message of the last failure on a batch. */
const char *nb_batch_last_error(nb_batch b);

/* ---- serving loop ----------------------------------------------------------
 * A device-resident request loop for subsystems of uneven N such as a hybrid
 * tree/direct code hands off (Sect. V-VI): each request is one force
 * evaluation of a subsystem on itself, or an integration of a subsystem with
 * block-step Hermite over t_span. A server thread admits queued requests in
 * arrival order while the device-memory budget and the in-flight limit
 * allow, keeps their particle state on the GPU, and runs ticks: every tick
 * evaluates, in ONE batched force launch, the new force requests and the
 * current due set of every integrating request, then corrects and schedules
 * each integrating request; finished requests are retired and their memory
 * reused. A request's arithmetic does not depend on what else is in flight.
 * FP32 kinds only (NB_F32DS or NB_F32). */
typedef struct nb_server_s *nb_server;

#define NB_REQ_FORCE 0
#define NB_REQ_EVOLVE 1

#define NB_STATUS_QUEUED 0
#define NB_STATUS_RUNNING 1
#define NB_STATUS_DONE 2
#define NB_STATUS_ERROR 3
#define NB_STATUS_CANCELLED 4

typedef struct nb_server_cfg {
    int device;            /* CUDA device */
    int variant;           /* NB_F32DS or NB_F32 */
    size_t budget_bytes;   /* device memory for request state; 0 = 4 GiB */
    int max_inflight;      /* requests on the GPU at once; 0 = 64 */
    int max_queue;         /* queued requests before nb_submit says NB_ERR_BUSY; 0 = 4096 */
    double eta;            /* step criterion of EVOLVE requests (0 = 0.01) */
    double dt_max;         /* largest block step of EVOLVE requests (0 = 1/16) */
    int flags;             /* NB_FLAG_* */
} nb_server_cfg;

typedef struct nb_request {
    int kind;              /* NB_REQ_FORCE or NB_REQ_EVOLVE */
    int n;                 /* particles, >= 1 */
    const double *m;       /* m[n] */
    const double *pos;     /* pos[3n] (x, y, z rows) */
    const double *vel;     /* vel[3n] */
    double eps;            /* softening, >= 0 */
    double t_span;         /* EVOLVE: time to integrate (a multiple of dt_max) */
} nb_request;

typedef struct nb_result {
    int status;            /* NB_STATUS_* */
    int error;             /* NB_OK or the failure's NB_ERR_* code */
    int n;
    const double *acc;     /* FORCE: acc[3n], jerk[3n], pot[n]; library-owned until */
    const double *jerk;    /* nb_result_release */
    const double *pot;
    const double *pos;     /* EVOLVE: final pos[3n], vel[3n] (library-owned) */
    const double *vel;
    double t_submit;       /* seconds on the server's clock */
    double t_start;        /* admitted to the GPU */
    double t_done;
    double interactions;   /* pair interactions spent on the request */
    long long block_steps; /* EVOLVE: block steps taken */
} nb_result;

typedef struct nb_server_stats {
    long long submitted, completed, cancelled, failed;
    long long ticks;            /* server ticks that launched work */
    long long force_launches;   /* batched force launches */
    double interactions;        /* total pair interactions */
    double busy_s;              /* time ticks spent on the GPU work */
    int queued, inflight;       /* right now */
    size_t bytes_in_use;        /* device bytes held for requests */
    long long kernel_launches;  /* kernels the server launched */
} nb_server_stats;

/* Start a server (one thread). Its device work runs on its own stream. */
int nb_server_create(const nb_server_cfg *cfg, nb_server *out);

/* Stop the thread (in-flight work finishes first), free everything; results
 * not yet released are freed too. NULL is a no-op. */
int nb_server_destroy(nb_server s);

/* Queue a request (its arrays are copied before the call returns); *ticket
 * identifies it. NB_ERR_BUSY when the queue is full, NB_ERR_BUDGET when the
 * request alone exceeds the budget, NB_ERR_ARG / NB_ERR_NONFINITE for bad
 * input. Thread-safe. */
int nb_submit(nb_server s, const nb_request *req, uint64_t *ticket);

/* Status (and, when done, the results) of a request. Thread-safe.
 * NB_ERR_NOTFOUND for an unknown or released ticket. */
int nb_poll(nb_server s, uint64_t ticket, nb_result *out);

/* nb_poll that waits up to timeout_s seconds for the request to finish. */
int nb_wait(nb_server s, uint64_t ticket, double timeout_s, nb_result *out);

/* Cancel a queued or running request (it ends as NB_STATUS_CANCELLED). */
int nb_cancel(nb_server s, uint64_t ticket);

/* Free a finished request's results and forget its ticket. */
int nb_result_release(nb_server s, uint64_t ticket);

int nb_server_get_stats(nb_server s, nb_server_stats *out);

/* ---- bridge coupling of two systems (Sect. V) ------------------------------
 * The paper's multi-scale method splits the Hamiltonian of two systems into
 * their own parts and the interaction, and advances them with a 2nd-order
 * kick-drift-kick "bridge": each system is kicked by the other's field, evolves
 * with its own integrator, and is kicked again. Here both systems are handles
 * of this library on the same device (for example a star cluster and the
 * field particles of its host galaxy).
 *
 * nb_kick_ext: the velocities of target change by dt_kick times the
 * acceleration of field's particles at target's positions (field's softening
 * and precision variant); then target's own acc and jerk are evaluated again
 * at the new velocities (the jerk depends on them); the steps dt_i stay. Both
 * systems must be synchronised at the same time (every particle's own time
 * equal to it), else NB_ERR_STATE; uninitialised systems are initialised
 * first. The field's force counts in field's statistics.
 *
 * nb_bridge_step: one bridge step of length dt: kick both systems by each
 * other for dt/2, advance each with nb_step to t + dt, kick both again for
 * dt/2. dt must be a multiple of both systems' dt_max (block steps) or shared
 * step, so both end synchronised; NB_ERR_ARG otherwise. Messages of a failure
 * of b are reported on a. */
int nb_kick_ext(nb_handle target, nb_handle field, double dt_kick);
int nb_bridge_step(nb_handle a, nb_handle b, double dt);

/* ---- self-check of the bounded device waits ---------------------------------
 * Every device-side wait of the library (a bulk copy's mbarrier, the
 * scheduler's look-back, the fused kernel's grid barriers) gives up after a
 * time limit, sets an error bit and returns, so the host reports NB_ERR_TIMEOUT
 * and the device stays usable. nb_selftest_wait runs one such wait that
 * nothing can complete, on device `device`, with a limit of limit_s seconds
 * (0 < limit_s <= 2): which = 0, an mbarrier phase that no copy or arrival
 * completes; which = 1, a grid barrier of a cooperative launch that one CTA
 * never reaches. It returns NB_ERR_TIMEOUT when the wait gave up and reported
 * it (the expected outcome), NB_ERR_STATE if the wait completed, NB_ERR_ARG /
 * NB_ERR_CUDA / NB_ERR_OOM otherwise. For tests of failure detection; the paper
 * has no counterpart. */
int nb_selftest_wait(int which, double limit_s, int device);

/* ---- allocation-free force evaluation -----------------------------------
 * The paper has no counterpart of this call; it exists for callers that
 * cannot call cudaMalloc: a host code that gives all of its device memory to
 * its own pool allocator (a tree code coupled to this library, say) and bars
 * other allocations, since cudaMalloc synchronises the device and fragments
 * the pool, or code that runs where no allocation is allowed.
 *
 * nb_force_static computes what nb_force computes with FP64 pair arithmetic
 * (NB_F64), but on caller-owned device buffers and with no handle:
 *   n_j            j-particles; m[n_j], pos and vel as 3 rows of stride ld
 *                  (x at pos[0..n_j), y at pos[ld..), z at pos[2 ld..)), ld >= n_j;
 *   n_i, idx       i-set: device int32 indices into the j-set (NULL: 0..n_i-1,
 *                  then n_i <= n_j); the pair i == j is left out;
 *   eps            softening (>= 0);
 *   acc, jerk      outputs, 3 rows of stride n_i each; pot: n_i values (device;
 *                  any may be NULL);
 *   stream         cudaStream_t of the work (NULL: the legacy default stream).
 * The call returns after the results are in the output buffers.
 * It calls no cudaMalloc, cudaFree or other allocating routine: the partial
 * sums of its j-split live in a file-scope device array of
 * NB_STATIC_SCRATCH_DOUBLES doubles (8 MiB). CUDA loads device code lazily, so
 * that array and the kernels of this call take their device memory on their
 * first use on a device, not when the library is loaded. The first call on a
 * device (any n_i, with that device current) is therefore a warm-up: it looks
 * up the array's device address (cudaGetSymbolAddress), loads the kernels and
 * runs them once on an empty i-set, and synchronises the stream. Make it with
 * n_i = 0 (acc, jerk, pot may be NULL then) before a pool allocator takes the
 * device memory and before any stream capture; from then on the device holds
 * the array until the process exits and no call allocates. All calls share
 * the one array, its error word and its split counter, so calls that overlap
 * on the GPU (other streams, other threads) race: serialise them. Sizes: n_i <= NB_STATIC_MAX_NI, else
 * NB_ERR_ARG; an index outside [0, n_j) gives NB_ERR_ARG, a non-finite result
 * NB_ERR_NONFINITE, a CUDA failure NB_ERR_CUDA. */
#define NB_STATIC_MAX_NI 1024
#define NB_STATIC_SCRATCH_DOUBLES (1 << 20)
int nb_force_static(int n_j, const double *m, const double *pos, const double *vel,
                    long long ld, int n_i, const int *idx, double eps, double *acc,
                    double *jerk, double *pot, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NBODY_H */
