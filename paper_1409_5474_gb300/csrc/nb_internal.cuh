// Internal declarations of libnbody: device helpers, launch plans and the
// kernel launchers shared by the engine, batch and server translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nbody.h"

namespace nb {

// ---- device error word bits (OR-ed by kernels, read by the host) ----------
enum : unsigned {
    DERR_NONFINITE = 1u,  // a force or corrected state that is not finite
    DERR_TIMEOUT = 2u,    // a bounded mbarrier wait gave up
    DERR_BACKWARD = 4u,   // prediction to a time before a particle's own time
    DERR_BADINDEX = 8u,   // an i-set index outside [0, n_j) (replaced by 0)
    DERR_UNSYNC = 16u,    // a particle's own time differs from the system time
    DERR_SCHED = 32u,     // the due set disagrees with the step-level histogram
};

// Double-single j-record, 48 bytes per particle (see DS_REC):
//   r[0] = {x_hi, y_hi, z_hi, m}, r[1] = {x_lo, y_lo, z_lo, id}, r[2] = {vx, vy, vz, 0}
// with x = x_hi + x_lo to ~48 bits, FP32 velocity, and id the particle index
// stored as int bits (read only to recognise the self pair of a gathered i-set).
constexpr int DS_REC = 3;  // float4 per record

// j-record of the 6th-order scheme, 64 bytes: the 48-byte record followed by
// r[3] = {ax, ay, az, 0}, the FP32 predicted acceleration (the snap term
// differentiates along it).
constexpr int DS6_REC = 4;

// Vector-field output with a row stride: component c of slot k is p[c*ld + k].
struct Out3 {
    double *acc;
    double *jerk;
    double *pot;
    long long ld;
};

// The i-set of an evaluation. Members of the j-set are given by idx (slot k ->
// particle idx[k], or k when idx is null) and read from the j-records; an
// external i-set brings its own records (rec32 / soa64) and has no self pair.
struct ISet {
    int n;
    const int *idx;        // member indices (nullptr: identity)
    bool member;           // true: i is a member of the j-set (self pair removed)
    const float4 *rec32;   // F32/DS records of the i-set (members: the j-records)
    const double *pos64;   // FP64 SoA [3][ld64] (members: predicted positions)
    const double *vel64;
    const double *m64;     // masses (members only; used for the self term)
    long long ld64;
    int nj;                // bound of member indices (the j-set size)
    bool gathered;         // FP32 kinds: rec32 holds one record per slot (a gathered
                           // copy) whose r[1].w carries the particle index bits
};

// The j-set of an evaluation: predicted FP64 SoA and the DS records.
struct JSet {
    int n;
    const float4 *rec32;   // n DS records
    const double *pos64;   // [3][ld]
    const double *vel64;
    const double *m64;
    long long ld;
};

// A force launch plan.
struct ForcePlan {
    int kind;     // 0: i-parallel tiles (K2 tile), 1: j-parallel warps (K2 jmode)
    int ipt;      // i-particles per thread
    int threads;  // CTA size
    int nsplit;   // j-splits (grid.y for tiles, grid.x for jmode)
    int jt;       // j-tile depth (tile kind)
    int nwj;      // warp rows sharing each j-tile (FP32 tile kind)
};

// Choose a plan for n_i i-particles against n_j j-particles.
ForcePlan plan_force(int variant, int n_i, int n_j, int num_sms);

// A plan from a plan-table entry (kind 0 or 1; sizes clamped to the sets).
ForcePlan plan_from_entry(const nb_plan &e, int variant, int n_i, int n_j);

// Resident CTAs per SM of the FP32 / double-single tile kernel with nwj warp rows.
int tile_blocks_per_sm(int variant, int nwj);

// Scratch doubles the plan needs for partial sums (0 when nsplit == 1).
size_t plan_partial_doubles(const ForcePlan &p, int n_i);

// Counters the split reduction needs: one per i-block (zero at allocation;
// every launch leaves them at zero again).
size_t plan_counters(const ForcePlan &p, int n_i);

// Launch K2 with the K3 reduction folded in: when nsplit > 1 each CTA writes
// its partial sums to part (plan_partial_doubles) and the last CTA of every
// i-block (counted in counters) sums them in the fixed order s = 0..nsplit-1.
// eps2: softening squared. Results go to out (slot-indexed). Non-finite
// results set DERR_NONFINITE in *err. ev (optional, 2 events) brackets the launch.
cudaError_t launch_force(int variant, const ForcePlan &plan, const JSet &js, const ISet &is,
                         double eps2, double *part, unsigned *counters, Out3 out, unsigned *err,
                         cudaStream_t st, cudaEvent_t *ev);

// Load the FP64 j-parallel force kernels (every i-per-thread variant) on the
// current device and run each once on an empty i-set, so that a later launch
// takes no lazy module load (a device allocation).
cudaError_t warm_force_jmode64(cudaStream_t st);

// ---- batched systems -------------------------------------------------------

// One work item of a batched evaluation: i-rows [i0, i0 + ni) of irec against
// the j-records [j0, j0 + nj) of jrec (one system; jrec points at its record 0,
// and the pair i == j is left out), outputs at slots i0.. of acc/jerk/pot (rows
// of stride ld). irec is either the system's own records (member rows: the
// particle index is the row) or a gathered copy of its due set (the index rides
// in each record).
//   kind 0: i-parallel - each thread holds 2 of up to 2 x CTA-size i-rows, the
//           j-records stream through the bulk-copy ring;
//   kind 1: j-parallel - for small i-sets (ni <= ITEM_JPAR_MAX_NI): the threads
//           stride over j, i-rows are taken four at a time.
// A j-split group (nsplit > 1 items with the same i-rows and consecutive
// j-ranges) writes double-single partials to part ([nsplit][7][ni] float2);
// launch_split_reduce, queued after the items, sums them in the order
// split = 0..nsplit-1 (SplitGroup). nsplit <= 1: the item writes its outputs.
struct WorkItem {
    const float4 *jrec;
    const float4 *irec;
    double *acc, *jerk, *pot;
    long long ld;
    int i0, ni, j0, nj;
    int gathered, kind;
    int split, nsplit;
    float eps2;
    int pad;
    float2 *part;
    unsigned *err;  // error word of the item's system
};

// A j-split group: outputs at slots i0 .. i0 + ni - 1 of acc/jerk/pot (rows of
// stride ld) are the fixed-order sums of the nsplit partials in part.
struct SplitGroup {
    const float2 *part;
    double *acc, *jerk, *pot;
    long long ld;
    int i0, ni, nsplit, pad;
    unsigned *err;
};

constexpr int ITEM_JPAR_MAX_NI = 64;

// CTA sizes the batched kernel is built for (the autotuner picks one).
constexpr int BATCH_THREADS[3] = {64, 128, 256};

// Batched force (FP32 / double-single) over a list of i-parallel items (kind 0);
// grid = number of persistent CTAs (items are taken round-robin, so sort them
// by decreasing work).
cudaError_t launch_force_items(int variant, int threads, const WorkItem *items, int nitems,
                               int grid, cudaStream_t st);

// Resident CTAs per SM of the batched kernel with `threads` threads.
int batch_blocks_per_sm(int variant, int threads);

// The j-parallel items (kind 1) of a batched evaluation, CTAs of JPAR_THREADS.
constexpr int JPAR_THREADS = 128;
cudaError_t launch_force_items_jpar(int variant, const WorkItem *items, int nitems, int grid,
                                    cudaStream_t st);
int jpar_blocks_per_sm(int variant);

// The fixed-order sums of j-split groups, after their items (same stream).
cudaError_t launch_split_reduce(const SplitGroup *groups, int ngroups, int grid,
                                cudaStream_t st);

// ---- per-particle kernels (K1, K4, K5) -------------------------------------

struct StateDev {
    int n;
    long long ld;      // row stride of the SoA vector fields (capacity)
    double *m;
    double *pos, *vel, *acc, *jerk;   // [3][ld]
    double *t, *dt;
    double *pos_p, *vel_p;            // predicted [3][ld]
    float4 *rec;                      // DS records [n][3]
    // 6th-order scheme only (null otherwise): snap, crackle and the predicted
    // acceleration [3][ld], and the 64-byte records [n][DS6_REC]
    double *snap, *crk, *acc_p;
    float4 *rec6;
};

struct StepParams {
    double eta, eta_s, dt_min, dt_max, shared_dt;
    double noise;  // 6th order: relative rounding noise of the forces (crackle floor); 0: none
};

// Step levels: dt = dt_max * 2^-k, k in [0, NLEVEL).
constexpr int NLEVEL = 64;

// Device-side state of the block scheduler.
struct SchedDev {
    double t_cur;                 // time of the last block step (max_i t_i)
    unsigned long long seq;       // number of the next scheduler launch (look-back epoch)
    unsigned ticket;              // tile tickets handed out in the running launch
    unsigned done;                // CTAs finished in the running launch
    int n_active;                 // due count, written by the CTA of the last tile
    int pad;
    int hist[NLEVEL];             // particles per step level
};

// Mailbox the scheduler writes (mapped host memory) after each launch: the
// host polls seq, then reads t_next and n_active.
struct Mailbox {
    volatile unsigned long long seq;
    volatile double t_next;
    volatile int n_active;
    volatile int pad;
};

// Particles per scheduler CTA (256 threads x 8).
constexpr int SCHED_THREADS = 256;
constexpr int SCHED_PER_THREAD = 1;
constexpr int SCHED_TILE = SCHED_THREADS * SCHED_PER_THREAD;

// K1: predict all particles of s to time t (FP64), writing pos_p, vel_p and,
// when want_rec, the DS records.
cudaError_t launch_predict(const StateDev &s, double t, bool want_rec, unsigned *err,
                           cudaStream_t st, const double *t_dev = nullptr);

// K4: Hermite corrector + new step for the n_a particles act[k] to time t_new,
// with the new acc/jerk in f (slot-indexed). dtmin_hits counts clamps. Keeps
// the level histogram of sd up to date and sets sd->t_cur = t_new.
cudaError_t launch_correct(const StateDev &s, const int *act, int n_a, double t_new,
                           const Out3 &f, const StepParams &p, SchedDev *sd, unsigned *err,
                           unsigned long long *dtmin_hits, cudaStream_t st,
                           const double *t_dev = nullptr, bool xp_from_state = false);

// The iterated corrector P(EC)^n: a trial correction of the n_a active
// particles writes their corrected x, v over their predicted ones (pos_p,
// vel_p, and with want_rec their j-records and, when irec is given, the
// gathered due-set records in slot order), keeping the start-of-step state;
// the next force evaluation then sees them. The final launch_correct of the
// step passes xp_from_state = true (its predicted values are recomputed).
cudaError_t launch_correct_trial(const StateDev &s, const int *act, int n_a, double t_new,
                                 const Out3 &f, const StepParams &p, bool want_rec, float4 *irec,
                                 unsigned *err, cudaStream_t st);

// K4 of many systems in one launch. Job q serves CTAs [block0, block0 +
// ceil(na / CORRECT_THREADS)) (jobs sorted by block0, nblocks CTAs in all).
constexpr int CORRECT_THREADS = 32;
struct CorrectJob {
    StateDev s;
    const int *act;
    int na, block0;
    double t_new;
    Out3 f;
    SchedDev *sd;
    unsigned *err;
};
cudaError_t launch_correct_multi(const CorrectJob *jobs, int njobs, int nblocks,
                                 const StepParams &p, unsigned long long *dtmin_hits,
                                 cudaStream_t st);

// With t_dev != nullptr the two kernels above take their time as *t_dev + t
// (resp. *t_dev + t_new) from device memory, so a captured graph can be
// replayed step after step; launch_advance then sets *t_dev += dt.
cudaError_t launch_advance(double *t_dev, double dt, cudaStream_t st);

// Per-system energies of a batch: kin[s] = sum m v^2/2, pot[s] = sum m pot/2
// over particles [off[s], off[s] + size[s]) (one CTA per system, fixed order).
cudaError_t launch_batch_energy(int n_sys, const int *off, const int *size, const double *m,
                                const double *vel, long long ld, const double *pot,
                                double *kin_out, double *pot_out, cudaStream_t st);

// K4 at start-up: initial steps from acc/jerk (slot k = particle k), or the
// shared step; adds every particle to the level histogram (zeroed by the caller).
cudaError_t launch_init_steps(const StateDev &s, const Out3 &f, const StepParams &p,
                              SchedDev *sd, unsigned *err, cudaStream_t st);

// K5 + K1 fused (block steps): t_next from the level histogram and t_cur (the
// next multiple of the smallest occupied step after t_cur, which equals
// min_i(t_i + dt_i) when every t_i is a multiple of dt_i and t_i <= t_cur <
// t_i + dt_i); predicts every particle to t_next (FP64 + DS records); writes
// the due particles (t_i + dt_i == t_next) to act in ascending index with a
// single-pass decoupled look-back scan over tiles, and (when want_rec) their
// records to irec in the same order; the last CTA publishes
// (seq, t_next, n_active) to the mailbox. status: one word per tile.
cudaError_t launch_sched_predict(const StateDev &s, SchedDev *sd, unsigned long long *status,
                                 int *act, float4 *irec, Mailbox *mail_dev, double dt_max,
                                 bool want_rec, unsigned *err, cudaStream_t st);

// K5 + K1 of many systems in one launch: job q serves CTAs [block0, block0 +
// ntiles) with ntiles = ceil(n / SCHED_TILE) (jobs sorted by block0).
struct SchedJob {
    StateDev s;
    SchedDev *sd;
    unsigned long long *status;
    int *act;
    float4 *irec;
    Mailbox *mail;
    unsigned *err;
    int block0, ntiles;
};
cudaError_t launch_sched_predict_multi(const SchedJob *jobs, int njobs, int nblocks,
                                       double dt_max, bool want_rec, cudaStream_t st);

// The same for the 6th-order scheme: the prediction runs through the crackle
// term and writes pos_p, vel_p, acc_p and (want_rec) the 64-byte records to
// rec6; act receives the due set in ascending index (no gathered records).
cudaError_t launch_sched_predict6(const StateDev &s, SchedDev *sd, unsigned long long *status,
                                  int *act, Mailbox *mail_dev, double dt_max, bool want_rec,
                                  unsigned *err, cudaStream_t st);

// ---- 6th-order Hermite (hermite6.cu) ------------------------------------------

// Outputs of a 6th-order evaluation (slot-indexed rows of stride ld).
struct Out6 {
    double *acc, *jerk, *snap, *pot;
    long long ld;
};

// K1 of the 6th-order scheme for all particles: pos_p, vel_p, acc_p at time t
// (Taylor series through the crackle) and, with want_rec, the 64-byte records.
cudaError_t launch_predict6(const StateDev &s, double t, bool want_rec, unsigned *err,
                            cudaStream_t st);

// Plan of a 6th-order evaluation: CTA shape and j-splits.
ForcePlan plan_force6(int variant, int n_i, int n_j, int num_sms);
// The 6th-order plan of a plan-table entry (kind 0: warp rows nwj, nsplit j-splits), and
// the resident CTAs per SM of the F32 / double-single tile kernel with nwj warp rows.
ForcePlan plan6_from_entry(int variant, int nwj, int nsplit, int n_i, int n_j);
int occ6_blocks(int variant, int nwj);
size_t plan6_partial_doubles(const ForcePlan &p, int n_i);

// K2 + K3 of the 6th-order scheme: acc, jerk, snap and pot of the members
// idx[k] (idx null: k) of the system s, from every other particle of s, at
// the predicted state (rec6 for the FP32 kinds; pos_p, vel_p, acc_p for FP64).
// part: plan6_partial_doubles scratch. ev (optional): {force start, force end,
// reduce start, reduce end}.
cudaError_t launch_force6(int variant, const ForcePlan &p, const StateDev &s, const int *idx,
                          int n_i, double eps2, double *part, const Out6 &out, unsigned *err,
                          cudaStream_t st, cudaEvent_t *ev);

// K4 of the 6th-order scheme for the n_a particles act[k] (act null: k) to
// time t_new: corrector, end-of-step crackle, the generalised step criterion
// and block quantization (or the shared step), level histogram, sd->t_cur.
cudaError_t launch_correct6(const StateDev &s, const int *act, int n_a, double t_new,
                            const Out6 &f, const StepParams &p, SchedDev *sd, unsigned *err,
                            unsigned long long *dtmin_hits, cudaStream_t st);

// ---- fused persistent block steps (persist.cu) ------------------------------

// Counters of the steps a fused launch took itself (added, not reset, by the kernel).
struct FusedStats {
    unsigned long long steps;
    double interactions;
    unsigned long long active_hist[32];
    unsigned long long phase_ns[4];     // CTA 0's time (globaltimer) in: prediction (and the
                                        // hand-off's gather), force (small due sets: with
                                        // their reduction and corrector), reduction +
                                        // corrector, the end-of-step barrier
    unsigned long long step_ns_hist[32];  // step time by floor(log2 N_active)
};

// One cooperative launch of the fused block-step kernel on a system whose
// state is corrected at sd->t_cur with a valid level histogram (as after K4):
// it takes block steps while the due set has at most na_max members and
// t_next <= t_end; at the first step that fails either test it has predicted
// every particle to that t_next and gathered the due set (act, and at order 4
// irec), then publishes (epoch, t_next, N_active) to the mailbox exactly as
// K5 + K1 do, so the caller continues with the planned kernels. part: j-chunk
// partials (fused_part_float2s(grid, na_max, order) float2); cnt:
// fused_cnt_ints(grid) ints; bar: 3 words, zero at launch (the launcher clears
// them). The order-6 kernel (na_max <= FUSED6_MAX_NA) uses neither irec nor f.
struct FusedArgs {
    StateDev s;
    SchedDev *sd;
    int *act;
    float4 *irec;
    Mailbox *mail;
    Out3 f;
    StepParams prm;
    float eps2f;
    int na_max;
    double t_end;
    float2 *part;
    int *cnt;      // fused_cnt_ints(grid): per-CTA due counts, then the two due-set
                   // counters and the tickets of the small-set groups (zeroed at launch)
    unsigned *bar;
    unsigned *err;
    unsigned long long *dtmin_hits;
    FusedStats *stats;
};

constexpr int FUSED_THREADS = 256;
constexpr int FUSED_MAX_WORDS = 256;  // due-flag words per CTA: n <= 8192 x grid
// Due sets of up to FUSED_SMALL_NA particles take the small-set path of the
// fused kernel (groups of four due particles, a ticket per group).
constexpr int FUSED_SMALL_NA = 16;
// The 6th-order fused kernel takes due sets of up to FUSED6_MAX_NA particles,
// all on its small-set path; larger ones go to the planned kernels.
constexpr int FUSED6_MAX_NA = NB_FUSED6_MAX_NA;

// Ints of the fused kernel's counter array: grid per-CTA counts, 2 due-set
// counters, the tickets of the small-set groups (at most FUSED6_MAX_NA / 4; padded).
inline size_t fused_cnt_ints(int grid) { return (size_t)grid + 64; }

// CTAs of the fused launch of the order-4 or order-6 kernel on this device (one
// or two per SM); 0 if the kernel cannot be launched cooperatively.
int fused_grid(int device, int order);
size_t fused_part_float2s(int grid, int na_max, int order);

// Self-checks of the bounded device waits: a wait that nothing completes (an
// mbarrier without arrivals; a grid barrier one CTA never reaches) gives up
// after limit_ns and sets DERR_TIMEOUT in *err. bar: 3 words (cleared here).
cudaError_t launch_selftest_mbar(unsigned *err, unsigned long long limit_ns, cudaStream_t st);
cudaError_t launch_selftest_barrier(unsigned *bar, unsigned *err, unsigned long long limit_ns,
                                    cudaStream_t st);
cudaError_t launch_fused_steps(const FusedArgs &a, int grid, bool ds, int order,
                               cudaStream_t st);

// Bridge kicks (Sect. V): vel += dt * acc (SoA rows of strides ld, lda);
// acc, jerk := a slot-indexed evaluation f for all particles; DERR_UNSYNC when
// some t[i] != tc.
cudaError_t launch_kick(int n, double *vel, long long ld, const double *acc, long long lda,
                        double dt, cudaStream_t st);
cudaError_t launch_set_derivs(const StateDev &s, const Out3 &f, cudaStream_t st);
cudaError_t launch_check_sync(int n, const double *t, double tc, unsigned *err, cudaStream_t st);

// Energy: K = sum m v^2 / 2 and W = sum m pot / 2 (single-CTA, fixed order).
cudaError_t launch_energy(int n, const double *m, const double *vel, long long ld,
                          const double *pot, double *out2, cudaStream_t st);

// DS records of an external i-set from FP64 SoA positions/velocities (mass 0).
cudaError_t launch_make_rec(int n, const double *pos, const double *vel, long long ld,
                            float4 *rec, cudaStream_t st);

// Check every value of n finite doubles (3 rows of stride ld, or 1 row when rows == 1).
cudaError_t launch_check_finite(const double *p, int n, int rows, long long ld, unsigned *err,
                                cudaStream_t st);

// ---- engine handles driven by the serving loop ------------------------------

// Device view of an engine handle (nb_handle) for code that launches the
// kernels itself.
struct HandleView {
    StateDev s;
    float4 *irec;
    int *act;
    double *f_acc, *f_jerk, *f_pot;
    long long ld;
    SchedDev *sd;
    unsigned long long *sched_status;
    Mailbox *mail_h, *mail_d;
    int n, cap;
};
void handle_view(nb_handle h, HandleView *v);
size_t handle_bytes(nb_handle h);
// Epoch of the next scheduler launch on h (advances the handle's mirror).
unsigned long long handle_take_epoch(nb_handle h);
// The caller has initialised h's steps and scheduler state at time t0.
void handle_mark_initialised(nb_handle h, double t0);
// The caller has written n particles into h's state (not yet initialised).
void handle_attach(nb_handle h, int n);
// The engine's planned force (K2 + folded K3) on h: all n members (due == false)
// or the first n_i gathered records of its due set, softening eps2, into h's
// f_acc / f_jerk / f_pot (slot-indexed); errors OR-ed into *err; queued on st.
// May grow h's split scratch (synchronising h's stream). NB_OK or NB_ERR_*.
int handle_force(nb_handle h, int n_i, bool due, double eps2, unsigned *err, cudaStream_t st);

}  // namespace nb
