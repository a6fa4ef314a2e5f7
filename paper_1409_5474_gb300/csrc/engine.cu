// C ABI of the single-system engine (nbody.h): handles, device state, the
// block-step Hermite loop and the host <-> device boundary.
//
// Device state of a handle is one slab of FP64 structure-of-arrays with row
// stride ld = capacity rounded up to 64 (plus 64 doubles of padding, so that
// bulk copies rounded up to 16 bytes stay inside the slab):
//   m[ld], pos/vel/acc/jerk[3][ld], t[ld], dt[ld], pos_p/vel_p[3][ld],
//   f_acc/f_jerk[3][ld], f_pot[ld], DS j-records rec[ld][3] (float4), act[ld],
//   and for the 6th-order scheme snap/crackle/acc_p/f_snap[3][ld] and the
//   64-byte j-records rec6[ld][4].
// The block-step loop (paper Sect. III, III.A) runs one scheduler kernel per
// block step, reads t_next and N_active from a mapped-memory mailbox, and
// launches predictor, force (+ reduction) and corrector for that N_active.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "nb_internal.cuh"

using namespace nb;

namespace {

std::mutex g_create_mu;
std::string g_create_msg;

bool is_pow2(double x)
{
    if (!(x > 0.0) || !std::isfinite(x)) return false;
    int e;
    double f = std::frexp(x, &e);
    return f == 0.5;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Timing: pairs of events recorded around launches, harvested at sync points.
enum TimerKind { T_FORCE = 0, T_REDUCE, T_PREDICT, T_CORRECT, T_SCHED, T_FUSED, T_NKIND };

struct Timer {
    std::vector<cudaEvent_t> free_ev;
    struct Pending {
        int kind;
        cudaEvent_t a, b;
        int bucket;  // floor(log2 n_i) for force launches, else -1
    };
    std::vector<Pending> pending;
    double ms[T_NKIND] = {0, 0, 0, 0, 0, 0};
    double force_hist[32] = {0};

    cudaEvent_t get()
    {
        if (!free_ev.empty()) {
            cudaEvent_t e = free_ev.back();
            free_ev.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void add(int kind, cudaEvent_t a, cudaEvent_t b, int bucket = -1)
    {
        pending.push_back({kind, a, b, bucket});
    }
    void harvest()
    {
        for (auto &p : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
                ms[p.kind] += t;
                if (p.bucket >= 0) force_hist[p.bucket] += t;
            }
            free_ev.push_back(p.a);
            free_ev.push_back(p.b);
        }
        pending.clear();
        cudaGetLastError();
    }
    ~Timer()
    {
        for (auto &p : pending) {
            free_ev.push_back(p.a);
            free_ev.push_back(p.b);
        }
        for (auto e : free_ev) cudaEventDestroy(e);
    }
};

}  // namespace

struct nb_handle_s {
    nb_config cfg{};
    int dev = 0;
    int num_sms = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;

    int n = 0;
    int cap = 0;
    long long ld = 0;
    void *slab = nullptr;
    size_t slab_bytes = 0;
    double *m = nullptr, *pos = nullptr, *vel = nullptr, *acc = nullptr, *jerk = nullptr;
    double *t = nullptr, *dt = nullptr, *pos_p = nullptr, *vel_p = nullptr;
    double *f_acc = nullptr, *f_jerk = nullptr, *f_pot = nullptr;
    float4 *rec = nullptr;
    float4 *irec = nullptr;  // records of the due set, gathered by the scheduler
    int *act = nullptr;
    // 6th-order scheme (order 6 only): snap, crackle, predicted acceleration,
    // the snap output of a force evaluation, and the 64-byte j-records
    double *snap = nullptr, *crk = nullptr, *acc_p = nullptr, *f_snap = nullptr;
    float4 *rec6 = nullptr;
    bool snap_valid = false;  // snap / crackle belong to the current state

    // growable scratch
    double *part = nullptr;
    size_t part_cap = 0;  // doubles
    unsigned *split_cnt = nullptr;  // per-i-block counters of the folded split reduction
    size_t split_cnt_cap = 0;
    double *io = nullptr; // host-API staging: [7][n_i] outputs, ext inputs
    size_t io_cap = 0;    // doubles
    int *d_idx = nullptr;
    size_t idx_cap = 0;   // ints
    float4 *ext_rec = nullptr;
    size_t ext_rec_cap = 0;  // records

    unsigned *d_err = nullptr;
    unsigned long long *d_dtmin = nullptr;
    double *d_energy = nullptr;
    Mailbox *mail_h = nullptr, *mail_d = nullptr;
    SchedDev *sd = nullptr;                // scheduler state on the device
    unsigned long long *sched_status = nullptr;  // look-back words, one per tile
    unsigned long long seq_next = 1;       // host mirror of sd->seq
    bool sched_valid = false;              // sd->t_cur / hist match the particles
    double t_cur = 0.0;                    // host mirror of the last block time
    cudaEvent_t ev_sched = nullptr;

    // fused persistent block steps (allocated at first use)
    int fused_grid = -1;                  // CTAs per launch; 0 = not available
    float2 *fused_part = nullptr;
    size_t fused_part_cap = 0;            // float2
    int *fused_cnt = nullptr;
    unsigned *fused_bar = nullptr;
    FusedStats *fused_stats = nullptr;

    size_t bytes = 0;  // device bytes held

    bool have_particles = false, initialised = false, predicted = false;
    double t_pred = 0.0;
    int last_force_n = -1;
    std::vector<int> last_idx;
    bool last_force_all = false;

    nb_stats stats{};
    Timer timer;
    std::string msg;
    nb_plan plans[32];  // plan table by bucket ceil(log2 n_i); kind -1 = heuristic
    bool plan_tuned[32] = {};  // entry b was timed by nb_autotune at n_i = min(2^b, n)
};

namespace {

int fail(nb_handle h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->msg = buf;
    else {
        std::lock_guard<std::mutex> lk(g_create_mu);
        g_create_msg = buf;
    }
    return code;
}

#define CK(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), NB_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

StateDev state_of(nb_handle h)
{
    StateDev s;
    s.n = h->n;
    s.ld = h->ld;
    s.m = h->m;
    s.pos = h->pos;
    s.vel = h->vel;
    s.acc = h->acc;
    s.jerk = h->jerk;
    s.t = h->t;
    s.dt = h->dt;
    s.pos_p = h->pos_p;
    s.vel_p = h->vel_p;
    s.rec = h->rec;
    s.snap = h->snap;
    s.crk = h->crk;
    s.acc_p = h->acc_p;
    s.rec6 = h->rec6;
    return s;
}

bool order6(nb_handle h) { return h->cfg.order == 6; }

StepParams params_of(nb_handle h)
{
    StepParams p{};
    p.eta = h->cfg.eta;
    p.eta_s = h->cfg.eta_s > 0.0 ? h->cfg.eta_s : h->cfg.eta;
    p.dt_min = h->cfg.dt_min;
    p.dt_max = h->cfg.dt_max;
    p.shared_dt = h->cfg.shared_dt;
    // double-single pairs round at 2^-23 relative (FP32 pair arithmetic); FP64: none
    p.noise = (h->cfg.order == 6 && h->cfg.variant == NB_F32DS) ? std::ldexp(1.0, -23) : 0.0;
    return p;
}

JSet jset_of(nb_handle h)
{
    JSet j;
    j.n = h->n;
    j.rec32 = h->rec;
    j.pos64 = h->pos_p;
    j.vel64 = h->vel_p;
    j.m64 = h->m;
    j.ld = h->ld;
    return j;
}

ISet members_of(nb_handle h, const int *idx_dev, int n_i)
{
    ISet is;
    is.n = n_i;
    is.idx = idx_dev;
    is.member = true;
    is.rec32 = h->rec;
    is.pos64 = h->pos_p;
    is.vel64 = h->vel_p;
    is.m64 = h->m;
    is.ld64 = h->ld;
    is.nj = h->n;
    is.gathered = false;
    return is;
}

// The due set of a block step: for FP32 kinds the gathered records (one row
// per slot, the index in the record); FP64 reads the predicted state by index.
ISet due_set(nb_handle h, int n_a)
{
    ISet is = members_of(h, h->act, n_a);
    if (h->cfg.variant != NB_F64) {
        is.gathered = true;
        is.rec32 = h->irec;
    }
    return is;
}

bool timing(nb_handle h) { return (h->cfg.flags & NB_FLAG_TIMING) != 0; }

// Grow a device buffer (synchronising first so no kernel still uses it).
template <typename T>
int grow(nb_handle h, T **buf, size_t *cap, size_t need)
{
    if (need <= *cap) return NB_OK;
    size_t want = std::max(need, *cap * 2);
    const size_t add = want * sizeof(T) - *cap * sizeof(T);
    if (h->cfg.budget_bytes && h->bytes + add > h->cfg.budget_bytes) {
        want = need;
        const size_t add2 = want * sizeof(T) - *cap * sizeof(T);
        if (h->bytes + add2 > h->cfg.budget_bytes)
            return fail(h, NB_ERR_BUDGET, "scratch of %zu bytes exceeds the budget of %zu bytes",
                        want * sizeof(T), h->cfg.budget_bytes);
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (*buf) {
        cudaFree(*buf);
        h->bytes -= *cap * sizeof(T);
        *buf = nullptr;
        *cap = 0;
    }
    T *p = nullptr;
    if (cudaMalloc(&p, want * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, NB_ERR_OOM, "cudaMalloc of %zu bytes failed", want * sizeof(T));
    }
    *buf = p;
    *cap = want;
    h->bytes += want * sizeof(T);
    return NB_OK;
}

// Read and clear the device error word; translate it into a status.
int check_err(nb_handle h)
{
    unsigned e = 0;
    CK(h, cudaMemcpyAsync(&e, h->d_err, sizeof e, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (timing(h)) h->timer.harvest();
    if (!e) return NB_OK;
    CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), h->stream));
    if (h->split_cnt)  // an aborted force launch may leave a split counter armed
        CK(h, cudaMemsetAsync(h->split_cnt, 0, h->split_cnt_cap * sizeof(unsigned), h->stream));
    if (e & DERR_TIMEOUT) return fail(h, NB_ERR_TIMEOUT, "a device-side wait timed out");
    if (e & DERR_BADINDEX) return fail(h, NB_ERR_ARG, "an i-set index is outside [0, n)");
    if (e & DERR_BACKWARD)
        return fail(h, NB_ERR_ARG, "prediction time is before some particle's own time");
    if (e & DERR_UNSYNC)
        return fail(h, NB_ERR_STATE, "the particles are not synchronised at the system time");
    if (e & DERR_SCHED)
        return fail(h, NB_ERR_STATE, "the due set disagrees with the step-level histogram");
    return fail(h, NB_ERR_NONFINITE,
                "non-finite force or state (coincident particles with eps = 0?)");
}

int ensure_part(nb_handle h, const ForcePlan &p, int n_i)
{
    int rc = grow(h, &h->part, &h->part_cap, std::max<size_t>(plan_partial_doubles(p, n_i), 1));
    if (rc) return rc;
    const size_t need = std::max<size_t>(plan_counters(p, n_i), 64);
    if (need > h->split_cnt_cap) {
        rc = grow(h, &h->split_cnt, &h->split_cnt_cap, need);
        if (rc) return rc;
        CK(h, cudaMemsetAsync(h->split_cnt, 0, h->split_cnt_cap * sizeof(unsigned), h->stream));
    }
    return NB_OK;
}

int bucket_of(int n_i)
{
    int b = 0;
    while ((1LL << b) < n_i && b < 31) ++b;
    return b;
}

// CTAs of one j-split of a plan on n_i i-particles (i-blocks or warp groups).
static long long blocks_of(const ForcePlan &p, int variant, int n_i)
{
    if (p.kind == 1) {
        if (variant == NB_F64) return 1;
        const long long groups = (n_i + p.ipt - 1) / p.ipt;
        const long long nw = p.threads / 32;
        return (groups + nw - 1) / nw;
    }
    const long long ib = (long long)(p.threads / p.nwj) * p.ipt;
    return (n_i + ib - 1) / ib;
}

ForcePlan plan_for(nb_handle h, int variant, int n_i)
{
    const int b = bucket_of(n_i);
    const nb_plan &e = h->plans[b];
    if (e.kind >= 0 && variant == h->cfg.variant) {
        ForcePlan p = plan_from_entry(e, variant, n_i, h->n);
        if (h->plan_tuned[b] && p.kind != 2) {
            // the tuner timed the bucket at n_i = min(2^b, n): keep that plan's CTA
            // count (its waves) for the other sizes of the bucket, rounded down (a
            // count rounded up past whole waves adds a nearly empty last wave)
            const int n_ref = (int)std::min<long long>(1LL << b, h->n);
            const long long ref = blocks_of(p, variant, n_ref), act = blocks_of(p, variant, n_i);
            if (ref != act && act > 0) {
                nb_plan scaled = e;
                scaled.nsplit = (int)std::max(1LL, ((long long)e.nsplit * ref) / act);
                p = plan_from_entry(scaled, variant, n_i, h->n);
            }
        }
        return p;
    }
    return plan_force(variant, n_i, h->n, h->num_sms);
}

nb_plan entry_of(const ForcePlan &p)
{
    nb_plan e;
    e.kind = p.kind;
    e.nwj = p.nwj;
    e.nsplit = p.nsplit;
    return e;
}

// Force on an i-set into out with a given plan; grows scratch, records timers.
int run_force_plan(nb_handle h, int variant, const ForcePlan &p, const ISet &is, Out3 out);

// Force on an i-set into out; plans, grows scratch, records timers.
int run_force(nb_handle h, int variant, const ISet &is, Out3 out)
{
    if (is.n <= 0) return NB_OK;
    return run_force_plan(h, variant, plan_for(h, variant, is.n), is, out);
}

int run_force_plan(nb_handle h, int variant, const ForcePlan &p, const ISet &is, Out3 out)
{
    if (is.n <= 0) return NB_OK;
    int rc = ensure_part(h, p, is.n);
    if (rc) return rc;
    cudaEvent_t ev[4];
    cudaEvent_t *evp = nullptr;
    if (timing(h)) {
        for (auto &e : ev) e = h->timer.get();
        evp = ev;
    }
    const double eps2 = h->cfg.eps * h->cfg.eps;
    CK(h, launch_force(variant, p, jset_of(h), is, eps2, h->part, h->split_cnt, out, h->d_err,
                       h->stream, evp));
    // the FP32 tile kernel's j-split partials are summed by a launch of their own
    h->stats.kernel_launches += (p.kind == 0 && p.nsplit > 1 && variant != NB_F64) ? 2 : 1;
    int lg = 0;
    while ((2LL << lg) <= is.n && lg < 31) ++lg;
    if (evp) {
        h->timer.add(T_FORCE, ev[0], ev[1], lg);
        h->timer.free_ev.push_back(ev[2]);
        h->timer.free_ev.push_back(ev[3]);
    }
    h->stats.force_launches++;
    h->stats.interactions += (double)is.n * (double)h->n;
    h->stats.inter_hist[lg] += (double)is.n * (double)h->n;
    return NB_OK;
}

template <typename F>
int timed(nb_handle h, int kind, F &&launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (timing(h)) {
        a = h->timer.get();
        b = h->timer.get();
        cudaEventRecord(a, h->stream);
    }
    cudaError_t e = launch();
    h->stats.kernel_launches++;
    if (timing(h)) {
        cudaEventRecord(b, h->stream);
        h->timer.add(kind, a, b);
    }
    if (e != cudaSuccess) return fail(h, NB_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return NB_OK;
}

int predict_to(nb_handle h, double t)
{
    const bool rec = h->cfg.variant != NB_F64;
    StateDev s = state_of(h);
    int rc = timed(h, T_PREDICT, [&] {
        return order6(h) ? launch_predict6(s, t, rec, h->d_err, h->stream)
                         : launch_predict(s, t, rec, h->d_err, h->stream);
    });
    if (rc) return rc;
    h->predicted = true;
    h->t_pred = t;
    return NB_OK;
}

int level_of(double dt, double dt_max)
{
    int k = std::ilogb(dt_max) - std::ilogb(dt);
    return k < 0 ? 0 : (k >= NLEVEL ? NLEVEL - 1 : k);
}

// Build the scheduler state from host copies of t and dt: the last block time
// t_cur = max t_i and the level histogram. Block steps need every t_i to be a
// multiple of its dt_i and t_cur < t_i + dt_i (no particle overdue); shared
// steps need all t_i equal.
int load_sched(nb_handle h, const double *t, const double *dt)
{
    const int n = h->n;
    double tc = t[0];
    for (int i = 1; i < n; ++i) tc = std::max(tc, t[i]);
    std::vector<int> hist(NLEVEL, 0);
    if (h->cfg.shared_dt > 0.0) {
        for (int i = 0; i < n; ++i)
            if (t[i] != tc) return fail(h, NB_ERR_STATE, "shared steps need equal particle times");
    } else {
        for (int i = 0; i < n; ++i) {
            if (std::fmod(t[i], dt[i]) != 0.0 || !(tc < t[i] + dt[i]))
                return fail(h, NB_ERR_STATE,
                            "particle %d: t = %.17g is not a block time of its step %.17g "
                            "(or it is overdue at t = %.17g)", i, t[i], dt[i], tc);
            if (dt[i] > h->cfg.dt_max || dt[i] < h->cfg.dt_min)
                return fail(h, NB_ERR_STATE, "particle %d: step outside [dt_min, dt_max]", i);
            hist[level_of(dt[i], h->cfg.dt_max)]++;
        }
    }
    CK(h, cudaMemcpyAsync(&h->sd->t_cur, &tc, sizeof tc, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->sd->hist, hist.data(), NLEVEL * sizeof(int), cudaMemcpyHostToDevice,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->t_cur = tc;
    h->sched_valid = true;
    return NB_OK;
}

int rebuild_sched(nb_handle h)
{
    const int n = h->n;
    std::vector<double> t(n), dt(n);
    CK(h, cudaMemcpyAsync(t.data(), h->t, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(dt.data(), h->dt, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return load_sched(h, t.data(), dt.data());
}

// Wait until the scheduler launch number `epoch` has published its mailbox.
int wait_mail(nb_handle h, unsigned long long epoch)
{
    volatile Mailbox *mb = h->mail_h;
    for (int spin = 0; spin < 20000; ++spin)
        if (mb->seq == epoch) return NB_OK;
    CK(h, cudaEventSynchronize(h->ev_sched));
    if (mb->seq != epoch) {
        int rc = check_err(h);
        if (rc) return rc;
        return fail(h, NB_ERR_CUDA, "scheduler %llu did not publish its result", epoch);
    }
    return NB_OK;
}

int do_init6(nb_handle h, double t0);

int do_init(nb_handle h)
{
    // all own times are equal at set-up: predict with d = 0 builds the records
    double t0 = 0.0;
    CK(h, cudaMemcpyAsync(&t0, h->t, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (order6(h)) return do_init6(h, t0);
    int rc = predict_to(h, t0);
    if (rc) return rc;
    Out3 f{h->f_acc, h->f_jerk, h->f_pot, h->ld};
    rc = run_force(h, h->cfg.variant, members_of(h, nullptr, h->n), f);
    if (rc) return rc;
    StateDev s = state_of(h);
    StepParams p = params_of(h);
    CK(h, cudaMemsetAsync(h->sd->hist, 0, NLEVEL * sizeof(int), h->stream));
    CK(h, launch_init_steps(s, f, p, h->sd, h->d_err, h->stream));
    h->stats.kernel_launches++;
    rc = check_err(h);
    if (rc) return rc;
    h->initialised = true;
    h->predicted = false;
    h->t_cur = t0;
    h->sched_valid = true;
    return NB_OK;
}

// ---- 6th-order scheme ---------------------------------------------------------

// The 6th-order plan of an evaluation of n_i i-particles: the plan table's entry of
// its bucket (kind 0) when one is set, else the built-in rule. An entry that
// nb_autotune timed at n_i = min(2^b, n) keeps its CTA count for the other sizes of
// the bucket (split count scaled by the ratio of i-blocks, rounded down).
ForcePlan plan_for6(nb_handle h, int variant, int n_i)
{
    const int b = bucket_of(n_i);
    const nb_plan &e = h->plans[b];
    if (e.kind == 0 && variant == h->cfg.variant) {
        nb_plan use = e;
        if (h->plan_tuned[b]) {
            const int n_ref = (int)std::min<long long>(1LL << b, h->n);
            const ForcePlan one = plan6_from_entry(variant, e.nwj, 1, n_i, h->n);
            const long long ib = (long long)one.threads * one.ipt;
            const long long ref = (n_ref + ib - 1) / ib, act = (n_i + ib - 1) / ib;
            if (ref != act && act > 0)
                use.nsplit = (int)std::max(1LL, ((long long)e.nsplit * ref) / act);
        }
        return plan6_from_entry(variant, use.nwj, use.nsplit, n_i, h->n);
    }
    return plan_force6(variant, n_i, h->n, h->num_sms);
}

int run_force6_plan(nb_handle h, int variant, const ForcePlan &p, const int *idx_dev, int n_i,
                    const Out6 &out);

// acc, jerk, snap and pot of the members idx_dev[k] (null: k) at the predicted
// state into out; plans, grows scratch, records timers and counters.
int run_force6(nb_handle h, int variant, const int *idx_dev, int n_i, const Out6 &out)
{
    if (n_i <= 0) return NB_OK;
    return run_force6_plan(h, variant, plan_for6(h, variant, n_i), idx_dev, n_i, out);
}

int run_force6_plan(nb_handle h, int variant, const ForcePlan &p, const int *idx_dev, int n_i,
                    const Out6 &out)
{
    if (n_i <= 0) return NB_OK;
    int rc = grow(h, &h->part, &h->part_cap, std::max<size_t>(plan6_partial_doubles(p, n_i), 1));
    if (rc) return rc;
    cudaEvent_t ev[4];
    cudaEvent_t *evp = nullptr;
    if (timing(h)) {
        for (auto &e : ev) e = h->timer.get();
        evp = ev;
    }
    const double eps2 = h->cfg.eps * h->cfg.eps;
    CK(h, launch_force6(variant, p, state_of(h), idx_dev, n_i, eps2, h->part, out, h->d_err,
                        h->stream, evp));
    h->stats.kernel_launches += p.nsplit > 1 ? 2 : 1;
    int lg = 0;
    while ((2LL << lg) <= n_i && lg < 31) ++lg;
    if (evp) {
        h->timer.add(T_FORCE, ev[0], ev[1], lg);
        h->timer.add(T_REDUCE, ev[2], ev[3]);
    }
    h->stats.force_launches++;
    h->stats.interactions += (double)n_i * (double)h->n;
    h->stats.inter_hist[lg] += (double)n_i * (double)h->n;
    return NB_OK;
}

Out6 out6_of(nb_handle h) { return Out6{h->f_acc, h->f_jerk, h->f_snap, h->f_pot, h->ld}; }

// Start-up of the 6th-order scheme at the common time t0: a first evaluation
// gives acc and jerk (they do not depend on the accelerations), a second one
// with those accelerations in the records gives the snap; crackle starts at
// zero; the initial steps come from acc and jerk as in the 4th-order path.
int do_init6(nb_handle h, double t0)
{
    const int n = h->n;
    CK(h, cudaMemsetAsync(h->acc, 0, 3 * h->ld * sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->jerk, 0, 3 * h->ld * sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->snap, 0, 3 * h->ld * sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->crk, 0, 3 * h->ld * sizeof(double), h->stream));
    const Out6 f = out6_of(h);
    const Out3 f3{h->f_acc, h->f_jerk, h->f_pot, h->ld};
    for (int pass = 0; pass < 2; ++pass) {
        int rc = predict_to(h, t0);
        if (rc) return rc;
        rc = run_force6(h, h->cfg.variant, nullptr, n, f);
        if (rc) return rc;
        if (pass == 0) CK(h, launch_set_derivs(state_of(h), f3, h->stream));
    }
    StateDev s = state_of(h);
    CK(h, cudaMemsetAsync(h->sd->hist, 0, NLEVEL * sizeof(int), h->stream));
    CK(h, launch_init_steps(s, f3, params_of(h), h->sd, h->d_err, h->stream));
    CK(h, cudaMemcpyAsync(h->snap, h->f_snap, 3 * h->ld * sizeof(double),
                          cudaMemcpyDeviceToDevice, h->stream));
    h->stats.kernel_launches += 2;
    int rc = check_err(h);
    if (rc) return rc;
    h->initialised = true;
    h->snap_valid = true;
    h->predicted = false;
    h->t_cur = t0;
    h->sched_valid = true;
    return NB_OK;
}

bool fused_ready(nb_handle h);
FusedArgs fused_args(nb_handle h, double t_end, const Out3 &f);

// Block (or shared) steps of the 6th-order scheme to t_end: the order-6
// scheduler + predictor (or the order-6 fused kernel, which takes the steps
// with small due sets itself) publishes (t_next, N_active), then the force on
// the due set and the corrector are queued; shared steps need no scheduler.
int step6_loop(nb_handle h, double t_end, const std::function<void(int)> &count_step)
{
    StateDev s = state_of(h);
    const StepParams prm = params_of(h);
    const bool rec = h->cfg.variant != NB_F64;
    const Out6 f = out6_of(h);
    int rc;
    if (prm.shared_dt > 0.0) {
        for (;;) {
            const double t_next = h->t_cur + prm.shared_dt;
            if (!(t_next <= t_end)) break;
            rc = timed(h, T_PREDICT,
                       [&] { return launch_predict6(s, t_next, rec, h->d_err, h->stream); });
            if (rc) return rc;
            rc = run_force6(h, h->cfg.variant, nullptr, h->n, f);
            if (rc) return rc;
            rc = timed(h, T_CORRECT, [&] {
                return launch_correct6(s, nullptr, h->n, t_next, f, prm, h->sd, h->d_err,
                                       h->d_dtmin, h->stream);
            });
            if (rc) return rc;
            h->t_cur = t_next;
            count_step(h->n);
        }
        return NB_OK;
    }
    const bool fused = fused_ready(h);
    const FusedArgs fa = fused ? fused_args(h, t_end, Out3{}) : FusedArgs{};
    auto launch_sched = [&]() -> int {
        h->seq_next++;
        int r;
        if (fused) {
            r = timed(h, T_FUSED, [&] {
                return launch_fused_steps(fa, h->fused_grid, true, 6, h->stream);
            });
            h->stats.fused_launches++;
        } else {
            r = timed(h, T_SCHED, [&] {
                return launch_sched_predict6(s, h->sd, h->sched_status, h->act, h->mail_d,
                                             prm.dt_max, rec, h->d_err, h->stream);
            });
        }
        if (r) return r;
        CK(h, cudaEventRecord(h->ev_sched, h->stream));
        return NB_OK;
    };
    rc = launch_sched();
    if (rc) return rc;
    for (;;) {
        rc = wait_mail(h, h->seq_next - 1);
        if (rc) return rc;
        const double t_next = h->mail_h->t_next;
        const int na = h->mail_h->n_active;
        if (!(t_next <= t_end)) break;
        if (na < 1 || na > h->n)
            return fail(h, NB_ERR_STATE, "scheduler returned %d due particles", na);
        rc = run_force6(h, h->cfg.variant, h->act, na, f);
        if (rc) return rc;
        rc = timed(h, T_CORRECT, [&] {
            return launch_correct6(s, h->act, na, t_next, f, prm, h->sd, h->d_err, h->d_dtmin,
                                   h->stream);
        });
        if (rc) return rc;
        h->t_cur = t_next;
        count_step(na);
        rc = launch_sched();
        if (rc) return rc;
    }
    if (fused) {
        // the fused kernel took steps of its own: the last block time is on the device
        CK(h, cudaMemcpyAsync(&h->t_cur, &h->sd->t_cur, sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
    }
    return NB_OK;
}

// Bridge kick (Sect. V): the velocities of tgt change by dt_kick times the
// acceleration of fld's particles at tgt's positions (fld's softening and
// precision variant), then tgt's own acc and jerk are evaluated again at the new
// velocities (jerk depends on them); the steps stay. Both systems must be
// initialised and synchronised at the same time.
int kick_by(nb_handle tgt, nb_handle fld, double dt_kick)
{
    const double t = tgt->t_cur;
    if (fld->t_cur != t)
        return fail(tgt, NB_ERR_STATE, "the two systems are at different times (%.17g, %.17g)",
                    t, fld->t_cur);
    // both synchronised at t (checked on the device)
    CK(tgt, launch_check_sync(tgt->n, tgt->t, t, tgt->d_err, tgt->stream));
    CK(fld, launch_check_sync(fld->n, fld->t, t, fld->d_err, fld->stream));
    int rc = check_err(tgt);
    if (rc) return rc;
    rc = check_err(fld);
    if (rc) return fail(tgt, rc, "field system: %s", fld->msg.c_str());
    // the field's force on tgt's particles (an external i-set of fld)
    rc = predict_to(fld, t);
    if (rc) return rc;
    const int n = tgt->n;
    rc = grow(fld, &fld->io, &fld->io_cap, 7 * (size_t)n);
    if (rc) return rc;
    ISet ext;
    ext.n = n;
    ext.idx = nullptr;
    ext.member = false;
    ext.rec32 = nullptr;
    ext.pos64 = tgt->pos;
    ext.vel64 = tgt->vel;
    ext.m64 = nullptr;
    ext.ld64 = tgt->ld;
    ext.nj = fld->n;
    ext.gathered = false;
    if (fld->cfg.variant != NB_F64) {
        rc = grow(fld, &fld->ext_rec, &fld->ext_rec_cap, (size_t)DS_REC * n);
        if (rc) return rc;
        CK(fld, launch_make_rec(n, tgt->pos, tgt->vel, tgt->ld, fld->ext_rec, fld->stream));
        ext.rec32 = fld->ext_rec;
    }
    const Out3 out{fld->io, fld->io + 3 * (size_t)n, fld->io + 6 * (size_t)n, n};
    rc = run_force(fld, fld->cfg.variant, ext, out);
    if (rc) return rc;
    CK(fld, launch_kick(n, tgt->vel, tgt->ld, out.acc, n, dt_kick, fld->stream));
    fld->stats.kernel_launches += 2;
    rc = check_err(fld);  // synchronises fld's stream: tgt's velocities are final
    if (rc) return fail(tgt, rc, "field system: %s", fld->msg.c_str());
    // tgt's own acc and jerk at the kicked velocities
    rc = predict_to(tgt, t);
    if (rc) return rc;
    const Out3 f{tgt->f_acc, tgt->f_jerk, tgt->f_pot, tgt->ld};
    rc = run_force(tgt, tgt->cfg.variant, members_of(tgt, nullptr, tgt->n), f);
    if (rc) return rc;
    CK(tgt, launch_set_derivs(state_of(tgt), f, tgt->stream));
    tgt->stats.kernel_launches++;
    tgt->predicted = false;
    tgt->last_force_n = -1;
    return check_err(tgt);
}

// The iterations of P(EC)^n (n = cfg.n_corr > 1) after a step's first force
// evaluation on the i-set `is` (n_a active particles act, or all when act is
// null): n - 1 times a trial correction that puts the corrected active
// particles into the j-set, and a new evaluation. The caller's final corrector
// then recomputes the predicted values.
int iterate_corrector(nb_handle h, const StateDev &s, const int *act, int n_a, double t_next,
                      const StepParams &prm, const ISet &is, const Out3 &f)
{
    const bool rec = h->cfg.variant != NB_F64;
    for (int it = 1; it < h->cfg.n_corr; ++it) {
        int rc = timed(h, T_CORRECT, [&] {
            return launch_correct_trial(s, act, n_a, t_next, f, prm, rec,
                                        (rec && is.gathered) ? h->irec : nullptr, h->d_err,
                                        h->stream);
        });
        if (rc) return rc;
        rc = run_force(h, h->cfg.variant, is, f);
        if (rc) return rc;
    }
    return NB_OK;
}

// Whether nb_step takes small block steps in the fused persistent kernel;
// allocates its scratch at first use.
bool fused_ready(nb_handle h)
{
    if (h->cfg.variant == NB_F64 || (h->cfg.flags & NB_FLAG_NO_FUSED) ||
        h->cfg.shared_dt > 0.0 || h->cfg.n_corr > 1)
        return false;
    if (h->fused_grid < 0) h->fused_grid = fused_grid(h->dev, h->cfg.order);
    const int g = h->fused_grid;
    if (g <= 0) return false;
    if ((h->n + g - 1) / g > FUSED_MAX_WORDS * 32) return false;
    if (!h->fused_cnt) {
        const size_t part = fused_part_float2s(g, NB_FUSED_MAX_NA, h->cfg.order);
        const size_t add =
            part * sizeof(float2) + fused_cnt_ints(g) * sizeof(int) + 256 + sizeof(FusedStats);
        if (h->cfg.budget_bytes && h->bytes + add > h->cfg.budget_bytes) return false;
        if (cudaMalloc(&h->fused_part, part * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&h->fused_cnt, fused_cnt_ints(g) * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&h->fused_bar, 256) != cudaSuccess ||
            cudaMalloc(&h->fused_stats, sizeof(FusedStats)) != cudaSuccess ||
            cudaMemset(h->fused_stats, 0, sizeof(FusedStats)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->fused_part);
            cudaFree(h->fused_cnt);
            cudaFree(h->fused_bar);
            cudaFree(h->fused_stats);
            h->fused_part = nullptr;
            h->fused_cnt = nullptr;
            h->fused_bar = nullptr;
            h->fused_stats = nullptr;
            h->fused_grid = 0;
            return false;
        }
        h->fused_part_cap = part;
        h->bytes += add;
    }
    return true;
}

// The arguments of the fused launches of nb_step to t_end (f: the order-4
// kernel's force outputs).
FusedArgs fused_args(nb_handle h, double t_end, const Out3 &f)
{
    FusedArgs fa{};
    fa.s = state_of(h);
    fa.sd = h->sd;
    fa.act = h->act;
    fa.irec = h->irec;
    fa.mail = h->mail_d;
    fa.f = f;
    fa.prm = params_of(h);
    fa.eps2f = (float)(h->cfg.eps * h->cfg.eps);
    fa.na_max = h->cfg.fused_max_na > 0 ? std::min(h->cfg.fused_max_na, NB_FUSED_MAX_NA)
                                        : NB_FUSED_DEFAULT_NA;
    if (order6(h)) fa.na_max = std::min(fa.na_max, FUSED6_MAX_NA);
    fa.t_end = t_end;
    fa.part = h->fused_part;
    fa.cnt = h->fused_cnt;
    fa.bar = h->fused_bar;
    fa.err = h->d_err;
    fa.dtmin_hits = h->d_dtmin;
    fa.stats = h->fused_stats;
    return fa;
}

// Add the steps the fused kernel took to the handle's counters (and clear them).
int fold_fused_stats(nb_handle h)
{
    if (!h->fused_stats) return NB_OK;
    FusedStats f{};
    CK(h, cudaMemcpyAsync(&f, h->fused_stats, sizeof f, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemsetAsync(h->fused_stats, 0, sizeof f, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->stats.block_steps += (long long)f.steps;
    h->stats.fused_steps += (long long)f.steps;
    h->stats.interactions += f.interactions;
    for (int k = 0; k < 32; ++k) {
        h->stats.active_hist[k] += (long long)f.active_hist[k];
        h->stats.fused_step_ms_hist[k] += 1e-6 * (double)f.step_ns_hist[k];
    }
    for (int k = 0; k < 4; ++k) h->stats.fused_stage_ms[k] += 1e-6 * (double)f.phase_ns[k];
    return NB_OK;
}

void sync_stats_counters(nb_handle h)
{
    unsigned long long hits = 0;
    if (cudaMemcpyAsync(&hits, h->d_dtmin, sizeof hits, cudaMemcpyDeviceToHost, h->stream) ==
            cudaSuccess &&
        cudaStreamSynchronize(h->stream) == cudaSuccess)
        h->stats.dt_min_hits = (long long)hits;
    if (timing(h)) {
        h->timer.harvest();
        h->stats.force_ms = h->timer.ms[T_FORCE];
        h->stats.reduce_ms = h->timer.ms[T_REDUCE];
        h->stats.predict_ms = h->timer.ms[T_PREDICT];
        h->stats.correct_ms = h->timer.ms[T_CORRECT];
        h->stats.sched_ms = h->timer.ms[T_SCHED];
        h->stats.fused_ms = h->timer.ms[T_FUSED];
        for (int k = 0; k < 32; ++k) h->stats.force_ms_hist[k] = h->timer.force_hist[k];
    }
}

int validate_host(nb_handle h, int n, const double *m, const double *pos, const double *vel)
{
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(m[i])) return fail(h, NB_ERR_NONFINITE, "mass %d is not finite", i);
        if (m[i] < 0.0) return fail(h, NB_ERR_ARG, "mass %d is negative", i);
    }
    for (long long q = 0; q < 3LL * n; ++q) {
        if (!std::isfinite(pos[q]) || !std::isfinite(vel[q]))
            return fail(h, NB_ERR_NONFINITE, "position/velocity entry %lld is not finite", q);
    }
    return NB_OK;
}

// Copy a host [rows][n] block into device rows of stride ld.
cudaError_t h2d_rows(double *dst, long long ld, const double *src, int n, int rows,
                     cudaStream_t st)
{
    return cudaMemcpy2DAsync(dst, ld * sizeof(double), src, n * sizeof(double), n * sizeof(double),
                             rows, cudaMemcpyHostToDevice, st);
}

cudaError_t d2h_rows(double *dst, const double *src, long long ld, int n, int rows,
                     cudaStream_t st)
{
    return cudaMemcpy2DAsync(dst, n * sizeof(double), src, ld * sizeof(double), n * sizeof(double),
                             rows, cudaMemcpyDeviceToHost, st);
}

}  // namespace

namespace nb {

void handle_view(nb_handle h, HandleView *v)
{
    v->s = state_of(h);
    v->irec = h->irec;
    v->act = h->act;
    v->f_acc = h->f_acc;
    v->f_jerk = h->f_jerk;
    v->f_pot = h->f_pot;
    v->ld = h->ld;
    v->sd = h->sd;
    v->sched_status = h->sched_status;
    v->mail_h = h->mail_h;
    v->mail_d = h->mail_d;
    v->n = h->n;
    v->cap = h->cap;
}

size_t handle_bytes(nb_handle h) { return h->bytes; }

unsigned long long handle_take_epoch(nb_handle h) { return h->seq_next++; }

void handle_attach(nb_handle h, int n)
{
    h->n = n;
    h->have_particles = true;
    h->initialised = false;
    h->predicted = false;
    h->sched_valid = false;
    h->last_force_n = -1;
}

int handle_force(nb_handle h, int n_i, bool due, double eps2, unsigned *err, cudaStream_t st)
{
    if (n_i <= 0) return NB_OK;
    const int variant = h->cfg.variant;
    const ISet is = due ? due_set(h, n_i) : members_of(h, nullptr, n_i);
    const ForcePlan p = plan_for(h, variant, n_i);
    int rc = ensure_part(h, p, n_i);
    if (rc) return rc;
    const Out3 out{h->f_acc, h->f_jerk, h->f_pot, h->ld};
    if (launch_force(variant, p, jset_of(h), is, eps2, h->part, h->split_cnt, out, err, st,
                     nullptr) != cudaSuccess)
        return NB_ERR_CUDA;
    return NB_OK;
}

void handle_mark_initialised(nb_handle h, double t0)
{
    h->initialised = true;
    h->sched_valid = true;
    h->predicted = false;
    h->t_cur = t0;
}

}  // namespace nb

extern "C" {

void nb_config_default(nb_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->n_max = 1024;
    cfg->variant = NB_F32DS;
    cfg->eps = 0.0;
    cfg->eta = 0.01;
    cfg->eta_s = 0.0;
    cfg->dt_max = 1.0 / 16;
    cfg->dt_min = std::ldexp(1.0, -30);
    cfg->shared_dt = 0.0;
    cfg->budget_bytes = 0;
    cfg->device = 0;
    cfg->flags = 0;
    cfg->order = 4;
}

const char *nb_status_string(int status)
{
    switch (status) {
    case NB_OK: return "NB_OK";
    case NB_ERR_ARG: return "NB_ERR_ARG";
    case NB_ERR_OOM: return "NB_ERR_OOM";
    case NB_ERR_BUDGET: return "NB_ERR_BUDGET";
    case NB_ERR_CUDA: return "NB_ERR_CUDA";
    case NB_ERR_TIMEOUT: return "NB_ERR_TIMEOUT";
    case NB_ERR_NONFINITE: return "NB_ERR_NONFINITE";
    case NB_ERR_BUSY: return "NB_ERR_BUSY";
    case NB_ERR_NOTFOUND: return "NB_ERR_NOTFOUND";
    case NB_ERR_STATE: return "NB_ERR_STATE";
    default: return "NB_ERR_UNKNOWN";
    }
}

const char *nb_last_error(nb_handle h)
{
    if (h) return h->msg.c_str();
    std::lock_guard<std::mutex> lk(g_create_mu);
    return g_create_msg.c_str();
}

const char *nb_version(void) { return "nbody-gb300 0.1 (sm_103a)"; }

int nb_create(const nb_config *cfg, nb_handle *out)
{
    if (!cfg || !out) return fail(nullptr, NB_ERR_ARG, "cfg and out must not be NULL");
    *out = nullptr;
    if (cfg->n_max < 1) return fail(nullptr, NB_ERR_ARG, "n_max must be >= 1");
    if (cfg->variant < NB_F32 || cfg->variant > NB_F64)
        return fail(nullptr, NB_ERR_ARG, "unknown variant %d", cfg->variant);
    if (!(cfg->eps >= 0.0) || !std::isfinite(cfg->eps))
        return fail(nullptr, NB_ERR_ARG, "eps must be finite and >= 0");
    if (!(cfg->eta > 0.0) || !std::isfinite(cfg->eta))
        return fail(nullptr, NB_ERR_ARG, "eta must be > 0");
    if (cfg->eta_s < 0.0) return fail(nullptr, NB_ERR_ARG, "eta_s must be >= 0");
    if (!is_pow2(cfg->dt_max)) return fail(nullptr, NB_ERR_ARG, "dt_max must be a power of two");
    if (!is_pow2(cfg->dt_min) || cfg->dt_min > cfg->dt_max)
        return fail(nullptr, NB_ERR_ARG, "dt_min must be a power of two <= dt_max");
    if (!(cfg->shared_dt >= 0.0) || !std::isfinite(cfg->shared_dt))
        return fail(nullptr, NB_ERR_ARG, "shared_dt must be finite and >= 0");
    if (cfg->fused_max_na < 0) return fail(nullptr, NB_ERR_ARG, "fused_max_na must be >= 0");
    if (cfg->n_corr < 0 || cfg->n_corr > NB_MAX_CORR)
        return fail(nullptr, NB_ERR_ARG, "n_corr must be in [0, %d]", NB_MAX_CORR);
    if (cfg->order != 0 && cfg->order != 4 && cfg->order != 6)
        return fail(nullptr, NB_ERR_ARG, "order must be 4 or 6 (0 = 4)");
    if (cfg->order == 6 && cfg->n_corr > 1)
        return fail(nullptr, NB_ERR_ARG, "the 6th-order scheme takes one evaluation per step");
    if (cfg->order == 6 && cfg->variant == NB_F32)
        return fail(nullptr, NB_ERR_ARG,
                    "the 6th-order scheme needs double-single or FP64 pairs (its end-of-step "
                    "derivatives amplify the FP32 position rounding)");

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, NB_ERR_CUDA, "no CUDA device available");
    }
    if (cfg->device < 0 || cfg->device >= ndev)
        return fail(nullptr, NB_ERR_ARG, "device %d out of range (%d devices)", cfg->device, ndev);

    nb_handle h = new nb_handle_s();
    h->cfg = *cfg;
    if (h->cfg.order == 0) h->cfg.order = 4;
    for (auto &e : h->plans) e = nb_plan{-1, 1, 1};
    h->dev = cfg->device;
    h->cap = cfg->n_max;
    h->ld = ((long long)cfg->n_max + 63) / 64 * 64;

    auto bail = [&](int code) {
        nb_destroy(h);
        return code;
    };
    if (cudaSetDevice(h->dev) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, NB_ERR_CUDA, "cudaSetDevice(%d) failed", cfg->device);
    }
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev);

    const size_t row = (size_t)h->ld;
    const size_t vec = align256((3 * row + 64) * sizeof(double));
    const size_t sca = align256((row + 64) * sizeof(double));
    const size_t recb = align256(row * DS_REC * sizeof(float4));
    const size_t actb = align256(row * sizeof(int));
    const size_t rec6b = align256(row * DS6_REC * sizeof(float4));
    h->slab_bytes = 6 * vec + 4 * sca + 2 * vec + 2 * recb + actb;  // see the file header
    if (h->cfg.order == 6) h->slab_bytes += 4 * vec + rec6b;
    const size_t small = 256 * 3;
    if (cfg->budget_bytes && h->slab_bytes + small > cfg->budget_bytes) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "state of %zu bytes exceeds the budget of %zu bytes",
                      h->slab_bytes, cfg->budget_bytes);
        delete h;
        return fail(nullptr, NB_ERR_BUDGET, "%s", msg);
    }
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, NB_ERR_CUDA, "cudaStreamCreate failed");
    }
    h->stream = h->own_stream;
    if (cudaMalloc(&h->slab, h->slab_bytes) != cudaSuccess) {
        cudaGetLastError();
        int code = fail(nullptr, NB_ERR_OOM, "cudaMalloc of %zu bytes failed", h->slab_bytes);
        bail(code);
        return code;
    }
    h->bytes = h->slab_bytes;
    char *p = static_cast<char *>(h->slab);
    auto take = [&](size_t b) {
        char *q = p;
        p += b;
        return q;
    };
    h->pos = (double *)take(vec);
    h->vel = (double *)take(vec);
    h->acc = (double *)take(vec);
    h->jerk = (double *)take(vec);
    h->pos_p = (double *)take(vec);
    h->vel_p = (double *)take(vec);
    h->m = (double *)take(sca);
    h->t = (double *)take(sca);
    h->dt = (double *)take(sca);
    h->f_pot = (double *)take(sca);
    h->f_acc = (double *)take(vec);
    h->f_jerk = (double *)take(vec);
    h->rec = (float4 *)take(recb);
    h->irec = (float4 *)take(recb);
    h->act = (int *)take(actb);
    if (h->cfg.order == 6) {
        h->snap = (double *)take(vec);
        h->crk = (double *)take(vec);
        h->acc_p = (double *)take(vec);
        h->f_snap = (double *)take(vec);
        h->rec6 = (float4 *)take(rec6b);
    }
    if (cudaMemsetAsync(h->slab, 0, h->slab_bytes, h->stream) != cudaSuccess ||
        cudaMalloc(&h->d_err, 256) != cudaSuccess || cudaMalloc(&h->d_dtmin, 256) != cudaSuccess ||
        cudaMalloc(&h->d_energy, 256) != cudaSuccess ||
        cudaMemsetAsync(h->d_err, 0, 256, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->d_dtmin, 0, 256, h->stream) != cudaSuccess ||
        cudaHostAlloc(&h->mail_h, sizeof(Mailbox), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&h->mail_d, h->mail_h, 0) != cudaSuccess ||
        cudaMalloc(&h->sd, sizeof(SchedDev)) != cudaSuccess ||
        cudaMemsetAsync(h->sd, 0, sizeof(SchedDev), h->stream) != cudaSuccess ||
        cudaMalloc(&h->sched_status, sizeof(unsigned long long) *
                                         ((h->cap + SCHED_TILE - 1) / SCHED_TILE)) != cudaSuccess ||
        cudaMemsetAsync(h->sched_status, 0, sizeof(unsigned long long) *
                                                ((h->cap + SCHED_TILE - 1) / SCHED_TILE),
                        h->stream) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_sched, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        int code = fail(nullptr, NB_ERR_CUDA, "device set-up failed");
        bail(code);
        return code;
    }
    h->bytes += 3 * 256 + sizeof(SchedDev) +
                sizeof(unsigned long long) * ((h->cap + SCHED_TILE - 1) / SCHED_TILE);
    {
        const unsigned long long one = 1;
        std::memset((void *)h->mail_h, 0, sizeof(Mailbox));
        if (cudaMemcpy(&h->sd->seq, &one, sizeof one, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            int code = fail(nullptr, NB_ERR_CUDA, "device set-up failed");
            bail(code);
            return code;
        }
        h->seq_next = 1;
    }
    *out = h;
    return NB_OK;
}

int nb_destroy(nb_handle h)
{
    if (!h) return NB_OK;
    cudaSetDevice(h->dev);
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->timer.harvest();
    cudaFree(h->slab);
    cudaFree(h->part);
    cudaFree(h->split_cnt);
    cudaFree(h->io);
    cudaFree(h->d_idx);
    cudaFree(h->ext_rec);
    cudaFree(h->d_err);
    cudaFree(h->d_dtmin);
    cudaFree(h->d_energy);
    cudaFree(h->sd);
    cudaFree(h->sched_status);
    cudaFree(h->fused_part);
    cudaFree(h->fused_cnt);
    cudaFree(h->fused_bar);
    cudaFree(h->fused_stats);
    if (h->ev_sched) cudaEventDestroy(h->ev_sched);
    if (h->mail_h) cudaFreeHost(h->mail_h);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    cudaGetLastError();
    delete h;
    return NB_OK;
}

int nb_set_stream(nb_handle h, void *stream)
{
    if (!h) return NB_ERR_ARG;
    cudaSetDevice(h->dev);
    CK(h, cudaStreamSynchronize(h->stream));
    h->stream = static_cast<cudaStream_t>(stream);  // NULL: the default stream
    return NB_OK;
}

int nb_set_particles(nb_handle h, int n, const double *m, const double *pos, const double *vel,
                     double t0)
{
    if (!h) return NB_ERR_ARG;
    if (n < 1 || n > h->cap) return fail(h, NB_ERR_ARG, "n = %d outside [1, n_max = %d]", n, h->cap);
    if (!m || !pos || !vel) return fail(h, NB_ERR_ARG, "m, pos and vel must not be NULL");
    if (!std::isfinite(t0)) return fail(h, NB_ERR_NONFINITE, "t0 is not finite");
    int rc = validate_host(h, n, m, pos, vel);
    if (rc) return rc;
    cudaSetDevice(h->dev);
    CK(h, cudaStreamSynchronize(h->stream));
    h->n = n;
    CK(h, cudaMemcpyAsync(h->m, m, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, h2d_rows(h->pos, h->ld, pos, n, 3, h->stream));
    CK(h, h2d_rows(h->vel, h->ld, vel, n, 3, h->stream));
    std::vector<double> tt(n, t0);
    CK(h, cudaMemcpyAsync(h->t, tt.data(), n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemsetAsync(h->dt, 0, n * sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->acc, 0, 3 * h->ld * sizeof(double), h->stream));
    CK(h, cudaMemsetAsync(h->jerk, 0, 3 * h->ld * sizeof(double), h->stream));
    if (order6(h)) {
        CK(h, cudaMemsetAsync(h->snap, 0, 3 * h->ld * sizeof(double), h->stream));
        CK(h, cudaMemsetAsync(h->crk, 0, 3 * h->ld * sizeof(double), h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    h->have_particles = true;
    h->snap_valid = false;
    h->initialised = false;
    h->predicted = false;
    h->sched_valid = false;
    h->last_force_n = -1;
    return NB_OK;
}

int nb_init(nb_handle h)
{
    if (!h) return NB_ERR_ARG;
    if (!h->have_particles) return fail(h, NB_ERR_STATE, "no particles set");
    cudaSetDevice(h->dev);
    return do_init(h);
}

int nb_get_particles(nb_handle h, double *m, double *pos, double *vel)
{
    if (!h) return NB_ERR_ARG;
    if (!h->have_particles) return fail(h, NB_ERR_STATE, "no particles set");
    cudaSetDevice(h->dev);
    const int n = h->n;
    if (m) CK(h, cudaMemcpyAsync(m, h->m, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (pos) CK(h, d2h_rows(pos, h->pos, h->ld, n, 3, h->stream));
    if (vel) CK(h, d2h_rows(vel, h->vel, h->ld, n, 3, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return NB_OK;
}

int nb_get_state(nb_handle h, int *n_out, double *m, double *pos, double *vel, double *acc,
                 double *jerk, double *t, double *dt)
{
    if (!h) return NB_ERR_ARG;
    if (n_out) *n_out = h->n;
    if (!h->have_particles) return fail(h, NB_ERR_STATE, "no particles set");
    cudaSetDevice(h->dev);
    const int n = h->n;
    if (m) CK(h, cudaMemcpyAsync(m, h->m, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (pos) CK(h, d2h_rows(pos, h->pos, h->ld, n, 3, h->stream));
    if (vel) CK(h, d2h_rows(vel, h->vel, h->ld, n, 3, h->stream));
    if (acc) CK(h, d2h_rows(acc, h->acc, h->ld, n, 3, h->stream));
    if (jerk) CK(h, d2h_rows(jerk, h->jerk, h->ld, n, 3, h->stream));
    if (t) CK(h, cudaMemcpyAsync(t, h->t, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (dt) CK(h, cudaMemcpyAsync(dt, h->dt, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return NB_OK;
}

int nb_set_state(nb_handle h, int n, const double *m, const double *pos, const double *vel,
                 const double *acc, const double *jerk, const double *t, const double *dt)
{
    if (!h) return NB_ERR_ARG;
    if (n < 1 || n > h->cap) return fail(h, NB_ERR_ARG, "n = %d outside [1, n_max = %d]", n, h->cap);
    if (!m || !pos || !vel || !acc || !jerk || !t || !dt)
        return fail(h, NB_ERR_ARG, "nb_set_state needs every array");
    int rc = validate_host(h, n, m, pos, vel);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(t[i]) || !(dt[i] > 0.0) || !std::isfinite(dt[i]))
            return fail(h, NB_ERR_ARG, "particle %d: t must be finite and dt > 0", i);
        if (h->cfg.shared_dt <= 0.0 && !is_pow2(dt[i]))
            return fail(h, NB_ERR_ARG, "particle %d: block steps must be powers of two", i);
    }
    cudaSetDevice(h->dev);
    CK(h, cudaStreamSynchronize(h->stream));
    const int n_prev = h->n;
    h->n = n;
    {
        int rc2 = load_sched(h, t, dt);
        if (rc2) {
            h->n = n_prev;
            return rc2 == NB_ERR_STATE ? fail(h, NB_ERR_ARG, "%s", h->msg.c_str()) : rc2;
        }
    }
    CK(h, cudaMemcpyAsync(h->m, m, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, h2d_rows(h->pos, h->ld, pos, n, 3, h->stream));
    CK(h, h2d_rows(h->vel, h->ld, vel, n, 3, h->stream));
    CK(h, h2d_rows(h->acc, h->ld, acc, n, 3, h->stream));
    CK(h, h2d_rows(h->jerk, h->ld, jerk, n, 3, h->stream));
    CK(h, cudaMemcpyAsync(h->t, t, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->dt, dt, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (order6(h)) {
        CK(h, cudaMemsetAsync(h->snap, 0, 3 * h->ld * sizeof(double), h->stream));
        CK(h, cudaMemsetAsync(h->crk, 0, 3 * h->ld * sizeof(double), h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    h->have_particles = true;
    h->snap_valid = false;  // order 6: nb_set_snap completes the state
    h->initialised = true;
    h->predicted = false;
    h->last_force_n = -1;
    return NB_OK;
}

int nb_predict(nb_handle h, double t)
{
    if (!h) return NB_ERR_ARG;
    if (!h->have_particles) return fail(h, NB_ERR_STATE, "no particles set");
    if (!std::isfinite(t)) return fail(h, NB_ERR_ARG, "t is not finite");
    cudaSetDevice(h->dev);
    int rc = predict_to(h, t);
    if (rc) return rc;
    rc = check_err(h);
    if (rc) h->predicted = false;
    return rc;
}

int nb_force_dev(nb_handle h, const int *idx_dev, int n_i, double *acc_dev, double *jerk_dev,
                 double *pot_dev)
{
    if (!h) return NB_ERR_ARG;
    if (!h->predicted) return fail(h, NB_ERR_STATE, "nb_force needs a preceding nb_predict");
    if (n_i < 0) return fail(h, NB_ERR_ARG, "n_i < 0");
    if (!idx_dev && n_i > h->n) return fail(h, NB_ERR_ARG, "n_i > n with idx == NULL");
    if (n_i == 0) return NB_OK;
    cudaSetDevice(h->dev);
    Out3 out{acc_dev, jerk_dev, pot_dev, n_i};
    h->last_force_n = -1;  // device buffers: nb_correct cannot use them
    if (order6(h)) {
        int rc = grow(h, &h->io, &h->io_cap, 3 * (size_t)n_i);  // the snap, not returned
        if (rc) return rc;
        return run_force6(h, h->cfg.variant, idx_dev, n_i,
                          Out6{acc_dev, jerk_dev, h->io, pot_dev, n_i});
    }
    return run_force(h, h->cfg.variant, members_of(h, idx_dev, n_i), out);
}

namespace {

// nb_force / nb_force_snap: the outputs go through the io staging buffer, rows
// acc 0-2, jerk 3-5, pot 6 and (order 6) snap 7-9 of stride n_i, where
// nb_correct finds them.
int host_force(nb_handle h, const int *idx, int n_i, double *acc, double *jerk, double *snap,
               double *pot)
{
    if (!h->predicted) return fail(h, NB_ERR_STATE, "nb_force needs a preceding nb_predict");
    if (n_i < 0) return fail(h, NB_ERR_ARG, "n_i < 0");
    if (!idx && n_i > h->n) return fail(h, NB_ERR_ARG, "n_i > n with idx == NULL");
    if (idx) {
        for (int k = 0; k < n_i; ++k)
            if (idx[k] < 0 || idx[k] >= h->n)
                return fail(h, NB_ERR_ARG, "idx[%d] = %d outside [0, %d)", k, idx[k], h->n);
    }
    h->last_force_n = -1;
    if (n_i == 0) return NB_OK;
    cudaSetDevice(h->dev);
    const int rows = order6(h) ? 10 : 7;
    int rc = grow(h, &h->io, &h->io_cap, rows * (size_t)n_i);
    if (rc) return rc;
    const int *idx_dev = nullptr;
    if (idx) {
        rc = grow(h, &h->d_idx, &h->idx_cap, (size_t)n_i);
        if (rc) return rc;
        CK(h, cudaMemcpyAsync(h->d_idx, idx, n_i * sizeof(int), cudaMemcpyHostToDevice, h->stream));
        idx_dev = h->d_idx;
    }
    Out3 out{h->io, h->io + 3 * (size_t)n_i, h->io + 6 * (size_t)n_i, n_i};
    if (order6(h))
        rc = run_force6(h, h->cfg.variant, idx_dev, n_i,
                        Out6{out.acc, out.jerk, h->io + 7 * (size_t)n_i, out.pot, n_i});
    else
        rc = run_force(h, h->cfg.variant, members_of(h, idx_dev, n_i), out);
    if (rc) return rc;
    std::vector<double> buf(rows * (size_t)n_i);
    CK(h, cudaMemcpyAsync(buf.data(), h->io, buf.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    rc = check_err(h);
    if (rc) return rc;
    if (acc) std::memcpy(acc, buf.data(), 3 * n_i * sizeof(double));
    if (jerk) std::memcpy(jerk, buf.data() + 3 * (size_t)n_i, 3 * n_i * sizeof(double));
    if (pot) std::memcpy(pot, buf.data() + 6 * (size_t)n_i, n_i * sizeof(double));
    if (snap) std::memcpy(snap, buf.data() + 7 * (size_t)n_i, 3 * n_i * sizeof(double));
    h->last_force_n = n_i;
    h->last_force_all = (idx == nullptr);
    if (idx)
        h->last_idx.assign(idx, idx + n_i);
    else
        h->last_idx.clear();
    return NB_OK;
}

}  // namespace

int nb_force(nb_handle h, const int *idx, int n_i, double *acc, double *jerk, double *pot)
{
    if (!h) return NB_ERR_ARG;
    return host_force(h, idx, n_i, acc, jerk, nullptr, pot);
}

int nb_force_snap(nb_handle h, const int *idx, int n_i, double *acc, double *jerk, double *snap,
                  double *pot)
{
    if (!h) return NB_ERR_ARG;
    if (!order6(h)) return fail(h, NB_ERR_ARG, "nb_force_snap needs a handle of order 6");
    return host_force(h, idx, n_i, acc, jerk, snap, pot);
}

int nb_get_snap(nb_handle h, double *snap, double *crackle)
{
    if (!h) return NB_ERR_ARG;
    if (!order6(h)) return fail(h, NB_ERR_ARG, "nb_get_snap needs a handle of order 6");
    if (!h->have_particles) return fail(h, NB_ERR_STATE, "no particles set");
    cudaSetDevice(h->dev);
    if (snap) CK(h, d2h_rows(snap, h->snap, h->ld, h->n, 3, h->stream));
    if (crackle) CK(h, d2h_rows(crackle, h->crk, h->ld, h->n, 3, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return NB_OK;
}

int nb_set_snap(nb_handle h, const double *snap, const double *crackle)
{
    if (!h) return NB_ERR_ARG;
    if (!order6(h)) return fail(h, NB_ERR_ARG, "nb_set_snap needs a handle of order 6");
    if (!h->have_particles || !h->initialised)
        return fail(h, NB_ERR_STATE, "nb_set_snap completes a state set by nb_set_state");
    if (!snap || !crackle) return fail(h, NB_ERR_ARG, "snap and crackle must not be NULL");
    for (long long q = 0; q < 3LL * h->n; ++q)
        if (!std::isfinite(snap[q]) || !std::isfinite(crackle[q]))
            return fail(h, NB_ERR_NONFINITE, "snap / crackle value %lld is not finite", q);
    cudaSetDevice(h->dev);
    CK(h, h2d_rows(h->snap, h->ld, snap, h->n, 3, h->stream));
    CK(h, h2d_rows(h->crk, h->ld, crackle, h->n, 3, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->snap_valid = true;
    h->predicted = false;
    return NB_OK;
}

int nb_force_ext(nb_handle h, int n_i, const double *pos, const double *vel, double *acc,
                 double *jerk, double *pot)
{
    if (!h) return NB_ERR_ARG;
    if (order6(h)) return fail(h, NB_ERR_ARG, "nb_force_ext is not available at order 6");
    if (!h->predicted) return fail(h, NB_ERR_STATE, "nb_force_ext needs a preceding nb_predict");
    if (n_i < 0 || (n_i > 0 && (!pos || !vel)))
        return fail(h, NB_ERR_ARG, "n_i < 0 or NULL pos/vel");
    for (long long q = 0; q < 3LL * n_i; ++q)
        if (!std::isfinite(pos[q]) || !std::isfinite(vel[q]))
            return fail(h, NB_ERR_NONFINITE, "external position/velocity %lld is not finite", q);
    if (n_i == 0) return NB_OK;
    cudaSetDevice(h->dev);
    // io layout: [7][n_i] outputs, then [6][n_i] inputs (pos rows, vel rows)
    int rc = grow(h, &h->io, &h->io_cap, 13 * (size_t)n_i);
    if (rc) return rc;
    double *in_pos = h->io + 7 * (size_t)n_i;
    double *in_vel = h->io + 10 * (size_t)n_i;
    CK(h, cudaMemcpyAsync(in_pos, pos, 3 * n_i * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(in_vel, vel, 3 * n_i * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    ISet is{};
    is.n = n_i;
    is.idx = nullptr;
    is.member = false;
    is.pos64 = in_pos;
    is.vel64 = in_vel;
    is.m64 = nullptr;
    is.ld64 = n_i;
    is.nj = h->n;
    is.gathered = false;
    if (h->cfg.variant != NB_F64) {
        rc = grow(h, &h->ext_rec, &h->ext_rec_cap, (size_t)n_i * DS_REC);
        if (rc) return rc;
        CK(h, launch_make_rec(n_i, in_pos, in_vel, n_i, h->ext_rec, h->stream));
        is.rec32 = h->ext_rec;
    }
    Out3 out{h->io, h->io + 3 * (size_t)n_i, h->io + 6 * (size_t)n_i, n_i};
    rc = run_force(h, h->cfg.variant, is, out);
    if (rc) return rc;
    std::vector<double> buf(7 * (size_t)n_i);
    CK(h, cudaMemcpyAsync(buf.data(), h->io, buf.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    rc = check_err(h);
    if (rc) return rc;
    if (acc) std::memcpy(acc, buf.data(), 3 * n_i * sizeof(double));
    if (jerk) std::memcpy(jerk, buf.data() + 3 * (size_t)n_i, 3 * n_i * sizeof(double));
    if (pot) std::memcpy(pot, buf.data() + 6 * (size_t)n_i, n_i * sizeof(double));
    h->last_force_n = -1;
    return NB_OK;
}

int nb_correct(nb_handle h, const int *idx, int n_i, double t)
{
    if (!h) return NB_ERR_ARG;
    if (h->last_force_n < 0 || !h->predicted)
        return fail(h, NB_ERR_STATE, "nb_correct needs a preceding host nb_force");
    if (n_i != h->last_force_n) return fail(h, NB_ERR_ARG, "idx must repeat the last nb_force list");
    if (!std::isfinite(t) || t != h->t_pred)
        return fail(h, NB_ERR_ARG, "t must equal the prediction time of the last nb_predict");
    if ((idx == nullptr) != h->last_force_all)
        return fail(h, NB_ERR_ARG, "idx must repeat the last nb_force list");
    if (idx) {
        if (!std::equal(idx, idx + n_i, h->last_idx.begin()))
            return fail(h, NB_ERR_ARG, "idx must repeat the last nb_force list");
        std::vector<char> seen(h->n, 0);
        for (int k = 0; k < n_i; ++k) {
            if (seen[idx[k]]) return fail(h, NB_ERR_ARG, "duplicate index %d in nb_correct", idx[k]);
            seen[idx[k]] = 1;
        }
    }
    if (n_i == 0) return NB_OK;
    cudaSetDevice(h->dev);
    Out3 f{h->io, h->io + 3 * (size_t)n_i, h->io + 6 * (size_t)n_i, n_i};
    StateDev s = state_of(h);
    StepParams p = params_of(h);
    int rc = timed(h, T_CORRECT, [&] {
        if (order6(h))
            return launch_correct6(s, idx ? h->d_idx : nullptr, n_i, t,
                                   Out6{f.acc, f.jerk, h->io + 7 * (size_t)n_i, f.pot, n_i}, p,
                                   h->sd, h->d_err, h->d_dtmin, h->stream);
        return launch_correct(s, idx ? h->d_idx : nullptr, n_i, t, f, p, h->sd, h->d_err,
                              h->d_dtmin, h->stream);
    });
    if (rc) return rc;
    h->predicted = false;
    h->last_force_n = -1;
    h->initialised = true;
    h->sched_valid = false;
    return check_err(h);
}

int nb_step(nb_handle h, double t_end, nb_stats *st)
{
    if (!h) return NB_ERR_ARG;
    if (!h->have_particles) return fail(h, NB_ERR_STATE, "no particles set");
    if (!std::isfinite(t_end)) return fail(h, NB_ERR_ARG, "t_end is not finite");
    cudaSetDevice(h->dev);
    sync_stats_counters(h);
    const nb_stats before = h->stats;
    int rc;
    if (!h->initialised) {
        rc = do_init(h);
        if (rc) return rc;
    }
    if (!h->sched_valid) {
        rc = rebuild_sched(h);
        if (rc) return rc;
    }
    StateDev s = state_of(h);
    StepParams prm = params_of(h);
    const bool rec = h->cfg.variant != NB_F64;
    Out3 f{h->f_acc, h->f_jerk, h->f_pot, h->ld};
    auto count_step = [&](int na) {
        h->stats.block_steps++;
        int lg = 0;
        while ((2LL << lg) <= na && lg < 31) ++lg;
        h->stats.active_hist[lg]++;
    };
    if (order6(h)) {
        if (!h->snap_valid)
            return fail(h, NB_ERR_STATE,
                        "6th-order state without snap and crackle (restore them with nb_set_snap)");
        rc = step6_loop(h, t_end, count_step);
        if (rc) return rc;
    } else if (prm.shared_dt > 0.0) {
        // shared steps: every particle is due at t_cur + dt; the host knows the
        // schedule, so the launches are queued without waiting on the device
        const ISet all = members_of(h, nullptr, h->n);
        for (;;) {
            const double t_next = h->t_cur + prm.shared_dt;
            if (!(t_next <= t_end)) break;
            rc = timed(h, T_PREDICT,
                       [&] { return launch_predict(s, t_next, rec, h->d_err, h->stream); });
            if (rc) return rc;
            rc = run_force(h, h->cfg.variant, all, f);
            if (rc) return rc;
            rc = iterate_corrector(h, s, nullptr, h->n, t_next, prm, all, f);
            if (rc) return rc;
            rc = timed(h, T_CORRECT, [&] {
                return launch_correct(s, nullptr, h->n, t_next, f, prm, h->sd, h->d_err,
                                      h->d_dtmin, h->stream, nullptr, h->cfg.n_corr > 1);
            });
            if (rc) return rc;
            h->t_cur = t_next;
            count_step(h->n);
        }
    } else {
        // block steps: the fused scheduler + predictor publishes (t_next, N_active)
        // to the mailbox; the force, corrector and the next scheduler launch are
        // queued as soon as it is read
        const bool fused = fused_ready(h);
        const FusedArgs fa = fused ? fused_args(h, t_end, f) : FusedArgs{};
        auto launch_sched = [&]() -> int {
            const unsigned long long ep = h->seq_next++;
            int r;
            if (fused) {
                r = timed(h, T_FUSED, [&] {
                    return launch_fused_steps(fa, h->fused_grid, h->cfg.variant == NB_F32DS, 4,
                                              h->stream);
                });
                h->stats.fused_launches++;
            } else {
                r = timed(h, T_SCHED, [&] {
                    return launch_sched_predict(s, h->sd, h->sched_status, h->act, h->irec,
                                                h->mail_d, prm.dt_max, rec, h->d_err, h->stream);
                });
            }
            if (r) return r;
            CK(h, cudaEventRecord(h->ev_sched, h->stream));
            (void)ep;
            return NB_OK;
        };
        rc = launch_sched();
        if (rc) return rc;
        for (;;) {
            rc = wait_mail(h, h->seq_next - 1);
            if (rc) return rc;
            const double t_next = h->mail_h->t_next;
            const int na = h->mail_h->n_active;
            if (!(t_next <= t_end)) break;
            if (na < 1 || na > h->n)
                return fail(h, NB_ERR_STATE, "scheduler returned %d due particles", na);
            rc = run_force(h, h->cfg.variant, due_set(h, na), f);
            if (rc) return rc;
            rc = iterate_corrector(h, s, h->act, na, t_next, prm, due_set(h, na), f);
            if (rc) return rc;
            rc = timed(h, T_CORRECT, [&] {
                return launch_correct(s, h->act, na, t_next, f, prm, h->sd, h->d_err, h->d_dtmin,
                                      h->stream, nullptr, h->cfg.n_corr > 1);
            });
            if (rc) return rc;
            h->t_cur = t_next;
            count_step(na);
            rc = launch_sched();
            if (rc) return rc;
        }
        if (fused) {
            // the fused kernel took steps of its own: the last block time is on the device
            CK(h, cudaMemcpyAsync(&h->t_cur, &h->sd->t_cur, sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream));
        }
    }
    h->predicted = false;
    h->last_force_n = -1;
    rc = check_err(h);
    {
        const int rc2 = fold_fused_stats(h);
        if (!rc) rc = rc2;
    }
    sync_stats_counters(h);
    if (st) {
        nb_stats d = h->stats;
        d.block_steps -= before.block_steps;
        d.force_launches -= before.force_launches;
        d.interactions -= before.interactions;
        d.force_ms -= before.force_ms;
        d.reduce_ms -= before.reduce_ms;
        d.predict_ms -= before.predict_ms;
        d.correct_ms -= before.correct_ms;
        d.sched_ms -= before.sched_ms;
        d.dt_min_hits -= before.dt_min_hits;
        for (int k = 0; k < 32; ++k) {
            d.active_hist[k] -= before.active_hist[k];
            d.force_ms_hist[k] -= before.force_ms_hist[k];
            d.inter_hist[k] -= before.inter_hist[k];
        }
        d.kernel_launches -= before.kernel_launches;
        d.fused_steps -= before.fused_steps;
        d.fused_launches -= before.fused_launches;
        d.fused_ms -= before.fused_ms;
        for (int k = 0; k < 4; ++k) d.fused_stage_ms[k] -= before.fused_stage_ms[k];
        for (int k = 0; k < 32; ++k) d.fused_step_ms_hist[k] -= before.fused_step_ms_hist[k];
        *st = d;
    }
    return rc;
}

int nb_energy(nb_handle h, double *kin, double *pot)
{
    if (!h) return NB_ERR_ARG;
    if (!h->have_particles) return fail(h, NB_ERR_STATE, "no particles set");
    cudaSetDevice(h->dev);
    const int n = h->n;
    std::vector<double> tt(n);
    CK(h, cudaMemcpyAsync(tt.data(), h->t, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 1; i < n; ++i)
        if (tt[i] != tt[0]) return fail(h, NB_ERR_STATE, "particles are not synchronised");
    int rc = predict_to(h, tt[0]);  // d = 0: the predicted state is the current state
    if (rc) return rc;
    const bool was_pred = h->predicted;
    (void)was_pred;
    Out3 f{h->f_acc, h->f_jerk, h->f_pot, h->ld};
    // FP64 pair potential: the diagnostic is kept in binary64 whatever the variant
    const int saved = h->cfg.variant;
    ISet is = members_of(h, nullptr, n);
    rc = run_force(h, NB_F64, is, f);
    h->cfg.variant = saved;
    if (rc) return rc;
    CK(h, launch_energy(n, h->m, h->vel, h->ld, h->f_pot, h->d_energy, h->stream));
    h->stats.kernel_launches++;
    double e2[2] = {0, 0};
    CK(h, cudaMemcpyAsync(e2, h->d_energy, sizeof e2, cudaMemcpyDeviceToHost, h->stream));
    rc = check_err(h);
    if (rc) return rc;
    if (kin) *kin = e2[0];
    if (pot) *pot = e2[1];
    h->predicted = false;
    return NB_OK;
}

int nb_get_stats(nb_handle h, nb_stats *st)
{
    if (!h || !st) return NB_ERR_ARG;
    cudaSetDevice(h->dev);
    cudaStreamSynchronize(h->stream);
    sync_stats_counters(h);
    *st = h->stats;
    return NB_OK;
}

int nb_reset_stats(nb_handle h)
{
    if (!h) return NB_ERR_ARG;
    cudaSetDevice(h->dev);
    cudaStreamSynchronize(h->stream);
    h->timer.harvest();
    for (double &x : h->timer.ms) x = 0.0;
    for (double &x : h->timer.force_hist) x = 0.0;
    std::memset(&h->stats, 0, sizeof h->stats);
    cudaMemsetAsync(h->d_dtmin, 0, sizeof(unsigned long long), h->stream);
    cudaStreamSynchronize(h->stream);
    return NB_OK;
}

int nb_plan_for(nb_handle h, int n_i, nb_plan *out)
{
    if (!h || !out || n_i < 1) return NB_ERR_ARG;
    if (!h->have_particles) return fail(h, NB_ERR_STATE, "no particles set");
    *out = entry_of(order6(h) ? plan_for6(h, h->cfg.variant, n_i)
                              : plan_for(h, h->cfg.variant, n_i));
    return NB_OK;
}

int nb_set_plan_table(nb_handle h, const nb_plan *table, int n)
{
    if (!h) return NB_ERR_ARG;
    if (!table) {
        for (int b = 0; b < 32; ++b) {
            h->plans[b] = nb_plan{-1, 1, 1};
            h->plan_tuned[b] = false;
        }
        return NB_OK;
    }
    if (n < 0 || n > 32) return fail(h, NB_ERR_ARG, "plan table has %d entries (max 32)", n);
    for (int b = 0; b < n; ++b) {
        const nb_plan &e = table[b];
        if (e.kind < -1 || e.kind > 2 || (e.kind >= 0 && e.nsplit < 1))
            return fail(h, NB_ERR_ARG, "plan entry %d is malformed", b);
        if (order6(h) && e.kind > 0)
            return fail(h, NB_ERR_ARG, "plan entry %d: order 6 has the tile kind only", b);
        if (order6(h) && e.kind == 0 && !(e.nwj == 1 || e.nwj == 2 || e.nwj == 4 || e.nwj == 8))
            return fail(h, NB_ERR_ARG, "plan entry %d: nwj must be 1, 2, 4 or 8", b);
        if (!order6(h) && e.kind == 0 && !(e.nwj == 1 || e.nwj == 4 || e.nwj == 8))
            return fail(h, NB_ERR_ARG, "plan entry %d: nwj must be 1, 4 or 8", b);
    }
    for (int b = 0; b < 32; ++b) {
        h->plans[b] = b < n ? table[b] : nb_plan{-1, 1, 1};
        h->plan_tuned[b] = false;
    }
    return NB_OK;
}

int nb_get_plan_table(nb_handle h, nb_plan *table)
{
    if (!h || !table) return NB_ERR_ARG;
    for (int b = 0; b < 32; ++b) table[b] = h->plans[b];
    return NB_OK;
}

int autotune6(nb_handle h, int reps);

int nb_autotune(nb_handle h, int reps)
{
    if (!h) return NB_ERR_ARG;
    if (!h->have_particles) return fail(h, NB_ERR_STATE, "no particles set");
    if (order6(h)) return autotune6(h, reps);
    if (reps < 1) reps = 1;
    cudaSetDevice(h->dev);
    const int n = h->n;
    const int variant = h->cfg.variant;
    // predict the j-set to the latest own time (valid for every particle)
    std::vector<double> tt(n);
    CK(h, cudaMemcpyAsync(tt.data(), h->t, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    double tmax = tt[0];
    for (int i = 1; i < n; ++i) tmax = std::max(tmax, tt[i]);
    int rc = predict_to(h, tmax);
    if (rc) return rc;
    const int saved_flags = h->cfg.flags;
    h->cfg.flags &= ~NB_FLAG_TIMING;  // the tuner's own events only
    const nb_stats saved_stats = h->stats;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    const int bmax = bucket_of(n);
    for (int b = 0; b <= bmax && rc == NB_OK; ++b) {
        const int n_i = (int)std::min<long long>(1LL << b, n);
        std::vector<int> idx(n_i);
        for (int k = 0; k < n_i; ++k) idx[k] = (int)((long long)k * n / n_i);
        rc = grow(h, &h->d_idx, &h->idx_cap, (size_t)n_i);
        if (rc) break;
        rc = grow(h, &h->io, &h->io_cap, 7 * (size_t)n_i);
        if (rc) break;
        CK(h, cudaMemcpyAsync(h->d_idx, idx.data(), n_i * sizeof(int), cudaMemcpyHostToDevice,
                              h->stream));
        const ISet is = members_of(h, h->d_idx, n_i);
        Out3 out{h->io, h->io + 3 * (size_t)n_i, h->io + 6 * (size_t)n_i, n_i};
        // candidates around the heuristic plan
        std::vector<ForcePlan> cand;
        const ForcePlan base = plan_force(variant, n_i, n, h->num_sms);
        std::vector<nb_plan> entries;
        if (variant != NB_F64 && n_i <= 32) entries.push_back(nb_plan{2, 1, 1});
        const int kinds_nwj[4][2] = {{1, 1}, {0, 1}, {0, 4}, {0, 8}};
        for (auto &kn : kinds_nwj) {
            const int kind = kn[0], nwj = kn[1];
            if (kind == 1 && n_i > 8192) continue;
            if (kind == 0 && n_i < 16) continue;
            if (variant == NB_F64 && nwj != 1) continue;
            if (variant == NB_F64 && kind == 1 && n_i > 32) continue;
            nb_plan probe{kind, nwj, 1};
            ForcePlan one = plan_from_entry(probe, variant, n_i, n);
            long long g;
            if (kind == 1) {
                const long long groups = variant == NB_F64 ? 1 : (n_i + one.ipt - 1) / one.ipt;
                g = std::max(1LL, (16LL * h->num_sms + groups - 1) / groups);
            } else {
                const long long ib = (long long)(one.threads / one.nwj) * one.ipt;
                const long long nblk = (n_i + ib - 1) / ib;
                g = std::max(1LL, (4LL * h->num_sms + nblk - 1) / nblk);
            }
            for (long long f : {1LL, 2LL, 4LL, 8LL, 16LL}) {
                for (int dir = 0; dir < 2; ++dir) {
                    long long ns = dir ? g * f : g / f;
                    if (ns < 1 || (dir && f == 1)) continue;
                    entries.push_back(nb_plan{kind, nwj, (int)ns});
                }
            }
            if (kind == 0 && variant != NB_F64) {
                // splits that fill whole waves of resident CTAs (no ragged last wave)
                const long long ib = (long long)(one.threads / one.nwj) * one.ipt;
                const long long nblk = (n_i + ib - 1) / ib;
                const long long slots = (long long)h->num_sms * tile_blocks_per_sm(variant, nwj);
                long long last = 0;
                for (long long k = 1; k <= 8; ++k) {
                    const long long ns = (k * slots + nblk / 2) / nblk;  // nearest
                    if (ns >= 1 && ns != last && ns <= 256)
                        entries.push_back(nb_plan{kind, nwj, (int)ns});
                    last = ns;
                }
            }
        }
        entries.push_back(entry_of(base));
        double best = 1e30;
        nb_plan best_e = entry_of(base);
        for (const nb_plan &e : entries) {
            const ForcePlan p = plan_from_entry(e, variant, n_i, n);
            rc = run_force_plan(h, variant, p, is, out);  // warm-up
            if (rc) break;
            std::vector<float> ms;
            for (int r = 0; r < reps; ++r) {
                CK(h, cudaEventRecord(e0, h->stream));
                rc = run_force_plan(h, variant, p, is, out);
                if (rc) break;
                CK(h, cudaEventRecord(e1, h->stream));
                CK(h, cudaEventSynchronize(e1));
                float t = 0.f;
                CK(h, cudaEventElapsedTime(&t, e0, e1));
                ms.push_back(t);
            }
            if (rc) break;
            std::sort(ms.begin(), ms.end());
            const double med = ms[ms.size() / 2];
            if (med < best) {
                best = med;
                best_e = entry_of(p);
            }
        }
        if (rc == NB_OK) {
            h->plans[b] = best_e;
            h->plan_tuned[b] = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cfg.flags = saved_flags;
    h->stats = saved_stats;
    h->predicted = false;
    h->last_force_n = -1;
    if (rc) return rc;
    return check_err(h);
}

// nb_autotune of a 6th-order handle (F32-DS pairs; FP64 keeps the built-in rule):
// for every bucket up to N, at n_i = min(2^b, N) evenly spread members, the
// 6th-order tile kernel with 1, 2, 4 and 8 warp rows, each with the split counts
// that fill 1..8 whole waves of resident CTAs (rounded down), and the built-in
// plan; the fastest median of reps timed launches goes into the plan table.
int autotune6(nb_handle h, int reps)
{
    if (reps < 1) reps = 1;
    const int variant = h->cfg.variant;
    if (variant == NB_F64) return NB_OK;
    cudaSetDevice(h->dev);
    const int n = h->n;
    std::vector<double> tt(n);
    CK(h, cudaMemcpyAsync(tt.data(), h->t, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    double tmax = tt[0];
    for (int i = 1; i < n; ++i) tmax = std::max(tmax, tt[i]);
    int rc = predict_to(h, tmax);
    if (rc) return rc;
    const int saved_flags = h->cfg.flags;
    h->cfg.flags &= ~NB_FLAG_TIMING;  // the tuner's own events only
    const nb_stats saved_stats = h->stats;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    const int bmax = bucket_of(n);
    const long long ntiles = (n + 127) / 128;
    for (int b = 0; b <= bmax && rc == NB_OK; ++b) {
        const int n_i = (int)std::min<long long>(1LL << b, n);
        std::vector<int> idx(n_i);
        for (int k = 0; k < n_i; ++k) idx[k] = (int)((long long)k * n / n_i);
        rc = grow(h, &h->d_idx, &h->idx_cap, (size_t)n_i);
        if (rc) break;
        rc = grow(h, &h->io, &h->io_cap, 10 * (size_t)n_i);
        if (rc) break;
        CK(h, cudaMemcpyAsync(h->d_idx, idx.data(), n_i * sizeof(int), cudaMemcpyHostToDevice,
                              h->stream));
        const Out6 out{h->io, h->io + 3 * (size_t)n_i, h->io + 6 * (size_t)n_i,
                       h->io + 9 * (size_t)n_i, n_i};
        const ForcePlan base = plan_force6(variant, n_i, n, h->num_sms);
        std::vector<nb_plan> entries{entry_of(base)};
        for (int nwj = 1; nwj <= 8; nwj *= 2) {
            const long long ib = 32LL * (8 / nwj);
            const long long nblk = (n_i + ib - 1) / ib;
            const long long slots = (long long)h->num_sms * occ6_blocks(variant, nwj);
            long long last = 0;
            for (long long k = 1; k <= 8; ++k) {
                const long long ns = std::min(std::min(ntiles, 1024LL), std::max(1LL, k * slots / nblk));
                if (ns != last) entries.push_back(nb_plan{0, nwj, (int)ns});
                last = ns;
            }
        }
        double best = 1e30;
        nb_plan best_e = entry_of(base);
        for (const nb_plan &e : entries) {
            const ForcePlan p = plan6_from_entry(variant, e.nwj, e.nsplit, n_i, n);
            rc = run_force6_plan(h, variant, p, h->d_idx, n_i, out);  // warm-up
            if (rc) break;
            std::vector<float> ms;
            for (int r = 0; r < reps; ++r) {
                CK(h, cudaEventRecord(e0, h->stream));
                rc = run_force6_plan(h, variant, p, h->d_idx, n_i, out);
                if (rc) break;
                CK(h, cudaEventRecord(e1, h->stream));
                CK(h, cudaEventSynchronize(e1));
                float t = 0.f;
                CK(h, cudaEventElapsedTime(&t, e0, e1));
                ms.push_back(t);
            }
            if (rc) break;
            std::sort(ms.begin(), ms.end());
            const double med = ms[ms.size() / 2];
            if (med < best) {
                best = med;
                best_e = entry_of(p);
            }
        }
        if (rc == NB_OK) {
            h->plans[b] = best_e;
            h->plan_tuned[b] = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cfg.flags = saved_flags;
    h->stats = saved_stats;
    h->predicted = false;
    h->last_force_n = -1;
    if (rc) return rc;
    return check_err(h);
}

int nb_kick_ext(nb_handle target, nb_handle field, double dt_kick)
{
    if (!target || !field || target == field) return NB_ERR_ARG;
    if (order6(target) || order6(field))
        return fail(target, NB_ERR_ARG, "bridge kicks take 4th-order systems");
    if (!std::isfinite(dt_kick)) return fail(target, NB_ERR_ARG, "dt_kick is not finite");
    if (target->dev != field->dev)
        return fail(target, NB_ERR_ARG, "the two systems are on different devices");
    if (!target->have_particles || !field->have_particles)
        return fail(target, NB_ERR_STATE, "no particles set");
    cudaSetDevice(target->dev);
    for (nb_handle h : {target, field})
        if (!h->initialised) {
            int rc = do_init(h);
            if (rc) return h == target ? rc : fail(target, rc, "field: %s", h->msg.c_str());
        }
    return kick_by(target, field, dt_kick);
}

// A step length that keeps a system synchronised: a multiple of its shared
// step, or of dt_max with block steps.
static bool keeps_sync(nb_handle h, double dt)
{
    const double unit = h->cfg.shared_dt > 0.0 ? h->cfg.shared_dt : h->cfg.dt_max;
    const double q = dt / unit;
    return q >= 1.0 && q == std::floor(q) && q < 1e15;
}

int nb_bridge_step(nb_handle a, nb_handle b, double dt)
{
    if (!a || !b || a == b) return NB_ERR_ARG;
    if (order6(a) || order6(b)) return fail(a, NB_ERR_ARG, "bridge steps take 4th-order systems");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(a, NB_ERR_ARG, "dt must be > 0");
    if (a->dev != b->dev) return fail(a, NB_ERR_ARG, "the two systems are on different devices");
    if (!a->have_particles || !b->have_particles) return fail(a, NB_ERR_STATE, "no particles set");
    if (!keeps_sync(a, dt) || !keeps_sync(b, dt))
        return fail(a, NB_ERR_ARG, "dt must be a multiple of both systems' dt_max (or shared step)");
    cudaSetDevice(a->dev);
    for (nb_handle h : {a, b})
        if (!h->initialised) {
            int rc = do_init(h);
            if (rc) return h == a ? rc : fail(a, rc, "second system: %s", h->msg.c_str());
        }
    const double t = a->t_cur;
    int rc;
    if ((rc = kick_by(a, b, 0.5 * dt))) return rc;
    if ((rc = kick_by(b, a, 0.5 * dt))) return fail(a, rc, "second system: %s", b->msg.c_str());
    if ((rc = nb_step(a, t + dt, nullptr))) return rc;
    if ((rc = nb_step(b, t + dt, nullptr))) return fail(a, rc, "second system: %s", b->msg.c_str());
    if ((rc = kick_by(a, b, 0.5 * dt))) return rc;
    if ((rc = kick_by(b, a, 0.5 * dt))) return fail(a, rc, "second system: %s", b->msg.c_str());
    return NB_OK;
}

int nb_selftest_wait(int which, double limit_s, int device)
{
    if (which < 0 || which > 1 || !(limit_s > 0.0) || limit_s > 2.0) return NB_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return NB_ERR_CUDA;
    unsigned *d = nullptr;  // [0..2] barrier words, [3] error word
    if (cudaMalloc(&d, 4 * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return NB_ERR_OOM;
    }
    cudaStream_t st = nullptr;
    unsigned e = 0;
    const unsigned long long limit_ns = (unsigned long long)(limit_s * 1e9);
    cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(d, 0, 4 * sizeof(unsigned), st);
    if (ce == cudaSuccess)
        ce = which == 0 ? launch_selftest_mbar(d + 3, limit_ns, st)
                        : launch_selftest_barrier(d, d + 3, limit_ns, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(&e, d + 3, sizeof e, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (st) cudaStreamDestroy(st);
    cudaFree(d);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    return (e & DERR_TIMEOUT) ? NB_ERR_TIMEOUT : NB_ERR_STATE;
}

}  // extern "C"
