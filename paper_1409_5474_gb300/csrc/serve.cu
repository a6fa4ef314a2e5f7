// The serving loop (nbody.h, nb_server_* / nb_submit / nb_poll): continuous
// batching of force and integration requests on subsystems of uneven N.
//
// A server thread owns the GPU work; submit/poll/cancel only touch the
// request table under a mutex. Each tick the thread
//   1. retires cancelled requests and admits queued ones (arrival order)
//      while the in-flight limit and the device-memory budget allow; an
//      admitted request gets an engine handle from a pool (by capacity
//      class) and its particles are copied in once - they stay on the GPU;
//   2. builds the tick's descriptors and uploads them in one copy: force work
//      items for new FORCE requests (every particle against every particle),
//      new EVOLVE requests (their initial evaluation) and the due set of every
//      stepping EVOLVE request (the records its scheduler gathered), with
//      j-splits for small i-sets; one corrector job and one scheduler job per
//      integration that goes on;
//   3. launches the batched force (i-parallel and j-parallel items on two
//      streams, then the fixed-order sums of the j-split groups), the initial
//      steps of new integrations, ONE corrector launch and ONE scheduler +
//      predictor launch over all integrations, and the copies of finished
//      results;
//   4. synchronises once, checks every request's error word and mailbox,
//      and retires finished requests, returning their handles to the pool.
// A request's items, splits and summation order depend only on the request
// itself (and the SM count), so its results are the same whatever else is in
// flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "nb_internal.cuh"

using namespace nb;

namespace {

enum Phase { PH_QUEUED = 0, PH_FORCE, PH_INIT, PH_STEP, PH_FINISHED };

struct Req {
    uint64_t id = 0;
    int kind = NB_REQ_FORCE;
    int n = 0;
    double eps = 0.0, t_span = 0.0;
    std::vector<double> m, pos, vel;  // the request's particles (host copy)
    int status = NB_STATUS_QUEUED;
    int error = NB_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
    double interactions = 0.0;
    long long block_steps = 0;
    bool cancel = false;
    // device side (server thread only)
    nb_handle h = nullptr;
    int cap = 0;
    size_t bytes = 0;
    int slot = -1;  // error word index
    int phase = PH_QUEUED;
    double t_end = 0.0;
    double t_next = 0.0;
    int n_active = 0;
    unsigned long long epoch = 0;
    bool final_copy = false;  // EVOLVE: t_end reached, results being copied out
    double tick_inter = 0.0;  // interactions / block steps of the running tick,
    long long tick_steps = 0; // published under the lock when it ends
    int pending = NB_OK;      // failure found on the host during the tick
    // results
    std::vector<double> acc, jerk, pot, out_pos, out_vel;
};

using ReqP = std::shared_ptr<Req>;

constexpr int NSIDE = 4;  // side streams of the engine-planned force launches

int capacity_class(int n)
{
    int c = 256;
    while (c < n) c <<= 1;
    return c;
}

}  // namespace

struct nb_server_s {
    nb_server_cfg cfg{};
    int dev = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;            // the j-parallel items, beside the rest
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t side[NSIDE] = {};             // engine-planned force launches
    cudaEvent_t ev_side[NSIDE] = {};
    std::chrono::steady_clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<uint64_t, ReqP> table;
    std::deque<ReqP> queue;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread thread;

    // server-thread state
    std::vector<ReqP> inflight;
    std::map<int, std::vector<nb_handle>> pool;  // idle handles by capacity class
    size_t bytes_in_use = 0;                      // in-flight + pooled handles
    std::vector<int> free_slots;
    unsigned *d_errs = nullptr;                   // one error word per slot
    unsigned *h_errs = nullptr;                   // their pinned host copy
    unsigned long long *d_dtmin = nullptr;        // corrector dt_min clamps
    char *d_stage = nullptr, *h_stage = nullptr;  // the tick's descriptors
    size_t stage_cap = 0;
    float2 *d_part = nullptr;          // j-split partials of the tick
    size_t part_cap = 0;               // float2
    int threads = 128, grid = 0, grid_jpar = 0;
    nb_server_stats st{};
    int fatal = NB_OK;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

size_t estimate_bytes(int cap)
{
    // the engine slab for cap particles plus its small buffers (see engine.cu)
    const size_t ld = ((size_t)cap + 63) / 64 * 64;
    const size_t vec = ((3 * ld + 64) * 8 + 255) & ~size_t(255);
    const size_t sca = ((ld + 64) * 8 + 255) & ~size_t(255);
    const size_t recb = (ld * 48 + 255) & ~size_t(255);
    const size_t actb = (ld * 4 + 255) & ~size_t(255);
    return 8 * vec + 4 * sca + 2 * recb + actb + 65536;
}

// A handle of capacity class cap: from the pool, else created (freeing pooled
// handles of other classes when the budget needs it). Server thread only.
nb_handle acquire_handle(nb_server s, int cap, size_t *bytes)
{
    auto &v = s->pool[cap];
    if (!v.empty()) {
        nb_handle h = v.back();
        v.pop_back();
        *bytes = handle_bytes(h);
        return h;
    }
    const size_t need = estimate_bytes(cap);
    for (auto &kv : s->pool) {
        while (s->bytes_in_use + need > s->cfg.budget_bytes && !kv.second.empty()) {
            nb_handle old = kv.second.back();
            kv.second.pop_back();
            s->bytes_in_use -= handle_bytes(old);
            nb_destroy(old);
        }
    }
    nb_config c;
    nb_config_default(&c);
    c.n_max = cap;
    c.variant = s->cfg.variant;
    c.eta = s->cfg.eta;
    c.dt_max = s->cfg.dt_max;
    c.device = s->dev;
    nb_handle h = nullptr;
    if (nb_create(&c, &h) != NB_OK) return nullptr;
    nb_set_stream(h, s->stream);
    *bytes = handle_bytes(h);
    s->bytes_in_use += *bytes;
    return h;
}

StepParams server_params(nb_server s)
{
    StepParams p{};
    p.eta = s->cfg.eta;
    p.eta_s = s->cfg.eta;
    p.dt_min = std::ldexp(1.0, -30);
    p.dt_max = s->cfg.dt_max;
    p.shared_dt = 0.0;
    return p;
}

}  // namespace

// ---------------------------------------------------------------------------
// Server thread
// ---------------------------------------------------------------------------

namespace {

#define CKS(call)                                              \
    do {                                                       \
        if ((call) != cudaSuccess) return NB_ERR_CUDA;         \
    } while (0)

int err_code(unsigned bits)
{
    if (bits & DERR_TIMEOUT) return NB_ERR_TIMEOUT;
    if (bits & DERR_NONFINITE) return NB_ERR_NONFINITE;
    return NB_ERR_STATE;
}

// Terminal status of r (lock held): counters, timestamps; frees nothing.
void finish_locked(nb_server s, Req &r, int status, int error)
{
    r.status = status;
    r.error = error;
    r.t_done = s->now();
    r.phase = PH_FINISHED;
    if (status == NB_STATUS_DONE)
        s->st.completed++;
    else if (status == NB_STATUS_CANCELLED)
        s->st.cancelled++;
    else
        s->st.failed++;
    // the particles are not needed any more
    std::vector<double>().swap(r.m);
    if (r.kind == NB_REQ_FORCE) {
        std::vector<double>().swap(r.pos);
        std::vector<double>().swap(r.vel);
    }
}

// Give r's handle back to the pool (reuse) or free it (after a failure, when
// its scheduler state may not match the host's epoch mirror).
void drop_handle(nb_server s, Req &r, bool reuse)
{
    if (r.h) {
        if (reuse) {
            s->pool[r.cap].push_back(r.h);
        } else {
            s->bytes_in_use -= handle_bytes(r.h);
            nb_destroy(r.h);
        }
    }
    r.h = nullptr;
    if (r.slot >= 0) s->free_slots.push_back(r.slot);
    r.slot = -1;
}

size_t inflight_bytes(nb_server s)
{
    size_t b = 0;
    for (auto &r : s->inflight) b += r->bytes;
    return b;
}

bool fits(nb_server s, const Req &r, size_t in_use)
{
    auto it = s->pool.find(r.cap);
    if (it != s->pool.end() && !it->second.empty()) return true;
    return in_use + estimate_bytes(r.cap) <= s->cfg.budget_bytes;
}

// The work items of one tick's batched force launch, with the scratch their
// j-split groups need (float2 offsets and counter indices until the buffers are
// sized; -1 = no split).
// A group large enough for the engine's own planned kernels (one launch).
struct EngineGroup {
    Req *r;
    int n_i;
    bool due;
};

struct TickItems {
    std::vector<EngineGroup> engine;
    std::vector<WorkItem> items;
    std::vector<long long> part_off;   // per item
    std::vector<SplitGroup> groups;
    std::vector<long long> group_off;  // per group
    size_t part_total = 0;
    double interactions = 0.0;
};

// Smallest j-range of an item in a j-split group (i-parallel, j-parallel).
constexpr int ITEM_MIN_J_IPAR = 1024;
constexpr int ITEM_MIN_J_JPAR = 2048;
// Groups of more i-rows than the j-parallel items take and at least this many
// interactions run on the engine's planned kernels (tile / warp-group kernels
// with their tuned j-splits) in a launch of their own, on one of the side
// streams; smaller work shares the batched item launch.
constexpr double ENGINE_MIN_INTERACTIONS = 4194304.0;

// Items of n_i i-rows of irec (member rows when !gathered) against all r.n
// j-records of r. Small i-sets become j-parallel items; the j-range is split
// so that the request alone yields about four items per SM, as long as every
// item keeps a minimum j-range. The split depends only on (n_i, r.n) and the
// SM count, never on the other requests of the tick, so a request's results
// are the same alone and in any mix.
void add_group(nb_server s, Req &r, const HandleView &v, const float4 *irec, int n_i,
               int gathered, TickItems &t)
{
    const double inter = (double)n_i * (double)r.n;
    r.tick_inter += inter;
    t.interactions += inter;
    if (n_i > ITEM_JPAR_MAX_NI && inter >= ENGINE_MIN_INTERACTIONS) {
        t.engine.push_back(EngineGroup{&r, n_i, gathered != 0});
        return;
    }
    const int ib = s->threads * 2;
    const bool jpar = n_i <= ITEM_JPAR_MAX_NI;
    const int nblk = jpar ? 1 : (n_i + ib - 1) / ib;
    const int jmin = jpar ? ITEM_MIN_J_JPAR : ITEM_MIN_J_IPAR;
    const int target = 4 * s->num_sms;
    int nsplit = std::max(1, std::min((r.n + jmin - 1) / jmin, (target + nblk - 1) / nblk));
    int chunk = (r.n + nsplit - 1) / nsplit;
    chunk = (chunk + 31) / 32 * 32;
    nsplit = (r.n + chunk - 1) / chunk;
    for (int blk = 0; blk < nblk; ++blk) {
        const int i0 = blk * ib;
        const int ni = jpar ? n_i : std::min(ib, n_i - i0);
        long long poff = -1;
        if (nsplit > 1) {
            poff = (long long)t.part_total;
            t.part_total += (size_t)nsplit * 7 * ni;
            SplitGroup g{};
            g.acc = v.f_acc;
            g.jerk = v.f_jerk;
            g.pot = v.f_pot;
            g.ld = v.ld;
            g.i0 = i0;
            g.ni = ni;
            g.nsplit = nsplit;
            g.err = s->d_errs + r.slot;
            t.groups.push_back(g);
            t.group_off.push_back(poff);
        }
        for (int sp = 0; sp < nsplit; ++sp) {
            WorkItem w{};
            w.jrec = v.s.rec;
            w.irec = irec;
            w.acc = v.f_acc;
            w.jerk = v.f_jerk;
            w.pot = v.f_pot;
            w.ld = v.ld;
            w.i0 = i0;
            w.ni = ni;
            w.j0 = sp * chunk;
            w.nj = std::min(chunk, r.n - w.j0);
            w.gathered = gathered;
            w.kind = jpar ? 1 : 0;
            w.split = sp;
            w.nsplit = nsplit;
            w.eps2 = (float)(r.eps * r.eps);
            w.err = s->d_errs + r.slot;
            t.items.push_back(w);
            t.part_off.push_back(poff);
        }
    }
}

// Per-thread work of an item, for ordering the list (longest first).
double item_cost(const WorkItem &w, int threads)
{
    if (w.kind == 1) return (double)((w.ni + 3) / 4 * 4) * w.nj / threads;
    return 2.0 * w.nj;
}

HandleView view_of(const Req &r)
{
    HandleView v;
    handle_view(r.h, &v);
    v.s.n = r.n;
    return v;
}

// Copy r's particles into its handle (time 0) and predict, which builds the
// j-records. Queued on the server stream.
int upload(nb_server s, Req &r)
{
    const HandleView v = view_of(r);
    cudaStream_t st = s->stream;
    const size_t row = (size_t)r.n * sizeof(double), pitch = (size_t)v.ld * sizeof(double);
    unsigned *err = s->d_errs + r.slot;
    handle_attach(r.h, r.n);
    CKS(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
    CKS(cudaMemcpyAsync(v.s.m, r.m.data(), row, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpy2DAsync(v.s.pos, pitch, r.pos.data(), row, row, 3, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpy2DAsync(v.s.vel, pitch, r.vel.data(), row, row, 3, cudaMemcpyHostToDevice, st));
    CKS(cudaMemsetAsync(v.s.t, 0, row, st));
    CKS(cudaMemsetAsync(v.s.dt, 0, row, st));
    CKS(launch_predict(v.s, 0.0, true, err, st));
    return NB_OK;
}

int grow_stage(nb_server s, size_t bytes)
{
    if (bytes <= s->stage_cap) return NB_OK;
    const size_t cap = std::max<size_t>(bytes, 2 * s->stage_cap);
    if (s->d_stage) cudaFree(s->d_stage);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    s->d_stage = nullptr;
    s->h_stage = nullptr;
    s->stage_cap = 0;
    CKS(cudaMalloc(&s->d_stage, cap));
    CKS(cudaMallocHost(&s->h_stage, cap));
    s->stage_cap = cap;
    return NB_OK;
}

int grow_scratch(nb_server s, size_t part, size_t)
{
    if (part > s->part_cap) {
        const size_t cap = std::max(part, 2 * s->part_cap);
        if (s->d_part) cudaFree(s->d_part);
        s->d_part = nullptr;
        s->part_cap = 0;
        CKS(cudaMalloc(&s->d_part, cap * sizeof(float2)));
        s->part_cap = cap;
    }
    return NB_OK;
}

}  // namespace

namespace {

// One tick (server thread): cancellations, admission, one batched force
// launch, the per-request kernels and copies, one synchronisation, and the
// bookkeeping of what finished. A CUDA failure returns NB_ERR_CUDA.
int tick(nb_server s)
{
    const cudaStream_t st = s->stream;
    std::vector<ReqP> admitted;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // running requests that were cancelled (none of their work is on the GPU)
        for (auto &r : s->inflight)
            if (r->cancel && r->phase != PH_FINISHED) {
                finish_locked(s, *r, NB_STATUS_CANCELLED, NB_OK);
                drop_handle(s, *r, true);
            }
        s->inflight.erase(std::remove_if(s->inflight.begin(), s->inflight.end(),
                                         [](const ReqP &r) { return r->phase == PH_FINISHED; }),
                          s->inflight.end());
        // admission in arrival order, while the in-flight limit and the budget allow
        size_t in_use = inflight_bytes(s);
        while (!s->queue.empty() && (int)s->inflight.size() < s->cfg.max_inflight) {
            ReqP r = s->queue.front();
            if (!s->inflight.empty() && !fits(s, *r, in_use)) break;
            s->queue.pop_front();
            r->status = NB_STATUS_RUNNING;
            r->t_start = s->now();
            admitted.push_back(r);
            s->inflight.push_back(r);
            in_use += estimate_bytes(r->cap);
        }
        s->st.queued = (int)s->queue.size();
        s->st.inflight = (int)s->inflight.size();
    }
    if (s->inflight.empty()) return NB_OK;
    const double t_begin = s->now();

    // handles and uploads of the admitted requests
    for (auto &r : admitted) {
        r->h = acquire_handle(s, r->cap, &r->bytes);
        if (!r->h) {
            r->pending = NB_ERR_OOM;
            continue;
        }
        r->slot = s->free_slots.back();
        s->free_slots.pop_back();
        int rc = upload(s, *r);
        if (rc) return rc;
    }

    // this tick's descriptors: force items, split groups, corrector jobs and
    // scheduler jobs (uploaded together)
    TickItems ti;
    std::vector<CorrectJob> cjobs;
    std::vector<SchedJob> sjobs;
    int c_blocks = 0, s_blocks = 0;
    const StepParams prm = server_params(s);
    for (auto &r : s->inflight) {
        if (r->pending) continue;
        const HandleView v = view_of(*r);
        unsigned *err = s->d_errs + r->slot;
        if (r->phase == PH_QUEUED) {
            add_group(s, *r, v, v.s.rec, r->n, 0, ti);
            r->phase = r->kind == NB_REQ_FORCE ? PH_FORCE : PH_INIT;
        } else if (r->phase == PH_STEP) {
            // the last scheduler launch finished before the previous tick ended
            if (v.mail_h->seq != r->epoch) {
                r->pending = NB_ERR_STATE;
                continue;
            }
            const double t_next = v.mail_h->t_next;
            const int na = v.mail_h->n_active;
            if (!(t_next <= r->t_end)) {
                r->final_copy = true;
                continue;
            }
            if (na < 1 || na > r->n) {
                r->pending = NB_ERR_STATE;
                continue;
            }
            r->t_next = t_next;
            r->n_active = na;
            add_group(s, *r, v, v.irec, na, 1, ti);
            CorrectJob j{};
            j.s = v.s;
            j.act = v.act;
            j.na = na;
            j.block0 = c_blocks;
            j.t_new = t_next;
            j.f = Out3{v.f_acc, v.f_jerk, v.f_pot, v.ld};
            j.sd = v.sd;
            j.err = err;
            cjobs.push_back(j);
            c_blocks += (na + CORRECT_THREADS - 1) / CORRECT_THREADS;
            r->tick_steps++;
        }
        if (r->phase == PH_INIT || r->phase == PH_STEP) {
            // the integration goes on: its next scheduler launch
            SchedJob q{};
            q.s = v.s;
            q.sd = v.sd;
            q.status = v.sched_status;
            q.act = v.act;
            q.irec = v.irec;
            q.mail = v.mail_d;
            q.err = err;
            q.block0 = s_blocks;
            q.ntiles = (r->n + SCHED_TILE - 1) / SCHED_TILE;
            sjobs.push_back(q);
            s_blocks += q.ntiles;
            r->epoch = handle_take_epoch(r->h);
        }
    }

    std::vector<WorkItem> &items = ti.items;
    int n0 = 0, n1 = 0;
    if (!items.empty()) {
        int rc = grow_scratch(s, ti.part_total, 0);
        if (rc) return rc;
        for (size_t k = 0; k < items.size(); ++k)
            if (ti.part_off[k] >= 0) items[k].part = s->d_part + ti.part_off[k];
        for (size_t g = 0; g < ti.groups.size(); ++g) ti.groups[g].part = s->d_part + ti.group_off[g];
        // i-parallel items, then j-parallel ones, each longest first (the
        // persistent CTAs take them round-robin)
        const int nt = s->threads;
        std::stable_sort(items.begin(), items.end(), [nt](const WorkItem &x, const WorkItem &y) {
            if (x.kind != y.kind) return x.kind < y.kind;
            return item_cost(x, nt) > item_cost(y, nt);
        });
        n0 = (int)(std::lower_bound(items.begin(), items.end(), 1,
                                    [](const WorkItem &w, int k) { return w.kind < k; }) -
                   items.begin());
        n1 = (int)items.size() - n0;
    }
    // one upload of every descriptor
    size_t off_items = 0, off_groups, off_c, off_s, total;
    {
        auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
        off_groups = up(off_items + items.size() * sizeof(WorkItem));
        off_c = up(off_groups + ti.groups.size() * sizeof(SplitGroup));
        off_s = up(off_c + cjobs.size() * sizeof(CorrectJob));
        total = up(off_s + sjobs.size() * sizeof(SchedJob));
    }
    if (total > 0) {
        int rc = grow_stage(s, total);
        if (rc) return rc;
        char *h = s->h_stage;
        if (!items.empty()) std::memcpy(h + off_items, items.data(), items.size() * sizeof(WorkItem));
        if (!ti.groups.empty())
            std::memcpy(h + off_groups, ti.groups.data(), ti.groups.size() * sizeof(SplitGroup));
        if (!cjobs.empty()) std::memcpy(h + off_c, cjobs.data(), cjobs.size() * sizeof(CorrectJob));
        if (!sjobs.empty()) std::memcpy(h + off_s, sjobs.data(), sjobs.size() * sizeof(SchedJob));
        CKS(cudaMemcpyAsync(s->d_stage, h, total, cudaMemcpyHostToDevice, st));
    }
    const WorkItem *d_items = reinterpret_cast<const WorkItem *>(s->d_stage + off_items);
    long long launches = 0;

    // the batched force
    if (n1 > 0 || !ti.engine.empty()) CKS(cudaEventRecord(s->ev_fork, st));
    if (n1 > 0) {
        CKS(cudaStreamWaitEvent(s->stream2, s->ev_fork, 0));
        CKS(launch_force_items_jpar(s->cfg.variant, d_items + n0, n1, std::min(n1, s->grid_jpar),
                                    s->stream2));
        ++launches;
        CKS(cudaEventRecord(s->ev_join, s->stream2));
    }
    if (n0 > 0) {
        CKS(launch_force_items(s->cfg.variant, s->threads, d_items, n0, std::min(n0, s->grid), st));
        ++launches;
    }
    if (!ti.engine.empty()) {
        // the large groups: the engine's planned kernels, spread over the side streams
        const int nside = std::min<int>(NSIDE, (int)ti.engine.size());
        for (int k = 0; k < nside; ++k) CKS(cudaStreamWaitEvent(s->side[k], s->ev_fork, 0));
        for (size_t g = 0; g < ti.engine.size(); ++g) {
            const EngineGroup &eg = ti.engine[g];
            Req &r = *eg.r;
            const int rc = handle_force(r.h, eg.n_i, eg.due, r.eps * r.eps, s->d_errs + r.slot,
                                        s->side[g % NSIDE]);
            if (rc == NB_ERR_CUDA) return rc;
            if (rc) r.pending = rc;
            ++launches;
        }
        for (int k = 0; k < nside; ++k) {
            CKS(cudaEventRecord(s->ev_side[k], s->side[k]));
            CKS(cudaStreamWaitEvent(st, s->ev_side[k], 0));
        }
    }
    if (n1 > 0) CKS(cudaStreamWaitEvent(st, s->ev_join, 0));
    if (!ti.groups.empty()) {
        const int ng = (int)ti.groups.size();
        CKS(launch_split_reduce(reinterpret_cast<const SplitGroup *>(s->d_stage + off_groups), ng,
                                std::min(ng, 4 * s->num_sms), st));
        ++launches;
    }

    // initial steps of new integrations, then one corrector launch and one
    // scheduler launch over all integrations
    for (auto &r : s->inflight) {
        if (r->pending || r->phase != PH_INIT) continue;
        const HandleView v = view_of(*r);
        CKS(cudaMemsetAsync(v.sd->hist, 0, NLEVEL * sizeof(int), st));
        CKS(launch_init_steps(v.s, Out3{v.f_acc, v.f_jerk, v.f_pot, v.ld}, prm, v.sd,
                              s->d_errs + r->slot, st));
        ++launches;
    }
    CKS(launch_correct_multi(reinterpret_cast<const CorrectJob *>(s->d_stage + off_c),
                             (int)cjobs.size(), c_blocks, prm, s->d_dtmin, st));
    CKS(launch_sched_predict_multi(reinterpret_cast<const SchedJob *>(s->d_stage + off_s),
                                   (int)sjobs.size(), s_blocks, prm.dt_max, true, st));
    launches += (cjobs.empty() ? 0 : 1) + (sjobs.empty() ? 0 : 1) + (long long)admitted.size();

    // results leave the GPU
    for (auto &r : s->inflight) {
        if (r->pending) continue;
        const HandleView v = view_of(*r);
        const size_t row = (size_t)r->n * sizeof(double), pitch = (size_t)v.ld * sizeof(double);
        if (r->phase == PH_FORCE) {
            r->acc.resize(3 * (size_t)r->n);
            r->jerk.resize(3 * (size_t)r->n);
            r->pot.resize(r->n);
            CKS(cudaMemcpy2DAsync(r->acc.data(), row, v.f_acc, pitch, row, 3,
                                  cudaMemcpyDeviceToHost, st));
            CKS(cudaMemcpy2DAsync(r->jerk.data(), row, v.f_jerk, pitch, row, 3,
                                  cudaMemcpyDeviceToHost, st));
            CKS(cudaMemcpyAsync(r->pot.data(), v.f_pot, row, cudaMemcpyDeviceToHost, st));
        } else if (r->phase == PH_STEP && r->final_copy) {
            r->out_pos.resize(3 * (size_t)r->n);
            r->out_vel.resize(3 * (size_t)r->n);
            CKS(cudaMemcpy2DAsync(r->out_pos.data(), row, v.s.pos, pitch, row, 3,
                                  cudaMemcpyDeviceToHost, st));
            CKS(cudaMemcpy2DAsync(r->out_vel.data(), row, v.s.vel, pitch, row, 3,
                                  cudaMemcpyDeviceToHost, st));
        }
    }
    CKS(cudaMemcpyAsync(s->h_errs, s->d_errs, s->cfg.max_inflight * sizeof(unsigned),
                        cudaMemcpyDeviceToHost, st));
    CKS(cudaStreamSynchronize(st));

    // bookkeeping
    const double inter = ti.interactions;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &r : s->inflight) {
            r->interactions += r->tick_inter;
            r->block_steps += r->tick_steps;
            r->tick_inter = 0.0;
            r->tick_steps = 0;
            const unsigned bits = r->slot >= 0 ? s->h_errs[r->slot] : 0u;
            if (r->pending || bits) {
                finish_locked(s, *r, NB_STATUS_ERROR, r->pending ? r->pending : err_code(bits));
                drop_handle(s, *r, false);
            } else if (r->phase == PH_FORCE || r->final_copy) {
                finish_locked(s, *r, NB_STATUS_DONE, NB_OK);
                drop_handle(s, *r, true);
            } else if (r->phase == PH_INIT) {
                r->phase = PH_STEP;
            }
        }
        s->inflight.erase(std::remove_if(s->inflight.begin(), s->inflight.end(),
                                         [](const ReqP &r) { return r->phase == PH_FINISHED; }),
                          s->inflight.end());
        s->st.ticks++;
        if (!items.empty() || !ti.engine.empty()) s->st.force_launches++;
        s->st.kernel_launches += launches;
        s->st.interactions += inter;
        s->st.busy_s += s->now() - t_begin;
        s->st.inflight = (int)s->inflight.size();
        s->st.bytes_in_use = s->bytes_in_use;
    }
    s->cv_done.notify_all();
    return NB_OK;
}

void fail_all(nb_server s, int error)
{
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = error;
    for (auto &r : s->inflight) {
        if (r->phase != PH_FINISHED) finish_locked(s, *r, NB_STATUS_ERROR, error);
        if (r->h) s->pool[r->cap].push_back(r->h);  // freed at nb_server_destroy
        r->h = nullptr;
    }
    s->inflight.clear();
    while (!s->queue.empty()) {
        finish_locked(s, *s->queue.front(), NB_STATUS_ERROR, error);
        s->queue.pop_front();
    }
    s->st.queued = 0;
    s->st.inflight = 0;
    s->cv_done.notify_all();
}

void run(nb_server s)
{
    cudaSetDevice(s->dev);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(
                lk, [&] { return s->stop || !s->queue.empty() || !s->inflight.empty(); });
            if (s->stop) {
                // queued requests are cancelled; in-flight ones run to their end
                while (!s->queue.empty()) {
                    finish_locked(s, *s->queue.front(), NB_STATUS_CANCELLED, NB_OK);
                    s->queue.pop_front();
                }
                s->st.queued = 0;
                s->cv_done.notify_all();
                if (s->inflight.empty()) break;
            }
        }
        if (tick(s) != NB_OK) {
            cudaGetLastError();
            fail_all(s, NB_ERR_CUDA);
            break;
        }
    }
}

}  // namespace

namespace {

bool make_side_streams(nb_server s)
{
    for (int k = 0; k < NSIDE; ++k)
        if (cudaStreamCreateWithFlags(&s->side[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->ev_side[k], cudaEventDisableTiming) != cudaSuccess)
            return false;
    return true;
}

void free_side_streams(nb_server s)
{
    for (int k = 0; k < NSIDE; ++k) {
        if (s->side[k]) cudaStreamDestroy(s->side[k]);
        if (s->ev_side[k]) cudaEventDestroy(s->ev_side[k]);
        s->side[k] = nullptr;
        s->ev_side[k] = nullptr;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

int nb_server_create(const nb_server_cfg *cfg, nb_server *out)
{
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    nb_server_cfg c{};
    if (cfg) c = *cfg;
    if (c.budget_bytes == 0) c.budget_bytes = size_t(4) << 30;
    if (c.max_inflight <= 0) c.max_inflight = 64;
    if (c.max_queue <= 0) c.max_queue = 4096;
    if (c.eta == 0.0) c.eta = 0.01;
    if (c.dt_max == 0.0) c.dt_max = 1.0 / 16;
    if (c.variant != NB_F32DS && c.variant != NB_F32) return NB_ERR_ARG;
    if (!(c.eta > 0.0) || !std::isfinite(c.eta)) return NB_ERR_ARG;
    if (!(c.dt_max > 0.0) || std::ilogb(c.dt_max) < -30 || c.dt_max != std::ldexp(1.0, std::ilogb(c.dt_max)))
        return NB_ERR_ARG;  // a power of two
    if (c.max_inflight > 4096) return NB_ERR_ARG;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    auto s = std::make_unique<nb_server_s>();
    s->cfg = c;
    s->dev = c.device;
    s->t0 = std::chrono::steady_clock::now();
    if (cudaSetDevice(s->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        !make_side_streams(s.get()) ||
        cudaMalloc(&s->d_errs, c.max_inflight * sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost(&s->h_errs, c.max_inflight * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&s->d_dtmin, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(s->d_errs, 0, c.max_inflight * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(s->d_dtmin, 0, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        if (s->stream) cudaStreamDestroy(s->stream);
        if (s->stream2) cudaStreamDestroy(s->stream2);
        if (s->ev_fork) cudaEventDestroy(s->ev_fork);
        if (s->ev_join) cudaEventDestroy(s->ev_join);
        free_side_streams(s.get());
        if (s->d_errs) cudaFree(s->d_errs);
        if (s->h_errs) cudaFreeHost(s->h_errs);
        if (s->d_dtmin) cudaFree(s->d_dtmin);
        return NB_ERR_CUDA;
    }
    s->threads = 128;
    s->grid = s->num_sms * batch_blocks_per_sm(c.variant, s->threads);
    s->grid_jpar = s->num_sms * jpar_blocks_per_sm(c.variant);
    for (int k = c.max_inflight - 1; k >= 0; --k) s->free_slots.push_back(k);
    nb_server raw = s.release();
    raw->thread = std::thread(run, raw);
    *out = raw;
    return NB_OK;
}

int nb_server_destroy(nb_server s)
{
    if (!s) return NB_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->thread.joinable()) s->thread.join();
    cudaSetDevice(s->dev);
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->pool)
        for (nb_handle h : kv.second) nb_destroy(h);
    s->pool.clear();
    if (s->d_stage) cudaFree(s->d_stage);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    if (s->d_part) cudaFree(s->d_part);
    cudaFree(s->d_errs);
    cudaFreeHost(s->h_errs);
    cudaFree(s->d_dtmin);
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->stream2);
    cudaEventDestroy(s->ev_fork);
    cudaEventDestroy(s->ev_join);
    free_side_streams(s);
    delete s;
    return NB_OK;
}

int nb_submit(nb_server s, const nb_request *req, uint64_t *ticket)
{
    if (!s || !req || !ticket) return NB_ERR_ARG;
    if (req->kind != NB_REQ_FORCE && req->kind != NB_REQ_EVOLVE) return NB_ERR_ARG;
    const int n = req->n;
    if (n < 1 || n > (1 << 26)) return NB_ERR_ARG;
    if (!req->m || !req->pos || !req->vel) return NB_ERR_ARG;
    if (!(req->eps >= 0.0) || !std::isfinite(req->eps)) return NB_ERR_ARG;
    if (req->kind == NB_REQ_EVOLVE) {
        const double q = req->t_span / s->cfg.dt_max;
        if (!(req->t_span > 0.0) || !std::isfinite(q) || q != std::floor(q) || q > 1e12)
            return NB_ERR_ARG;  // a positive multiple of dt_max
    }
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(req->m[i]) || req->m[i] < 0.0) return NB_ERR_NONFINITE;
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(req->pos[(size_t)c * n + i]) ||
                !std::isfinite(req->vel[(size_t)c * n + i]))
                return NB_ERR_NONFINITE;
    }
    auto r = std::make_shared<Req>();
    r->kind = req->kind;
    r->n = n;
    r->eps = req->eps;
    r->t_span = req->t_span;
    r->t_end = req->t_span;
    r->cap = capacity_class(n);
    if (estimate_bytes(r->cap) > s->cfg.budget_bytes) return NB_ERR_BUDGET;
    r->m.assign(req->m, req->m + n);
    r->pos.assign(req->pos, req->pos + 3 * (size_t)n);
    r->vel.assign(req->vel, req->vel + 3 * (size_t)n);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal) return s->fatal;
        if (s->stop) return NB_ERR_STATE;
        if ((int)s->queue.size() >= s->cfg.max_queue) return NB_ERR_BUSY;
        r->id = s->next_id++;
        r->t_submit = s->now();
        s->table[r->id] = r;
        s->queue.push_back(r);
        s->st.submitted++;
        s->st.queued = (int)s->queue.size();
        *ticket = r->id;
    }
    s->cv_work.notify_one();
    return NB_OK;
}

namespace {

void fill_result(const Req &r, nb_result *out)
{
    std::memset(out, 0, sizeof *out);
    out->status = r.status;
    out->error = r.error;
    out->n = r.n;
    out->t_submit = r.t_submit;
    out->t_start = r.t_start;
    out->t_done = r.t_done;
    out->interactions = r.interactions;
    out->block_steps = r.block_steps;
    if (r.status == NB_STATUS_DONE) {
        if (r.kind == NB_REQ_FORCE) {
            out->acc = r.acc.data();
            out->jerk = r.jerk.data();
            out->pot = r.pot.data();
        } else {
            out->pos = r.out_pos.data();
            out->vel = r.out_vel.data();
        }
    }
}

bool terminal(int status)
{
    return status == NB_STATUS_DONE || status == NB_STATUS_ERROR ||
           status == NB_STATUS_CANCELLED;
}

}  // namespace

int nb_poll(nb_server s, uint64_t ticket, nb_result *out)
{
    if (!s || !out) return NB_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return NB_ERR_NOTFOUND;
    fill_result(*it->second, out);
    return NB_OK;
}

int nb_wait(nb_server s, uint64_t ticket, double timeout_s, nb_result *out)
{
    if (!s || !out) return NB_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return NB_ERR_NOTFOUND;
    ReqP r = it->second;
    const auto limit = std::chrono::duration<double>(std::max(0.0, timeout_s));
    const bool done = s->cv_done.wait_for(lk, limit, [&] { return terminal(r->status); });
    fill_result(*r, out);
    return done ? NB_OK : NB_ERR_TIMEOUT;
}

int nb_cancel(nb_server s, uint64_t ticket)
{
    if (!s) return NB_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->table.find(ticket);
        if (it == s->table.end()) return NB_ERR_NOTFOUND;
        Req &r = *it->second;
        if (terminal(r.status)) return NB_ERR_STATE;
        if (r.status == NB_STATUS_QUEUED) {
            auto q = std::find(s->queue.begin(), s->queue.end(), it->second);
            if (q != s->queue.end()) s->queue.erase(q);
            finish_locked(s, r, NB_STATUS_CANCELLED, NB_OK);
            s->st.queued = (int)s->queue.size();
        } else {
            r.cancel = true;  // the server thread retires it before its next tick
        }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_one();
    return NB_OK;
}

int nb_result_release(nb_server s, uint64_t ticket)
{
    if (!s) return NB_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return NB_ERR_NOTFOUND;
    if (!terminal(it->second->status)) return NB_ERR_STATE;
    s->table.erase(it);
    return NB_OK;
}

int nb_server_get_stats(nb_server s, nb_server_stats *out)
{
    if (!s || !out) return NB_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    return NB_OK;
}

}  // extern "C"
