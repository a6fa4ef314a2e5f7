// C ABI of batched systems (nbody.h, nb_batch_*): many independent clusters
// advanced together with shared-step 4th-order Hermite.
//
// Device state is one slab of concatenated FP64 structure-of-arrays (row
// stride ld = Ntot rounded up to 64) plus the double-single records. A step
// of all systems is three kernels, captured once into a CUDA graph and
// replayed: predictor over all particles (time read from device memory), the
// batched force kernel over a work list of (system, i-block) items sorted by
// decreasing work, corrector over all particles; a one-thread kernel then
// advances the device time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "nb_internal.cuh"

using namespace nb;

struct nb_batch_s {
    nb_config cfg{};
    int dev = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    int n_sys = 0;
    long long ntot = 0, ld = 0;
    std::vector<int> sizes, offs;
    std::vector<double> eps;
    double dt = 0.0;
    double interactions_per_step = 0.0;

    void *slab = nullptr;
    double *m = nullptr, *pos = nullptr, *vel = nullptr, *acc = nullptr, *jerk = nullptr;
    double *t = nullptr, *dtv = nullptr, *pos_p = nullptr, *vel_p = nullptr;
    double *f_acc = nullptr, *f_jerk = nullptr, *f_pot = nullptr;
    float4 *rec = nullptr;
    WorkItem *d_items = nullptr;
    int nitems = 0;
    float *d_eps2 = nullptr;
    int *d_off = nullptr, *d_size = nullptr;
    double *d_time = nullptr;  // the shared time of every system
    double *d_energy = nullptr;
    unsigned *d_err = nullptr;
    SchedDev *sd = nullptr;    // unused by shared steps; the corrector takes one

    int threads = 128;         // batched-kernel CTA size (autotuned)
    int grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    bool have = false, initialised = false;
    double t_host = 0.0;
    nb_stats stats{};
    std::string msg;
};

namespace {

int bfail(nb_batch b, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->msg = buf;
    return code;
}

#define BCK(b, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail((b), NB_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

StateDev bstate(nb_batch b)
{
    StateDev s;
    s.n = (int)b->ntot;
    s.ld = b->ld;
    s.m = b->m;
    s.pos = b->pos;
    s.vel = b->vel;
    s.acc = b->acc;
    s.jerk = b->jerk;
    s.t = b->t;
    s.dt = b->dtv;
    s.pos_p = b->pos_p;
    s.vel_p = b->vel_p;
    s.rec = b->rec;
    return s;
}

StepParams bparams(nb_batch b)
{
    StepParams p{};
    p.eta = 0.01;
    p.eta_s = 0.01;
    p.dt_min = b->dt;
    p.dt_max = b->dt;
    p.shared_dt = b->dt;
    return p;
}

Out3 bout(nb_batch b) { return Out3{b->f_acc, b->f_jerk, b->f_pot, b->ld}; }

// Work list for CTAs of `threads` threads (i-blocks of 2 * threads), sorted
// by decreasing work (ni * nj), ties by position.
int build_items(nb_batch b)
{
    const int ib = 2 * b->threads;
    std::vector<WorkItem> items;
    for (int s = 0; s < b->n_sys; ++s) {
        const int n = b->sizes[s], o = b->offs[s];
        const float4 *base = b->rec + (size_t)DS_REC * o;  // the system's records
        const float e2 = (float)(b->eps[s] * b->eps[s]);
        for (int i0 = 0; i0 < n; i0 += ib) {
            WorkItem w{};
            w.jrec = base;
            w.irec = base;
            w.acc = b->f_acc + o;
            w.jerk = b->f_jerk + o;
            w.pot = b->f_pot + o;
            w.ld = b->ld;
            w.i0 = i0;
            w.ni = std::min(ib, n - i0);
            w.nj = n;
            w.gathered = 0;
            w.eps2 = e2;
            w.err = b->d_err;
            items.push_back(w);
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const WorkItem &x, const WorkItem &y) {
        return (long long)x.ni * x.nj > (long long)y.ni * y.nj;
    });
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    BCK(b, cudaMalloc(&b->d_items, sizeof(WorkItem) * std::max<size_t>(items.size(), 1)));
    BCK(b, cudaMemcpy(b->d_items, items.data(), sizeof(WorkItem) * items.size(),
                      cudaMemcpyHostToDevice));
    b->nitems = (int)items.size();
    b->grid = b->num_sms * batch_blocks_per_sm(b->cfg.variant, b->threads);
    return NB_OK;
}

void drop_graph(nb_batch b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
}

int launch_batch_force(nb_batch b)
{
    BCK(b, launch_force_items(b->cfg.variant, b->threads, b->d_items, b->nitems, b->grid,
                              b->stream));
    return NB_OK;
}

int check_berr(nb_batch b)
{
    unsigned e = 0;
    BCK(b, cudaMemcpyAsync(&e, b->d_err, sizeof e, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (!e) return NB_OK;
    BCK(b, cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->stream));
    if (e & DERR_TIMEOUT) return bfail(b, NB_ERR_TIMEOUT, "a device-side wait timed out");
    return bfail(b, NB_ERR_NONFINITE, "non-finite force or state in the batch");
}

// Initial acc/jerk of every system at its (common) time and the shared steps.
int binit(nb_batch b)
{
    StateDev s = bstate(b);
    BCK(b, launch_predict(s, b->t_host, true, b->d_err, b->stream));
    int rc = launch_batch_force(b);
    if (rc) return rc;
    BCK(b, launch_init_steps(s, bout(b), bparams(b), b->sd, b->d_err, b->stream));
    b->stats.kernel_launches += 3;
    b->stats.force_launches += 1;
    b->stats.interactions += b->interactions_per_step;
    rc = check_berr(b);
    if (rc) return rc;
    b->initialised = true;
    return NB_OK;
}

// Capture one shared step of all systems into a graph.
int capture_step(nb_batch b)
{
    drop_graph(b);
    StateDev s = bstate(b);
    const StepParams p = bparams(b);
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_predict(s, b->dt, true, b->d_err, b->stream, b->d_time);
    if (e == cudaSuccess && (b->cfg.flags & NB_FLAG_TIMING)) e = cudaEventRecordWithFlags(b->ev[0], b->stream, cudaEventRecordExternal);
    if (e == cudaSuccess)
        e = launch_force_items(b->cfg.variant, b->threads, b->d_items, b->nitems, b->grid,
                               b->stream);
    if (e == cudaSuccess && (b->cfg.flags & NB_FLAG_TIMING)) e = cudaEventRecordWithFlags(b->ev[1], b->stream, cudaEventRecordExternal);
    if (e == cudaSuccess)
        e = launch_correct(s, nullptr, (int)b->ntot, b->dt, bout(b), p, b->sd, b->d_err, nullptr,
                           b->stream, b->d_time);
    if (e == cudaSuccess) e = launch_advance(b->d_time, b->dt, b->stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return bfail(b, NB_ERR_CUDA, "graph capture failed: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    b->graph = g;
    BCK(b, cudaGraphInstantiate(&b->gexec, g, 0));
    return NB_OK;
}

}  // namespace

extern "C" {

const char *nb_batch_last_error(nb_batch b) { return b ? b->msg.c_str() : "NULL batch"; }

int nb_batch_create(const nb_config *cfg, int n_sys, const int *sizes, const double *eps,
                    double dt, nb_batch *out)
{
    if (!cfg || !out || !sizes || !eps || n_sys < 1) return NB_ERR_ARG;
    *out = nullptr;
    if (cfg->variant != NB_F32DS && cfg->variant != NB_F32) return NB_ERR_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return NB_ERR_ARG;
    long long ntot = 0;
    for (int s = 0; s < n_sys; ++s) {
        if (sizes[s] < 1 || !(eps[s] >= 0.0) || !std::isfinite(eps[s])) return NB_ERR_ARG;
        ntot += sizes[s];
    }
    if (ntot > (1LL << 30)) return NB_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    if (cfg->device < 0 || cfg->device >= ndev) return NB_ERR_ARG;
    nb_batch b = new nb_batch_s();
    b->cfg = *cfg;
    b->dev = cfg->device;
    b->n_sys = n_sys;
    b->ntot = ntot;
    b->ld = (ntot + 63) / 64 * 64;
    b->dt = dt;
    b->sizes.assign(sizes, sizes + n_sys);
    b->eps.assign(eps, eps + n_sys);
    b->offs.resize(n_sys);
    long long o = 0;
    for (int s = 0; s < n_sys; ++s) {
        b->offs[s] = (int)o;
        o += sizes[s];
        b->interactions_per_step += (double)sizes[s] * (double)sizes[s];
    }
    cudaSetDevice(b->dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->dev);
    auto bail = [&](int code) {
        nb_batch_destroy(b);
        return code;
    };
    const size_t vec = ((3 * (size_t)b->ld + 64) * sizeof(double) + 255) & ~size_t(255);
    const size_t sca = (((size_t)b->ld + 64) * sizeof(double) + 255) & ~size_t(255);
    const size_t recb = ((size_t)b->ld * DS_REC * sizeof(float4) + 255) & ~size_t(255);
    const size_t bytes = 8 * vec + 4 * sca + recb;
    if (cfg->budget_bytes && bytes > cfg->budget_bytes) {
        delete b;
        return NB_ERR_BUDGET;
    }
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&b->slab, bytes) != cudaSuccess) {
        cudaGetLastError();
        return bail(NB_ERR_OOM);
    }
    char *p = static_cast<char *>(b->slab);
    auto take = [&](size_t n) {
        char *q = p;
        p += n;
        return q;
    };
    b->pos = (double *)take(vec);
    b->vel = (double *)take(vec);
    b->acc = (double *)take(vec);
    b->jerk = (double *)take(vec);
    b->pos_p = (double *)take(vec);
    b->vel_p = (double *)take(vec);
    b->f_acc = (double *)take(vec);
    b->f_jerk = (double *)take(vec);
    b->m = (double *)take(sca);
    b->t = (double *)take(sca);
    b->dtv = (double *)take(sca);
    b->f_pot = (double *)take(sca);
    b->rec = (float4 *)take(recb);
    std::vector<float> e2(n_sys);
    for (int s = 0; s < n_sys; ++s) e2[s] = (float)(eps[s] * eps[s]);
    if (cudaMalloc(&b->d_eps2, sizeof(float) * n_sys) != cudaSuccess ||
        cudaMalloc(&b->d_off, sizeof(int) * n_sys) != cudaSuccess ||
        cudaMalloc(&b->d_size, sizeof(int) * n_sys) != cudaSuccess ||
        cudaMalloc(&b->d_time, 256) != cudaSuccess ||
        cudaMalloc(&b->d_energy, sizeof(double) * 2 * n_sys) != cudaSuccess ||
        cudaMalloc(&b->d_err, 256) != cudaSuccess || cudaMalloc(&b->sd, sizeof(SchedDev)) != cudaSuccess ||
        cudaMemcpy(b->d_eps2, e2.data(), sizeof(float) * n_sys, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_off, b->offs.data(), sizeof(int) * n_sys, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_size, sizes, sizeof(int) * n_sys, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_err, 0, 256) != cudaSuccess || cudaMemset(b->sd, 0, sizeof(SchedDev)) != cudaSuccess ||
        cudaMemset(b->slab, 0, bytes) != cudaSuccess ||
        cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess) {
        cudaGetLastError();
        return bail(NB_ERR_OOM);
    }
    if (build_items(b) != NB_OK) return bail(NB_ERR_CUDA);
    *out = b;
    return NB_OK;
}

int nb_batch_destroy(nb_batch b)
{
    if (!b) return NB_OK;
    cudaSetDevice(b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    cudaFree(b->slab);
    cudaFree(b->d_items);
    cudaFree(b->d_eps2);
    cudaFree(b->d_off);
    cudaFree(b->d_size);
    cudaFree(b->d_time);
    cudaFree(b->d_energy);
    cudaFree(b->d_err);
    cudaFree(b->sd);
    for (auto e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
    return NB_OK;
}

int nb_batch_set(nb_batch b, const double *m, const double *pos, const double *vel, double t0)
{
    if (!b || !m || !pos || !vel) return NB_ERR_ARG;
    const long long n = b->ntot;
    for (long long i = 0; i < n; ++i) {
        if (!std::isfinite(m[i]) || m[i] < 0.0)
            return bfail(b, m[i] < 0.0 ? NB_ERR_ARG : NB_ERR_NONFINITE, "bad mass %lld", i);
    }
    for (long long q = 0; q < 3 * n; ++q)
        if (!std::isfinite(pos[q]) || !std::isfinite(vel[q]))
            return bfail(b, NB_ERR_NONFINITE, "non-finite position/velocity %lld", q);
    if (!std::isfinite(t0)) return bfail(b, NB_ERR_NONFINITE, "t0 is not finite");
    cudaSetDevice(b->dev);
    BCK(b, cudaStreamSynchronize(b->stream));
    BCK(b, cudaMemcpyAsync(b->m, m, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpy2DAsync(b->pos, b->ld * sizeof(double), pos, n * sizeof(double),
                             n * sizeof(double), 3, cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpy2DAsync(b->vel, b->ld * sizeof(double), vel, n * sizeof(double),
                             n * sizeof(double), 3, cudaMemcpyHostToDevice, b->stream));
    std::vector<double> tt(n, t0);
    BCK(b, cudaMemcpyAsync(b->t, tt.data(), n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_time, &t0, sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    b->t_host = t0;
    b->have = true;
    b->initialised = false;
    return NB_OK;
}

int nb_batch_step(nb_batch b, int n_steps, nb_stats *st)
{
    if (!b || n_steps < 0) return NB_ERR_ARG;
    if (!b->have) return bfail(b, NB_ERR_STATE, "no particles set");
    cudaSetDevice(b->dev);
    const nb_stats before = b->stats;
    int rc;
    if (!b->initialised) {
        rc = binit(b);
        if (rc) return rc;
    }
    if (!b->gexec) {
        rc = capture_step(b);
        if (rc) return rc;
    }
    const bool timing = (b->cfg.flags & NB_FLAG_TIMING) != 0;
    for (int k = 0; k < n_steps; ++k) {
        BCK(b, cudaGraphLaunch(b->gexec, b->stream));
        if (timing) {
            BCK(b, cudaEventSynchronize(b->ev[1]));
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess) b->stats.force_ms += ms;
        }
        b->stats.block_steps++;
        b->stats.force_launches++;
        b->stats.kernel_launches += 4;
        b->stats.interactions += b->interactions_per_step;
        b->t_host += b->dt;
    }
    rc = check_berr(b);
    if (st) {
        nb_stats d = b->stats;
        d.block_steps -= before.block_steps;
        d.force_launches -= before.force_launches;
        d.kernel_launches -= before.kernel_launches;
        d.interactions -= before.interactions;
        d.force_ms -= before.force_ms;
        *st = d;
    }
    return rc;
}

int nb_batch_get(nb_batch b, double *pos, double *vel, double *t)
{
    if (!b) return NB_ERR_ARG;
    if (!b->have) return bfail(b, NB_ERR_STATE, "no particles set");
    cudaSetDevice(b->dev);
    const long long n = b->ntot;
    if (pos)
        BCK(b, cudaMemcpy2DAsync(pos, n * sizeof(double), b->pos, b->ld * sizeof(double),
                                 n * sizeof(double), 3, cudaMemcpyDeviceToHost, b->stream));
    if (vel)
        BCK(b, cudaMemcpy2DAsync(vel, n * sizeof(double), b->vel, b->ld * sizeof(double),
                                 n * sizeof(double), 3, cudaMemcpyDeviceToHost, b->stream));
    if (t) BCK(b, cudaMemcpyAsync(t, b->d_time, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return NB_OK;
}

int nb_batch_energy(nb_batch b, double *kin, double *pot)
{
    if (!b || !kin || !pot) return NB_ERR_ARG;
    if (!b->have) return bfail(b, NB_ERR_STATE, "no particles set");
    cudaSetDevice(b->dev);
    double tnow = 0.0;
    BCK(b, cudaMemcpyAsync(&tnow, b->d_time, sizeof tnow, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    StateDev s = bstate(b);
    BCK(b, launch_predict(s, tnow, true, b->d_err, b->stream));  // d = 0: current state
    int rc = launch_batch_force(b);
    if (rc) return rc;
    BCK(b, launch_batch_energy(b->n_sys, b->d_off, b->d_size, b->m, b->vel, b->ld, b->f_pot,
                               b->d_energy, b->d_energy + b->n_sys, b->stream));
    BCK(b, cudaMemcpyAsync(kin, b->d_energy, sizeof(double) * b->n_sys, cudaMemcpyDeviceToHost,
                           b->stream));
    BCK(b, cudaMemcpyAsync(pot, b->d_energy + b->n_sys, sizeof(double) * b->n_sys,
                           cudaMemcpyDeviceToHost, b->stream));
    return check_berr(b);
}

int nb_batch_autotune(nb_batch b, int *threads)
{
    if (!b) return NB_ERR_ARG;
    if (!b->have) return bfail(b, NB_ERR_STATE, "no particles set");
    cudaSetDevice(b->dev);
    double tnow = 0.0;
    BCK(b, cudaMemcpyAsync(&tnow, b->d_time, sizeof tnow, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    StateDev s = bstate(b);
    BCK(b, launch_predict(s, tnow, true, b->d_err, b->stream));
    // the force outputs are scratch: every step (and the first step's
    // initialisation) recomputes them before use
    float best = 1e30f;
    int best_t = b->threads;
    for (int cand : BATCH_THREADS) {
        b->threads = cand;
        int rc = build_items(b);
        if (rc) return rc;
        float tot = 0.f;
        for (int r = 0; r < 3; ++r) {
            BCK(b, cudaEventRecord(b->ev[0], b->stream));
            rc = launch_batch_force(b);
            if (rc) return rc;
            BCK(b, cudaEventRecord(b->ev[1], b->stream));
            BCK(b, cudaEventSynchronize(b->ev[1]));
            float ms = 0.f;
            BCK(b, cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
            if (r > 0) tot += ms;
        }
        if (tot < best) {
            best = tot;
            best_t = cand;
        }
    }
    b->threads = best_t;
    int rc = build_items(b);
    if (rc) return rc;
    drop_graph(b);
    if (threads) *threads = best_t;
    return check_berr(b);
}

}  // extern "C"
