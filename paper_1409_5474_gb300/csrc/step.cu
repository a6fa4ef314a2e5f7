// Per-particle kernels of the block-step Hermite integrator:
//  K1 predict  - Taylor prediction of every j-particle to the block time
//                (paper Sect. III.A: the prediction step on the j particles),
//                emitting FP64 positions/velocities and the double-single
//                j-records the FP32 pair kernels read;
//  K4 correct  - 4th-order Hermite corrector (Sect. II, VI: ph4) and the new
//                individual step (Aarseth's criterion, quantized to a power of
//                two that divides the new time: block steps, Sect. III);
//  K5 sched    - the next block time t_next = min_i(t_i + dt_i) and the list
//                of due particles in ascending index (Sect. III.A: only the
//                particles due at time t are updated, N_i << N_j);
//  energy      - K and W sums for the diagnostics.
// All state is FP64 structure-of-arrays with row stride ld.
#include <cuda_runtime.h>
#include <math.h>

#include "nb_internal.cuh"
#include "step_body.cuh"

namespace nb {

// ---- K1 --------------------------------------------------------------------

template <bool REC>
__global__ void k_predict(StateDev s, double t, unsigned *err, const double *t_dev)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    if (t_dev) t = *t_dev + t;
    const double d = t - s.t[i];
    const double d6 = d * (1.0 / 6.0), d2h = 0.5 * d;
    if (d < 0.0) atomicOr(err, DERR_BACKWARD);
    double xp[3], vp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long q = c * s.ld + i;
        const double x = s.pos[q], v = s.vel[q], a = s.acc[q], j = s.jerk[q];
        xp[c] = fma(fma(fma(j, d6, 0.5 * a), d, v), d, x);  // x + v d + a d^2/2 + j d^3/6
        vp[c] = fma(fma(j, d2h, a), d, v);                   // v + a d + j d^2/2
        s.pos_p[q] = xp[c];
        s.vel_p[q] = vp[c];
    }
    if (REC) {
        float4 rec[DS_REC];
        make_record(xp, vp, s.m[i], i, rec);
        float4 *r = s.rec + (size_t)DS_REC * i;
        r[0] = rec[0];
        r[1] = rec[1];
        r[2] = rec[2];
    }
}

cudaError_t launch_predict(const StateDev &s, double t, bool want_rec, unsigned *err,
                           cudaStream_t st, const double *t_dev)
{
    if (s.n <= 0) return cudaSuccess;
    const int bs = 256;
    const int g = (s.n + bs - 1) / bs;
    if (want_rec)
        k_predict<true><<<g, bs, 0, st>>>(s, t, err, t_dev);
    else
        k_predict<false><<<g, bs, 0, st>>>(s, t, err, t_dev);
    return cudaGetLastError();
}

__global__ void k_advance(double *t_dev, double dt) { *t_dev = *t_dev + dt; }

cudaError_t launch_advance(double *t_dev, double dt, cudaStream_t st)
{
    k_advance<<<1, 1, 0, st>>>(t_dev, dt);
    return cudaGetLastError();
}

__global__ void k_correct(StateDev s, const int *__restrict__ act, int na, double t_new, Out3 f,
                          StepParams prm, SchedDev *sd, unsigned *err,
                          unsigned long long *dtmin_hits, const double *t_dev, bool xp_from_state)
{
    correct_body(s, act, na, t_new, f, prm, sd, err, dtmin_hits, t_dev,
                 blockIdx.x * blockDim.x + threadIdx.x, xp_from_state);
}

// A trial correction of the iterated corrector P(EC)^n: the corrected x, v of
// each active particle replace its predicted ones (pos_p, vel_p and, for the
// FP32 kinds, its j-record and the gathered copy of its due-set record), so
// that the next evaluation sees them; the start-of-step state is kept.
template <bool REC>
__global__ void k_correct_trial(StateDev s, const int *act, int na, double t_new, Out3 f,
                                StepParams prm, float4 *irec, unsigned *err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const int i = act ? act[k] : k;
    const double dt = t_new - s.t[i];
    double dt2, idt2, idt3;
    step_factors(dt, prm, dt2, idt2, idt3);
    double x1[3], v1[3];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double a1, j1, a2e, a3e;
        correct_values(s, f, i, k, c, dt, dt2, idt2, idt3, true, x1[c], v1[c], a1, j1, a2e, a3e);
        s.pos_p[c * s.ld + i] = x1[c];
        s.vel_p[c * s.ld + i] = v1[c];
        finite = finite && isfinite(x1[c]) && isfinite(v1[c]);
    }
    if (!finite) atomicOr(err, DERR_NONFINITE);
    if (REC) {
        float4 rec[DS_REC];
        make_record(x1, v1, s.m[i], i, rec);
        float4 *r = s.rec + (size_t)DS_REC * i;
        r[0] = rec[0];
        r[1] = rec[1];
        r[2] = rec[2];
        if (irec) {
            float4 *g = irec + (size_t)DS_REC * k;
            g[0] = rec[0];
            g[1] = rec[1];
            g[2] = rec[2];
        }
    }
}

// The job of CTA b in a list sorted by first CTA (block0 ascending).
template <class Job>
__device__ __forceinline__ int job_of(const Job *jobs, int njobs, int b)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// K4 of many systems in one launch: CTA b serves the job whose CTA range holds b.
__global__ void k_correct_multi(const CorrectJob *__restrict__ jobs, int njobs, StepParams prm,
                                unsigned long long *dtmin_hits)
{
    const int q = job_of(jobs, njobs, blockIdx.x);
    const CorrectJob &jb = jobs[q];
    correct_body(jb.s, jb.act, jb.na, jb.t_new, jb.f, prm, jb.sd, jb.err, dtmin_hits, nullptr,
                 (blockIdx.x - jb.block0) * blockDim.x + threadIdx.x);
}

cudaError_t launch_correct(const StateDev &s, const int *act, int n_a, double t_new, const Out3 &f,
                           const StepParams &p, SchedDev *sd, unsigned *err,
                           unsigned long long *dtmin_hits, cudaStream_t st, const double *t_dev,
                           bool xp_from_state)
{
    if (n_a <= 0) return cudaSuccess;
    const int bs = CORRECT_THREADS;  // FP64-heavy: spread small active sets over many SMs
    k_correct<<<(n_a + bs - 1) / bs, bs, 0, st>>>(s, act, n_a, t_new, f, p, sd, err, dtmin_hits,
                                                   t_dev, xp_from_state);
    return cudaGetLastError();
}

cudaError_t launch_correct_trial(const StateDev &s, const int *act, int n_a, double t_new,
                                 const Out3 &f, const StepParams &p, bool want_rec, float4 *irec,
                                 unsigned *err, cudaStream_t st)
{
    if (n_a <= 0) return cudaSuccess;
    const int bs = CORRECT_THREADS;
    if (want_rec)
        k_correct_trial<true><<<(n_a + bs - 1) / bs, bs, 0, st>>>(s, act, n_a, t_new, f, p, irec,
                                                                   err);
    else
        k_correct_trial<false><<<(n_a + bs - 1) / bs, bs, 0, st>>>(s, act, n_a, t_new, f, p,
                                                                    irec, err);
    return cudaGetLastError();
}

cudaError_t launch_correct_multi(const CorrectJob *jobs, int njobs, int nblocks,
                                 const StepParams &p, unsigned long long *dtmin_hits,
                                 cudaStream_t st)
{
    if (njobs <= 0 || nblocks <= 0) return cudaSuccess;
    k_correct_multi<<<nblocks, CORRECT_THREADS, 0, st>>>(jobs, njobs, p, dtmin_hits);
    return cudaGetLastError();
}

constexpr int BENERGY_T = 256;

__global__ void __launch_bounds__(BENERGY_T)
    k_batch_energy(const int *__restrict__ off, const int *__restrict__ size,
                   const double *__restrict__ m, const double *__restrict__ vel, long long ld,
                   const double *__restrict__ pot, double *kin_out, double *pot_out)
{
    __shared__ double sk[BENERGY_T], sw[BENERGY_T];
    const int sys = blockIdx.x, tid = threadIdx.x;
    const int o = off[sys], n = size[sys];
    double k = 0.0, w = 0.0;
    for (int q = tid; q < n; q += BENERGY_T) {
        const int i = o + q;
        const double vx = vel[i], vy = vel[ld + i], vz = vel[2 * ld + i];
        k += 0.5 * m[i] * (vx * vx + vy * vy + vz * vz);
        w += 0.5 * m[i] * pot[i];
    }
    sk[tid] = k;
    sw[tid] = w;
    __syncthreads();
    for (int h = BENERGY_T / 2; h > 0; h >>= 1) {
        if (tid < h) {
            sk[tid] += sk[tid + h];
            sw[tid] += sw[tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) {
        kin_out[sys] = sk[0];
        pot_out[sys] = sw[0];
    }
}

cudaError_t launch_batch_energy(int n_sys, const int *off, const int *size, const double *m,
                                const double *vel, long long ld, const double *pot,
                                double *kin_out, double *pot_out, cudaStream_t st)
{
    if (n_sys <= 0) return cudaSuccess;
    k_batch_energy<<<n_sys, BENERGY_T, 0, st>>>(off, size, m, vel, ld, pot, kin_out, pot_out);
    return cudaGetLastError();
}

// Initial step: acc/jerk of particle k are in f (slot k = particle k) and in s.
__global__ void k_init_steps(StateDev s, Out3 f, StepParams prm, SchedDev *sd, unsigned *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    double a[3], j[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a[c] = f.acc[c * f.ld + i];
        j[c] = f.jerk[c * f.ld + i];
        s.acc[c * s.ld + i] = a[c];
        s.jerk[c * s.ld + i] = j[c];
    }
    double dt;
    if (prm.shared_dt > 0.0) {
        dt = prm.shared_dt;
    } else {
        const double nj_ = norm3(j[0], j[1], j[2]);
        const double raw = (nj_ == 0.0) ? INFINITY : prm.eta_s * norm3(a[0], a[1], a[2]) / nj_;
        bool clamped;
        dt = quantize(raw, 0.0, s.t[i], prm.dt_min, prm.dt_max, &clamped);
        hist_add(sd->hist, step_level(dt, prm.dt_max), 1);
    }
    s.dt[i] = dt;
    if (i == 0) sd->t_cur = s.t[0];
}

cudaError_t launch_init_steps(const StateDev &s, const Out3 &f, const StepParams &p, SchedDev *sd,
                              unsigned *err, cudaStream_t st)
{
    if (s.n <= 0) return cudaSuccess;
    const int bs = 256;
    k_init_steps<<<(s.n + bs - 1) / bs, bs, 0, st>>>(s, f, p, sd, err);
    return cudaGetLastError();
}

// ---- K5 + K1: fused block scheduler and predictor -----------------------

// K5 + K1 for one tile of one system (ntiles CTAs serve the system; each takes
// its tile number from a ticket, so tiles start in order).
template <bool REC, int ORD = 4>
__device__ __forceinline__ void sched_body(const StateDev &s, SchedDev *sd,
                                           unsigned long long *status, int *act, float4 *irec,
                                           Mailbox *mail, double dt_max, unsigned *err,
                                           int ntiles)
{
    constexpr int NWORD = SCHED_TILE / 32;
    __shared__ unsigned s_flags[NWORD];
    __shared__ int s_woff[NWORD];
    __shared__ int s_wtot[(NWORD + 31) / 32];
    __shared__ int s_tile, s_agg, s_excl;
    __shared__ unsigned s_epoch;
    __shared__ unsigned s_occ[NLEVEL / 32];
    __shared__ double s_tnext, s_tcur;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // occupied step levels -> t_next
    static_assert(NLEVEL % 32 == 0 && NLEVEL / 32 <= SCHED_THREADS / 32, "levels");
    if (warp < NLEVEL / 32) {
        const bool occ = ((volatile int *)sd->hist)[warp * 32 + lane] > 0;
        const unsigned b = __ballot_sync(0xffffffffu, occ);
        if (lane == 0) s_occ[warp] = b;
    }
    // the start-up reads go out together (different warps), one round trip
    if (tid == 64) s_tile = (int)atomicAdd(&sd->ticket, 1u);  // tiles in start order
    if (tid == 96) s_epoch = (unsigned)(*(volatile unsigned long long *)&sd->seq);
    if (tid == 128) s_tcur = *(volatile double *)&sd->t_cur;
    __syncthreads();
    if (tid == 0) {
        int kmax = 0;
        for (int w = 0; w < NLEVEL / 32; ++w)
            if (s_occ[w]) kmax = w * 32 + 31 - __clz(s_occ[w]);
        const double dm = ldexp(dt_max, -kmax);
        const double tc = s_tcur;
        // next multiple of the power of two dm after tc: tc / dm is exact, so
        // floor(tc / dm) + 1 times dm is too (no fmod, which is slow in FP64)
        s_tnext = (floor(tc * (1.0 / dm)) + 1.0) * dm;
    }
    __syncthreads();
    const int tile = s_tile;
    const double tn = s_tnext;
    const int base = tile * SCHED_TILE;

    // predict + due flags (one ballot word per warp and round); the records stay
    // in registers for the gathered copy of the due set
    float4 keep[SCHED_PER_THREAD][DS_REC];
#pragma unroll
    for (int r = 0; r < SCHED_PER_THREAD; ++r) {
        const int i = base + r * SCHED_THREADS + tid;
        bool due = false;
        if (i < s.n) {
            if (ORD == 6)
                due = predict6_one<REC>(s, i, tn);
            else
                due = predict_one<REC>(s, i, tn, keep[r]);
        }
        const unsigned b = __ballot_sync(0xffffffffu, due);
        if (lane == 0) s_flags[r * (SCHED_THREADS / 32) + warp] = b;
    }
    __syncthreads();

    // exclusive offsets of the flag words in index order, and the tile aggregate
    constexpr int NSW = (NWORD + 31) / 32;  // warps that scan the words
    static_assert(NSW <= SCHED_THREADS / 32, "flag words");
    if (warp < NSW) {
        const int w = warp * 32 + lane;
        const int v = (w < NWORD) ? __popc(s_flags[w]) : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (w < NWORD) s_woff[w] = incl - v;
        if (lane == 31) s_wtot[warp] = incl;
    }
    __syncthreads();
    if (warp < NSW && warp > 0) {
        int carry = 0;
        for (int q = 0; q < warp; ++q) carry += s_wtot[q];
        const int w = warp * 32 + lane;
        if (w < NWORD) s_woff[w] += carry;
    }
    if (tid == 0) {
        int a = 0;
        for (int q = 0; q < NSW; ++q) a += s_wtot[q];
        s_agg = a;
    }
    __syncthreads();
    const int agg = s_agg;

    // decoupled look-back over the tiles in front of this one, 32 tiles per
    // round trip: lane l reads tile (top - l); tiles before 0 count as a prefix 0
    if (warp == 0) {
        const unsigned ep = s_epoch;
        if (tile == 0) {
            if (lane == 0) st_release_u64(status, st_word(ep, ST_PREFIX, (unsigned)agg));
            if (lane == 0) s_excl = 0;
        } else {
            if (lane == 0) st_release_u64(status + tile, st_word(ep, ST_AGG, (unsigned)agg));
            int excl = 0;
            int top = tile - 1;
            const unsigned long long t0 = globaltimer_ns();
            bool ok = true;
            for (;;) {
                const int t = top - lane;
                unsigned long long wd = st_word(ep, ST_PREFIX, 0u);
                bool ready = true;
                if (t >= 0) {
                    wd = ld_acquire_u64(status + t);
                    ready = (unsigned)(wd >> 32) == ep;
                }
                if (!__all_sync(0xffffffffu, ready)) {
                    if (globaltimer_ns() - t0 > LOOKBACK_LIMIT_NS) {
                        ok = false;
                        break;
                    }
                    continue;
                }
                const unsigned flag = (unsigned)(wd >> 30) & 3u;
                const int val = (int)(wd & 0x3fffffffu);
                const unsigned pre = __ballot_sync(0xffffffffu, flag == ST_PREFIX);
                if (pre) {
                    const int pl = __ffs(pre) - 1;  // nearest tile with a full prefix
                    int c = lane <= pl ? val : 0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                    excl += c;
                    break;
                }
                int c = val;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                excl += c;
                top -= 32;
            }
            if (lane == 0) {
                if (!ok) atomicOr(err, DERR_TIMEOUT);
                st_release_u64(status + tile, st_word(ep, ST_PREFIX, (unsigned)(excl + agg)));
                s_excl = excl;
            }
        }
        if (lane == 0 && tile == ntiles - 1) sd->n_active = s_excl + agg;
    }
    __syncthreads();
    const int excl = s_excl;

    // scatter the due indices (and records) in ascending order
#pragma unroll
    for (int r = 0; r < SCHED_PER_THREAD; ++r) {
        const int w = r * (SCHED_THREADS / 32) + warp;
        const unsigned b = s_flags[w];
        if (b & (1u << lane)) {
            const int i = base + r * SCHED_THREADS + tid;
            const int slot = excl + s_woff[w] + __popc(b & ((1u << lane) - 1u));
            act[slot] = i;
            if (REC && ORD == 4) {
                float4 *g = irec + (size_t)DS_REC * slot;
                g[0] = keep[r][0];
                g[1] = keep[r][1];
                g[2] = keep[r][2];
            }
        }
    }

    // the last CTA to finish publishes the result and re-arms the launch state
    if (tid == 0) {
        __threadfence();
        const unsigned fin = atomicAdd(&sd->done, 1u);
        if (fin == (unsigned)ntiles - 1) {
            __threadfence();
            const int na = *(volatile int *)&sd->n_active;
            mail->t_next = tn;
            mail->n_active = na;
            __threadfence_system();
            mail->seq = (unsigned long long)s_epoch;
            sd->ticket = 0;
            sd->done = 0;
            sd->seq = (unsigned long long)s_epoch + 1ull;
        }
    }
}

template <bool REC, int ORD>
__global__ void __launch_bounds__(SCHED_THREADS)
    k_sched_predict(StateDev s, SchedDev *sd, unsigned long long *status, int *act,
                    float4 *irec, Mailbox *mail, double dt_max, unsigned *err)
{
    sched_body<REC, ORD>(s, sd, status, act, irec, mail, dt_max, err, gridDim.x);
}

// K5 + K1 of many systems in one launch (each system's tiles as above).
template <bool REC>
__global__ void __launch_bounds__(SCHED_THREADS)
    k_sched_predict_multi(const SchedJob *__restrict__ jobs, int njobs, double dt_max)
{
    const int q = job_of(jobs, njobs, blockIdx.x);
    const SchedJob &jb = jobs[q];
    sched_body<REC>(jb.s, jb.sd, jb.status, jb.act, jb.irec, jb.mail, dt_max, jb.err,
                    jb.ntiles);
}

cudaError_t launch_sched_predict(const StateDev &s, SchedDev *sd, unsigned long long *status,
                                 int *act, float4 *irec, Mailbox *mail_dev, double dt_max,
                                 bool want_rec, unsigned *err, cudaStream_t st)
{
    const int g = (s.n + SCHED_TILE - 1) / SCHED_TILE;
    if (want_rec)
        k_sched_predict<true, 4><<<g, SCHED_THREADS, 0, st>>>(s, sd, status, act, irec,
                                                              mail_dev, dt_max, err);
    else
        k_sched_predict<false, 4><<<g, SCHED_THREADS, 0, st>>>(s, sd, status, act, irec,
                                                               mail_dev, dt_max, err);
    return cudaGetLastError();
}

cudaError_t launch_sched_predict6(const StateDev &s, SchedDev *sd, unsigned long long *status,
                                  int *act, Mailbox *mail_dev, double dt_max, bool want_rec,
                                  unsigned *err, cudaStream_t st)
{
    const int g = (s.n + SCHED_TILE - 1) / SCHED_TILE;
    if (want_rec)
        k_sched_predict<true, 6><<<g, SCHED_THREADS, 0, st>>>(s, sd, status, act, nullptr,
                                                              mail_dev, dt_max, err);
    else
        k_sched_predict<false, 6><<<g, SCHED_THREADS, 0, st>>>(s, sd, status, act, nullptr,
                                                               mail_dev, dt_max, err);
    return cudaGetLastError();
}

cudaError_t launch_sched_predict_multi(const SchedJob *jobs, int njobs, int nblocks,
                                       double dt_max, bool want_rec, cudaStream_t st)
{
    if (njobs <= 0 || nblocks <= 0) return cudaSuccess;
    if (want_rec)
        k_sched_predict_multi<true><<<nblocks, SCHED_THREADS, 0, st>>>(jobs, njobs, dt_max);
    else
        k_sched_predict_multi<false><<<nblocks, SCHED_THREADS, 0, st>>>(jobs, njobs, dt_max);
    return cudaGetLastError();
}

// ---- bridge kicks (Sect. V) ---------------------------------------------------

// vel[c][i] += dt * acc[c][i] for the n particles (SoA rows of stride ld / lda).
__global__ void k_kick(int n, double *__restrict__ vel, long long ld,
                       const double *__restrict__ acc, long long lda, double dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) vel[c * ld + i] = fma(dt, acc[c * lda + i], vel[c * ld + i]);
}

cudaError_t launch_kick(int n, double *vel, long long ld, const double *acc, long long lda,
                        double dt, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_kick<<<(n + 255) / 256, 256, 0, st>>>(n, vel, ld, acc, lda, dt);
    return cudaGetLastError();
}

// acc, jerk of every particle from a slot-indexed evaluation f (the steps stay).
__global__ void k_set_derivs(StateDev s, Out3 f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s.acc[c * s.ld + i] = f.acc[c * f.ld + i];
        s.jerk[c * s.ld + i] = f.jerk[c * f.ld + i];
    }
}

cudaError_t launch_set_derivs(const StateDev &s, const Out3 &f, cudaStream_t st)
{
    if (s.n <= 0) return cudaSuccess;
    k_set_derivs<<<(s.n + 255) / 256, 256, 0, st>>>(s, f);
    return cudaGetLastError();
}

// Flags DERR_UNSYNC when some particle's own time is not tc.
__global__ void k_check_sync(int n, const double *__restrict__ t, double tc, unsigned *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && t[i] != tc) atomicOr(err, DERR_UNSYNC);
}

cudaError_t launch_check_sync(int n, const double *t, double tc, unsigned *err, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_check_sync<<<(n + 255) / 256, 256, 0, st>>>(n, t, tc, err);
    return cudaGetLastError();
}

// ---- energy ----------------------------------------------------------------

constexpr int ENERGY_T = 512;

__global__ void __launch_bounds__(ENERGY_T)
    k_energy(int n, const double *__restrict__ m, const double *__restrict__ vel, long long ld,
             const double *__restrict__ pot, double *out2)
{
    __shared__ double sk[ENERGY_T], sw[ENERGY_T];
    const int tid = threadIdx.x;
    double k = 0.0, w = 0.0;
    for (int i = tid; i < n; i += ENERGY_T) {
        const double vx = vel[i], vy = vel[ld + i], vz = vel[2 * ld + i];
        k += 0.5 * m[i] * (vx * vx + vy * vy + vz * vz);
        w += 0.5 * m[i] * pot[i];
    }
    sk[tid] = k;
    sw[tid] = w;
    __syncthreads();
    for (int o = ENERGY_T / 2; o > 0; o >>= 1) {
        if (tid < o) {
            sk[tid] += sk[tid + o];
            sw[tid] += sw[tid + o];
        }
        __syncthreads();
    }
    if (tid == 0) {
        out2[0] = sk[0];
        out2[1] = sw[0];
    }
}

cudaError_t launch_energy(int n, const double *m, const double *vel, long long ld,
                          const double *pot, double *out2, cudaStream_t st)
{
    k_energy<<<1, ENERGY_T, 0, st>>>(n, m, vel, ld, pot, out2);
    return cudaGetLastError();
}

__global__ void k_make_rec(int n, const double *__restrict__ pos, const double *__restrict__ vel,
                           long long ld, float4 *__restrict__ rec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float hi[3], lo[3], v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double x = pos[c * ld + i];
        split_ds(x, hi[c], lo[c]);
        v[c] = f32_trunc(vel[c * ld + i]);
    }
    float4 *r = rec + (size_t)DS_REC * i;
    r[0] = make_float4(hi[0], hi[1], hi[2], 0.f);
    r[1] = make_float4(lo[0], lo[1], lo[2], 0.f);
    r[2] = make_float4(v[0], v[1], v[2], 0.f);
}

cudaError_t launch_make_rec(int n, const double *pos, const double *vel, long long ld, float4 *rec,
                            cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int bs = 256;
    k_make_rec<<<(n + bs - 1) / bs, bs, 0, st>>>(n, pos, vel, ld, rec);
    return cudaGetLastError();
}

__global__ void k_check_finite(const double *p, int n, int rows, long long ld, unsigned *err)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)n * rows) return;
    const int r = (int)(q / n), i = (int)(q % n);
    if (!isfinite(p[r * ld + i])) atomicOr(err, DERR_NONFINITE);
}

cudaError_t launch_check_finite(const double *p, int n, int rows, long long ld, unsigned *err,
                                cudaStream_t st)
{
    const long long tot = (long long)n * rows;
    if (tot <= 0) return cudaSuccess;
    const int bs = 256;
    k_check_finite<<<(unsigned)((tot + bs - 1) / bs), bs, 0, st>>>(p, n, rows, ld, err);
    return cudaGetLastError();
}

}  // namespace nb
