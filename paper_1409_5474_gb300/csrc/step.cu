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

namespace nb {

// ---- double -> double-single split without FP64 instructions ------------
//
// GB300's FP64 pipe is narrow (a warp-wide FP64 instruction occupies it for
// ~64 cycles), so the records are split with integer operations: hi keeps the
// leading 24 significant bits of x (truncated), lo is the remaining 29 bits,
// converted to FP32 (rounded to 24 bits); x = hi + lo to ~48 bits. Values
// below 2^-74 in magnitude keep hi only (their lo is < 2^-98); zero gives 0.

__device__ __forceinline__ void split_ds(double x, float &hi, float &lo)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ff) - 1023;  // unbiased exponent
    if (e < -126) {                                 // zero or below the float range
        hi = __uint_as_float(sign);
        lo = __uint_as_float(sign);
        return;
    }
    if (e > 127) {                                  // beyond the float range
        hi = __uint_as_float(sign | 0x7f800000u);
        lo = 0.f;
        return;
    }
    const unsigned mant_hi = (unsigned)((u >> 29) & 0x7fffffu);
    hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | mant_hi);
    const unsigned rem = (unsigned)(u & ((1ull << 29) - 1ull));  // weight 2^(e-52)
    if (e - 52 + 127 < 1 || rem == 0u) {             // 2^(e-52) not a normal float
        lo = __uint_as_float(sign);
        return;
    }
    const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);
    lo = __uint_as_float(sign | __float_as_uint(__uint2float_rn(rem) * scale));
}

// FP32 value of x truncated to 24 significant bits (integer operations only).
__device__ __forceinline__ float f32_trunc(double x)
{
    float hi, lo;
    split_ds(x, hi, lo);
    return hi;
}

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
        float hi[3], lo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            split_ds(xp[c], hi[c], lo[c]);
        }
        float4 *r = s.rec + (size_t)DS_REC * i;
        r[0] = make_float4(hi[0], hi[1], hi[2], f32_trunc(s.m[i]));
        r[1] = make_float4(lo[0], lo[1], lo[2], __int_as_float(i));
        r[2] = make_float4(f32_trunc(vp[0]), f32_trunc(vp[1]), f32_trunc(vp[2]), 0.f);
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

// ---- step criterion and block quantization ---------------------------------

__device__ __forceinline__ double norm3(double x, double y, double z)
{
    return sqrt(x * x + y * y + z * z);
}

// t is a whole multiple of the power of two d: t / d is exact, so test it for an
// integer (equivalent to fmod(t, d) == 0 for power-of-two d, and cheaper).
__device__ __forceinline__ bool divides(double t, double d)
{
    const double q = t * ldexp(1.0, -ilogb(d));
    return q == trunc(q);
}

// Largest power of two <= raw (dt_max for raw >= dt_max or +inf), at most twice
// dt_old, clamped to [dt_min, dt_max], halved until it divides t_new.
__device__ double quantize(double raw, double dt_old, double t_new, double dt_min, double dt_max,
                           bool *clamped)
{
    double d;
    if (!(raw < dt_max)) {
        d = dt_max;
    } else {
        int e;
        frexp(raw, &e);
        d = ldexp(1.0, e - 1);
    }
    if (dt_old > 0.0 && d > 2.0 * dt_old) d = 2.0 * dt_old;
    if (d > dt_max) d = dt_max;
    *clamped = false;
    if (d < dt_min) {
        d = dt_min;
        *clamped = true;
    }
    while (d > dt_min && !divides(t_new, d)) d = 0.5 * d;
    return d;
}

// Level of a power-of-two step: dt = dt_max * 2^-k.
__device__ __forceinline__ int step_level(double dt, double dt_max)
{
    int k = ilogb(dt_max) - ilogb(dt);
    return k < 0 ? 0 : (k >= NLEVEL ? NLEVEL - 1 : k);
}

// hist[level] += delta, one atomic per group of lanes with the same level.
__device__ __forceinline__ void hist_add(int *hist, int level, int delta)
{
    const unsigned act = __activemask();
    const unsigned same = __match_any_sync(act, level);
    const int lane = threadIdx.x & 31;
    if (lane == __ffs(same) - 1) atomicAdd(hist + level, delta * __popc(same));
}

__device__ __forceinline__ double dot3(const double *u, const double *v)
{
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}

// quantize() for raw = sqrt(num / den) without forming the ratio: the largest
// power of two <= raw is 2^floor(floor(log2(num / den)) / 2), and
// floor(log2(num / den)) comes from the exponents and the significands of num
// and den. den == 0 means raw = +inf (dt_max); num == 0 means raw = 0 (dt_min).
__device__ double quantize_sq(double num, double den, double dt_old, double t_new,
                              double dt_min, double dt_max, bool *clamped)
{
    double d;
    if (!(den > 0.0) || !(num == num)) {
        d = dt_max;
    } else if (!(num > 0.0)) {
        d = 0.0;
    } else {
        const int en = ilogb(num), ed = ilogb(den);
        const double mn = scalbn(num, -en), md = scalbn(den, -ed);  // in [1, 2)
        const int e = en - ed - (mn < md ? 1 : 0);                   // floor(log2(num/den))
        const int half = e >= 0 ? e / 2 : -((1 - e) / 2);            // floor(e / 2)
        d = (half >= ilogb(dt_max)) ? dt_max : ldexp(1.0, half);
    }
    if (dt_old > 0.0 && d > 2.0 * dt_old) d = 2.0 * dt_old;
    if (d > dt_max) d = dt_max;
    *clamped = false;
    if (d < dt_min) {
        d = dt_min;
        *clamped = true;
    }
    while (d > dt_min && !divides(t_new, d)) d = 0.5 * d;
    return d;
}

// quantize() given e = floor(log2(raw^2)) (raw > 0 finite): the largest power of
// two <= raw is 2^floor(e / 2).
__device__ double quantize_log2(int e, double dt_old, double t_new, double dt_min, double dt_max,
                                bool *clamped)
{
    const int half = e >= 0 ? e / 2 : -((1 - e) / 2);  // floor(e / 2)
    double d = (half >= ilogb(dt_max)) ? dt_max : ldexp(1.0, half);
    if (dt_old > 0.0 && d > 2.0 * dt_old) d = 2.0 * dt_old;
    if (d > dt_max) d = dt_max;
    *clamped = false;
    if (d < dt_min) {
        d = dt_min;
        *clamped = true;
    }
    while (d > dt_min && !divides(t_new, d)) d = 0.5 * d;
    return d;
}

// ---- K4 --------------------------------------------------------------------

// K4 for active slot k (thread k of the corrector's grid).
__device__ __forceinline__ void correct_body(const StateDev &s, const int *__restrict__ act, int na,
                                             double t_new, const Out3 &f, const StepParams &prm,
                                             SchedDev *sd, unsigned *err,
                                             unsigned long long *dtmin_hits, const double *t_dev,
                                             int k)
{
    if (t_dev)
        t_new = *t_dev + t_new;
    else if (k == 0)
        sd->t_cur = t_new;
    if (k >= na) return;
    const int i = act ? act[k] : k;
    const double dt = t_new - s.t[i];
    const double dt_old = s.dt[i];
    // block steps are powers of two, whose reciprocal is exact by exponent
    // arithmetic; a shared step may be any number
    const double idt = prm.shared_dt > 0.0 ? 1.0 / dt : ldexp(1.0, -ilogb(dt));
    const double idt2 = idt * idt, idt3 = idt2 * idt;
    const double dt2 = dt * dt;
    double a1v[3], j1v[3], a2e[3], a3e[3];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long q = c * s.ld + i;
        const double a0 = s.acc[q], j0 = s.jerk[q];
        const double a1 = f.acc[c * f.ld + k], j1 = f.jerk[c * f.ld + k];
        // with A2 = a2 dt^2 and A3 = a3 dt^3 (the Hermite interpolant's 2nd and
        // 3rd derivatives, scaled): A2 = -6 (a0 - a1) - dt (4 j0 + 2 j1),
        // A3 = 12 (a0 - a1) + 6 dt (j0 + j1); x1 = xp + dt^2 (A2/24 + A3/120),
        // v1 = vp + dt (A2/6 + A3/24) - the same corrector in fewer FP64 steps
        const double da = a0 - a1;
        const double A3 = fma(6.0 * dt, j0 + j1, 12.0 * da);
        const double A2 = fma(-dt, fma(4.0, j0, 2.0 * j1), -6.0 * da);
        const double x1 = fma(dt2, fma(A3, 1.0 / 120.0, A2 * (1.0 / 24.0)), s.pos_p[q]);
        const double v1 = fma(dt, fma(A3, 1.0 / 24.0, A2 * (1.0 / 6.0)), s.vel_p[q]);
        const double a2 = A2 * idt2, a3 = A3 * idt3;
        s.pos[q] = x1;
        s.vel[q] = v1;
        s.acc[q] = a1;
        s.jerk[q] = j1;
        a1v[c] = a1;
        j1v[c] = j1;
        a2e[c] = a2 + dt * a3;
        a3e[c] = a3;
        finite = finite && isfinite(x1) && isfinite(v1);
    }
    if (!finite) atomicOr(err, DERR_NONFINITE);
    double dt_new;
    if (prm.shared_dt > 0.0) {
        dt_new = prm.shared_dt;
    } else {
        // Aarseth: dt^2 = eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2). Only the
        // power-of-two floor of dt is needed: estimate floor(log2(dt^2)) in
        // FP32 (relative error ~1e-6) and redo it exactly in FP64 only when the
        // estimate lies within 1e-5 of a power of two, where the two could differ.
        float af[3], jf[3], a2f[3], a3f[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            af[c] = f32_trunc(a1v[c]);
            jf[c] = f32_trunc(j1v[c]);
            a2f[c] = f32_trunc(a2e[c]);
            a3f[c] = f32_trunc(a3e[c]);
        }
        const float Af = af[0] * af[0] + af[1] * af[1] + af[2] * af[2];
        const float Jf = jf[0] * jf[0] + jf[1] * jf[1] + jf[2] * jf[2];
        const float A2f = a2f[0] * a2f[0] + a2f[1] * a2f[1] + a2f[2] * a2f[2];
        const float A3f = a3f[0] * a3f[0] + a3f[1] * a3f[1] + a3f[2] * a3f[2];
        const float numf = (float)prm.eta * (sqrtf(Af * A2f) + Jf);
        const float denf = sqrtf(Jf * A3f) + A2f;
        const float qf = numf / denf;
        int e2 = 0;
        bool exact_needed = !(qf > 1e-30f && qf < 1e30f) || !(denf > 0.f);
        if (!exact_needed) {
            const int eb = (int)((__float_as_uint(qf) >> 23) & 0xffu) - 127;
            const float mant = __uint_as_float((__float_as_uint(qf) & 0x007fffffu) | 0x3f800000u);
            e2 = eb;
            exact_needed = mant < 1.00001f || mant > 1.99998f;
        }
        bool clamped;
        if (exact_needed) {
            const double A = dot3(a1v, a1v), J = dot3(j1v, j1v);
            const double A2 = dot3(a2e, a2e), A3 = dot3(a3e, a3e);
            const double num = prm.eta * (sqrt(A * A2) + J);
            const double den = sqrt(J * A3) + A2;
            dt_new = quantize_sq(num, den, dt, t_new, prm.dt_min, prm.dt_max, &clamped);
        } else {
            dt_new = quantize_log2(e2, dt, t_new, prm.dt_min, prm.dt_max, &clamped);
        }
        if (clamped && dtmin_hits) atomicAdd(dtmin_hits, 1ull);
        const int lo = step_level(dt_old, prm.dt_max), ln = step_level(dt_new, prm.dt_max);
        if (lo != ln) {
            hist_add(sd->hist, lo, -1);
            hist_add(sd->hist, ln, +1);
        }
    }
    s.t[i] = t_new;
    s.dt[i] = dt_new;
}

__global__ void k_correct(StateDev s, const int *__restrict__ act, int na, double t_new, Out3 f,
                          StepParams prm, SchedDev *sd, unsigned *err,
                          unsigned long long *dtmin_hits, const double *t_dev)
{
    correct_body(s, act, na, t_new, f, prm, sd, err, dtmin_hits, t_dev,
                 blockIdx.x * blockDim.x + threadIdx.x);
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
                           unsigned long long *dtmin_hits, cudaStream_t st, const double *t_dev)
{
    if (n_a <= 0) return cudaSuccess;
    const int bs = CORRECT_THREADS;  // FP64-heavy: spread small active sets over many SMs
    k_correct<<<(n_a + bs - 1) / bs, bs, 0, st>>>(s, act, n_a, t_new, f, p, sd, err, dtmin_hits,
                                                   t_dev);
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

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long LOOKBACK_LIMIT_NS = 4000000000ull;  // 4 s

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
constexpr unsigned ST_AGG = 1u, ST_PREFIX = 2u;

__device__ __forceinline__ unsigned long long st_word(unsigned epoch, unsigned flag, unsigned v)
{
    return ((unsigned long long)epoch << 32) | ((unsigned long long)flag << 30) | v;
}

// K5 + K1 for one tile of one system (ntiles CTAs serve the system; each takes
// its tile number from a ticket, so tiles start in order).
template <bool REC>
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
            const double ti = s.t[i];
            const double d = tn - ti;
            const double d6 = d * (1.0 / 6.0), d2h = 0.5 * d;
            due = (ti + s.dt[i] == tn);
            double xp[3], vp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long q = c * s.ld + i;
                const double x = s.pos[q], v = s.vel[q], a = s.acc[q], j = s.jerk[q];
                xp[c] = fma(fma(fma(j, d6, 0.5 * a), d, v), d, x);
                vp[c] = fma(fma(j, d2h, a), d, v);
                s.pos_p[q] = xp[c];
                s.vel_p[q] = vp[c];
            }
            if (REC) {
                float hi[3], lo[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    split_ds(xp[c], hi[c], lo[c]);
                }
                float4 *rr = s.rec + (size_t)DS_REC * i;
                keep[r][0] = make_float4(hi[0], hi[1], hi[2], f32_trunc(s.m[i]));
                keep[r][1] = make_float4(lo[0], lo[1], lo[2], __int_as_float(i));
                keep[r][2] =
                    make_float4(f32_trunc(vp[0]), f32_trunc(vp[1]), f32_trunc(vp[2]), 0.f);
                rr[0] = keep[r][0];
                rr[1] = keep[r][1];
                rr[2] = keep[r][2];
            }
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
            if (REC) {
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

template <bool REC>
__global__ void __launch_bounds__(SCHED_THREADS)
    k_sched_predict(StateDev s, SchedDev *sd, unsigned long long *status, int *act,
                    float4 *irec, Mailbox *mail, double dt_max, unsigned *err)
{
    sched_body<REC>(s, sd, status, act, irec, mail, dt_max, err, gridDim.x);
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
        k_sched_predict<true><<<g, SCHED_THREADS, 0, st>>>(s, sd, status, act, irec, mail_dev,
                                                           dt_max, err);
    else
        k_sched_predict<false><<<g, SCHED_THREADS, 0, st>>>(s, sd, status, act, irec, mail_dev,
                                                            dt_max, err);
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
