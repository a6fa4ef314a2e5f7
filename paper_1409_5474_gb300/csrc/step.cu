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

// ---- K1 --------------------------------------------------------------------

template <bool REC>
__global__ void k_predict(StateDev s, double t, unsigned *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const double d = t - s.t[i];
    if (d < 0.0) atomicOr(err, DERR_BACKWARD);
    double xp[3], vp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long q = c * s.ld + i;
        const double x = s.pos[q], v = s.vel[q], a = s.acc[q], j = s.jerk[q];
        xp[c] = x + d * (v + d * (0.5 * a + d * (j / 6.0)));
        vp[c] = v + d * (a + d * (0.5 * j));
        s.pos_p[q] = xp[c];
        s.vel_p[q] = vp[c];
    }
    if (REC) {
        float hi[3], lo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            hi[c] = (float)xp[c];
            lo[c] = (float)(xp[c] - (double)hi[c]);
        }
        float4 *r = s.rec + (size_t)DS_REC * i;
        r[0] = make_float4(hi[0], hi[1], hi[2], (float)s.m[i]);
        r[1] = make_float4(lo[0], lo[1], lo[2], 0.f);
        r[2] = make_float4((float)vp[0], (float)vp[1], (float)vp[2], 0.f);
    }
}

cudaError_t launch_predict(const StateDev &s, double t, bool want_rec, unsigned *err,
                           cudaStream_t st)
{
    if (s.n <= 0) return cudaSuccess;
    const int bs = 256;
    const int g = (s.n + bs - 1) / bs;
    if (want_rec)
        k_predict<true><<<g, bs, 0, st>>>(s, t, err);
    else
        k_predict<false><<<g, bs, 0, st>>>(s, t, err);
    return cudaGetLastError();
}

// ---- step criterion and block quantization ---------------------------------

__device__ __forceinline__ double norm3(double x, double y, double z)
{
    return sqrt(x * x + y * y + z * z);
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
    while (d > dt_min && fmod(t_new, d) != 0.0) d = 0.5 * d;
    return d;
}

// ---- K4 --------------------------------------------------------------------

__global__ void k_correct(StateDev s, const int *__restrict__ act, int na, double t_new, Out3 f,
                          StepParams prm, unsigned *err, unsigned long long *dtmin_hits)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const int i = act ? act[k] : k;
    const double dt = t_new - s.t[i];
    const double dt2 = dt * dt, dt3 = dt2 * dt, dt4 = dt3 * dt, dt5 = dt4 * dt;
    double a1v[3], j1v[3], a2e[3], a3e[3];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long q = c * s.ld + i;
        const double a0 = s.acc[q], j0 = s.jerk[q];
        const double a1 = f.acc[c * f.ld + k], j1 = f.jerk[c * f.ld + k];
        const double a2 = (-6.0 * (a0 - a1) - dt * (4.0 * j0 + 2.0 * j1)) / dt2;
        const double a3 = (12.0 * (a0 - a1) + 6.0 * dt * (j0 + j1)) / dt3;
        const double x1 = s.pos_p[q] + a2 * dt4 / 24.0 + a3 * dt5 / 120.0;
        const double v1 = s.vel_p[q] + a2 * dt3 / 6.0 + a3 * dt4 / 24.0;
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
        const double na_ = norm3(a1v[0], a1v[1], a1v[2]);
        const double nj_ = norm3(j1v[0], j1v[1], j1v[2]);
        const double n2 = norm3(a2e[0], a2e[1], a2e[2]);
        const double n3 = norm3(a3e[0], a3e[1], a3e[2]);
        const double num = na_ * n2 + nj_ * nj_;
        const double den = nj_ * n3 + n2 * n2;
        const double raw = (den == 0.0) ? INFINITY : sqrt(prm.eta * num / den);
        bool clamped;
        dt_new = quantize(raw, dt, t_new, prm.dt_min, prm.dt_max, &clamped);
        if (clamped && dtmin_hits) atomicAdd(dtmin_hits, 1ull);
    }
    s.t[i] = t_new;
    s.dt[i] = dt_new;
}

cudaError_t launch_correct(const StateDev &s, const int *act, int n_a, double t_new, const Out3 &f,
                           const StepParams &p, unsigned *err, unsigned long long *dtmin_hits,
                           cudaStream_t st)
{
    if (n_a <= 0) return cudaSuccess;
    const int bs = 128;
    k_correct<<<(n_a + bs - 1) / bs, bs, 0, st>>>(s, act, n_a, t_new, f, p, err, dtmin_hits);
    return cudaGetLastError();
}

// Initial step: acc/jerk of particle k are in f (slot k = particle k) and in s.
__global__ void k_init_steps(StateDev s, Out3 f, StepParams prm, unsigned *err)
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
    }
    s.dt[i] = dt;
}

cudaError_t launch_init_steps(const StateDev &s, const Out3 &f, const StepParams &p, unsigned *err,
                              cudaStream_t st)
{
    if (s.n <= 0) return cudaSuccess;
    const int bs = 256;
    k_init_steps<<<(s.n + bs - 1) / bs, bs, 0, st>>>(s, f, p, err);
    return cudaGetLastError();
}

// ---- K5 --------------------------------------------------------------------

constexpr int SCHED_T = 1024;

// One CTA: min reduction, then an ordered compaction in chunks of SCHED_T.
__global__ void __launch_bounds__(SCHED_T) k_sched(StateDev s, int *__restrict__ act, Mailbox *mail)
{
    __shared__ double s_min[SCHED_T / 32];
    __shared__ int s_cnt[SCHED_T / 32];
    __shared__ int s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = s.n;

    double mn = INFINITY;
    for (int i = tid; i < n; i += SCHED_T) mn = fmin(mn, s.t[i] + s.dt[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if (lane == 0) s_min[warp] = mn;
    __syncthreads();
    if (warp == 0) {
        double v = s_min[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) s_min[0] = v;
    }
    __syncthreads();
    const double tn = s_min[0];

    int base = 0;
    const unsigned lt = (1u << lane) - 1u;
    for (int c0 = 0; c0 < n; c0 += SCHED_T) {
        const int i = c0 + tid;
        const bool due = (i < n) && (s.t[i] + s.dt[i] == tn);
        const unsigned b = __ballot_sync(0xffffffffu, due);
        if (lane == 0) s_cnt[warp] = __popc(b);
        __syncthreads();
        if (warp == 0) {
            const int v = s_cnt[lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            s_cnt[lane] = incl - v;
            if (lane == 31) s_total = incl;
        }
        __syncthreads();
        if (due) act[base + s_cnt[warp] + __popc(b & lt)] = i;
        base += s_total;
        __syncthreads();
    }
    if (tid == 0) {
        mail->t_next = tn;
        mail->n_active = base;
    }
}

cudaError_t launch_sched(const StateDev &s, int *act, Mailbox *mail_dev, cudaStream_t st)
{
    k_sched<<<1, SCHED_T, 0, st>>>(s, act, mail_dev);
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
        hi[c] = (float)x;
        lo[c] = (float)(x - (double)hi[c]);
        v[c] = (float)vel[c * ld + i];
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
