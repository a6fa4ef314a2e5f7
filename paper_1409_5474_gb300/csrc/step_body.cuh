// Device-side arithmetic of the per-particle steps, shared by the per-step
// kernels (step.cu) and the fused persistent block-step kernel (persist.cu):
// the double-single split of FP64 values, the step criterion and block
// quantization, the Hermite corrector of one active slot, and the helpers of
// bounded inter-CTA waits.
#pragma once

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

// ---- K1 for one particle ------------------------------------------------------

// The double-single j-record of particle i at position x, velocity v:
// {x_hi, y_hi, z_hi, m}, {x_lo, y_lo, z_lo, index bits}, {vx, vy, vz, 0}.
__device__ __forceinline__ void make_record(const double x[3], const double v[3], double m, int i,
                                            float4 rec[3])
{
    float hi[3], lo[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) split_ds(x[c], hi[c], lo[c]);
    rec[0] = make_float4(hi[0], hi[1], hi[2], f32_trunc(m));
    rec[1] = make_float4(lo[0], lo[1], lo[2], __int_as_float(i));
    rec[2] = make_float4(f32_trunc(v[0]), f32_trunc(v[1]), f32_trunc(v[2]), 0.f);
}

// Predict particle i to time tn (FP64 Taylor series to the jerk term), write
// pos_p / vel_p (unless !STORE_P) and, when REC, its double-single j-record
// (also left in rec[]); returns whether the particle is due at tn
// (t_i + dt_i == tn).
template <bool REC, bool STORE_P = true>
__device__ __forceinline__ bool predict_one(const StateDev &s, int i, double tn, float4 rec[3])
{
    const double ti = s.t[i];
    const double d = tn - ti;
    const double d6 = d * (1.0 / 6.0), d2h = 0.5 * d;
    const bool due = (ti + s.dt[i] == tn);
    double xp[3], vp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long q = c * s.ld + i;
        const double x = s.pos[q], v = s.vel[q], a = s.acc[q], j = s.jerk[q];
        xp[c] = fma(fma(fma(j, d6, 0.5 * a), d, v), d, x);
        vp[c] = fma(fma(j, d2h, a), d, v);
        if (STORE_P) {
            s.pos_p[q] = xp[c];
            s.vel_p[q] = vp[c];
        }
    }
    if (REC) {
        make_record(xp, vp, s.m[i], i, rec);
        float4 *rr = s.rec + (size_t)DS_REC * i;
        rr[0] = rec[0];
        rr[1] = rec[1];
        rr[2] = rec[2];
    }
    return due;
}

// The state K1 reads for one particle, so that a thread can have the loads of
// several particles in flight before any arithmetic.
struct PState {
    double t, dt, m, x[3], v[3], a[3], j[3];
};

__device__ __forceinline__ void pstate_load(const StateDev &s, int i, PState &q)
{
    q.t = s.t[i];
    q.dt = s.dt[i];
    q.m = s.m[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long k = c * s.ld + i;
        q.x[c] = s.pos[k];
        q.v[c] = s.vel[k];
        q.a[c] = s.acc[k];
        q.j[c] = s.jerk[k];
    }
}

// K1 on a loaded state: the same arithmetic (and bits) as predict_one, the
// double-single j-record written to s.rec and left in rec[]; whether the
// particle is due at tn.
__device__ __forceinline__ bool predict_rec_from(const StateDev &s, const PState &q, int i,
                                                 double tn, float4 rec[3])
{
    const double d = tn - q.t;
    const double d6 = d * (1.0 / 6.0), d2h = 0.5 * d;
    double xp[3], vp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xp[c] = fma(fma(fma(q.j[c], d6, 0.5 * q.a[c]), d, q.v[c]), d, q.x[c]);
        vp[c] = fma(fma(q.j[c], d2h, q.a[c]), d, q.v[c]);
    }
    make_record(xp, vp, q.m, i, rec);
    float4 *rr = s.rec + (size_t)DS_REC * i;
    rr[0] = rec[0];
    rr[1] = rec[1];
    rr[2] = rec[2];
    return q.t + q.dt == tn;
}

// The 6th-order prediction of particle i to time tn (FP64 Taylor series through
// the crackle term, in Horner form): pos_p, vel_p, acc_p and, when REC, its
// 64-byte record (the 48-byte record plus the FP32 predicted acceleration).
// Returns whether the particle is due at tn.
template <bool REC>
__device__ __forceinline__ bool predict6_one(const StateDev &s, int i, double tn)
{
    const double ti = s.t[i];
    const double d = tn - ti;
    const double h2 = d * 0.5, h3 = d * (1.0 / 3.0), h4 = d * 0.25, h5 = d * 0.2;
    const bool due = (ti + s.dt[i] == tn);
    double xp[3], vp[3], ap[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long q = c * s.ld + i;
        const double x = s.pos[q], v = s.vel[q], a = s.acc[q], j = s.jerk[q];
        const double sn = s.snap[q], cr = s.crk[q];
        // x + d (v + d/2 (a + d/3 (j + d/4 (s + d/5 c)))) and likewise for v, a
        xp[c] = fma(d, fma(h2, fma(h3, fma(h4, fma(h5, cr, sn), j), a), v), x);
        vp[c] = fma(d, fma(h2, fma(h3, fma(h4, cr, sn), j), a), v);
        ap[c] = fma(d, fma(h2, fma(h3, cr, sn), j), a);
        s.pos_p[q] = xp[c];
        s.vel_p[q] = vp[c];
        s.acc_p[q] = ap[c];
    }
    if (REC) {
        float4 r[3];
        make_record(xp, vp, s.m[i], i, r);
        float4 *rr = s.rec6 + (size_t)DS6_REC * i;
        rr[0] = r[0];
        rr[1] = r[1];
        rr[2] = r[2];
        rr[3] = make_float4(f32_trunc(ap[0]), f32_trunc(ap[1]), f32_trunc(ap[2]), 0.f);
    }
    return due;
}

// The state the 6th-order K1 reads for one particle (loads of several particles
// in flight before any arithmetic).
struct PState6 {
    double t, dt, m, x[3], v[3], a[3], j[3], sn[3], cr[3];
};

__device__ __forceinline__ void pstate6_load(const StateDev &s, int i, PState6 &q)
{
    q.t = s.t[i];
    q.dt = s.dt[i];
    q.m = s.m[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long k = c * s.ld + i;
        q.x[c] = s.pos[k];
        q.v[c] = s.vel[k];
        q.a[c] = s.acc[k];
        q.j[c] = s.jerk[k];
        q.sn[c] = s.snap[k];
        q.cr[c] = s.crk[k];
    }
}

// predict6_one on a loaded state, the 64-byte record only (the same arithmetic
// and bits; no FP64 pos_p / vel_p / acc_p: the order-6 corrector starts from
// the start-of-step state); whether the particle is due at tn.
__device__ __forceinline__ bool predict6_rec_from(const StateDev &s, const PState6 &q, int i,
                                                  double tn)
{
    const double d = tn - q.t;
    const double h2 = d * 0.5, h3 = d * (1.0 / 3.0), h4 = d * 0.25, h5 = d * 0.2;
    double xp[3], vp[3], ap[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xp[c] = fma(d, fma(h2, fma(h3, fma(h4, fma(h5, q.cr[c], q.sn[c]), q.j[c]), q.a[c]),
                           q.v[c]), q.x[c]);
        vp[c] = fma(d, fma(h2, fma(h3, fma(h4, q.cr[c], q.sn[c]), q.j[c]), q.a[c]), q.v[c]);
        ap[c] = fma(d, fma(h2, fma(h3, q.cr[c], q.sn[c]), q.j[c]), q.a[c]);
    }
    float4 r[3];
    make_record(xp, vp, q.m, i, r);
    float4 *rr = s.rec6 + (size_t)DS6_REC * i;
    rr[0] = r[0];
    rr[1] = r[1];
    rr[2] = r[2];
    rr[3] = make_float4(f32_trunc(ap[0]), f32_trunc(ap[1]), f32_trunc(ap[2]), 0.f);
    return q.t + q.dt == tn;
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
static __device__ double quantize(double raw, double dt_old, double t_new, double dt_min, double dt_max,
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
static __device__ double quantize_sq(double num, double den, double dt_old, double t_new,
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
static __device__ double quantize_log2(int e, double dt_old, double t_new, double dt_min, double dt_max,
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

// The Hermite corrector of one component from the start-of-step x, v, a0, j0,
// the predicted xp, vp and the new a1, j1: x1, v1 and the end-of-step a2
// (a2 + dt a3) and a3 for the step criterion.
__device__ __forceinline__ void hermite_correct(double xp, double vp, double a0, double j0,
                                                double a1, double j1, double dt, double dt2,
                                                double idt2, double idt3, double &x1,
                                                double &v1, double &a2eo, double &a3eo)
{
    // with A2 = a2 dt^2 and A3 = a3 dt^3 (the Hermite interpolant's 2nd and
    // 3rd derivatives, scaled): A2 = -6 (a0 - a1) - dt (4 j0 + 2 j1),
    // A3 = 12 (a0 - a1) + 6 dt (j0 + j1); x1 = xp + dt^2 (A2/24 + A3/120),
    // v1 = vp + dt (A2/6 + A3/24) - the same corrector in fewer FP64 steps
    const double da = a0 - a1;
    const double A3 = fma(6.0 * dt, j0 + j1, 12.0 * da);
    const double A2 = fma(-dt, fma(4.0, j0, 2.0 * j1), -6.0 * da);
    x1 = fma(dt2, fma(A3, 1.0 / 120.0, A2 * (1.0 / 24.0)), xp);
    v1 = fma(dt, fma(A3, 1.0 / 24.0, A2 * (1.0 / 6.0)), vp);
    const double a2 = A2 * idt2, a3 = A3 * idt3;
    a2eo = a2 + dt * a3;
    a3eo = a3;
}

// The FP64 prediction over dt from the start-of-step state (the K1 formula,
// the same bits as the predictor).
__device__ __forceinline__ void predict_xv(double x, double v, double a0, double j0, double dt,
                                           double &xp, double &vp)
{
    const double d = dt, d6 = d * (1.0 / 6.0), d2h = 0.5 * d;
    xp = fma(fma(fma(j0, d6, 0.5 * a0), d, v), d, x);
    vp = fma(fma(j0, d2h, a0), d, v);
}

// K4, component c of active slot k (particle i): the Hermite corrector of x, v
// with the new acc/jerk f (slot-indexed). The predicted x_p, v_p are read from
// pos_p / vel_p, or, with xp_from_state (the iterated corrector, which has
// overwritten them), recomputed from the start-of-step state with the K1
// formula, which gives the same bits. Returns x1, v1, the new acc/jerk and the
// end-of-step a2 (a2 + dt a3) and a3 for the step criterion.
__device__ __forceinline__ void correct_values(const StateDev &s, const Out3 &f, int i, int k,
                                               int c, double dt, double dt2, double idt2,
                                               double idt3, bool xp_from_state, double &x1,
                                               double &v1, double &a1o, double &j1o,
                                               double &a2eo, double &a3eo)
{
    const long long q = c * s.ld + i;
    const double a0 = s.acc[q], j0 = s.jerk[q];
    const double a1 = f.acc[c * f.ld + k], j1 = f.jerk[c * f.ld + k];
    double xp, vp;
    if (xp_from_state)
        predict_xv(s.pos[q], s.vel[q], a0, j0, dt, xp, vp);
    else {
        xp = s.pos_p[q];
        vp = s.vel_p[q];
    }
    hermite_correct(xp, vp, a0, j0, a1, j1, dt, dt2, idt2, idt3, x1, v1, a2eo, a3eo);
    a1o = a1;
    j1o = j1;
}

// K4, component c of active slot k: correct_values, then the new pos, vel,
// acc, jerk of particle i are stored. Whether x and v stayed finite.
__device__ __forceinline__ bool correct_component(const StateDev &s, const Out3 &f, int i, int k,
                                                  int c, double dt, double dt2, double idt2,
                                                  double idt3, double &a1o, double &j1o,
                                                  double &a2eo, double &a3eo,
                                                  bool xp_from_state = false)
{
    const long long q = c * s.ld + i;
    double x1, v1;
    correct_values(s, f, i, k, c, dt, dt2, idt2, idt3, xp_from_state, x1, v1, a1o, j1o, a2eo,
                   a3eo);
    s.pos[q] = x1;
    s.vel[q] = v1;
    s.acc[q] = a1o;
    s.jerk[q] = j1o;
    return isfinite(x1) && isfinite(v1);
}

// K4, the new step of particle i from its new acc, jerk, a2 and a3 (Aarseth's
// criterion, block quantization, level histogram), and its new time.
__device__ __forceinline__ void correct_step(const StateDev &s, int i, double t_new, double dt,
                                             double dt_old, const double a1v[3],
                                             const double j1v[3], const double a2e[3],
                                             const double a3e[3], const StepParams &prm,
                                             SchedDev *sd, unsigned long long *dtmin_hits)
{
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

// The step of a particle whose time is t_i (block steps: a power of two, whose
// reciprocal is exact by exponent arithmetic; a shared step may be any number).
__device__ __forceinline__ void step_factors(double dt, const StepParams &prm, double &dt2,
                                             double &idt2, double &idt3)
{
    const double idt = prm.shared_dt > 0.0 ? 1.0 / dt : ldexp(1.0, -ilogb(dt));
    idt2 = idt * idt;
    idt3 = idt2 * idt;
    dt2 = dt * dt;
}

// K4 for active slot k (thread k of the corrector's grid).
__device__ __forceinline__ void correct_body(const StateDev &s, const int *act, int na,
                                             double t_new, const Out3 &f, const StepParams &prm,
                                             SchedDev *sd, unsigned *err,
                                             unsigned long long *dtmin_hits, const double *t_dev,
                                             int k, bool xp_from_state = false)
{
    if (t_dev)
        t_new = *t_dev + t_new;
    else if (k == 0)
        sd->t_cur = t_new;
    if (k >= na) return;
    const int i = act ? act[k] : k;
    const double dt = t_new - s.t[i];
    const double dt_old = s.dt[i];
    double dt2, idt2, idt3;
    step_factors(dt, prm, dt2, idt2, idt3);
    double a1v[3], j1v[3], a2e[3], a3e[3];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        finite = correct_component(s, f, i, k, c, dt, dt2, idt2, idt3, a1v[c], j1v[c], a2e[c],
                                   a3e[c], xp_from_state) &&
                 finite;
    if (!finite) atomicOr(err, DERR_NONFINITE);
    correct_step(s, i, t_new, dt, dt_old, a1v, j1v, a2e, a3e, prm, sd, dtmin_hits);
}

// K4 for active slot k by three lanes of a warp (component c = lane - lane0 on
// lanes lane0 .. lane0 + 2; every lane of the warp calls this, valid marks the
// three that hold a slot): the same arithmetic as correct_body, the FP64
// dependency chain split over the components.
__device__ __forceinline__ void correct_lanes(const StateDev &s, const int *act, int na,
                                              double t_new, const Out3 &f, const StepParams &prm,
                                              SchedDev *sd, unsigned *err,
                                              unsigned long long *dtmin_hits, int k, int lane0,
                                              bool valid, bool xp_from_state = false)
{
    const int lane = threadIdx.x & 31;
    const int c = lane - lane0;
    const bool mine = valid && k < na && c >= 0 && c < 3;
    double a1 = 0.0, j1 = 0.0, a2e = 0.0, a3e = 0.0, dt = 1.0, dt_old = 0.0;
    int i = 0;
    bool fin = true;
    if (mine) {
        if (k == 0 && c == 0) sd->t_cur = t_new;
        i = act ? act[k] : k;
        dt = t_new - s.t[i];
        dt_old = s.dt[i];
        double dt2, idt2, idt3;
        step_factors(dt, prm, dt2, idt2, idt3);
        fin = correct_component(s, f, i, k, c, dt, dt2, idt2, idt3, a1, j1, a2e, a3e,
                                xp_from_state);
    }
    double a1v[3], j1v[3], a2v[3], a3v[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int src = min(31, lane0 + q);
        a1v[q] = __shfl_sync(0xffffffffu, a1, src);
        j1v[q] = __shfl_sync(0xffffffffu, j1, src);
        a2v[q] = __shfl_sync(0xffffffffu, a2e, src);
        a3v[q] = __shfl_sync(0xffffffffu, a3e, src);
    }
    const unsigned bad = __ballot_sync(0xffffffffu, mine && !fin);
    if (mine && c == 0) {
        if (bad & (7u << lane0)) atomicOr(err, DERR_NONFINITE);
        correct_step(s, i, t_new, dt, dt_old, a1v, j1v, a2v, a3v, prm, sd, dtmin_hits);
    }
}

// The start-of-step state of component c of a particle, loaded ahead of its
// corrector (so that the loads overlap other work).
struct CState {
    double x, v, a0, j0, t, dt;
};

__device__ __forceinline__ void cstate_load(const StateDev &s, int i, int c, CState &q)
{
    const long long k = c * s.ld + i;
    q.x = s.pos[k];
    q.v = s.vel[k];
    q.a0 = s.acc[k];
    q.j0 = s.jerk[k];
    q.t = s.t[i];
    q.dt = s.dt[i];
}

// K4 for active slot k (particle i) by three lanes of a warp (component
// c = lane - lane0 on the lanes where mine holds; every lane of the warp calls
// this) from a preloaded state q and the new acc / jerk component a1, j1: the
// same arithmetic as correct_lanes with the prediction recomputed from the
// state.
__device__ __forceinline__ void correct_lanes_pre(const StateDev &s, int i, int k, int c,
                                                  int lane0, bool mine, double t_new,
                                                  const CState &q, double a1, double j1,
                                                  const StepParams &prm, SchedDev *sd,
                                                  unsigned *err, unsigned long long *dtmin_hits)
{
    const int lane = threadIdx.x & 31;
    double a2e = 0.0, a3e = 0.0, dt = 1.0;
    bool fin = true;
    if (mine) {
        if (k == 0 && c == 0) sd->t_cur = t_new;
        dt = t_new - q.t;
        double dt2, idt2, idt3, xp, vp, x1, v1;
        step_factors(dt, prm, dt2, idt2, idt3);
        predict_xv(q.x, q.v, q.a0, q.j0, dt, xp, vp);
        hermite_correct(xp, vp, q.a0, q.j0, a1, j1, dt, dt2, idt2, idt3, x1, v1, a2e, a3e);
        const long long qq = c * s.ld + i;
        s.pos[qq] = x1;
        s.vel[qq] = v1;
        s.acc[qq] = a1;
        s.jerk[qq] = j1;
        fin = isfinite(x1) && isfinite(v1);
    }
    double a1v[3], j1v[3], a2v[3], a3v[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int src = min(31, lane0 + u);
        a1v[u] = __shfl_sync(0xffffffffu, a1, src);
        j1v[u] = __shfl_sync(0xffffffffu, j1, src);
        a2v[u] = __shfl_sync(0xffffffffu, a2e, src);
        a3v[u] = __shfl_sync(0xffffffffu, a3e, src);
    }
    const unsigned bad = __ballot_sync(0xffffffffu, mine && !fin);
    if (mine && c == 0) {
        if (bad & (7u << lane0)) atomicOr(err, DERR_NONFINITE);
        correct_step(s, i, t_new, dt, q.dt, a1v, j1v, a2v, a3v, prm, sd, dtmin_hits);
    }
    (void)lane;
}

// ---- K4 of the 6th-order scheme ---------------------------------------------

// The start-of-step state of component c of a particle for the order-6 corrector.
struct C6State {
    double x, v, a0, j0, s0, t, dt;
};

__device__ __forceinline__ void c6state_load(const StateDev &s, int i, int c, C6State &q)
{
    const long long k = c * s.ld + i;
    q.x = s.pos[k];
    q.v = s.vel[k];
    q.a0 = s.acc[k];
    q.j0 = s.jerk[k];
    q.s0 = s.snap[k];
    q.t = s.t[i];
    q.dt = s.dt[i];
}

// The order-6 corrector of slot k (particle i) by three lanes of a warp
// (component c on lane lane0 + c where mine holds; every lane of the warp calls
// this) from the start-of-step state q and the new a1, j1, s1: x1 and v1 from
// the two-point expansion through (a, jerk, snap) at both ends, the crackle at
// the end of the step from the quintic through both ends (mid-point expansion,
// T = dt/2); the new step from Aarseth's criterion on (a, jerk, snap, crackle),
// quantized as in the 4th-order path. The quintic's k-th derivative carries the
// force rounding (~1e-7 of |a| for double-single pairs) divided by T^k: a
// criterion on the 4th and 5th collapses the steps to dt_min, and the crackle
// is used above its rounding floor only (prm.noise), else a particle whose step
// once got small (a close encounter) could not grow it again.
__device__ __forceinline__ void correct6_lanes_pre(const StateDev &s, int i, int k, int c,
                                                   int lane0, bool mine, double t_new,
                                                   const C6State &q, double a1, double j1,
                                                   double s1, const StepParams &prm,
                                                   SchedDev *sd, unsigned *err,
                                                   unsigned long long *dtmin_hits)
{
    double a3 = 0.0, dt = 1.0, dt_old = 0.0, T = 0.5;
    bool fin = true;
    if (mine) {
        if (k == 0 && c == 0) sd->t_cur = t_new;
        dt = t_new - q.t;
        dt_old = q.dt;
        T = 0.5 * dt;
        const double iT = prm.shared_dt > 0.0 ? 1.0 / T : ldexp(1.0, -ilogb(T));
        const double iT3 = iT * iT * iT, iT5 = iT3 * iT * iT;
        const double x0 = q.x, v0 = q.v, a0 = q.a0, j0 = q.j0, s0 = q.s0;
        // v1 = v0 + dt/2 (a0 + a1) - dt^2/10 (j1 - j0) + dt^3/120 (s0 + s1)
        const double v1 = v0 + dt * fma(dt, fma(dt, (s0 + s1) * (1.0 / 120.0),
                                                -0.1 * (j1 - j0)), 0.5 * (a0 + a1));
        // x1 = x0 + dt/2 (v0 + v1) - dt^2/10 (a1 - a0) + dt^3/120 (j0 + j1)
        const double x1 = x0 + dt * fma(dt, fma(dt, (j0 + j1) * (1.0 / 120.0),
                                                -0.1 * (a1 - a0)), 0.5 * (v0 + v1));
        const double Am = 0.5 * (a1 - a0);
        const double Jp = 0.5 * (j1 + j0), Jm = 0.5 * (j1 - j0);
        const double Sp = 0.5 * (s1 + s0), Sm = 0.5 * (s1 - s0);
        const double c5 = (45.0 * Am - 45.0 * T * Jp + 15.0 * T * T * Sm) * iT5;
        const double c3 = (7.5 * (T * Jp - Am) - 1.5 * T * T * Sm) * iT3;
        const double c4 = 3.0 * (T * Sp - Jm) * iT3;
        a3 = c3 + T * (c4 + 0.5 * T * c5);
        const long long qq = c * s.ld + i;
        s.pos[qq] = x1;
        s.vel[qq] = v1;
        s.acc[qq] = a1;
        s.jerk[qq] = j1;
        s.snap[qq] = s1;
        s.crk[qq] = a3;
        fin = isfinite(x1) && isfinite(v1);
    }
    // the slot's three components on its first lane
    double a1v[3], j1v[3], s1v[3], a3v[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int src = min(31, lane0 + u);
        a1v[u] = __shfl_sync(0xffffffffu, a1, src);
        j1v[u] = __shfl_sync(0xffffffffu, j1, src);
        s1v[u] = __shfl_sync(0xffffffffu, s1, src);
        a3v[u] = __shfl_sync(0xffffffffu, a3, src);
    }
    const unsigned bad = __ballot_sync(0xffffffffu, mine && !fin);
    if (!mine || c != 0) return;
    if (bad & (7u << lane0)) atomicOr(err, DERR_NONFINITE);
    double dt_new;
    if (prm.shared_dt > 0.0) {
        dt_new = prm.shared_dt;
    } else {
        // Aarseth's criterion with the evaluated snap as a2 and the crackle as a3:
        // dt^2 = eta (|a||s| + |j|^2) / (|j||c| + |s|^2), the crackle's magnitude
        // reduced by its rounding floor 30 noise |a| / T^3 (the forces' relative
        // rounding enters it through (a1 - a0) / T^3 with coefficients 7.5 + 22.5);
        // below the floor it counts as zero
        const double A = dot3(a1v, a1v), J = dot3(j1v, j1v), S = dot3(s1v, s1v);
        const double cn = sqrt(dot3(a3v, a3v));
        const double cfl = 30.0 * prm.noise * sqrt(A) / (T * T * T);
        const double ce = cn > cfl ? cn - cfl : 0.0;
        const double num = prm.eta * (sqrt(A * S) + J);
        const double den = sqrt(J) * ce + S;
        bool clamped;
        dt_new = quantize_sq(num, den, dt, t_new, prm.dt_min, prm.dt_max, &clamped);
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

// ---- bounded waits and ordered status words ---------------------------------

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

}  // namespace nb
