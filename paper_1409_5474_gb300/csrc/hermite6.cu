// The 6th-order Hermite scheme on the GPU (Sect. II: direct-summation codes
// pair with integrators of 4th or higher order and individual time steps; the
// scheme is the two-point Hermite one of Nitadori & Makino's 6th-order paper,
// which the same passage cites).
//
// What differs from the 4th-order path: every pair also yields the snap, the
// second time derivative of its acceleration,
//   alpha = (r.v) / r2,   beta = (|v|^2 + r.a) / r2 + alpha^2,
//   A = m r / r2^(3/2),   J = m v / r2^(3/2) - 3 alpha A,
//   S = m a / r2^(3/2) - 6 alpha J - 3 beta A,
// with r, v, a the j-minus-i position, velocity and predicted acceleration and
// r2 = |r|^2 + eps^2. The FP32 kernels evaluate it expanded in r, v and a, so
// that every term is one FMA into its running sum: with q = m / r2^(3/2),
// a3 = -3 alpha and u3 = -3 (|v|^2 + r.a) / r2,
//   J = q v + (a3 q) r,   S = q a + (2 a3 q) v + ((5/3) a3^2 + u3) q r
// (57 FP32 operations per pair against 64 for the nested form). So the j-records carry the predicted acceleration (64
// bytes instead of 48), the prediction runs through the crackle term, and the
// corrector is the order-6 two-point quadrature with the crackle, pop and 5th
// derivative of the acceleration taken from the quintic through (a, jerk,
// snap) at both ends of the step; the step criterion uses the crackle only (see
// k_correct6).
//
// Kernels:
//   k_predict6           K1 for all particles (the block scheduler has its own
//                        order-6 instantiation in step.cu)
//   k_force6_tile32<DS, IPT, NWJ>
//                        K2, FP32 / double-single pairs: a CTA of 8 warps holds
//                        IPT i-particles per thread in 8/NWJ warp columns, NWJ
//                        warp rows share each j-tile; j-tiles of 128 records
//                        stream through a 3-stage ring of bulk copies (TMA
//                        engine, mbarrier completion, bounded waits); a full
//                        tile is transposed into j-pairs and its pair terms run
//                        on packed FP32x2 arithmetic, two j per instruction;
//                        FP32 sums per tile are folded into double-single
//                        totals; grid.y splits the j-range
//   k_force6_tile64      K2, FP64 pairs (the correctness variant)
//   k_force6_reduce<DS>  K3: the splits of each output added in fixed order
//   k_correct6           K4: corrector, end-of-step crackle, step criterion,
//                        block quantization
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "ds.cuh"
#include "nb_internal.cuh"
#include "step_body.cuh"
#include "tma.cuh"

namespace nb {

namespace {

constexpr int H6_VALS = 10;     // acc 3, jerk 3, snap 3, pot 1 per i-particle
constexpr int H6_JT = 128;      // j-records per tile
constexpr int H6_NS = 3;        // ring stages
constexpr int H6_NWARP = 8;     // warps per FP32 CTA
constexpr int H6_T64 = 128;     // threads per FP64 CTA
constexpr int H6_JT64 = 128;    // j per FP64 shared tile
constexpr int CORRECT6_THREADS = 128;  // 4 warps x 10 slots (3 lanes per slot)
constexpr float F53 = 5.f / 3.f;        // S's r coefficient: (15 alpha^2 - 3 u) = 5/3 a3^2 + u3

// ---- K1 ----------------------------------------------------------------------

template <bool REC>
__global__ void k_predict6(StateDev s, double t, unsigned *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    if (t < s.t[i]) atomicOr(err, DERR_BACKWARD);
    predict6_one<REC>(s, i, t);
}

// Member index of slot k; an index outside [0, n) is flagged and replaced by 0.
__device__ __forceinline__ int member6(const int *idx, int k, int n, unsigned *err)
{
    const int r = idx ? __ldg(idx + k) : k;
    if ((unsigned)r >= (unsigned)n) {
        atomicOr(err, DERR_BADINDEX);
        return 0;
    }
    return r;
}

// Store the 10 totals of slot k (v[9] is the positive potential sum P; pot = -P).
__device__ __forceinline__ void store6(const Out6 &out, int k, double v[H6_VALS], unsigned *err)
{
    v[9] = -v[9];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < H6_VALS; ++c) ok = ok && isfinite(v[c]);
    if (!ok) atomicOr(err, DERR_NONFINITE);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (out.acc) out.acc[c * out.ld + k] = v[c];
        if (out.jerk) out.jerk[c * out.ld + k] = v[3 + c];
        if (out.snap) out.snap[c * out.ld + k] = v[6 + c];
    }
    if (out.pot) out.pot[k] = v[9];
}

// ---- K2, FP32 / double-single ---------------------------------------------------

// IPT i-particles per thread share each j-record loaded from shared memory. The
// CTA's 8 warps are NWI warp columns (different i-particles) x NWJ warp rows
// (the same i-particles, sharing out each j-tile: row g takes j = g, g + NWJ,
// ...), so that a small due set still spreads over the SM; rows are added in
// shared memory at the end, in fixed order. Two CTAs per SM (16 warps) hide the
// pair arithmetic's latencies better than one. A full j-tile is rewritten once in
// shared memory as j-pairs (each float4 part of records 2q and 2q + 1 interleaved
// component by component), so that the pair terms of two j run on the packed
// FP32x2 instructions (half the issue slots of scalar FP32 at the same lane rate),
// with the i-particle's values duplicated in both lanes; a tile that holds the
// i-particle itself, or the ragged last tile, takes the scalar body. One
// i-particle per thread: a second one with the packed sums spills registers.
template <bool DS, int IPT, int NWJ>
__global__ void __launch_bounds__(32 * H6_NWARP, 2)
    k_force6_tile32(const float4 *__restrict__ jrec, int nj, const int *__restrict__ idx,
                    int n_i, float eps2f, int ntiles, float2 *__restrict__ part, long long pld,
                    Out6 out, unsigned *err)
{
    // H6_NS ring stages of H6_JT records, then the current tile as j-pairs
    extern __shared__ __align__(128) float4 s_tile6[];
    __shared__ __align__(8) uint64_t s_full[H6_NS];
    __shared__ int s_abort;

    constexpr int NWI = H6_NWARP / NWJ;
    constexpr int IB = 32 * NWI * IPT;
    static_assert(NWI * NWJ == H6_NWARP, "warp grid");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wi = warp % NWI, wj = warp / NWI;
    const int nsplit = gridDim.y, split = blockIdx.y;
    const int tile0 = (int)((long long)ntiles * split / nsplit);
    const int tile1 = (int)((long long)ntiles * (split + 1) / nsplit);
    const int my_tiles = tile1 - tile0;

    // this thread's i-particles (idle slots past n_i compute a copy of the last one)
    int ii[IPT];
    float xh[IPT], yh[IPT], zh[IPT], xl[IPT], yl[IPT], zl[IPT];
    float vx[IPT], vy[IPT], vz[IPT], ax[IPT], ay[IPT], az[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
        const int k = min(blockIdx.x * IB + p * (32 * NWI) + wi * 32 + lane, n_i - 1);
        ii[p] = member6(idx, k, nj, err);
        const float4 *r = jrec + (size_t)DS6_REC * ii[p];
        const float4 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2), d = __ldg(r + 3);
        xh[p] = a.x; yh[p] = a.y; zh[p] = a.z;
        xl[p] = b.x; yl[p] = b.y; zl[p] = b.z;
        vx[p] = c.x; vy[p] = c.y; vz[p] = c.z;
        ax[p] = d.x; ay[p] = d.y; az[p] = d.z;
    }
    constexpr int NPAIR = H6_JT / 2;
    float4 *s_pair = s_tile6 + (size_t)H6_NS * H6_JT * DS6_REC;
    const float2 e2 = make_float2(eps2f, eps2f);

    // double-single totals (hi, lo) and the FP32 sums of the current tile (folded
    // after every tile: 128 pairs per sum)
    float H[IPT][H6_VALS], L[IPT][H6_VALS], t[IPT][H6_VALS];
    float2 t2[IPT][H6_VALS];  // the packed path's sums: even and odd j of the pairs
#pragma unroll
    for (int p = 0; p < IPT; ++p)
#pragma unroll
        for (int c = 0; c < H6_VALS; ++c) {
            H[p][c] = L[p][c] = t[p][c] = 0.f;
            t2[p][c] = make_float2(0.f, 0.f);
        }

    if (tid == 0) {
        s_abort = 0;
#pragma unroll
        for (int q = 0; q < H6_NS; ++q) mbar_init(&s_full[q], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int kt) {
        const int stage = kt % H6_NS;
        const int tt = tile0 + kt;
        const int cnt = min(H6_JT, nj - tt * H6_JT);
        const uint32_t bytes = (uint32_t)cnt * DS6_REC * 16u;
        mbar_expect_tx(&s_full[stage], bytes);
        bulk_g2s(s_tile6 + (size_t)stage * H6_JT * DS6_REC, jrec + (size_t)tt * H6_JT * DS6_REC,
                 bytes, &s_full[stage]);
    };
    if (tid == 0)
        for (int kt = 0; kt < H6_NS && kt < my_tiles; ++kt) issue(kt);

    for (int kt = 0; kt < my_tiles; ++kt) {
        const int stage = kt % H6_NS;
        if (!mbar_wait(&s_full[stage], (uint32_t)((kt / H6_NS) & 1))) s_abort = 1;
        const float4 *T = s_tile6 + (size_t)stage * H6_JT * DS6_REC;
        const int jbase = (tile0 + kt) * H6_JT;
        const int cnt = min(H6_JT, nj - jbase);
        bool mine = false;
#pragma unroll
        for (int p = 0; p < IPT; ++p) mine = mine || (ii[p] >= jbase && ii[p] < jbase + cnt);
        const bool own = __any_sync(0xffffffffu, mine);

        auto body = [&](int jj, auto masked_tag) {
            constexpr bool MASKED = decltype(masked_tag)::value;
            const float4 P = T[DS6_REC * jj];
            const float4 V = T[DS6_REC * jj + 2];
            const float4 W = T[DS6_REC * jj + 3];
            float4 Q;
            if (DS) Q = T[DS6_REC * jj + 1];
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
                float dx, dy, dz;
                if (DS) {
                    dx = (P.x - xh[p]) + (Q.x - xl[p]);
                    dy = (P.y - yh[p]) + (Q.y - yl[p]);
                    dz = (P.z - zh[p]) + (Q.z - zl[p]);
                } else {
                    dx = P.x - xh[p];
                    dy = P.y - yh[p];
                    dz = P.z - zh[p];
                }
                const float dvx = V.x - vx[p], dvy = V.y - vy[p], dvz = V.z - vz[p];
                const float dax = W.x - ax[p], day = W.y - ay[p], daz = W.z - az[p];
                float r2 = fmaf(dx, dx, eps2f);
                r2 = fmaf(dy, dy, r2);
                r2 = fmaf(dz, dz, r2);
                float rv = dx * dvx;
                rv = fmaf(dy, dvy, rv);
                rv = fmaf(dz, dvz, rv);
                float w2 = dvx * dvx;  // |v|^2 + r.a
                w2 = fmaf(dvy, dvy, w2);
                w2 = fmaf(dvz, dvz, w2);
                w2 = fmaf(dx, dax, w2);
                w2 = fmaf(dy, day, w2);
                w2 = fmaf(dz, daz, w2);
                float rinv = rsqrtf(r2);
                if (MASKED) rinv = (jbase + jj == ii[p]) ? 0.f : rinv;
                const float rinv2 = rinv * rinv;
                const float mrinv = P.w * rinv;
                const float mr3 = mrinv * rinv2;
                const float r3 = rinv2 * -3.f;
                const float m3a = rv * r3;  // -3 alpha
                const float m3u = w2 * r3;  // -3 (|v|^2 + r.a) / r^2
                const float k1 = m3a * mr3;
                const float c1 = k1 + k1;
                const float c2 = fmaf(m3a, m3a * F53, m3u) * mr3;
                t[p][0] = fmaf(mr3, dx, t[p][0]);
                t[p][1] = fmaf(mr3, dy, t[p][1]);
                t[p][2] = fmaf(mr3, dz, t[p][2]);
                t[p][3] = fmaf(k1, dx, fmaf(mr3, dvx, t[p][3]));
                t[p][4] = fmaf(k1, dy, fmaf(mr3, dvy, t[p][4]));
                t[p][5] = fmaf(k1, dz, fmaf(mr3, dvz, t[p][5]));
                t[p][6] = fmaf(c2, dx, fmaf(c1, dvx, fmaf(mr3, dax, t[p][6])));
                t[p][7] = fmaf(c2, dy, fmaf(c1, dvy, fmaf(mr3, day, t[p][7])));
                t[p][8] = fmaf(c2, dz, fmaf(c1, dvz, fmaf(mr3, daz, t[p][8])));
                t[p][9] += mrinv;
            }
        };
        if (cnt == H6_JT) {
            // full tile: transposed into j-pairs (each float4 part of records 2q and
            // 2q + 1 side by side) for the packed FP32x2 pair terms, two j at a time
            for (int x = tid; x < DS6_REC * NPAIR; x += 32 * H6_NWARP) {
                const int q = x % NPAIR, part6 = x / NPAIR;
                const float4 u = T[DS6_REC * (2 * q) + part6];
                const float4 v = T[DS6_REC * (2 * q + 1) + part6];
                float4 *Pp = s_pair + 2 * DS6_REC * q + 2 * part6;
                Pp[0] = make_float4(u.x, v.x, u.y, v.y);
                Pp[1] = make_float4(u.z, v.z, u.w, v.w);
            }
            __syncthreads();
            if (own) {
                for (int jj = wj; jj < H6_JT; jj += NWJ) body(jj, std::true_type{});
            } else {
#pragma unroll 2
                for (int q = wj; q < NPAIR; q += NWJ) {
                    const float4 *Pp = s_pair + 2 * DS6_REC * q;
                    const float4 q0 = Pp[0], q1 = Pp[1], q4 = Pp[4], q5 = Pp[5], q6 = Pp[6],
                                 q7 = Pp[7];
                    float4 q2, q3;
                    if (DS) {
                        q2 = Pp[2];
                        q3 = Pp[3];
                    }
#pragma unroll
                    for (int p = 0; p < IPT; ++p) {
                        float2 dx, dy, dz;
                        if (DS) {
                            dx = __fadd2_rn(__fadd2_rn(make_float2(q0.x, q0.y), make_float2(-xh[p], -xh[p])),
                                            __fadd2_rn(make_float2(q2.x, q2.y), make_float2(-xl[p], -xl[p])));
                            dy = __fadd2_rn(__fadd2_rn(make_float2(q0.z, q0.w), make_float2(-yh[p], -yh[p])),
                                            __fadd2_rn(make_float2(q2.z, q2.w), make_float2(-yl[p], -yl[p])));
                            dz = __fadd2_rn(__fadd2_rn(make_float2(q1.x, q1.y), make_float2(-zh[p], -zh[p])),
                                            __fadd2_rn(make_float2(q3.x, q3.y), make_float2(-zl[p], -zl[p])));
                        } else {
                            dx = __fadd2_rn(make_float2(q0.x, q0.y), make_float2(-xh[p], -xh[p]));
                            dy = __fadd2_rn(make_float2(q0.z, q0.w), make_float2(-yh[p], -yh[p]));
                            dz = __fadd2_rn(make_float2(q1.x, q1.y), make_float2(-zh[p], -zh[p]));
                        }
                        const float2 dvx = __fadd2_rn(make_float2(q4.x, q4.y), make_float2(-vx[p], -vx[p]));
                        const float2 dvy = __fadd2_rn(make_float2(q4.z, q4.w), make_float2(-vy[p], -vy[p]));
                        const float2 dvz = __fadd2_rn(make_float2(q5.x, q5.y), make_float2(-vz[p], -vz[p]));
                        const float2 dax = __fadd2_rn(make_float2(q6.x, q6.y), make_float2(-ax[p], -ax[p]));
                        const float2 day = __fadd2_rn(make_float2(q6.z, q6.w), make_float2(-ay[p], -ay[p]));
                        const float2 daz = __fadd2_rn(make_float2(q7.x, q7.y), make_float2(-az[p], -az[p]));
                        float2 r2 = __ffma2_rn(dx, dx, e2);
                        r2 = __ffma2_rn(dy, dy, r2);
                        r2 = __ffma2_rn(dz, dz, r2);
                        float2 rv = __fmul2_rn(dx, dvx);
                        rv = __ffma2_rn(dy, dvy, rv);
                        rv = __ffma2_rn(dz, dvz, rv);
                        float2 w2 = __fmul2_rn(dvx, dvx);  // |v|^2 + r.a
                        w2 = __ffma2_rn(dvy, dvy, w2);
                        w2 = __ffma2_rn(dvz, dvz, w2);
                        w2 = __ffma2_rn(dx, dax, w2);
                        w2 = __ffma2_rn(dy, day, w2);
                        w2 = __ffma2_rn(dz, daz, w2);
                        const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                        const float2 rinv2 = __fmul2_rn(rinv, rinv);
                        const float2 mrinv = __fmul2_rn(make_float2(q1.z, q1.w), rinv);
                        const float2 mr3 = __fmul2_rn(mrinv, rinv2);
                        const float2 r3 = __fmul2_rn(rinv2, make_float2(-3.f, -3.f));
                        const float2 m3a = __fmul2_rn(rv, r3);  // -3 alpha
                        const float2 m3u = __fmul2_rn(w2, r3);  // -3 (|v|^2 + r.a) / r^2
                        const float2 k1 = __fmul2_rn(m3a, mr3);
                        const float2 c1 = __fadd2_rn(k1, k1);
                        const float2 c2 = __fmul2_rn(
                            __ffma2_rn(m3a, __fmul2_rn(m3a, make_float2(F53, F53)), m3u), mr3);
                        t2[p][0] = __ffma2_rn(mr3, dx, t2[p][0]);
                        t2[p][1] = __ffma2_rn(mr3, dy, t2[p][1]);
                        t2[p][2] = __ffma2_rn(mr3, dz, t2[p][2]);
                        t2[p][3] = __ffma2_rn(k1, dx, __ffma2_rn(mr3, dvx, t2[p][3]));
                        t2[p][4] = __ffma2_rn(k1, dy, __ffma2_rn(mr3, dvy, t2[p][4]));
                        t2[p][5] = __ffma2_rn(k1, dz, __ffma2_rn(mr3, dvz, t2[p][5]));
                        t2[p][6] = __ffma2_rn(c2, dx, __ffma2_rn(c1, dvx, __ffma2_rn(mr3, dax, t2[p][6])));
                        t2[p][7] = __ffma2_rn(c2, dy, __ffma2_rn(c1, dvy, __ffma2_rn(mr3, day, t2[p][7])));
                        t2[p][8] = __ffma2_rn(c2, dz, __ffma2_rn(c1, dvz, __ffma2_rn(mr3, daz, t2[p][8])));
                        t2[p][9] = __fadd2_rn(t2[p][9], mrinv);
                    }
                }
            }
        } else if (own) {
            for (int jj = wj; jj < cnt; jj += NWJ) body(jj, std::true_type{});
        } else {
#pragma unroll 2
            for (int jj = wj; jj < cnt; jj += NWJ) body(jj, std::false_type{});
        }
#pragma unroll
        for (int p = 0; p < IPT; ++p)
#pragma unroll
            for (int c = 0; c < H6_VALS; ++c) {
                const float sum = t[p][c] + (t2[p][c].x + t2[p][c].y);
                if (DS)
                    ds_add(H[p][c], L[p][c], sum);
                else
                    H[p][c] += sum;
                t[p][c] = 0.f;
                t2[p][c] = make_float2(0.f, 0.f);
            }

        __syncthreads();  // every warp is done with this stage
        if (s_abort) {
            if (tid == 0) drain_ring<H6_NS>(s_full, 0u, kt, my_tiles);
            break;
        }
        if (tid == 0 && kt + H6_NS < my_tiles) issue(kt + H6_NS);
    }
    if (s_abort) {
        if (tid == 0) atomicOr(err, DERR_TIMEOUT);
        return;
    }
    if (NWJ > 1) {
        // add the warp rows in order 0..NWJ-1 (the tile ring is free: every copy has landed)
        float2 *s_red = reinterpret_cast<float2 *>(s_tile6);  // [NWJ][H6_VALS][IB]
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
            const int slot = p * (32 * NWI) + wi * 32 + lane;
#pragma unroll
            for (int c = 0; c < H6_VALS; ++c)
                s_red[(wj * H6_VALS + c) * IB + slot] = make_float2(H[p][c], L[p][c]);
        }
        __syncthreads();
        if (wj != 0) return;
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
            const int slot = p * (32 * NWI) + wi * 32 + lane;
#pragma unroll
            for (int c = 0; c < H6_VALS; ++c) {
                dsf v{H[p][c], L[p][c]};
                for (int g = 1; g < NWJ; ++g) {
                    const float2 w = s_red[(g * H6_VALS + c) * IB + slot];
                    ds_acc(v, dsf{w.x, w.y});
                }
                H[p][c] = v.hi;
                L[p][c] = v.lo;
            }
        }
    }
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
        const int kk = blockIdx.x * IB + p * (32 * NWI) + wi * 32 + lane;
        if (kk >= n_i) continue;
        if (nsplit == 1) {
            double v[H6_VALS];
#pragma unroll
            for (int c = 0; c < H6_VALS; ++c) v[c] = ds_to_double(dsf{H[p][c], L[p][c]});
            store6(out, kk, v, err);
        } else {
#pragma unroll
            for (int c = 0; c < H6_VALS; ++c)
                part[((size_t)split * H6_VALS + c) * pld + kk] = make_float2(H[p][c], L[p][c]);
        }
    }
}

// ---- K2, FP64 ---------------------------------------------------------------

// One i-particle per thread; the j-set (predicted FP64 position, velocity,
// acceleration and mass: 80 bytes per particle) goes through shared memory in
// tiles of H6_JT64. grid.y splits the j-range.
__global__ void __launch_bounds__(H6_T64)
    k_force6_tile64(StateDev s, const int *__restrict__ idx, int n_i, double eps2,
                    double *__restrict__ part, long long pld, Out6 out, unsigned *err)
{
    __shared__ double sj[10][H6_JT64];
    const int nj = s.n;
    const int nsplit = gridDim.y, split = blockIdx.y;
    const int ntiles = (nj + H6_JT64 - 1) / H6_JT64;
    const int tile0 = (int)((long long)ntiles * split / nsplit);
    const int tile1 = (int)((long long)ntiles * (split + 1) / nsplit);
    const int k = min(blockIdx.x * H6_T64 + (int)threadIdx.x, n_i - 1);
    const int ii = member6(idx, k, nj, err);
    double xi[3], vi[3], ai[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xi[c] = s.pos_p[c * s.ld + ii];
        vi[c] = s.vel_p[c * s.ld + ii];
        ai[c] = s.acc_p[c * s.ld + ii];
    }
    double acc[H6_VALS];
#pragma unroll
    for (int c = 0; c < H6_VALS; ++c) acc[c] = 0.0;
    for (int tt = tile0; tt < tile1; ++tt) {
        const int jbase = tt * H6_JT64;
        const int cnt = min(H6_JT64, nj - jbase);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += H6_T64) {
            const int j = jbase + q;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sj[c][q] = s.pos_p[c * s.ld + j];
                sj[3 + c][q] = s.vel_p[c * s.ld + j];
                sj[6 + c][q] = s.acc_p[c * s.ld + j];
            }
            sj[9][q] = s.m[j];
        }
        __syncthreads();
        for (int q = 0; q < cnt; ++q) {
            if (jbase + q == ii) continue;
            const double dx = sj[0][q] - xi[0], dy = sj[1][q] - xi[1], dz = sj[2][q] - xi[2];
            const double dvx = sj[3][q] - vi[0], dvy = sj[4][q] - vi[1], dvz = sj[5][q] - vi[2];
            const double dax = sj[6][q] - ai[0], day = sj[7][q] - ai[1], daz = sj[8][q] - ai[2];
            const double r2 = eps2 + dx * dx + dy * dy + dz * dz;
            const double rinv = rsqrt(r2);
            const double rinv2 = rinv * rinv;
            const double mrinv = sj[9][q] * rinv;
            const double mr3 = mrinv * rinv2;
            const double alpha = (dx * dvx + dy * dvy + dz * dvz) * rinv2;
            const double beta =
                (dvx * dvx + dvy * dvy + dvz * dvz + dx * dax + dy * day + dz * daz) * rinv2 +
                alpha * alpha;
            const double A[3] = {mr3 * dx, mr3 * dy, mr3 * dz};
            const double dv[3] = {dvx, dvy, dvz}, da[3] = {dax, day, daz};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double J = mr3 * dv[c] - 3.0 * alpha * A[c];
                acc[c] += A[c];
                acc[3 + c] += J;
                acc[6 + c] += mr3 * da[c] - 6.0 * alpha * J - 3.0 * beta * A[c];
            }
            acc[9] += mrinv;
        }
    }
    const int kk = blockIdx.x * H6_T64 + threadIdx.x;
    if (kk >= n_i) return;
    if (nsplit == 1) {
        store6(out, kk, acc, err);
    } else {
#pragma unroll
        for (int c = 0; c < H6_VALS; ++c) part[((size_t)split * H6_VALS + c) * pld + kk] = acc[c];
    }
}

// ---- K3 --------------------------------------------------------------------------

// One warp per (component, slot): lane l adds splits l, l + 32, ... in order, then
// a fixed xor tree, so the result does not depend on the order the CTAs ran in.
template <bool DS>
__global__ void k_force6_reduce(const void *__restrict__ part, long long pld, int nsplit, int n_i,
                                Out6 out, unsigned *err)
{
    const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= (long long)n_i * H6_VALS) return;  // whole warps leave together
    const int c = (int)(q / n_i), k = (int)(q % n_i);
    double v;
    if (DS) {
        const float2 *p = static_cast<const float2 *>(part);
        dsf a{0.f, 0.f};
        for (int sp = lane; sp < nsplit; sp += 32) {
            const float2 w = __ldg(p + ((size_t)sp * H6_VALS + c) * pld + k);
            ds_acc(a, dsf{w.x, w.y});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ds_acc(a, ds_shfl_xor(a, o));
        v = ds_to_double(a);
    } else {
        const double *p = static_cast<const double *>(part);
        v = 0.0;
        for (int sp = lane; sp < nsplit; sp += 32) v += __ldg(p + ((size_t)sp * H6_VALS + c) * pld + k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    if (lane != 0) return;
    if (c == 9) {
        v = -v;
        if (out.pot) out.pot[k] = v;
    } else {
        double *dst = c < 3 ? out.acc : (c < 6 ? out.jerk : out.snap);
        if (dst) dst[(c % 3) * out.ld + k] = v;
    }
    if (!isfinite(v)) atomicOr(err, DERR_NONFINITE);
}

// ---- K4 --------------------------------------------------------------------------

// Slot k: the order-6 corrector (correct6_lanes_pre) from the start-of-step state
// and the new a1, j1, s1 (f, slot-indexed).
__global__ void __launch_bounds__(CORRECT6_THREADS)
    k_correct6(StateDev s, const int *__restrict__ act, int na, double t_new, Out6 f,
               StepParams prm, SchedDev *sd, unsigned *err, unsigned long long *dtmin_hits)
{
    // three lanes per slot (component c = lane % 3 of slot lane / 3; lanes 30, 31
    // idle), so that the FP64 dependency chains of the three components run side by side
    const int lane = threadIdx.x & 31;
    const int warp_g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int k = warp_g * 10 + lane / 3;
    const int c = lane % 3;
    const bool mine = lane < 30 && k < na;
    C6State q{};
    double a1 = 0.0, j1 = 0.0, s1 = 0.0;
    int i = 0;
    if (mine) {
        i = act ? act[k] : k;
        c6state_load(s, i, c, q);
        a1 = f.acc[c * f.ld + k];
        j1 = f.jerk[c * f.ld + k];
        s1 = f.snap[c * f.ld + k];
    }
    correct6_lanes_pre(s, i, k, c, lane - c, mine, t_new, q, a1, j1, s1, prm, sd, err,
                       dtmin_hits);
}

// Resident CTAs per SM of a FP32 / double-single variant (occupancy API, cached).
template <bool DS, int IPT, int NWJ>
int occ6()
{
    static int v = -1;
    if (v < 0) {
        int b = 0;
        const size_t smem = (size_t)(H6_NS + 1) * H6_JT * DS6_REC * sizeof(float4);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_force6_tile32<DS, IPT, NWJ>,
                                                          32 * H6_NWARP, smem) != cudaSuccess) {
            cudaGetLastError();
            b = 1;
        }
        v = std::max(b, 1);
    }
    return v;
}

int occ6_of(bool ds, int ipt, int nwj)
{
    switch (nwj) {
    case 8: return ds ? occ6<true, 1, 8>() : occ6<false, 1, 8>();
    case 4: return ds ? occ6<true, 1, 4>() : occ6<false, 1, 4>();
    case 2: return ds ? occ6<true, 1, 2>() : occ6<false, 1, 2>();
    default: return ds ? occ6<true, 1, 1>() : occ6<false, 1, 1>();
    }
}

}  // namespace

// ---- host side ---------------------------------------------------------------------

cudaError_t launch_predict6(const StateDev &s, double t, bool want_rec, unsigned *err,
                            cudaStream_t st)
{
    if (s.n <= 0) return cudaSuccess;
    const int bs = 256, g = (s.n + bs - 1) / bs;
    if (want_rec)
        k_predict6<true><<<g, bs, 0, st>>>(s, t, err);
    else
        k_predict6<false><<<g, bs, 0, st>>>(s, t, err);
    return cudaGetLastError();
}


// The CTA shape from the size of the due set: one i-particle per thread, warp
// rows sharing each j-tile below 256 (8 rows for 32 or fewer). Then the
// j-splits: at least two waves of resident CTAs (one for the warp-row shapes,
// whose CTAs are short: 8-14% faster there), then the fewest splits, up to
// eight times that many, whose last wave is at least 97% full, else the
// fullest (256 i-blocks on 304 slots fill 84% of their last wave at 3 to 6
// splits: the SMs idled 16% of a full N = 65536 evaluation); at most one split
// per j-tile.
ForcePlan plan_force6(int variant, int n_i, int n_j, int num_sms)
{
    ForcePlan p{};
    p.kind = 0;
    const bool f64 = (variant == NB_F64);
    p.ipt = 1;  // the packed pair terms already give each thread two j per step
    if (!f64 && n_i > 256 && n_i < 512) {
        // 257-511 due particles: the shape (warp rows) and split count of least
        // estimated time, waves x (i per CTA x j per CTA + about 16384 pair terms of
        // fixed cost per CTA: prologue, pipeline fill, epilogue), with at least 4 j-tiles
        // per split; candidates: the split counts just within 1..8 whole waves. The rule
        // below gives these sizes two half-used i-blocks in two waves of CTAs of 1.7
        // j-tiles each (87 us per launch at N = 65536, 200 G/s); this model gives 8 warp
        // rows and one wave (66 us). For 128-255 and 2048-4095 due particles the same
        // model chose shapes 5% slower than the rule's, so it is not used there.
        const long long ntiles = (n_j + H6_JT - 1) / H6_JT;
        const long long cap = std::max(1LL, std::min(ntiles / 4, 1024LL));
        const bool ds = variant == NB_F32DS;
        double best_t = -1.0;
        for (int nwj = 1; nwj <= 8; nwj *= 2) {
            const long long ib = 32LL * (H6_NWARP / nwj);
            const long long nblk = (n_i + ib - 1) / ib;
            const long long slots = (long long)std::max(num_sms, 1) * occ6_of(ds, 1, nwj);
            for (int k = 0; k <= 9; ++k) {
                const long long ns =
                    k == 0 ? 1 : (k == 9 ? cap : std::max(1LL, std::min(cap, k * slots / nblk)));
                const long long jpc = (ntiles + ns - 1) / ns * H6_JT;
                const double t = (double)((nblk * ns + slots - 1) / slots) *
                                 ((double)ib * (double)jpc + 16384.0);
                if (best_t < 0.0 || t < best_t * (1.0 - 1e-12)) {
                    best_t = t;
                    p.nwj = nwj;
                    p.nsplit = (int)ns;
                }
            }
        }
        p.threads = 32 * (H6_NWARP / p.nwj);
        p.jt = H6_JT;
        return p;
    }
    p.nwj = f64 ? 1 : (n_i <= 32 ? 8 : n_i <= 64 ? 4 : n_i <= 128 ? 2 : 1);
    p.threads = f64 ? H6_T64 : 32 * (H6_NWARP / p.nwj) * p.ipt;  // i-particles per CTA
    p.jt = f64 ? H6_JT64 : H6_JT;
    const long long nblk = (n_i + p.threads - 1) / p.threads;
    const long long ntiles = (n_j + p.jt - 1) / p.jt;
    const long long cap = std::max(1LL, f64 ? ntiles / 4 : ntiles);
    const long long slots =
        (long long)std::max(num_sms, 1) * (f64 ? 4 : occ6_of(variant == NB_F32DS, p.ipt, p.nwj));
    const long long waves = p.nwj > 1 ? 1 : 2;
    const long long ns0 = std::min(cap, std::max(1LL, (waves * slots + nblk - 1) / nblk));
    long long best = ns0;
    double best_eff = 0.0;
    for (long long ns = ns0; ns <= std::min(cap, 8 * ns0); ++ns) {
        const double waves = (double)(nblk * ns) / (double)slots;
        const double eff = waves / std::ceil(waves);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = ns;
        }
        if (eff >= 0.97) break;  // the fewest splits whose last wave is nearly full
    }
    p.nsplit = (int)std::min(best, 1024LL);
    return p;
}

// The plan of a table entry (F32 / double-single kinds: warp rows nwj in {1, 2, 4,
// 8}, nsplit j-splits clamped to the j-tiles and to 1024; FP64: one warp row).
ForcePlan plan6_from_entry(int variant, int nwj, int nsplit, int n_i, int n_j)
{
    ForcePlan p{};
    p.kind = 0;
    p.ipt = 1;
    if (variant == NB_F64) {
        p.nwj = 1;
        p.threads = H6_T64;
        p.jt = H6_JT64;
    } else {
        p.nwj = (nwj == 2 || nwj == 4 || nwj == 8) ? nwj : 1;
        p.threads = 32 * (H6_NWARP / p.nwj);
        p.jt = H6_JT;
    }
    const long long ntiles = std::max(1LL, ((long long)n_j + p.jt - 1) / p.jt);
    p.nsplit = (int)std::max(1LL, std::min<long long>({(long long)nsplit, ntiles, 1024LL}));
    (void)n_i;
    return p;
}

int occ6_blocks(int variant, int nwj)
{
    return occ6_of(variant == NB_F32DS, 1, nwj);
}

size_t plan6_partial_doubles(const ForcePlan &p, int n_i)
{
    if (p.nsplit <= 1) return 0;
    return (size_t)p.nsplit * H6_VALS * (size_t)n_i;  // float2 (DS) or double: 8 bytes each
}

cudaError_t launch_force6(int variant, const ForcePlan &p, const StateDev &s, const int *idx,
                          int n_i, double eps2, double *part, const Out6 &out, unsigned *err,
                          cudaStream_t st, cudaEvent_t *ev)
{
    if (n_i <= 0) return cudaSuccess;
    const long long pld = n_i;
    if (ev) cudaEventRecord(ev[0], st);
    if (variant == NB_F64) {
        dim3 grid((n_i + H6_T64 - 1) / H6_T64, p.nsplit);
        k_force6_tile64<<<grid, H6_T64, 0, st>>>(s, idx, n_i, eps2, part, pld, out, err);
    } else {
        const int ntiles = (s.n + H6_JT - 1) / H6_JT;
        const int nt = 32 * H6_NWARP;
        const int ib = 32 * (H6_NWARP / p.nwj) * p.ipt;
        dim3 grid((n_i + ib - 1) / ib, p.nsplit);
        const size_t smem = (size_t)(H6_NS + 1) * H6_JT * DS6_REC * sizeof(float4);
        float2 *pp = reinterpret_cast<float2 *>(part);
        const float e2 = (float)eps2;
        auto go = [&](auto kern) {
            kern<<<grid, nt, smem, st>>>(s.rec6, s.n, idx, n_i, e2, ntiles, pp, pld, out, err);
        };
        const bool ds = (variant == NB_F32DS);
        if (p.nwj == 8)
            ds ? go(k_force6_tile32<true, 1, 8>) : go(k_force6_tile32<false, 1, 8>);
        else if (p.nwj == 4)
            ds ? go(k_force6_tile32<true, 1, 4>) : go(k_force6_tile32<false, 1, 4>);
        else if (p.nwj == 2)
            ds ? go(k_force6_tile32<true, 1, 2>) : go(k_force6_tile32<false, 1, 2>);
        else
            ds ? go(k_force6_tile32<true, 1, 1>) : go(k_force6_tile32<false, 1, 1>);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) {
        cudaEventRecord(ev[1], st);
        cudaEventRecord(ev[2], st);
    }
    if (p.nsplit > 1) {
        const long long total = (long long)n_i * H6_VALS * 32;  // a warp per output
        const int bs = 256;
        const int g = (int)((total + bs - 1) / bs);
        if (variant == NB_F64)
            k_force6_reduce<false><<<g, bs, 0, st>>>(part, pld, p.nsplit, n_i, out, err);
        else
            k_force6_reduce<true><<<g, bs, 0, st>>>(part, pld, p.nsplit, n_i, out, err);
        e = cudaGetLastError();
    }
    if (ev) cudaEventRecord(ev[3], st);
    return e;
}

cudaError_t launch_correct6(const StateDev &s, const int *act, int n_a, double t_new,
                            const Out6 &f, const StepParams &p, SchedDev *sd, unsigned *err,
                            unsigned long long *dtmin_hits, cudaStream_t st)
{
    const int slots = 10 * (CORRECT6_THREADS / 32);
    const int g = std::max(1, (n_a + slots - 1) / slots);
    k_correct6<<<g, CORRECT6_THREADS, 0, st>>>(s, act, n_a, t_new, f, p, sd, err, dtmin_hits);
    return cudaGetLastError();
}

}  // namespace nb
