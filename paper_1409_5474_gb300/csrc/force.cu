// Pair-force kernels (K2) and the partial-sum reduction (K3).
//
// Direct summation of softened gravity from a j-set onto an i-set (paper
// Sect. III.A): for every i and every j != i,
//   r = x_j - x_i, v = v_j - v_i, s2 = |r|^2 + eps^2, rinv = s2^(-1/2),
//   acc += m_j rinv^3 r,  jerk += m_j rinv^3 (v - 3 (r.v) rinv^2 r),  pot -= m_j rinv.
//
// Two mappings of the (i, j) work onto the GPU, as the paper discusses:
//  - tile kernels ("i-parallel", Sect. III.A): each thread owns IPT
//    i-particles in registers; the CTA streams its j-range through shared
//    memory in tiles of JT records, staged by 1-D bulk copies (the TMA engine,
//    cp.async.bulk) into an NS-deep ring of mbarrier-guarded buffers. The
//    j-range is split across grid.y (the paper's j-parallel split for small
//    N_i, after Makino's scheme), and the partial sums are reduced by K3.
//  - j-parallel warp kernels for tiny i-sets (N_i <= 32, block-step tails):
//    every thread holds the same few i-particles and a different j; partial
//    sums are combined by warp shuffles, then across warps in FP64, then
//    across CTAs by K3.
//
// Precision variants (Sect. III.A: emulated double precision for the
// inter-particle distance, native FP64 for extreme mass ratios):
//  - NB_F32DS: positions as double-single (hi + lo FP32) records; the relative
//    coordinate is (x_j.hi - x_i.hi) + (x_j.lo - x_i.lo), which keeps close
//    pairs far from the origin accurate; pair math in FP32 with rsqrtf on the
//    SFU; per-tile FP32 sums folded into double-single accumulators (TwoSum).
//  - NB_F32: the same kernel with FP32 positions (hi only) and FP32 sums.
//  - NB_F64: IEEE binary64 throughout.
//
// Self pair: for i-particles that are members of the j-set the i == j pair is
// masked by index (its potential term m_i/eps would otherwise swamp the FP32
// sums, and with eps = 0 it is 0/0). The mask is applied only in the j-tiles
// that contain one of the warp's own i-particles (a warp-uniform branch), so
// the inner loop of every other tile carries no compare.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "nb_internal.cuh"
#include "ds.cuh"
#include "tma.cuh"

namespace nb {

__device__ __forceinline__ bool finite7(const double *v)
{
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 7; ++c) ok = ok && isfinite(v[c]);
    return ok;
}

// Write the 7 totals of slot k: acc (3), jerk (3) and the positive potential
// sum P (pot = -P).
__device__ __forceinline__ void write_final(const Out3 &out, int k, double v[7], unsigned *err)
{
    v[6] = -v[6];
    if (!finite7(v)) atomicOr(err, DERR_NONFINITE);
    if (out.acc) {
        out.acc[k] = v[0];
        out.acc[out.ld + k] = v[1];
        out.acc[2 * out.ld + k] = v[2];
    }
    if (out.jerk) {
        out.jerk[k] = v[3];
        out.jerk[out.ld + k] = v[4];
        out.jerk[2 * out.ld + k] = v[5];
    }
    if (out.pot) out.pot[k] = v[6];
}

// Member index of slot k; an index outside the j-set is flagged and replaced by 0.
// Store the reduced value s of component c of slot k (c == 6: the positive
// potential sum, stored negated).
__device__ __forceinline__ void store_component(const Out3 &out, int c, int k, double s,
                                                unsigned *err)
{
    if (c == 6) {
        s = -s;
        if (out.pot) out.pot[k] = s;
    } else if (c < 3) {
        if (out.acc) out.acc[c * out.ld + k] = s;
    } else {
        if (out.jerk) out.jerk[(c - 3) * out.ld + k] = s;
    }
    if (!isfinite(s)) atomicOr(err, DERR_NONFINITE);
}

// K3, folded into the force kernels: after a CTA has written its partial sums
// for slots [slot0, slot0 + nslots), the last of the nsplit CTAs that share
// these slots (counted in *counter) reduces them and re-arms the counter. One
// warp per (slot, component): lane l adds splits l, l + 32, ... in order, then a
// fixed xor tree, so the result does not depend on which CTA finished last.
// The same with double-single partials (float2 {hi, lo} in the part buffer)
// combined in FP32 arithmetic; the final value is converted once.
template <int NT, int U = 8>
__device__ __forceinline__ void finish_split_ds(int nsplit, int slot0, int nslots, int n_i,
                                                const float2 *part, long long pld,
                                                unsigned *counter, const Out3 &out,
                                                unsigned *err)
{
    __shared__ int s_last_ds;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last_ds = (atomicAdd(counter, 1u) == (unsigned)nsplit - 1u);
    __syncthreads();
    if (!s_last_ds) return;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int valid = min(nslots, n_i - slot0);
    const int total = valid * 7;
    for (int q0 = warp * U; q0 < total; q0 += (NT / 32) * U) {
        dsf acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = dsf{0.f, 0.f};
        for (int sp = lane; sp < nsplit; sp += 32) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + u;
                if (q < total) {
                    const int c = q / valid, k = slot0 + q % valid;
                    const float2 v = __ldcg(part + ((size_t)sp * 7 + c) * pld + k);
                    ds_acc(acc[u], dsf{v.x, v.y});
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            dsf v = acc[u];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ds_acc(v, ds_shfl_xor(v, o));
            const int q = q0 + u;
            if (lane == 0 && q < total)
                store_component(out, q / valid, slot0 + q % valid, ds_to_double(v), err);
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

template <int NT>
__device__ __forceinline__ void finish_split(int nsplit, int slot0, int nslots, int n_i,
                                             const double *part, long long pld,
                                             unsigned *counter, const Out3 &out, unsigned *err)
{
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == (unsigned)nsplit - 1u);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int valid = min(nslots, n_i - slot0);
    const int total = valid * 7;
    constexpr int U = 8;  // outputs per warp pass: 8 independent loads in flight per lane
    for (int q0 = warp * U; q0 < total; q0 += (NT / 32) * U) {
        double acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = 0.0;
        for (int sp = lane; sp < nsplit; sp += 32) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + u;
                if (q < total) {
                    const int c = q / valid, k = slot0 + q % valid;
                    acc[u] += __ldcg(part + ((size_t)sp * 7 + c) * pld + k);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            double v = acc[u];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            const int q = q0 + u;
            if (lane == 0 && q < total) store_component(out, q / valid, slot0 + q % valid, v, err);
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// Record row of i-slot k: the slot itself for a gathered or external i-set,
// else the member's particle index.
__device__ __forceinline__ int member_index(const ISet &is, int k, unsigned *err);
__device__ __forceinline__ int i_row(const ISet &is, int k, unsigned *err)
{
    if (is.gathered || !is.member) return k;
    return member_index(is, k, err);
}

// Particle index of an i-record (self-pair mask): from the record for a
// gathered set, the row for members, none (-1) for an external set.
__device__ __forceinline__ int i_id(const ISet &is, int row, float id_bits)
{
    if (is.gathered) return __float_as_int(id_bits);
    return is.member ? row : -1;
}

__device__ __forceinline__ int member_index(const ISet &is, int k, unsigned *err)
{
    const int r = is.idx ? __ldg(is.idx + k) : k;
    if ((unsigned)r >= (unsigned)is.nj) {
        atomicOr(err, DERR_BADINDEX);
        return 0;
    }
    return r;
}

// ---------------------------------------------------------------------------
// FP32 / double-single tile kernel.
//
// A CTA is NWI x NWJ warps. The NWI warp columns own different i-particles
// (IPT per lane, an i-block of IB = 32 NWI IPT); the NWJ warp rows hold the
// same i-particles and share out every j-tile (row g takes j = g, g + NWJ,
// ...), so that a few hundred i-particles still fill an SM without cutting
// the j-range into many grid-level pieces. Rows are added in shared memory at
// the end, in fixed order.
// ---------------------------------------------------------------------------

template <int VAR, int IPT, int NWI, int NWJ, int JT, int NS>
__global__ void __launch_bounds__(32 * NWI * NWJ, 2)
    k_force_tile32(const float4 *__restrict__ jrec, int nj, ISet is, float eps2f, int ntiles,
                   double *__restrict__ part, long long pld, unsigned *counters, Out3 out,
                   unsigned *err)
{
    // NS ring stages of JT records (bulk-copy destinations), then the current
    // tile transposed into j-pairs (JT / 2 pairs x 6 float4)
    extern __shared__ __align__(128) float4 s_tile[];
    __shared__ __align__(8) uint64_t s_full[NS];
    __shared__ int s_abort;

    constexpr bool DS = (VAR == NB_F32DS);
    constexpr int NT = 32 * NWI * NWJ;
    constexpr int IB = 32 * NWI * IPT;
    constexpr int NPAIR = JT / 2;
    // tiles per FP32 partial sum: about 128 terms in each half of a packed sum between folds
    constexpr int FOLD = (256 * NWJ / JT) > 1 ? (256 * NWJ / JT) : 1;
    float4 *s_pair = s_tile + (size_t)NS * JT * DS_REC;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wi = warp % NWI, wj = warp / NWI;
    const int nsplit = gridDim.y;
    const int split = blockIdx.y;
    const int tile0 = (int)((long long)ntiles * split / nsplit);
    const int tile1 = (int)((long long)ntiles * (split + 1) / nsplit);
    const int my_tiles = tile1 - tile0;

    // i-particles of this thread, negated and duplicated into both halves of a
    // float2 (the packed pair arithmetic takes two j at a time)
    float2 nxh[IPT], nyh[IPT], nzh[IPT], nxl[IPT], nyl[IPT], nzl[IPT], nvx[IPT], nvy[IPT],
        nvz[IPT];
    int iid[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
        int k = blockIdx.x * IB + p * (32 * NWI) + wi * 32 + lane;
        if (k >= is.n) k = is.n - 1;  // idle slots compute a copy, never written
        const int r = i_row(is, k, err);
        const float4 a = __ldg(is.rec32 + (size_t)DS_REC * r);
        const float4 b = __ldg(is.rec32 + (size_t)DS_REC * r + 1);
        const float4 c = __ldg(is.rec32 + (size_t)DS_REC * r + 2);
        nxh[p] = make_float2(-a.x, -a.x);
        nyh[p] = make_float2(-a.y, -a.y);
        nzh[p] = make_float2(-a.z, -a.z);
        nxl[p] = make_float2(-b.x, -b.x);
        nyl[p] = make_float2(-b.y, -b.y);
        nzl[p] = make_float2(-b.z, -b.z);
        nvx[p] = make_float2(-c.x, -c.x);
        nvy[p] = make_float2(-c.y, -c.y);
        nvz[p] = make_float2(-c.z, -c.z);
        iid[p] = i_id(is, r, b.w);
    }
    const float2 e2 = make_float2(eps2f, eps2f);

    // running totals: double-single (DS) or plain FP32
    float A_h[IPT][3], A_l[IPT][3], J_h[IPT][3], J_l[IPT][3], P_h[IPT], P_l[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
#pragma unroll
        for (int c = 0; c < 3; ++c) A_h[p][c] = A_l[p][c] = J_h[p][c] = J_l[p][c] = 0.f;
        P_h[p] = P_l[p] = 0.f;
    }
    // FP32 partial sums between folds, two lanes each (even and odd j of a pair;
    // the masked scalar path adds into .x)
    float2 ta[IPT][3], tja[IPT][3], tjb[IPT][3], tp[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
#pragma unroll
        for (int c = 0; c < 3; ++c) ta[p][c] = tja[p][c] = tjb[p][c] = make_float2(0.f, 0.f);
        tp[p] = make_float2(0.f, 0.f);
    }

    if (tid == 0) {
        s_abort = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) mbar_init(&s_full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int kt) {
        const int stage = kt % NS;
        const int t = tile0 + kt;
        const int cnt = min(JT, nj - t * JT);
        const uint32_t bytes = (uint32_t)cnt * DS_REC * 16u;
        mbar_expect_tx(&s_full[stage], bytes);
        bulk_g2s(s_tile + (size_t)stage * JT * DS_REC, jrec + (size_t)t * JT * DS_REC, bytes,
                 &s_full[stage]);
    };
    if (tid == 0) {
        for (int kt = 0; kt < NS && kt < my_tiles; ++kt) issue(kt);
    }

    for (int kt = 0; kt < my_tiles; ++kt) {
        const int stage = kt % NS;
        const uint32_t parity = (uint32_t)((kt / NS) & 1);
        if (!mbar_wait(&s_full[stage], parity)) s_abort = 1;
        const float4 *T = s_tile + (size_t)stage * JT * DS_REC;
        const int jbase = (tile0 + kt) * JT;
        const int cnt = min(JT, nj - jbase);

        // self pair in this tile for any lane of the warp? (warp-uniform)
        bool own = false;
#pragma unroll
        for (int p = 0; p < IPT; ++p) own = own || (iid[p] >= jbase && iid[p] < jbase + cnt);
        own = __any_sync(0xffffffffu, own);

        // scalar pair term of record jj (the self pair masked when MASKED)
        auto body = [&](int jj, auto masked_tag) {
            constexpr bool MASKED = decltype(masked_tag)::value;
            const float4 a = T[DS_REC * jj];
            const float4 c = T[DS_REC * jj + 2];
            float4 b;
            if (DS) b = T[DS_REC * jj + 1];
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
                float dx, dy, dz;
                if (DS) {
                    dx = (a.x + nxh[p].x) + (b.x + nxl[p].x);
                    dy = (a.y + nyh[p].x) + (b.y + nyl[p].x);
                    dz = (a.z + nzh[p].x) + (b.z + nzl[p].x);
                } else {
                    dx = a.x + nxh[p].x;
                    dy = a.y + nyh[p].x;
                    dz = a.z + nzh[p].x;
                }
                const float dvx = c.x + nvx[p].x, dvy = c.y + nvy[p].x, dvz = c.z + nvz[p].x;
                float r2 = fmaf(dx, dx, eps2f);
                r2 = fmaf(dy, dy, r2);
                r2 = fmaf(dz, dz, r2);
                float rv = dx * dvx;
                rv = fmaf(dy, dvy, rv);
                rv = fmaf(dz, dvz, rv);
                float rinv = rsqrtf(r2);
                if (MASKED) rinv = (jbase + jj == iid[p]) ? 0.f : rinv;
                const float rinv2 = rinv * rinv;
                const float mrinv = a.w * rinv;
                const float mr3 = mrinv * rinv2;
                const float beta = (mr3 * rinv2) * rv;
                tp[p].x += mrinv;
                ta[p][0].x = fmaf(mr3, dx, ta[p][0].x);
                ta[p][1].x = fmaf(mr3, dy, ta[p][1].x);
                ta[p][2].x = fmaf(mr3, dz, ta[p][2].x);
                tja[p][0].x = fmaf(mr3, dvx, tja[p][0].x);
                tja[p][1].x = fmaf(mr3, dvy, tja[p][1].x);
                tja[p][2].x = fmaf(mr3, dvz, tja[p][2].x);
                tjb[p][0].x = fmaf(beta, dx, tjb[p][0].x);
                tjb[p][1].x = fmaf(beta, dy, tjb[p][1].x);
                tjb[p][2].x = fmaf(beta, dz, tjb[p][2].x);
            }
        };
        if (cnt == JT) {
            // full tile: transpose it into j-pairs, {x_hi} {y_hi} {z_hi} {m} {x_lo}
            // {y_lo} {z_lo} {index} {vx} {vy} {vz} of j = 2q, 2q + 1 side by side
            for (int x = tid; x < 3 * NPAIR; x += NT) {
                const int q = x % NPAIR, part = x / NPAIR;
                const float4 u = T[DS_REC * (2 * q) + part];
                const float4 v = T[DS_REC * (2 * q + 1) + part];
                float4 *P = s_pair + 6 * q + 2 * part;
                P[0] = make_float4(u.x, v.x, u.y, v.y);
                P[1] = make_float4(u.z, v.z, u.w, v.w);
            }
            __syncthreads();
            if (own) {
                for (int jj = wj; jj < JT; jj += NWJ) body(jj, std::true_type{});
            } else {
#pragma unroll 2
                for (int q = wj; q < NPAIR; q += NWJ) {
                    const float4 *P = s_pair + 6 * q;
                    const float4 q0 = P[0], q1 = P[1], q4 = P[4], q5 = P[5];
                    float4 q2, q3;
                    if (DS) {
                        q2 = P[2];
                        q3 = P[3];
                    }
                    const float2 XH = make_float2(q0.x, q0.y), YH = make_float2(q0.z, q0.w);
                    const float2 ZH = make_float2(q1.x, q1.y), MJ = make_float2(q1.z, q1.w);
                    const float2 VX = make_float2(q4.x, q4.y), VY = make_float2(q4.z, q4.w);
                    const float2 VZ = make_float2(q5.x, q5.y);
#pragma unroll
                    for (int p = 0; p < IPT; ++p) {
                        float2 dx, dy, dz;
                        if (DS) {
                            dx = __fadd2_rn(__fadd2_rn(XH, nxh[p]),
                                            __fadd2_rn(make_float2(q2.x, q2.y), nxl[p]));
                            dy = __fadd2_rn(__fadd2_rn(YH, nyh[p]),
                                            __fadd2_rn(make_float2(q2.z, q2.w), nyl[p]));
                            dz = __fadd2_rn(__fadd2_rn(ZH, nzh[p]),
                                            __fadd2_rn(make_float2(q3.x, q3.y), nzl[p]));
                        } else {
                            dx = __fadd2_rn(XH, nxh[p]);
                            dy = __fadd2_rn(YH, nyh[p]);
                            dz = __fadd2_rn(ZH, nzh[p]);
                        }
                        const float2 dvx = __fadd2_rn(VX, nvx[p]);
                        const float2 dvy = __fadd2_rn(VY, nvy[p]);
                        const float2 dvz = __fadd2_rn(VZ, nvz[p]);
                        float2 r2 = __ffma2_rn(dx, dx, e2);
                        r2 = __ffma2_rn(dy, dy, r2);
                        r2 = __ffma2_rn(dz, dz, r2);
                        float2 rv = __fmul2_rn(dx, dvx);
                        rv = __ffma2_rn(dy, dvy, rv);
                        rv = __ffma2_rn(dz, dvz, rv);
                        const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                        const float2 rinv2 = __fmul2_rn(rinv, rinv);
                        const float2 mrinv = __fmul2_rn(MJ, rinv);
                        const float2 mr3 = __fmul2_rn(mrinv, rinv2);
                        const float2 beta = __fmul2_rn(__fmul2_rn(mr3, rinv2), rv);
                        tp[p] = __fadd2_rn(tp[p], mrinv);
                        ta[p][0] = __ffma2_rn(mr3, dx, ta[p][0]);
                        ta[p][1] = __ffma2_rn(mr3, dy, ta[p][1]);
                        ta[p][2] = __ffma2_rn(mr3, dz, ta[p][2]);
                        tja[p][0] = __ffma2_rn(mr3, dvx, tja[p][0]);
                        tja[p][1] = __ffma2_rn(mr3, dvy, tja[p][1]);
                        tja[p][2] = __ffma2_rn(mr3, dvz, tja[p][2]);
                        tjb[p][0] = __ffma2_rn(beta, dx, tjb[p][0]);
                        tjb[p][1] = __ffma2_rn(beta, dy, tjb[p][1]);
                        tjb[p][2] = __ffma2_rn(beta, dz, tjb[p][2]);
                    }
                }
            }
        } else if (own) {
            for (int jj = wj; jj < cnt; jj += NWJ) body(jj, std::true_type{});
        } else {
#pragma unroll 2
            for (int jj = wj; jj < cnt; jj += NWJ) body(jj, std::false_type{});
        }

        // fold the FP32 partial sums (both lanes) into the running totals
        if ((kt + 1) % FOLD == 0 || kt + 1 == my_tiles) {
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float sa = ta[p][c].x + ta[p][c].y;
                    const float jt = fmaf(-3.f, tjb[p][c].x + tjb[p][c].y,
                                          tja[p][c].x + tja[p][c].y);
                    if (DS) {
                        ds_add(A_h[p][c], A_l[p][c], sa);
                        ds_add(J_h[p][c], J_l[p][c], jt);
                    } else {
                        A_h[p][c] += sa;
                        J_h[p][c] += jt;
                    }
                }
                const float sp = tp[p].x + tp[p].y;
                if (DS)
                    ds_add(P_h[p], P_l[p], sp);
                else
                    P_h[p] += sp;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    ta[p][c] = tja[p][c] = tjb[p][c] = make_float2(0.f, 0.f);
                tp[p] = make_float2(0.f, 0.f);
            }
        }

        __syncthreads();  // every warp is done with this stage and the j-pairs
        if (s_abort) {
            if (tid == 0) drain_ring<NS>(s_full, 0u, kt, my_tiles);
            break;
        }
        if (tid == 0 && kt + NS < my_tiles) issue(kt + NS);
    }
    if (s_abort) {
        if (tid == 0) atomicOr(err, DERR_TIMEOUT);
        return;
    }

    dsf v[IPT][7];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[p][c] = dsf{A_h[p][c], A_l[p][c]};
            v[p][3 + c] = dsf{J_h[p][c], J_l[p][c]};
        }
        v[p][6] = dsf{P_h[p], P_l[p]};
    }
    if (NWJ > 1) {
        // add the warp rows in order 0..NWJ-1 (the tile ring is free: all tiles consumed)
        float2 *s_red = reinterpret_cast<float2 *>(s_tile);  // [NWJ][7][IB]
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
            const int slot = p * (32 * NWI) + wi * 32 + lane;
#pragma unroll
            for (int c = 0; c < 7; ++c)
                s_red[(wj * 7 + c) * IB + slot] = make_float2(v[p][c].hi, v[p][c].lo);
        }
        __syncthreads();
        if (wj == 0) {
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
                const int slot = p * (32 * NWI) + wi * 32 + lane;
#pragma unroll
                for (int c = 0; c < 7; ++c)
                    for (int g = 1; g < NWJ; ++g) {
                        const float2 w = s_red[(g * 7 + c) * IB + slot];
                        ds_acc(v[p][c], dsf{w.x, w.y});
                    }
            }
        }
    }
    if (wj == 0) {
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
            const int k = blockIdx.x * IB + p * (32 * NWI) + wi * 32 + lane;
            if (k >= is.n) continue;
            if (nsplit == 1) {
                double d[7];
#pragma unroll
                for (int c = 0; c < 7; ++c) d[c] = ds_to_double(v[p][c]);
                write_final(out, k, d, err);
            } else {
                float2 *pp = reinterpret_cast<float2 *>(part);
#pragma unroll
                for (int c = 0; c < 7; ++c)
                    pp[((size_t)split * 7 + c) * pld + k] = make_float2(v[p][c].hi, v[p][c].lo);
            }
        }
    }
    // with nsplit > 1 the partials are summed by k_tile_split_reduce, launched next
    (void)counters;
}

// K3 of the tile kernel: one thread per output (component c of slot k) adds the
// nsplit double-single partials in the order s = 0, 1, ... (the partials of
// consecutive slots are adjacent, so the loads of a warp are coalesced), eight
// loads in flight at a time.
__global__ void __launch_bounds__(256)
    k_tile_split_reduce(const float2 *__restrict__ part, long long pld, int nsplit, int n_i,
                        Out3 out, unsigned *err)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 7LL * n_i) return;
    const int c = (int)(q / n_i), k = (int)(q % n_i);
    const float2 *p = part + (size_t)c * pld + k;
    const size_t stride = (size_t)7 * pld;
    dsf sum{0.f, 0.f};
    int sp = 0;
    for (; sp + 8 <= nsplit; sp += 8) {
        float2 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = __ldcg(p + (size_t)(sp + u) * stride);
#pragma unroll
        for (int u = 0; u < 8; ++u) ds_acc(sum, dsf{x[u].x, x[u].y});
    }
    for (; sp < nsplit; ++sp) {
        const float2 x = __ldcg(p + (size_t)sp * stride);
        ds_acc(sum, dsf{x.x, x.y});
    }
    store_component(out, c, k, ds_to_double(sum), err);
}


// ---------------------------------------------------------------------------
// FP64 tile kernel.
// ---------------------------------------------------------------------------

template <int IPT, int NT, int JT, int NS>
__global__ void __launch_bounds__(NT)
    k_force_tile64(JSet js, ISet is, double eps2, int ntiles, double *__restrict__ part,
                   long long pld, unsigned *counters, Out3 out, unsigned *err)
{
    extern __shared__ __align__(128) double s_t64[];  // NS * 7 * JT
    __shared__ __align__(8) uint64_t s_full[NS];
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int nsplit = gridDim.y;
    const int split = blockIdx.y;
    const int tile0 = (int)((long long)ntiles * split / nsplit);
    const int tile1 = (int)((long long)ntiles * (split + 1) / nsplit);
    const int my_tiles = tile1 - tile0;
    const int nj = js.n;

    double xi[IPT][3], vi[IPT][3], mi[IPT];
    int iid[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
        int k = blockIdx.x * (NT * IPT) + p * NT + tid;
        if (k >= is.n) k = is.n - 1;
        const int r = is.member ? member_index(is, k, err) : k;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xi[p][c] = __ldg(is.pos64 + c * is.ld64 + r);
            vi[p][c] = __ldg(is.vel64 + c * is.ld64 + r);
        }
        mi[p] = is.member ? __ldg(is.m64 + r) : 0.0;
        iid[p] = is.member ? r : -1;
    }

    double A[IPT][3], J[IPT][3], P[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
#pragma unroll
        for (int c = 0; c < 3; ++c) A[p][c] = J[p][c] = 0.0;
        P[p] = 0.0;
    }

    if (tid == 0) {
        s_abort = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) mbar_init(&s_full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // 7 rows per stage: x, y, z, vx, vy, vz, m
    auto issue = [&](int kt) {
        const int stage = kt % NS;
        const int t = tile0 + kt;
        const int cnt = min(JT, nj - t * JT);
        const uint32_t bytes = (uint32_t)(((cnt * 8) + 15) & ~15);  // rows are padded
        mbar_expect_tx(&s_full[stage], 7u * bytes);
        double *dst = s_t64 + (size_t)stage * 7 * JT;
        const size_t off = (size_t)t * JT;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            bulk_g2s(dst + c * JT, js.pos64 + c * js.ld + off, bytes, &s_full[stage]);
            bulk_g2s(dst + (3 + c) * JT, js.vel64 + c * js.ld + off, bytes, &s_full[stage]);
        }
        bulk_g2s(dst + 6 * JT, js.m64 + off, bytes, &s_full[stage]);
    };
    if (tid == 0) {
        for (int kt = 0; kt < NS && kt < my_tiles; ++kt) issue(kt);
    }

    for (int kt = 0; kt < my_tiles; ++kt) {
        const int stage = kt % NS;
        const uint32_t parity = (uint32_t)((kt / NS) & 1);
        if (!mbar_wait(&s_full[stage], parity)) s_abort = 1;
        const double *T = s_t64 + (size_t)stage * 7 * JT;
        const int jbase = (tile0 + kt) * JT;
        const int cnt = min(JT, nj - jbase);
        double ta[IPT][3], tja[IPT][3], tjb[IPT][3], tp[IPT];
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
#pragma unroll
            for (int c = 0; c < 3; ++c) ta[p][c] = tja[p][c] = tjb[p][c] = 0.0;
            tp[p] = 0.0;
        }
        bool own = false;
#pragma unroll
        for (int p = 0; p < IPT; ++p) own = own || (iid[p] >= jbase && iid[p] < jbase + cnt);
        own = __any_sync(0xffffffffu, own);
#pragma unroll 2
        for (int jj = 0; jj < cnt; ++jj) {
            const double xj = T[jj], yj = T[JT + jj], zj = T[2 * JT + jj];
            const double uj = T[3 * JT + jj], wj = T[4 * JT + jj], qj = T[5 * JT + jj];
            const double mj = T[6 * JT + jj];
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
                const double dx = xj - xi[p][0], dy = yj - xi[p][1], dz = zj - xi[p][2];
                const double dvx = uj - vi[p][0], dvy = wj - vi[p][1], dvz = qj - vi[p][2];
                double r2 = fma(dx, dx, eps2);
                r2 = fma(dy, dy, r2);
                r2 = fma(dz, dz, r2);
                double rv = dx * dvx;
                rv = fma(dy, dvy, rv);
                rv = fma(dz, dvz, rv);
                double rinv = rsqrt(r2);
                if (own) rinv = (jbase + jj == iid[p]) ? 0.0 : rinv;
                const double rinv2 = rinv * rinv;
                const double mrinv = mj * rinv;
                const double mr3 = mrinv * rinv2;
                const double beta = (mr3 * rinv2) * rv;
                tp[p] += mrinv;
                ta[p][0] = fma(mr3, dx, ta[p][0]);
                ta[p][1] = fma(mr3, dy, ta[p][1]);
                ta[p][2] = fma(mr3, dz, ta[p][2]);
                tja[p][0] = fma(mr3, dvx, tja[p][0]);
                tja[p][1] = fma(mr3, dvy, tja[p][1]);
                tja[p][2] = fma(mr3, dvz, tja[p][2]);
                tjb[p][0] = fma(beta, dx, tjb[p][0]);
                tjb[p][1] = fma(beta, dy, tjb[p][1]);
                tjb[p][2] = fma(beta, dz, tjb[p][2]);
            }
        }
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                A[p][c] += ta[p][c];
                J[p][c] += fma(-3.0, tjb[p][c], tja[p][c]);
            }
            P[p] += tp[p];
        }
        __syncthreads();
        if (s_abort) {
            if (tid == 0) drain_ring<NS>(s_full, 0u, kt, my_tiles);
            break;
        }
        if (tid == 0 && kt + NS < my_tiles) issue(kt + NS);
    }
    if (s_abort) {
        if (tid == 0) atomicOr(err, DERR_TIMEOUT);
        return;
    }

#pragma unroll
    for (int p = 0; p < IPT; ++p) {
        const int k = blockIdx.x * (NT * IPT) + p * NT + tid;
        if (k >= is.n) continue;
        double v[7] = {A[p][0], A[p][1], A[p][2], J[p][0], J[p][1], J[p][2], P[p]};
        if (nsplit == 1) {
            write_final(out, k, v, err);
        } else {
#pragma unroll
            for (int c = 0; c < 7; ++c) part[((size_t)split * 7 + c) * pld + k] = v[c];
        }
    }
    if (nsplit > 1)
        finish_split<NT>(nsplit, blockIdx.x * (NT * IPT), NT * IPT, is.n, part, pld,
                         counters + blockIdx.x, out, err);
}

// ---------------------------------------------------------------------------
// j-parallel kernels for small i-sets (lanes over j).
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP32 / double-single warp-group kernel for small and mid-size i-sets: each
// warp owns its own IPT i-particles (every lane holds the same ones) and its
// lanes stride over the CTA's j-range, reading the j-records straight from
// L1/L2 (the warps of a CTA share one j-range, so it is read from L2 once per
// CTA). A warp needs no block barrier: its lanes' sums meet in one xor tree.
// Grid: i-groups of NWARP warps (x) times j-splits (y); the splits are reduced
// by the last CTA of each group (finish_split).
template <int VAR, int IPT, int NWARP>
__global__ void __launch_bounds__(32 * NWARP)
    k_force_wgrp32(const float4 *__restrict__ jrec, int nj, ISet is, float eps2f,
                   double *__restrict__ part, long long pld, unsigned *counters, Out3 out,
                   unsigned *err)
{
    constexpr bool DS = (VAR == NB_F32DS);
    constexpr int NT = 32 * NWARP;
    constexpr int CHUNK = 32 * 32;  // j per FP32 partial sum (32 per lane)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nsplit = gridDim.y, split = blockIdx.y;
    const int j0 = (int)((long long)nj * split / nsplit);
    const int j1 = (int)((long long)nj * (split + 1) / nsplit);
    const int slot0 = (blockIdx.x * NWARP + warp) * IPT;

    float xh[IPT], yh[IPT], zh[IPT], xl[IPT], yl[IPT], zl[IPT], vx[IPT], vy[IPT], vz[IPT];
    int iid[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
        const int k = min(slot0 + p, is.n - 1);
        const int r = i_row(is, k, err);
        const float4 a = __ldg(is.rec32 + (size_t)DS_REC * r);
        const float4 b = __ldg(is.rec32 + (size_t)DS_REC * r + 1);
        const float4 c = __ldg(is.rec32 + (size_t)DS_REC * r + 2);
        xh[p] = a.x; yh[p] = a.y; zh[p] = a.z;
        xl[p] = b.x; yl[p] = b.y; zl[p] = b.z;
        vx[p] = c.x; vy[p] = c.y; vz[p] = c.z;
        iid[p] = i_id(is, r, b.w);
    }
    float A_h[IPT][3], A_l[IPT][3], J_h[IPT][3], J_l[IPT][3], P_h[IPT], P_l[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
#pragma unroll
        for (int c = 0; c < 3; ++c) A_h[p][c] = A_l[p][c] = J_h[p][c] = J_l[p][c] = 0.f;
        P_h[p] = P_l[p] = 0.f;
    }

    for (int c0 = j0; c0 < j1; c0 += CHUNK) {
        const int c1 = min(c0 + CHUNK, j1);
        float ta[IPT][3], tja[IPT][3], tjb[IPT][3], tp[IPT];
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
#pragma unroll
            for (int c = 0; c < 3; ++c) ta[p][c] = tja[p][c] = tjb[p][c] = 0.f;
            tp[p] = 0.f;
        }
#pragma unroll 4
        for (int j = c0 + lane; j < c1; j += 32) {
            const float4 a = __ldg(jrec + (size_t)DS_REC * j);
            const float4 c = __ldg(jrec + (size_t)DS_REC * j + 2);
            float4 b;
            if (DS) b = __ldg(jrec + (size_t)DS_REC * j + 1);
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
                float dx, dy, dz;
                if (DS) {
                    dx = (a.x - xh[p]) + (b.x - xl[p]);
                    dy = (a.y - yh[p]) + (b.y - yl[p]);
                    dz = (a.z - zh[p]) + (b.z - zl[p]);
                } else {
                    dx = a.x - xh[p];
                    dy = a.y - yh[p];
                    dz = a.z - zh[p];
                }
                const float dvx = c.x - vx[p], dvy = c.y - vy[p], dvz = c.z - vz[p];
                float r2 = fmaf(dx, dx, eps2f);
                r2 = fmaf(dy, dy, r2);
                r2 = fmaf(dz, dz, r2);
                float rv = dx * dvx;
                rv = fmaf(dy, dvy, rv);
                rv = fmaf(dz, dvz, rv);
                float rinv = rsqrtf(r2);
                rinv = (j == iid[p]) ? 0.f : rinv;
                const float rinv2 = rinv * rinv;
                const float mrinv = a.w * rinv;
                const float mr3 = mrinv * rinv2;
                const float beta = (mr3 * rinv2) * rv;
                tp[p] += mrinv;
                ta[p][0] = fmaf(mr3, dx, ta[p][0]);
                ta[p][1] = fmaf(mr3, dy, ta[p][1]);
                ta[p][2] = fmaf(mr3, dz, ta[p][2]);
                tja[p][0] = fmaf(mr3, dvx, tja[p][0]);
                tja[p][1] = fmaf(mr3, dvy, tja[p][1]);
                tja[p][2] = fmaf(mr3, dvz, tja[p][2]);
                tjb[p][0] = fmaf(beta, dx, tjb[p][0]);
                tjb[p][1] = fmaf(beta, dy, tjb[p][1]);
                tjb[p][2] = fmaf(beta, dz, tjb[p][2]);
            }
        }
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float jt = fmaf(-3.f, tjb[p][c], tja[p][c]);
                if (DS) {
                    ds_add(A_h[p][c], A_l[p][c], ta[p][c]);
                    ds_add(J_h[p][c], J_l[p][c], jt);
                } else {
                    A_h[p][c] += ta[p][c];
                    J_h[p][c] += jt;
                }
            }
            if (DS)
                ds_add(P_h[p], P_l[p], tp[p]);
            else
                P_h[p] += tp[p];
        }
    }

    // lanes -> warp total (double-single xor tree); lane 0 stores
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
        dsf v[7];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c] = dsf{A_h[p][c], A_l[p][c]};
            v[3 + c] = dsf{J_h[p][c], J_l[p][c]};
        }
        v[6] = dsf{P_h[p], P_l[p]};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 7; ++c) ds_acc(v[c], ds_shfl_xor(v[c], o));
        const int k = slot0 + p;
        if (lane == 0 && k < is.n) {
            if (nsplit == 1) {
                double d[7];
#pragma unroll
                for (int c = 0; c < 7; ++c) d[c] = ds_to_double(v[c]);
                write_final(out, k, d, err);
            } else {
                float2 *pp = reinterpret_cast<float2 *>(part);
#pragma unroll
                for (int c = 0; c < 7; ++c)
                    pp[((size_t)split * 7 + c) * pld + k] = make_float2(v[c].hi, v[c].lo);
            }
        }
    }
    if (nsplit > 1)
        finish_split_ds<NT>(nsplit, blockIdx.x * NWARP * IPT, NWARP * IPT, is.n,
                            reinterpret_cast<float2 *>(part), pld, counters + blockIdx.x, out,
                            err);
}


// FP32 / double-single kernel for tiny i-sets (block-step tails): every thread
// holds the same IPT i-particles and JPT j-records of its own, all loaded
// before any arithmetic so the whole j-set costs one L2 round trip; sums go
// through a double-single warp tree, then across the CTA's warps, one
// partial per CTA.
// Groups of IPT (<= 4) i-particles are processed in turn (the j-records stay
// in registers).
template <int VAR, int IPT, int JPT>
__global__ void __launch_bounds__(256)
    k_force_tiny32(const float4 *__restrict__ jrec, int nj, ISet is, float eps2f,
                   double *__restrict__ part, long long pld, unsigned *counters, Out3 out,
                   unsigned *err)
{
    constexpr bool DS = (VAR == NB_F32DS);
    constexpr int NT = 256, NW = NT / 32;
    __shared__ float2 s_red[NW][IPT * 7];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nsplit = gridDim.x, split = blockIdx.x;

    // this thread's j-records: j = split * NT * JPT + r * NT + tid
    float4 ja[JPT], jb[JPT], jc[JPT];
    int jidx[JPT];
#pragma unroll
    for (int r = 0; r < JPT; ++r) {
        const int j = split * NT * JPT + r * NT + tid;
        jidx[r] = j;
        if (j < nj) {
            ja[r] = __ldg(jrec + (size_t)DS_REC * j);
            jc[r] = __ldg(jrec + (size_t)DS_REC * j + 2);
            if (DS) jb[r] = __ldg(jrec + (size_t)DS_REC * j + 1);
        } else {
            ja[r] = make_float4(0.f, 0.f, 0.f, 0.f);  // massless: contributes nothing
            jc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            jb[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            jidx[r] = -2;
        }
    }

    for (int g0 = 0; g0 < is.n; g0 += IPT) {
        float xh[IPT], yh[IPT], zh[IPT], xl[IPT], yl[IPT], zl[IPT], vx[IPT], vy[IPT], vz[IPT];
        int iid[IPT];
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
            const int k = min(g0 + p, is.n - 1);
            const int r = i_row(is, k, err);
            const float4 a = __ldg(is.rec32 + (size_t)DS_REC * r);
            const float4 b = __ldg(is.rec32 + (size_t)DS_REC * r + 1);
            const float4 c = __ldg(is.rec32 + (size_t)DS_REC * r + 2);
            xh[p] = a.x; yh[p] = a.y; zh[p] = a.z;
            xl[p] = b.x; yl[p] = b.y; zl[p] = b.z;
            vx[p] = c.x; vy[p] = c.y; vz[p] = c.z;
            iid[p] = i_id(is, r, b.w);
        }
        dsf v[IPT][7];
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
            float ta0 = 0.f, ta1 = 0.f, ta2 = 0.f, tj0 = 0.f, tj1 = 0.f, tj2 = 0.f;
            float tb0 = 0.f, tb1 = 0.f, tb2 = 0.f, tp = 0.f;
#pragma unroll
            for (int r = 0; r < JPT; ++r) {
                float dx, dy, dz;
                if (DS) {
                    dx = (ja[r].x - xh[p]) + (jb[r].x - xl[p]);
                    dy = (ja[r].y - yh[p]) + (jb[r].y - yl[p]);
                    dz = (ja[r].z - zh[p]) + (jb[r].z - zl[p]);
                } else {
                    dx = ja[r].x - xh[p];
                    dy = ja[r].y - yh[p];
                    dz = ja[r].z - zh[p];
                }
                const float dvx = jc[r].x - vx[p], dvy = jc[r].y - vy[p], dvz = jc[r].z - vz[p];
                float r2 = fmaf(dx, dx, eps2f);
                r2 = fmaf(dy, dy, r2);
                r2 = fmaf(dz, dz, r2);
                float rv = dx * dvx;
                rv = fmaf(dy, dvy, rv);
                rv = fmaf(dz, dvz, rv);
                float rinv = rsqrtf(r2);
                // self pair and padding records (jidx -2) contribute nothing
                rinv = (jidx[r] == iid[p] || jidx[r] < 0) ? 0.f : rinv;
                const float rinv2 = rinv * rinv;
                const float mrinv = ja[r].w * rinv;
                const float mr3 = mrinv * rinv2;
                const float beta = (mr3 * rinv2) * rv;
                tp += mrinv;
                ta0 = fmaf(mr3, dx, ta0);
                ta1 = fmaf(mr3, dy, ta1);
                ta2 = fmaf(mr3, dz, ta2);
                tj0 = fmaf(mr3, dvx, tj0);
                tj1 = fmaf(mr3, dvy, tj1);
                tj2 = fmaf(mr3, dvz, tj2);
                tb0 = fmaf(beta, dx, tb0);
                tb1 = fmaf(beta, dy, tb1);
                tb2 = fmaf(beta, dz, tb2);
            }
            v[p][0] = dsf{ta0, 0.f};
            v[p][1] = dsf{ta1, 0.f};
            v[p][2] = dsf{ta2, 0.f};
            v[p][3] = dsf{fmaf(-3.f, tb0, tj0), 0.f};
            v[p][4] = dsf{fmaf(-3.f, tb1, tj1), 0.f};
            v[p][5] = dsf{fmaf(-3.f, tb2, tj2), 0.f};
            v[p][6] = dsf{tp, 0.f};
        }
        // double-single xor tree across the lanes, all chains interleaved
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int p = 0; p < IPT; ++p)
#pragma unroll
                for (int c = 0; c < 7; ++c) ds_acc(v[p][c], ds_shfl_xor(v[p][c], o));
        }
        if (lane == 0) {
#pragma unroll
            for (int p = 0; p < IPT; ++p)
#pragma unroll
                for (int c = 0; c < 7; ++c)
                    s_red[warp][p * 7 + c] = make_float2(v[p][c].hi, v[p][c].lo);
        }
        __syncthreads();
        if (tid < IPT * 7) {
            const int p = tid / 7, c = tid % 7;
            const int k = g0 + p;
            dsf sum{0.f, 0.f};
#pragma unroll
            for (int w = 0; w < NW; ++w) ds_acc(sum, dsf{s_red[w][tid].x, s_red[w][tid].y});
            if (k < is.n) {
                if (nsplit == 1)
                    store_component(out, c, k, ds_to_double(sum), err);
                else
                    reinterpret_cast<float2 *>(part)[((size_t)split * 7 + c) * pld + k] =
                        make_float2(sum.hi, sum.lo);
            }
        }
        __syncthreads();
    }
    if (nsplit > 1)
        finish_split_ds<NT>(nsplit, 0, is.n, is.n, reinterpret_cast<float2 *>(part), pld, counters,
                            out, err);
}

// FP64 j-parallel kernel: thread = j, all threads share IPT i's.
template <int IPT, int NT>
__global__ void __launch_bounds__(NT)
    k_force_jmode64(JSet js, ISet is, double eps2, double *__restrict__ part, long long pld,
                    unsigned *counters, Out3 out, unsigned *err)
{
    constexpr int NW = NT / 32;
    __shared__ double s_red[NW][IPT][7];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nsplit = gridDim.x, split = blockIdx.x;
    const int nj = js.n;
    const int j0 = (int)((long long)nj * split / nsplit);
    const int j1 = (int)((long long)nj * (split + 1) / nsplit);

    for (int g0 = 0; g0 < is.n; g0 += IPT) {
        double xi[IPT][3], vi[IPT][3], mi[IPT];
        int iid[IPT];
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
            const int k = min(g0 + p, is.n - 1);
            const int r = is.member ? member_index(is, k, err) : k;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xi[p][c] = __ldg(is.pos64 + c * is.ld64 + r);
                vi[p][c] = __ldg(is.vel64 + c * is.ld64 + r);
            }
            mi[p] = is.member ? __ldg(is.m64 + r) : 0.0;
            iid[p] = is.member ? r : -1;
        }
        double ta[IPT][3], tja[IPT][3], tjb[IPT][3], tp[IPT];
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
#pragma unroll
            for (int c = 0; c < 3; ++c) ta[p][c] = tja[p][c] = tjb[p][c] = 0.0;
            tp[p] = 0.0;
        }
        for (int j = j0 + tid; j < j1; j += NT) {
            const double xj = __ldg(js.pos64 + j), yj = __ldg(js.pos64 + js.ld + j),
                         zj = __ldg(js.pos64 + 2 * js.ld + j);
            const double uj = __ldg(js.vel64 + j), wj = __ldg(js.vel64 + js.ld + j),
                         qj = __ldg(js.vel64 + 2 * js.ld + j);
            const double mj = __ldg(js.m64 + j);
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
                const double dx = xj - xi[p][0], dy = yj - xi[p][1], dz = zj - xi[p][2];
                const double dvx = uj - vi[p][0], dvy = wj - vi[p][1], dvz = qj - vi[p][2];
                double r2 = fma(dx, dx, eps2);
                r2 = fma(dy, dy, r2);
                r2 = fma(dz, dz, r2);
                double rv = dx * dvx;
                rv = fma(dy, dvy, rv);
                rv = fma(dz, dvz, rv);
                double rinv = rsqrt(r2);
                rinv = (j == iid[p]) ? 0.0 : rinv;
                const double rinv2 = rinv * rinv;
                const double mrinv = mj * rinv;
                const double mr3 = mrinv * rinv2;
                const double beta = (mr3 * rinv2) * rv;
                tp[p] += mrinv;
                ta[p][0] = fma(mr3, dx, ta[p][0]);
                ta[p][1] = fma(mr3, dy, ta[p][1]);
                ta[p][2] = fma(mr3, dz, ta[p][2]);
                tja[p][0] = fma(mr3, dvx, tja[p][0]);
                tja[p][1] = fma(mr3, dvy, tja[p][1]);
                tja[p][2] = fma(mr3, dvz, tja[p][2]);
                tjb[p][0] = fma(beta, dx, tjb[p][0]);
                tjb[p][1] = fma(beta, dy, tjb[p][1]);
                tjb[p][2] = fma(beta, dz, tjb[p][2]);
            }
        }
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
            double v[7];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[c] = ta[p][c];
                v[3 + c] = fma(-3.0, tjb[p][c], tja[p][c]);
            }
            v[6] = tp[p];
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                const double w = warp_sum(v[c]);
                if (lane == 0) s_red[warp][p][c] = w;
            }
        }
        __syncthreads();
        if (tid < IPT * 7) {
            const int p = tid / 7, c = tid % 7;
            const int k = g0 + p;
            if (k < is.n) {
                double s = 0.0;
#pragma unroll
                for (int w = 0; w < NW; ++w) s += s_red[w][p][c];
                if (nsplit == 1) {
                    if (c == 6) {
                        s = -s;
                        if (out.pot) out.pot[k] = s;
                    } else if (c < 3) {
                        if (out.acc) out.acc[c * out.ld + k] = s;
                    } else {
                        if (out.jerk) out.jerk[(c - 3) * out.ld + k] = s;
                    }
                    if (!isfinite(s)) atomicOr(err, DERR_NONFINITE);
                } else {
                    part[((size_t)split * 7 + c) * pld + k] = s;
                }
            }
        }
        __syncthreads();
    }
    if (nsplit > 1) finish_split<NT>(nsplit, 0, is.n, is.n, part, pld, counters, out, err);
}

// ---------------------------------------------------------------------------
// Batched force kernel: many independent systems in one launch (the batched
// clusters, and the requests of the serving loop). A work item is a block of
// i-rows of one system against a range of the same system's j-records, with
// its own pointers (WorkItem). The persistent CTAs walk the item list (sorted
// by decreasing work on the host, so the round-robin assignment is balanced).
// i-parallel items stage the j-tiles through the same bulk-copy ring as the
// tile kernel (the mbarrier phases run on across items); j-parallel items read
// the j-records straight from L1/L2. Items of a j-split group leave
// double-single partials that the group's last item sums in split order.
// ---------------------------------------------------------------------------

// One j-parallel item (kind 1): every thread takes j = j0 + tid, j0 + tid + NT,
// ... against the same four i-rows at a time. FP32 sums over at most JPAR_RUN
// j per thread meet in a fixed xor tree per warp (double-single) and a
// fixed-order sum over the warps, added to double-single totals in shared
// memory; the totals are the item's outputs, or its partials when its j-range
// is one split of a group.
constexpr int JPAR_RUN = 32;

template <bool DS, int NT>
__device__ __forceinline__ void item_jpar(const WorkItem &w, float2 (*s_red)[28], float2 *s_tot)
{
    constexpr int G = 4;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float eps2f = w.eps2;
    const int jend = w.j0 + w.nj;
    for (int g0 = 0; g0 < w.ni; g0 += G) {
        float xh[G], yh[G], zh[G], xl[G], yl[G], zl[G], vx[G], vy[G], vz[G];
        int iid[G];
#pragma unroll
        for (int p = 0; p < G; ++p) {
            const int r = w.i0 + min(g0 + p, w.ni - 1);  // idle slots copy the last i
            const float4 a = __ldg(w.irec + (size_t)DS_REC * r);
            const float4 b = __ldg(w.irec + (size_t)DS_REC * r + 1);
            const float4 c = __ldg(w.irec + (size_t)DS_REC * r + 2);
            xh[p] = a.x; yh[p] = a.y; zh[p] = a.z;
            xl[p] = b.x; yl[p] = b.y; zl[p] = b.z;
            vx[p] = c.x; vy[p] = c.y; vz[p] = c.z;
            iid[p] = w.gathered ? __float_as_int(b.w) : r;
        }
        if (tid < G * 7) s_tot[tid] = make_float2(0.f, 0.f);
        for (int jb = w.j0; jb < jend; jb += NT * JPAR_RUN) {
            float ta[G][3], tjv[G][3], tp[G];
#pragma unroll
            for (int p = 0; p < G; ++p) {
#pragma unroll
                for (int c = 0; c < 3; ++c) ta[p][c] = tjv[p][c] = 0.f;
                tp[p] = 0.f;
            }
            const int jstop = min(jend, jb + NT * JPAR_RUN);
#pragma unroll 2
            for (int j = jb + tid; j < jstop; j += NT) {
                const float4 a = __ldg(w.jrec + (size_t)DS_REC * j);
                const float4 c = __ldg(w.jrec + (size_t)DS_REC * j + 2);
                float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
                if (DS) b = __ldg(w.jrec + (size_t)DS_REC * j + 1);
#pragma unroll
                for (int p = 0; p < G; ++p) {
                    float dx, dy, dz;
                    if (DS) {
                        dx = (a.x - xh[p]) + (b.x - xl[p]);
                        dy = (a.y - yh[p]) + (b.y - yl[p]);
                        dz = (a.z - zh[p]) + (b.z - zl[p]);
                    } else {
                        dx = a.x - xh[p];
                        dy = a.y - yh[p];
                        dz = a.z - zh[p];
                    }
                    const float dvx = c.x - vx[p], dvy = c.y - vy[p], dvz = c.z - vz[p];
                    float r2 = fmaf(dx, dx, eps2f);
                    r2 = fmaf(dy, dy, r2);
                    r2 = fmaf(dz, dz, r2);
                    float rv = dx * dvx;
                    rv = fmaf(dy, dvy, rv);
                    rv = fmaf(dz, dvz, rv);
                    float rinv = rsqrtf(r2);
                    rinv = (j == iid[p]) ? 0.f : rinv;
                    const float rinv2 = rinv * rinv;
                    const float mrinv = a.w * rinv;
                    const float mr3 = mrinv * rinv2;
                    const float beta = -3.f * ((mr3 * rinv2) * rv);
                    tp[p] += mrinv;
                    ta[p][0] = fmaf(mr3, dx, ta[p][0]);
                    ta[p][1] = fmaf(mr3, dy, ta[p][1]);
                    ta[p][2] = fmaf(mr3, dz, ta[p][2]);
                    // per pair: m v / s^3 - 3 m (r.v) r / s^5
                    tjv[p][0] = fmaf(beta, dx, fmaf(mr3, dvx, tjv[p][0]));
                    tjv[p][1] = fmaf(beta, dy, fmaf(mr3, dvy, tjv[p][1]));
                    tjv[p][2] = fmaf(beta, dz, fmaf(mr3, dvz, tjv[p][2]));
                }
            }
            // lanes -> warp (fixed xor tree), warps -> CTA (fixed order) -> totals
#pragma unroll
            for (int p = 0; p < G; ++p)
#pragma unroll
                for (int c = 0; c < 7; ++c) {
                    dsf v{c < 3 ? ta[p][c] : (c < 6 ? tjv[p][c - 3] : tp[p]), 0.f};
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) ds_acc(v, ds_shfl_xor(v, o));
                    if (lane == 0) s_red[warp][p * 7 + c] = make_float2(v.hi, v.lo);
                }
            __syncthreads();
            if (tid < G * 7) {
                dsf sum{s_tot[tid].x, s_tot[tid].y};
#pragma unroll
                for (int q = 0; q < NW; ++q) ds_acc(sum, dsf{s_red[q][tid].x, s_red[q][tid].y});
                s_tot[tid] = make_float2(sum.hi, sum.lo);
            }
            __syncthreads();
        }
        if (tid < G * 7) {
            const int p = tid / 7, c = tid % 7, k = g0 + p;
            if (k < w.ni) {
                const float2 t = s_tot[tid];
                if (w.nsplit <= 1) {
                    const Out3 out{w.acc, w.jerk, w.pot, w.ld};
                    store_component(out, c, w.i0 + k, ds_to_double(dsf{t.x, t.y}), w.err);
                } else {
                    w.part[((size_t)w.split * 7 + c) * w.ni + k] = t;
                }
            }
        }
        __syncthreads();
    }
}

// The j-parallel items of a batched evaluation (kind 1), in a kernel of their
// own so that their register needs do not lower the occupancy of the
// i-parallel kernel; the two run concurrently on two streams.
template <int VAR, int NT>
__global__ void __launch_bounds__(NT)
    k_force_items_jpar32(const WorkItem *__restrict__ items, int nitems)
{
    __shared__ float2 s_red[NT / 32][28];
    __shared__ float2 s_tot[28];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        item_jpar<VAR == NB_F32DS, NT>(w, s_red, s_tot);
    }
}

// The j-split groups of a batched evaluation, after the items: each group's
// outputs are the sums of its nsplit double-single partials in the order
// split = 0..nsplit-1 (one thread per output, consecutive outputs coalesced).
__global__ void __launch_bounds__(256)
    k_split_reduce(const SplitGroup *__restrict__ groups, int ngroups)
{
    for (int gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
        const SplitGroup g = groups[gi];
        const int total = 7 * g.ni;
        const Out3 out{g.acc, g.jerk, g.pot, g.ld};
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            const int c = q / g.ni, k = q % g.ni;
            dsf sum{0.f, 0.f};
            for (int sp = 0; sp < g.nsplit; ++sp) {
                const float2 v = __ldcg(g.part + ((size_t)sp * 7 + c) * g.ni + k);
                ds_acc(sum, dsf{v.x, v.y});
            }
            store_component(out, c, g.i0 + k, ds_to_double(sum), g.err);
        }
    }
}


template <int VAR, int IPT, int NT, int JT, int NS>
__global__ void __launch_bounds__(NT, 512 / NT)
    k_force_items32(const WorkItem *__restrict__ items, int nitems)
{
    // NS ring stages of JT records, then the current full tile as j-pairs
    extern __shared__ __align__(128) float4 s_tile[];
    __shared__ __align__(8) uint64_t s_full[NS];
    __shared__ int s_abort;
    constexpr bool DS = (VAR == NB_F32DS);
    constexpr int NPAIR = JT / 2;
    float4 *s_pair = s_tile + (size_t)NS * JT * DS_REC;
    const int tid = threadIdx.x;

    if (tid == 0) {
        s_abort = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) mbar_init(&s_full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    unsigned seq = 0;  // tiles consumed so far by this CTA (ring position and phase)
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const WorkItem w = items[it];
        unsigned *err = w.err;
        const float eps2f = w.eps2;
        const float2 e2 = make_float2(eps2f, eps2f);
        const float4 *__restrict__ jrec = w.jrec;
        const int ntiles = (w.nj + JT - 1) / JT;

        // the i-particles, negated and duplicated into both halves of a float2 (the
        // packed pair terms take two j at a time; the scalar path uses .x)
        float2 nxh[IPT], nyh[IPT], nzh[IPT], nxl[IPT], nyl[IPT], nzl[IPT], nvx[IPT], nvy[IPT],
            nvz[IPT];
        int iid[IPT];
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
            const int k = min(p * NT + tid, w.ni - 1);  // idle slots copy the last i
            const int r = w.i0 + k;
            const float4 a = __ldg(w.irec + (size_t)DS_REC * r);
            const float4 b = __ldg(w.irec + (size_t)DS_REC * r + 1);
            const float4 c = __ldg(w.irec + (size_t)DS_REC * r + 2);
            nxh[p] = make_float2(-a.x, -a.x);
            nyh[p] = make_float2(-a.y, -a.y);
            nzh[p] = make_float2(-a.z, -a.z);
            nxl[p] = make_float2(-b.x, -b.x);
            nyl[p] = make_float2(-b.y, -b.y);
            nzl[p] = make_float2(-b.z, -b.z);
            nvx[p] = make_float2(-c.x, -c.x);
            nvy[p] = make_float2(-c.y, -c.y);
            nvz[p] = make_float2(-c.z, -c.z);
            iid[p] = w.gathered ? __float_as_int(b.w) : r;
        }
        float A_h[IPT][3], A_l[IPT][3], J_h[IPT][3], J_l[IPT][3], P_h[IPT], P_l[IPT];
#pragma unroll
        for (int p = 0; p < IPT; ++p) {
#pragma unroll
            for (int c = 0; c < 3; ++c) A_h[p][c] = A_l[p][c] = J_h[p][c] = J_l[p][c] = 0.f;
            P_h[p] = P_l[p] = 0.f;
        }

        auto issue = [&](int kt) {
            const unsigned sq = seq + (unsigned)kt;
            const int stage = (int)(sq % NS);
            const int cnt = min(JT, w.nj - kt * JT);
            const uint32_t bytes = (uint32_t)cnt * DS_REC * 16u;
            mbar_expect_tx(&s_full[stage], bytes);
            bulk_g2s(s_tile + (size_t)stage * JT * DS_REC,
                     jrec + ((size_t)w.j0 + (size_t)kt * JT) * DS_REC, bytes, &s_full[stage]);
        };
        if (tid == 0) {
            for (int kt = 0; kt < NS && kt < ntiles; ++kt) issue(kt);
        }
        for (int kt = 0; kt < ntiles; ++kt) {
            const unsigned sq = seq + (unsigned)kt;
            const int stage = (int)(sq % NS);
            if (!mbar_wait(&s_full[stage], (sq / NS) & 1u)) s_abort = 1;
            const float4 *T = s_tile + (size_t)stage * JT * DS_REC;
            const int jbase = w.j0 + kt * JT;
            const int cnt = min(JT, w.nj - kt * JT);
            bool own = false;
#pragma unroll
            for (int p = 0; p < IPT; ++p) own = own || (iid[p] >= jbase && iid[p] < jbase + cnt);
            own = __any_sync(0xffffffffu, own);
            // FP32 sums of this tile, two lanes each (even and odd j of a pair; the
            // scalar path adds into .x)
            float2 ta[IPT][3], tja[IPT][3], tjb[IPT][3], tp[IPT];
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
#pragma unroll
                for (int c = 0; c < 3; ++c) ta[p][c] = tja[p][c] = tjb[p][c] = make_float2(0.f, 0.f);
                tp[p] = make_float2(0.f, 0.f);
            }
            auto body = [&](int jj, auto masked_tag) {
                constexpr bool MASKED = decltype(masked_tag)::value;
                const float4 a = T[DS_REC * jj];
                const float4 c = T[DS_REC * jj + 2];
                float4 b;
                if (DS) b = T[DS_REC * jj + 1];
#pragma unroll
                for (int p = 0; p < IPT; ++p) {
                    float dx, dy, dz;
                    if (DS) {
                        dx = (a.x + nxh[p].x) + (b.x + nxl[p].x);
                        dy = (a.y + nyh[p].x) + (b.y + nyl[p].x);
                        dz = (a.z + nzh[p].x) + (b.z + nzl[p].x);
                    } else {
                        dx = a.x + nxh[p].x;
                        dy = a.y + nyh[p].x;
                        dz = a.z + nzh[p].x;
                    }
                    const float dvx = c.x + nvx[p].x, dvy = c.y + nvy[p].x, dvz = c.z + nvz[p].x;
                    float r2 = fmaf(dx, dx, eps2f);
                    r2 = fmaf(dy, dy, r2);
                    r2 = fmaf(dz, dz, r2);
                    float rv = dx * dvx;
                    rv = fmaf(dy, dvy, rv);
                    rv = fmaf(dz, dvz, rv);
                    float rinv = rsqrtf(r2);
                    if (MASKED) rinv = (jbase + jj == iid[p]) ? 0.f : rinv;
                    const float rinv2 = rinv * rinv;
                    const float mrinv = a.w * rinv;
                    const float mr3 = mrinv * rinv2;
                    const float beta = (mr3 * rinv2) * rv;
                    tp[p].x += mrinv;
                    ta[p][0].x = fmaf(mr3, dx, ta[p][0].x);
                    ta[p][1].x = fmaf(mr3, dy, ta[p][1].x);
                    ta[p][2].x = fmaf(mr3, dz, ta[p][2].x);
                    tja[p][0].x = fmaf(mr3, dvx, tja[p][0].x);
                    tja[p][1].x = fmaf(mr3, dvy, tja[p][1].x);
                    tja[p][2].x = fmaf(mr3, dvz, tja[p][2].x);
                    tjb[p][0].x = fmaf(beta, dx, tjb[p][0].x);
                    tjb[p][1].x = fmaf(beta, dy, tjb[p][1].x);
                    tjb[p][2].x = fmaf(beta, dz, tjb[p][2].x);
                }
            };
            if (cnt == JT) {
                // full tile: transposed into j-pairs for the packed FP32x2 pair terms
                for (int x = tid; x < 3 * NPAIR; x += NT) {
                    const int q = x % NPAIR, part = x / NPAIR;
                    const float4 u = T[DS_REC * (2 * q) + part];
                    const float4 v = T[DS_REC * (2 * q + 1) + part];
                    float4 *P = s_pair + 6 * q + 2 * part;
                    P[0] = make_float4(u.x, v.x, u.y, v.y);
                    P[1] = make_float4(u.z, v.z, u.w, v.w);
                }
                __syncthreads();
                if (own) {
                    for (int jj = 0; jj < JT; ++jj) body(jj, std::true_type{});
                } else {
#pragma unroll 2
                    for (int q = 0; q < NPAIR; ++q) {
                        const float4 *P = s_pair + 6 * q;
                        const float4 q0 = P[0], q1 = P[1], q4 = P[4], q5 = P[5];
                        float4 q2, q3;
                        if (DS) {
                            q2 = P[2];
                            q3 = P[3];
                        }
                        const float2 XH = make_float2(q0.x, q0.y), YH = make_float2(q0.z, q0.w);
                        const float2 ZH = make_float2(q1.x, q1.y), MJ = make_float2(q1.z, q1.w);
                        const float2 VX = make_float2(q4.x, q4.y), VY = make_float2(q4.z, q4.w);
                        const float2 VZ = make_float2(q5.x, q5.y);
#pragma unroll
                        for (int p = 0; p < IPT; ++p) {
                            float2 dx, dy, dz;
                            if (DS) {
                                dx = __fadd2_rn(__fadd2_rn(XH, nxh[p]),
                                                __fadd2_rn(make_float2(q2.x, q2.y), nxl[p]));
                                dy = __fadd2_rn(__fadd2_rn(YH, nyh[p]),
                                                __fadd2_rn(make_float2(q2.z, q2.w), nyl[p]));
                                dz = __fadd2_rn(__fadd2_rn(ZH, nzh[p]),
                                                __fadd2_rn(make_float2(q3.x, q3.y), nzl[p]));
                            } else {
                                dx = __fadd2_rn(XH, nxh[p]);
                                dy = __fadd2_rn(YH, nyh[p]);
                                dz = __fadd2_rn(ZH, nzh[p]);
                            }
                            const float2 dvx = __fadd2_rn(VX, nvx[p]);
                            const float2 dvy = __fadd2_rn(VY, nvy[p]);
                            const float2 dvz = __fadd2_rn(VZ, nvz[p]);
                            float2 r2 = __ffma2_rn(dx, dx, e2);
                            r2 = __ffma2_rn(dy, dy, r2);
                            r2 = __ffma2_rn(dz, dz, r2);
                            float2 rv = __fmul2_rn(dx, dvx);
                            rv = __ffma2_rn(dy, dvy, rv);
                            rv = __ffma2_rn(dz, dvz, rv);
                            const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                            const float2 rinv2 = __fmul2_rn(rinv, rinv);
                            const float2 mrinv = __fmul2_rn(MJ, rinv);
                            const float2 mr3 = __fmul2_rn(mrinv, rinv2);
                            const float2 beta = __fmul2_rn(__fmul2_rn(mr3, rinv2), rv);
                            tp[p] = __fadd2_rn(tp[p], mrinv);
                            ta[p][0] = __ffma2_rn(mr3, dx, ta[p][0]);
                            ta[p][1] = __ffma2_rn(mr3, dy, ta[p][1]);
                            ta[p][2] = __ffma2_rn(mr3, dz, ta[p][2]);
                            tja[p][0] = __ffma2_rn(mr3, dvx, tja[p][0]);
                            tja[p][1] = __ffma2_rn(mr3, dvy, tja[p][1]);
                            tja[p][2] = __ffma2_rn(mr3, dvz, tja[p][2]);
                            tjb[p][0] = __ffma2_rn(beta, dx, tjb[p][0]);
                            tjb[p][1] = __ffma2_rn(beta, dy, tjb[p][1]);
                            tjb[p][2] = __ffma2_rn(beta, dz, tjb[p][2]);
                        }
                    }
                }
            } else if (own) {
                for (int jj = 0; jj < cnt; ++jj) body(jj, std::true_type{});
            } else {
#pragma unroll 2
                for (int jj = 0; jj < cnt; ++jj) body(jj, std::false_type{});
            }
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float sa = ta[p][c].x + ta[p][c].y;
                    const float jt = fmaf(-3.f, tjb[p][c].x + tjb[p][c].y,
                                          tja[p][c].x + tja[p][c].y);
                    if (DS) {
                        ds_add(A_h[p][c], A_l[p][c], sa);
                        ds_add(J_h[p][c], J_l[p][c], jt);
                    } else {
                        A_h[p][c] += sa;
                        J_h[p][c] += jt;
                    }
                }
                const float sp = tp[p].x + tp[p].y;
                if (DS)
                    ds_add(P_h[p], P_l[p], sp);
                else
                    P_h[p] += sp;
            }
            __syncthreads();  // the stage and the pair buffer are free
            if (s_abort) {
                if (tid == 0) {
                    drain_ring<NS>(s_full, seq, kt, ntiles);
                    atomicOr(err, DERR_TIMEOUT);
                }
                return;
            }
            if (tid == 0 && kt + NS < ntiles) issue(kt + NS);
        }
        seq += (unsigned)ntiles;
        if (w.nsplit <= 1) {
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
                const int k = p * NT + tid;
                if (k >= w.ni) continue;
                double d[7];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    d[c] = ds_to_double(dsf{A_h[p][c], A_l[p][c]});
                    d[3 + c] = ds_to_double(dsf{J_h[p][c], J_l[p][c]});
                }
                d[6] = ds_to_double(dsf{P_h[p], P_l[p]});
                write_final(Out3{w.acc, w.jerk, w.pot, w.ld}, w.i0 + k, d, err);
            }
        } else {
            float2 *pp = w.part + (size_t)w.split * 7 * w.ni;
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
                const int k = p * NT + tid;
                if (k >= w.ni) continue;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    pp[(size_t)c * w.ni + k] = make_float2(A_h[p][c], A_l[p][c]);
                    pp[(size_t)(3 + c) * w.ni + k] = make_float2(J_h[p][c], J_l[p][c]);
                }
                pp[(size_t)6 * w.ni + k] = make_float2(P_h[p], P_l[p]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Plans and launchers.
// ---------------------------------------------------------------------------

constexpr int JT32 = 128;    // j-tile of the batched items
constexpr int JT_TILE = 256;  // j-tile of the tile kernel
constexpr int NS32 = 3;
constexpr int JT64 = 64;
constexpr int NS64 = 3;

// Warp-group layout (FP32 kind 1): ipt i-particles per warp, nwarp warps per CTA.
static void wgrp_shape(int n_i, ForcePlan &p)
{
    p.ipt = n_i <= 1 ? 1 : 2;
    const int groups = (n_i + p.ipt - 1) / p.ipt;
    const int nwarp = groups <= 1 ? 1 : groups <= 2 ? 2 : groups <= 4 ? 4 : 8;
    p.threads = 32 * nwarp;
}

static long long clampll(long long v, long long lo, long long hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

// Tiny-set layout (FP32 kind 2): ipt i-particles per pass, jt = j per thread;
// one j-split per CTA of 256 threads.
static void tiny_shape(int n_i, int n_j, ForcePlan &p)
{
    p.kind = 2;
    p.ipt = n_i <= 1 ? 1 : (n_i <= 2 ? 2 : 4);
    p.threads = 256;
    p.jt = n_j >= 256 * 4 * 32 ? 4 : (n_j >= 256 * 2 * 32 ? 2 : 1);
    p.nsplit = (n_j + 256 * p.jt - 1) / (256 * p.jt);
}

ForcePlan plan_force(int variant, int n_i, int n_j, int num_sms)
{
    ForcePlan p{};
    p.nwj = 1;
    if (variant == NB_F64) {
        if (n_i <= 32) {  // FP64 j-parallel kernel
            p.kind = 1;
            p.ipt = n_i <= 1 ? 1 : n_i <= 2 ? 2 : 4;
            p.threads = 128;
            p.nsplit = (int)clampll((n_j + 128LL * 4 - 1) / (128LL * 4), 1, 2LL * num_sms);
            return p;
        }
        p.kind = 0;
        p.ipt = 1;
        p.threads = 128;
        p.jt = JT64;
        const long long nblk = (n_i + 127) / 128;
        const long long ntiles = (n_j + JT64 - 1) / JT64;
        p.nsplit = (int)clampll((16LL * num_sms + nblk - 1) / nblk, 1,
                                ntiles / 2 > 1 ? ntiles / 2 : 1);
        return p;
    }
    if (n_i <= 4) {
        tiny_shape(n_i, n_j, p);
        return p;
    }
    if (n_i < 4096) {
        // warp groups: about 14 warps per SM in total, at least 1024 j per split
        // (the best plans a sweep over N_i at N = 65536 found on GB300)
        p.kind = 1;
        wgrp_shape(n_i, p);
        const long long groups = (n_i + p.ipt - 1) / p.ipt;
        const long long cap = n_j / 1024 > 1 ? n_j / 1024 : 1;
        p.nsplit = (int)clampll((14LL * num_sms + groups - 1) / groups, 1, cap);
        return p;
    }
    // tiles: 256 threads, 2 i per thread; 8 or 4 warp rows share each j-tile
    // below 65536 i; about 40 CTAs per SM, at least 16 tiles per split; then, up
    // to twice that many splits, the fewest whose last wave of resident CTAs is at
    // least 97% full, else the fullest (N = 2^20: 2048 i-blocks x 3 splits fill
    // 21% of their 21st wave on 304 slots, x 4 splits 95% of their 27th)
    p.kind = 0;
    p.ipt = 2;
    p.threads = 256;
    p.jt = JT_TILE;
    p.nwj = n_i >= 65536 ? 1 : (n_i >= 8192 ? 4 : 8);
    const long long ib = (long long)(p.threads / p.nwj) * p.ipt;
    const long long nblk = (n_i + ib - 1) / ib;
    const long long ntiles = (n_j + p.jt - 1) / p.jt;
    const long long cap = ntiles / 16 > 1 ? ntiles / 16 : 1;
    const long long ns0 = clampll((40LL * num_sms + nblk - 1) / nblk, 1, cap);
    const long long slots = (long long)num_sms * tile_blocks_per_sm(variant, p.nwj);
    long long best = ns0;
    double best_eff = 0.0;
    for (long long ns = ns0; ns <= std::min(cap, 2 * ns0); ++ns) {
        const double waves = (double)(nblk * ns) / (double)slots;
        const double eff = waves / std::ceil(waves);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = ns;
        }
        if (eff >= 0.97) break;
    }
    p.nsplit = (int)best;
    return p;
}

ForcePlan plan_from_entry(const nb_plan &e, int variant, int n_i, int n_j)
{
    ForcePlan p{};
    p.nwj = 1;
    if (e.kind == 2 && variant != NB_F64) {
        tiny_shape(n_i, n_j, p);  // its split count follows from the j per thread
        return p;
    }
    if (e.kind == 1 || e.kind == 2) {
        p.kind = 1;
        if (variant == NB_F64) {
            p.ipt = n_i <= 1 ? 1 : n_i <= 2 ? 2 : 4;
            p.threads = 128;
        } else {
            wgrp_shape(n_i, p);
        }
        p.nsplit = (int)clampll(e.nsplit, 1, n_j);
        return p;
    }
    p.kind = 0;
    if (variant == NB_F64) {
        p.ipt = 1;
        p.threads = 128;
        p.jt = JT64;
    } else {
        p.ipt = 2;
        p.threads = 256;
        p.jt = JT_TILE;
        p.nwj = (e.nwj == 4 || e.nwj == 8) ? e.nwj : 1;
    }
    const int ntiles = (n_j + p.jt - 1) / p.jt;
    p.nsplit = (int)clampll(e.nsplit, 1, ntiles);
    return p;
}

size_t plan_partial_doubles(const ForcePlan &p, int n_i)
{
    if (p.nsplit <= 1) return 0;
    return (size_t)p.nsplit * 7 * (size_t)n_i;
}

template <int VAR, int IPT, int NWI, int NWJ>
static cudaError_t go_tile32(const JSet &js, const ISet &is, float eps2f, int nsplit,
                             double *part, unsigned *cnt, Out3 out, unsigned *err,
                             cudaStream_t st)
{
    auto kern = k_force_tile32<VAR, IPT, NWI, NWJ, JT_TILE, NS32>;
    constexpr int NT = 32 * NWI * NWJ;
    constexpr int IB = 32 * NWI * IPT;
    // the ring (36 KB) and the transposed tile (12 KB); the warp-row sums reuse them
    const size_t ring = (size_t)(NS32 + 1) * JT_TILE * DS_REC * sizeof(float4);
    const size_t red = NWJ > 1 ? (size_t)NWJ * 7 * IB * sizeof(double) : 0;  // <= 28 KB
    const size_t smem = ring > red ? ring : red;
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    const int ntiles = (js.n + JT_TILE - 1) / JT_TILE;
    dim3 grid((is.n + IB - 1) / IB, nsplit);
    kern<<<grid, NT, smem, st>>>(js.rec32, js.n, is, eps2f, ntiles, part, is.n, cnt, out, err);
    if (nsplit > 1) {
        const long long outs = 7LL * is.n;
        k_tile_split_reduce<<<(unsigned)((outs + 255) / 256), 256, 0, st>>>(
            reinterpret_cast<const float2 *>(part), is.n, nsplit, is.n, out, err);
    }
    return cudaGetLastError();
}

template <int VAR, int IPT, int NWARP>
static cudaError_t go_wgrp32(const JSet &js, const ISet &is, float eps2f, int nsplit,
                             double *part, unsigned *cnt, Out3 out, unsigned *err,
                             cudaStream_t st)
{
    const int groups = (is.n + IPT - 1) / IPT;
    dim3 grid((groups + NWARP - 1) / NWARP, nsplit);
    k_force_wgrp32<VAR, IPT, NWARP><<<grid, 32 * NWARP, 0, st>>>(js.rec32, js.n, is, eps2f, part,
                                                                  is.n, cnt, out, err);
    return cudaGetLastError();
}

template <int VAR, int IPT, int JPT>
static cudaError_t go_tiny32(const JSet &js, const ISet &is, float eps2f, double *part,
                             unsigned *cnt, Out3 out, unsigned *err, cudaStream_t st)
{
    const int g = (js.n + 256 * JPT - 1) / (256 * JPT);
    k_force_tiny32<VAR, IPT, JPT><<<g, 256, 0, st>>>(js.rec32, js.n, is, eps2f, part, is.n, cnt,
                                                      out, err);
    return cudaGetLastError();
}

template <int VAR, int IPT>
static cudaError_t go_tiny32_j(int jpt, const JSet &js, const ISet &is, float eps2f,
                               double *part, unsigned *cnt, Out3 out, unsigned *err,
                               cudaStream_t st)
{
    switch (jpt) {
    case 1: return go_tiny32<VAR, IPT, 1>(js, is, eps2f, part, cnt, out, err, st);
    case 2: return go_tiny32<VAR, IPT, 2>(js, is, eps2f, part, cnt, out, err, st);
    default: return go_tiny32<VAR, IPT, 4>(js, is, eps2f, part, cnt, out, err, st);
    }
}

template <int IPT, int NT>
static cudaError_t go_tile64(const JSet &js, const ISet &is, double eps2, int nsplit, double *part,
                             unsigned *cnt, Out3 out, unsigned *err, cudaStream_t st)
{
    auto kern = k_force_tile64<IPT, NT, JT64, NS64>;
    const size_t smem = (size_t)NS64 * 7 * JT64 * sizeof(double);  // 10.5 KB
    const int ntiles = (js.n + JT64 - 1) / JT64;
    dim3 grid((is.n + NT * IPT - 1) / (NT * IPT), nsplit);
    kern<<<grid, NT, smem, st>>>(js, is, eps2, ntiles, part, is.n, cnt, out, err);
    return cudaGetLastError();
}

template <int VAR>
static cudaError_t dispatch32(const ForcePlan &p, const JSet &js, const ISet &is, float eps2f,
                              double *part, unsigned *cnt, Out3 out, unsigned *err,
                              cudaStream_t st)
{
    if (p.kind == 2) {
        switch (p.ipt) {
        case 1: return go_tiny32_j<VAR, 1>(p.jt, js, is, eps2f, part, cnt, out, err, st);
        case 2: return go_tiny32_j<VAR, 2>(p.jt, js, is, eps2f, part, cnt, out, err, st);
        default: return go_tiny32_j<VAR, 4>(p.jt, js, is, eps2f, part, cnt, out, err, st);
        }
    }
    if (p.kind == 1) {
        const int nw = p.threads / 32;
        if (p.ipt == 1) return go_wgrp32<VAR, 1, 1>(js, is, eps2f, p.nsplit, part, cnt, out, err, st);
        switch (nw) {
        case 1: return go_wgrp32<VAR, 2, 1>(js, is, eps2f, p.nsplit, part, cnt, out, err, st);
        case 2: return go_wgrp32<VAR, 2, 2>(js, is, eps2f, p.nsplit, part, cnt, out, err, st);
        case 4: return go_wgrp32<VAR, 2, 4>(js, is, eps2f, p.nsplit, part, cnt, out, err, st);
        default: return go_wgrp32<VAR, 2, 8>(js, is, eps2f, p.nsplit, part, cnt, out, err, st);
        }
    }
    switch (p.nwj) {
    case 1: return go_tile32<VAR, 2, 8, 1>(js, is, eps2f, p.nsplit, part, cnt, out, err, st);
    case 4: return go_tile32<VAR, 2, 2, 4>(js, is, eps2f, p.nsplit, part, cnt, out, err, st);
    default: return go_tile32<VAR, 2, 1, 8>(js, is, eps2f, p.nsplit, part, cnt, out, err, st);
    }
}

cudaError_t warm_force_jmode64(cudaStream_t st)
{
    cudaFuncAttributes fa;
    cudaError_t e;
    if ((e = cudaFuncGetAttributes(&fa, k_force_jmode64<1, 128>)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, k_force_jmode64<2, 128>)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, k_force_jmode64<4, 128>)) != cudaSuccess)
        return e;
    // an empty i-set: the i-loop does not run and one CTA writes nothing
    const JSet js{};
    ISet is{};
    is.member = true;
    k_force_jmode64<1, 128><<<1, 128, 0, st>>>(js, is, 0.0, nullptr, 0, nullptr, Out3{}, nullptr);
    k_force_jmode64<2, 128><<<1, 128, 0, st>>>(js, is, 0.0, nullptr, 0, nullptr, Out3{}, nullptr);
    k_force_jmode64<4, 128><<<1, 128, 0, st>>>(js, is, 0.0, nullptr, 0, nullptr, Out3{}, nullptr);
    return cudaGetLastError();
}

static cudaError_t dispatch64(const ForcePlan &p, const JSet &js, const ISet &is, double eps2,
                              double *part, unsigned *cnt, Out3 out, unsigned *err,
                              cudaStream_t st)
{
    if (p.kind == 1) {
        const int g = p.nsplit;
#define JM(I) k_force_jmode64<I, 128><<<g, 128, 0, st>>>(js, is, eps2, part, is.n, cnt, out, err)
        switch (p.ipt) {
        case 1: JM(1); break;
        case 2: JM(2); break;
        default: JM(4); break;
        }
#undef JM
        return cudaGetLastError();
    }
    return go_tile64<1, 128>(js, is, eps2, p.nsplit, part, cnt, out, err, st);
}

template <int VAR, int NT>
static cudaError_t go_items(const WorkItem *items, int nitems, int grid, cudaStream_t st)
{
    const size_t smem = (size_t)(NS32 + 1) * JT32 * DS_REC * sizeof(float4);
    k_force_items32<VAR, 2, NT, JT32, NS32><<<grid, NT, smem, st>>>(items, nitems);
    return cudaGetLastError();
}

cudaError_t launch_force_items(int variant, int threads, const WorkItem *items, int nitems,
                               int grid, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (variant == NB_F32DS) {
        switch (threads) {
        case 64: return go_items<NB_F32DS, 64>(items, nitems, grid, st);
        case 128: return go_items<NB_F32DS, 128>(items, nitems, grid, st);
        default: return go_items<NB_F32DS, 256>(items, nitems, grid, st);
        }
    }
    switch (threads) {
    case 64: return go_items<NB_F32, 64>(items, nitems, grid, st);
    case 128: return go_items<NB_F32, 128>(items, nitems, grid, st);
    default: return go_items<NB_F32, 256>(items, nitems, grid, st);
    }
}

cudaError_t launch_force_items_jpar(int variant, const WorkItem *items, int nitems, int grid,
                                    cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (variant == NB_F32DS)
        k_force_items_jpar32<NB_F32DS, JPAR_THREADS><<<grid, JPAR_THREADS, 0, st>>>(items, nitems);
    else
        k_force_items_jpar32<NB_F32, JPAR_THREADS><<<grid, JPAR_THREADS, 0, st>>>(items, nitems);
    return cudaGetLastError();
}

cudaError_t launch_split_reduce(const SplitGroup *groups, int ngroups, int grid,
                                cudaStream_t st)
{
    if (ngroups <= 0) return cudaSuccess;
    k_split_reduce<<<grid, 256, 0, st>>>(groups, ngroups);
    return cudaGetLastError();
}

int jpar_blocks_per_sm(int variant)
{
    int nb = 0;
    const cudaError_t e =
        variant == NB_F32DS
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &nb, k_force_items_jpar32<NB_F32DS, JPAR_THREADS>, JPAR_THREADS, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &nb, k_force_items_jpar32<NB_F32, JPAR_THREADS>, JPAR_THREADS, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

// Self-check of the bounded copy wait: an mbarrier that no copy or arrival
// completes; the wait gives up after limit_ns and reports DERR_TIMEOUT.
__global__ void k_selftest_mbar(unsigned *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, limit_ns)) atomicOr(err, DERR_TIMEOUT);
}

cudaError_t launch_selftest_mbar(unsigned *err, unsigned long long limit_ns, cudaStream_t st)
{
    k_selftest_mbar<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

template <int VAR, int NWI, int NWJ>
static int tile_occ()
{
    constexpr int NT = 32 * NWI * NWJ;
    constexpr int IB = 32 * NWI * 2;
    const size_t ring = (size_t)(NS32 + 1) * JT_TILE * DS_REC * sizeof(float4);
    const size_t red = NWJ > 1 ? (size_t)NWJ * 7 * IB * sizeof(double) : 0;
    const size_t smem = ring > red ? ring : red;
    auto kern = k_force_tile32<VAR, 2, NWI, NWJ, JT_TILE, NS32>;
    int nb = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

int tile_blocks_per_sm(int variant, int nwj)
{
    if (variant == NB_F32DS)
        return nwj == 1 ? tile_occ<NB_F32DS, 8, 1>()
                        : (nwj == 4 ? tile_occ<NB_F32DS, 2, 4>() : tile_occ<NB_F32DS, 1, 8>());
    return nwj == 1 ? tile_occ<NB_F32, 8, 1>()
                    : (nwj == 4 ? tile_occ<NB_F32, 2, 4>() : tile_occ<NB_F32, 1, 8>());
}

int batch_blocks_per_sm(int variant, int threads)
{
    int nb = 0;
    const size_t smem = (size_t)(NS32 + 1) * JT32 * DS_REC * sizeof(float4);
    cudaError_t e;
    if (variant == NB_F32DS) {
        e = threads == 64    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &nb, k_force_items32<NB_F32DS, 2, 64, JT32, NS32>, 64, smem)
            : threads == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                   &nb, k_force_items32<NB_F32DS, 2, 128, JT32, NS32>, 128, smem)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                   &nb, k_force_items32<NB_F32DS, 2, 256, JT32, NS32>, 256, smem);
    } else {
        e = threads == 64    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &nb, k_force_items32<NB_F32, 2, 64, JT32, NS32>, 64, smem)
            : threads == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                   &nb, k_force_items32<NB_F32, 2, 128, JT32, NS32>, 128, smem)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                   &nb, k_force_items32<NB_F32, 2, 256, JT32, NS32>, 256, smem);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

size_t plan_counters(const ForcePlan &p, int n_i)
{
    if (p.nsplit <= 1) return 1;
    if (p.kind == 2) return 1;
    long long ib;
    if (p.kind == 1)
        ib = (long long)(p.threads / 32) * p.ipt;  // FP32 warp groups (FP64 j-parallel: one)
    else
        ib = (long long)(p.threads / p.nwj) * p.ipt;
    return (size_t)((n_i + ib - 1) / ib);
}

cudaError_t launch_force(int variant, const ForcePlan &plan, const JSet &js, const ISet &is,
                         double eps2, double *part, unsigned *counters, Out3 out, unsigned *err,
                         cudaStream_t st, cudaEvent_t *ev)
{
    if (is.n <= 0) return cudaSuccess;
    const float eps2f = (float)eps2;
    cudaError_t e;
    if (ev) cudaEventRecord(ev[0], st);
    if (variant == NB_F64)
        e = dispatch64(plan, js, is, eps2, part, counters, out, err, st);
    else if (variant == NB_F32DS)
        e = dispatch32<NB_F32DS>(plan, js, is, eps2f, part, counters, out, err, st);
    else
        e = dispatch32<NB_F32>(plan, js, is, eps2f, part, counters, out, err, st);
    if (ev) cudaEventRecord(ev[1], st);
    return e;
}

}  // namespace nb
