// Fused persistent block steps: one cooperative launch takes block step after
// block step of one system with grid-wide barriers between the stages, so a
// step with a small due set (the common case of block time steps, Sect. III:
// most block times have only a few particles due) costs no host round trip
// and no launch gaps:
//   A  t_next and the due count from the level histogram; if t_next > t_end
//      or the due set is larger than na_max, every CTA predicts its range in
//      full, the due set is gathered in ascending index (CTA counts, prefix)
//      and the kernel publishes (epoch, t_next, N_active) to the mailbox like
//      K5 + K1 and returns; else every CTA predicts its contiguous range of
//      particles (K1, double-single records only) and its due particles take
//      slots of the due set by warp-aggregated atomics;  -- barrier
//   C  small due sets: items of four due slots against a j-chunk (lanes over
//      j); the CTA that completes a group's last chunk (a ticket) sums its
//      double-single partials in chunk order (K3) and corrects its particles
//      (K4), three lanes for the three components; larger due sets (order 4):
//      CTA items of 32 (64) due slots whose j-chunk is staged through shared memory
//      as j-pairs, double-single partials per chunk;   -- barrier
//   D  (larger due sets) one warp per due particle sums its chunk partials in
//      chunk order (K3) and corrects it (K4: Hermite corrector, Aarseth step,
//      histogram);                                          -- barrier
// k_fused_steps6 runs the same loop for the 6th-order scheme with the small
// path only (64-byte records, ten outputs per slot, the order-6 corrector).
// Every inter-CTA wait is bounded; a CTA that gives up raises the abort flag
// and all CTAs leave at their next barrier (the host then reports a timeout).
// This file is compiled with global loads cached in L2 only (-dlcm=cg): data
// written by other CTAs in the same launch must not be served from a stale L1.
#include <cuda_runtime.h>
#include <math.h>

#include "ds.cuh"
#include "nb_internal.cuh"
#include "step_body.cuh"

namespace nb {

constexpr unsigned long long BARRIER_LIMIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch: bar[0] counts the arrivals of the
// whole launch (generation g is complete once it reaches g x gridDim.x; the
// comparison is wrap-safe), bar[2] is the abort flag (both zero at launch).
// Thread 0 of every CTA adds its arrival after a fence (a release) and polls
// the count with acquire loads, so the last arrival itself releases the
// waiters; the abort flag and the time limit (BARRIER_LIMIT_NS) are checked
// every 32 polls. Returns false once this CTA gave up or saw the abort flag; a
// CTA that gives up never arrives again, so the others stop at their next
// barrier at the latest. gen: thread 0's generation.
__device__ bool grid_barrier(unsigned *bar, unsigned &gen,
                             unsigned long long limit_ns = BARRIER_LIMIT_NS)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = (gen + 1u) * gridDim.x;
        __threadfence();
        atomicAdd(&bar[0], 1u);
        const unsigned long long t0 = globaltimer_ns();
        for (unsigned it = 1;; ++it) {
            if ((int)(ld_acquire_u32(&bar[0]) - target) >= 0) break;
            if ((it & 31u) == 0u) {
                if (ld_acquire_u32(&bar[2]) != 0u) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > limit_ns) {
                    atomicExch(&bar[2], 1u);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        gen += 1u;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// K2 for one tile item (due sets larger than FUSED_SMALL_NA): 32 IPT due slots
// (slots k0 + 32 p + lane, p < IPT; idle slots copy the last due one)
// against the j-records [j0, j1), staged through shared memory in tiles of
// FUSED_TILE records (double-buffered: the next tile's loads are in flight
// during the arithmetic). A tile is stored as j-pairs, the values of records
// 2q and 2q + 1 side by side, so that the pair terms of two j run in one
// packed FP32x2 instruction (__fadd2_rn / __fmul2_rn / __ffma2_rn; each lane
// holds its due particles in both halves). The CTA's eight warps hold the same
// slots and split every tile (warp w takes pairs w, w + 8, ...), so no lane
// sums have to meet in a shuffle tree; FP32 sums (about 128 terms per half)
// are folded into double-single totals, and the warps' totals are added in
// fixed order through shared memory: one partial per (slot, chunk).
constexpr int FUSED_TILE = 256;
constexpr int FUSED_IB = 64;        // most due slots per tile item (two per lane)
// Due sets of at least FUSED_IPT2_NA particles take items of two due slots per lane
// (64 per item: half the shared-memory reads per pair term, two independent chains);
// smaller ones one slot per lane (32 per item: more items to spread over the CTAs).
constexpr int FUSED_IPT2_NA = 256;
constexpr int FUSED_TILE_FOLD = 8;  // tiles per FP32 partial sum (8 x 16 terms per half)

template <bool DS, int IPT>
__device__ __forceinline__ void tile_item(const FusedArgs &a, int na, int k0, int j0, int j1,
                                          int chunk, float4 (*s_tile)[DS_REC * FUSED_TILE])
{
    constexpr int NT = FUSED_THREADS, NW = NT / 32, PF = (DS_REC * FUSED_TILE + NT - 1) / NT;
    constexpr int NPAIR = FUSED_TILE / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the lane's due particles (slots k0 + 32 p + lane), negated, in both halves
    float2 nxh[IPT], nyh[IPT], nzh[IPT], nxl[IPT], nyl[IPT], nzl[IPT], nvx[IPT], nvy[IPT],
        nvz[IPT];
    int iid[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
        const float4 *ir = a.irec + (size_t)DS_REC * min(k0 + 32 * p + lane, na - 1);
        const float4 I0 = __ldcg(ir), I1 = __ldcg(ir + 1), I2 = __ldcg(ir + 2);
        nxh[p] = make_float2(-I0.x, -I0.x);
        nyh[p] = make_float2(-I0.y, -I0.y);
        nzh[p] = make_float2(-I0.z, -I0.z);
        nxl[p] = make_float2(-I1.x, -I1.x);
        nyl[p] = make_float2(-I1.y, -I1.y);
        nzl[p] = make_float2(-I1.z, -I1.z);
        nvx[p] = make_float2(-I2.x, -I2.x);
        nvy[p] = make_float2(-I2.y, -I2.y);
        nvz[p] = make_float2(-I2.z, -I2.z);
        iid[p] = __float_as_int(I1.w);
    }
    const float2 e2 = make_float2(a.eps2f, a.eps2f);
    float A_h[IPT][3], A_l[IPT][3], J_h[IPT][3], J_l[IPT][3], P_h[IPT], P_l[IPT];
    float2 ta[IPT][3], tja[IPT][3], tjb[IPT][3], tp[IPT];
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            A_h[p][c] = A_l[p][c] = J_h[p][c] = J_l[p][c] = 0.f;
            ta[p][c] = tja[p][c] = tjb[p][c] = make_float2(0.f, 0.f);
        }
        P_h[p] = P_l[p] = 0.f;
        tp[p] = make_float2(0.f, 0.f);
    }
    const float4 *jr = a.s.rec;
    const int ntile = (j1 - j0 + FUSED_TILE - 1) / FUSED_TILE;
    float4 pf[PF];
    auto fetch = [&](int t) {
        const int tb = j0 + t * FUSED_TILE;
        const int m = DS_REC * min(FUSED_TILE, j1 - tb);
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int q = tid + u * NT;
            pf[u] = q < m ? __ldcg(jr + (size_t)DS_REC * tb + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    // float4 part p of record r goes to the pair layout: {p.x of 2q, p.x of 2q+1,
    // p.y of 2q, p.y of 2q+1} and {p.z ..., p.w ...} at float4 6q + 2p, 6q + 2p + 1
    auto stash = [&](int buf) {
        float *P = reinterpret_cast<float *>(s_tile[buf]);
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int q = tid + u * NT;
            if (q < DS_REC * FUSED_TILE) {
                const int r = q / DS_REC, part = q % DS_REC, h = r & 1;
                float *d = P + 4 * (6 * (r >> 1) + 2 * part);
                d[h] = pf[u].x;
                d[2 + h] = pf[u].y;
                d[4 + h] = pf[u].z;
                d[6 + h] = pf[u].w;
            }
        }
    };
    __syncthreads();  // the buffers are free (a previous item may still read them)
    fetch(0);
    stash(0);
    __syncthreads();
    for (int t = 0; t < ntile; ++t) {
        const int tb = j0 + t * FUSED_TILE;
        const int cnt = min(FUSED_TILE, j1 - tb);
        if (t + 1 < ntile) fetch(t + 1);
        const float4 *T = s_tile[t & 1];
        // a tile with a lane's own particle or a ragged end masks per half (warp-uniform)
        bool own = false;
#pragma unroll
        for (int p = 0; p < IPT; ++p) own = own || (iid[p] >= tb && iid[p] < tb + cnt);
        const bool masked = __any_sync(0xffffffffu, own) || cnt < FUSED_TILE;
        auto body = [&](int q, bool msk) {
            const float4 *P = T + 6 * q;
            const float4 q0 = P[0], q1 = P[1], q4 = P[4], q5 = P[5];
            float4 q2, q3;
            if (DS) {
                q2 = P[2];
                q3 = P[3];
            }
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
                float2 dx, dy, dz;
                if (DS) {
                    dx = __fadd2_rn(__fadd2_rn(make_float2(q0.x, q0.y), nxh[p]),
                                    __fadd2_rn(make_float2(q2.x, q2.y), nxl[p]));
                    dy = __fadd2_rn(__fadd2_rn(make_float2(q0.z, q0.w), nyh[p]),
                                    __fadd2_rn(make_float2(q2.z, q2.w), nyl[p]));
                    dz = __fadd2_rn(__fadd2_rn(make_float2(q1.x, q1.y), nzh[p]),
                                    __fadd2_rn(make_float2(q3.x, q3.y), nzl[p]));
                } else {
                    dx = __fadd2_rn(make_float2(q0.x, q0.y), nxh[p]);
                    dy = __fadd2_rn(make_float2(q0.z, q0.w), nyh[p]);
                    dz = __fadd2_rn(make_float2(q1.x, q1.y), nzh[p]);
                }
                const float2 dvx = __fadd2_rn(make_float2(q4.x, q4.y), nvx[p]);
                const float2 dvy = __fadd2_rn(make_float2(q4.z, q4.w), nvy[p]);
                const float2 dvz = __fadd2_rn(make_float2(q5.x, q5.y), nvz[p]);
                float2 r2 = __ffma2_rn(dx, dx, e2);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                float2 rv = __fmul2_rn(dx, dvx);
                rv = __ffma2_rn(dy, dvy, rv);
                rv = __ffma2_rn(dz, dvz, rv);
                float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                if (msk) {
                    const int ja = tb + 2 * q;  // the self pair and records past the end: nothing
                    rinv.x = (ja == iid[p] || 2 * q >= cnt) ? 0.f : rinv.x;
                    rinv.y = (ja + 1 == iid[p] || 2 * q + 1 >= cnt) ? 0.f : rinv.y;
                }
                const float2 rinv2 = __fmul2_rn(rinv, rinv);
                const float2 mrinv = __fmul2_rn(make_float2(q1.z, q1.w), rinv);
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
        };
        const int npair = (cnt + 1) / 2;
        if (masked) {
            for (int q = warp; q < npair; q += NW) body(q, true);
        } else {
#pragma unroll 2
            for (int q = warp; q < NPAIR; q += NW) body(q, false);
        }
        if ((t + 1) % FUSED_TILE_FOLD == 0 || t + 1 == ntile) {
#pragma unroll
            for (int p = 0; p < IPT; ++p) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float sa = ta[p][c].x + ta[p][c].y;
                    const float jt = fmaf(-3.f, tjb[p][c].x + tjb[p][c].y, tja[p][c].x + tja[p][c].y);
                    if (DS) {
                        ds_add(A_h[p][c], A_l[p][c], sa);
                        ds_add(J_h[p][c], J_l[p][c], jt);
                    } else {
                        A_h[p][c] += sa;
                        J_h[p][c] += jt;
                    }
                    ta[p][c] = tja[p][c] = tjb[p][c] = make_float2(0.f, 0.f);
                }
                const float sp = tp[p].x + tp[p].y;
                if (DS)
                    ds_add(P_h[p], P_l[p], sp);
                else
                    P_h[p] += sp;
                tp[p] = make_float2(0.f, 0.f);
            }
        }
        if (t + 1 < ntile) stash((t + 1) & 1);
        __syncthreads();
    }
    // the warps' totals, added in order 0..7, one group of 32 slots at a time (the tile
    // buffers are free now)
    float2 *s_red = reinterpret_cast<float2 *>(&s_tile[0][0]);  // [NW][7][32]
#pragma unroll
    for (int p = 0; p < IPT; ++p) {
        const float2 mine[7] = {make_float2(A_h[p][0], A_l[p][0]), make_float2(A_h[p][1], A_l[p][1]),
                                make_float2(A_h[p][2], A_l[p][2]), make_float2(J_h[p][0], J_l[p][0]),
                                make_float2(J_h[p][1], J_l[p][1]), make_float2(J_h[p][2], J_l[p][2]),
                                make_float2(P_h[p], P_l[p])};
#pragma unroll
        for (int c = 0; c < 7; ++c) s_red[(warp * 7 + c) * 32 + lane] = mine[c];
        __syncthreads();
        const int k = k0 + 32 * p + lane;
        if (warp == 0 && k < na) {
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                dsf v{mine[c].x, mine[c].y};
#pragma unroll
                for (int w = 1; w < NW; ++w) {
                    const float2 x = s_red[(w * 7 + c) * 32 + lane];
                    ds_acc(v, dsf{x.x, x.y});
                }
                a.part[((size_t)chunk * 7 + c) * na + k] = make_float2(v.hi, v.lo);
            }
        }
        __syncthreads();  // s_red is free for the next group (or the next item's tiles)
    }
}

// The j-chunks of a step with na (> FUSED_SMALL_NA) due particles on n (a
// function of (na, n, grid) only): one round of items over the grid, at most
// FUSED_MAX_CHUNKS chunks (the reduction's lanes hold four each) of at least
// FUSED_TILE j.
constexpr int FUSED_MAX_CHUNKS = 128;

__device__ __forceinline__ void tile_chunking(int na, int n, int grid, int ib, int &nchunk,
                                              int &jc)
{
    const int nib = (na + ib - 1) / ib;
    int nc = max(1, grid / nib);
    nc = max(1, min(min(nc, (n + FUSED_TILE - 1) / FUSED_TILE), FUSED_MAX_CHUNKS));
    jc = (n + nc - 1) / nc;
    jc = (jc + 31) & ~31;
    nchunk = (n + jc - 1) / jc;
}

// ---- small due sets: groups of four due slots, a ticket per group ----------

// An item of a small due set is one group of four due slots (slots 4g ..
// 4g + 3; idle slots copy the last due one) against one j-chunk; the CTA's
// eight warps split the chunk, every lane loads up to SMALL_JPL j-records at
// once before any arithmetic (one L2 round trip per batch), FP32 sums per lane
// meet in a fixed FP32 xor tree per warp, and the warps' sums in a fixed-order
// double-single sum: one double-single partial per (group, chunk) and output
// q = 7 p + component. The CTA that completes a
// group's last chunk (its ticket) sums the group's partials in a fixed order
// and corrects the group's particles, so no grid barrier separates the force
// from the corrector.
constexpr int SMALL_JPL = 2;
constexpr int SMALL_CHUNK_MAX_J = 2048;  // j per small-set chunk: 8 per lane
constexpr int SMALL_Q = 28;  // outputs of a group: 4 slots x 7 components

// The j-chunks of a small due set (a function of (na, n, grid) only): at most one
// item per CTA while the chunks hold at most SMALL_CHUNK_MAX_J j (at most two
// batches per lane), at least 32 j per chunk.
__device__ __forceinline__ void small_chunking(int na, int n, int grid, int &nchunk, int &jc)
{
    const int ng = (na + 3) / 4;
    int nc = max(grid / ng, (n + SMALL_CHUNK_MAX_J - 1) / SMALL_CHUNK_MAX_J);
    nc = max(1, min(nc, (n + 31) / 32));
    jc = (n + nc - 1) / nc;
    jc = (jc + 31) & ~31;
    nchunk = (n + jc - 1) / jc;
}

// Output q of slot k (component c = q % 7; c == 6 is the positive potential sum).
__device__ __forceinline__ void store_out(const Out3 &f, int k, int c, double v, unsigned *err)
{
    if (c < 3)
        f.acc[c * f.ld + k] = v;
    else if (c < 6)
        f.jerk[(c - 3) * f.ld + k] = v;
    else
        f.pot[k] = v = -v;
    if (!isfinite(v)) atomicOr(err, DERR_NONFINITE);
}

// The group's sums (each of SMALL_SUBS threads per output adds a contiguous
// range of chunks in order, all its loads in flight at once; the ranges are
// then added in order) and the corrector of its due particles.
constexpr int SMALL_SUBS = FUSED_THREADS / SMALL_Q;  // 9 ranges per output
// loads in flight per thread: every range of up to 9 x 24 = 216 chunks (the grid's
// 152 and more) in one L2 round trip
constexpr int SMALL_BATCH = 24;

__device__ __forceinline__ void small_finish(const FusedArgs &a, int na, int g, int nchunk,
                                             double tn, float *s_fin)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __threadfence();
    // warps 0..3, lanes 0..2: the start-of-step state of slot 4 g + warp, component
    // lane, requested before the partial sums
    const int k = 4 * g + warp, c = lane;
    const bool mine = warp < 4 && lane < 3 && k < na;
    CState q{};
    int i = 0;
    if (mine) {
        i = __ldcg(a.act + k);
        cstate_load(a.s, i, c, q);
    }
    if (tid < SMALL_SUBS * SMALL_Q) {
        const int o = tid % SMALL_Q, sub = tid / SMALL_Q;
        const int len = (nchunk + SMALL_SUBS - 1) / SMALL_SUBS;
        const int c0 = sub * len, c1 = min(nchunk, c0 + len);
        const float2 *base = a.part + (size_t)g * nchunk * SMALL_Q + o;
        dsf acc{0.f, 0.f};
        for (int cb = c0; cb < c1; cb += SMALL_BATCH) {
            float2 x[SMALL_BATCH];
#pragma unroll
            for (int u = 0; u < SMALL_BATCH; ++u)
                x[u] = cb + u < c1 ? __ldcg(base + (size_t)(cb + u) * SMALL_Q)
                                   : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < SMALL_BATCH; ++u) ds_acc(acc, dsf{x[u].x, x[u].y});
        }
        s_fin[2 * tid] = acc.hi;
        s_fin[2 * tid + 1] = acc.lo;
    }
    __syncthreads();
    double *s_res = reinterpret_cast<double *>(s_fin + 512);  // [28]: acc, jerk, P per slot
    if (tid < SMALL_Q) {
        dsf v{s_fin[2 * tid], s_fin[2 * tid + 1]};
#pragma unroll
        for (int sub = 1; sub < SMALL_SUBS; ++sub) {
            const int r = sub * SMALL_Q + tid;
            ds_acc(v, dsf{s_fin[2 * r], s_fin[2 * r + 1]});
        }
        const double x = ds_to_double(v);
        s_res[tid] = x;
        if (4 * g + tid / 7 < na && !isfinite(x)) atomicOr(a.err, DERR_NONFINITE);
    }
    if (tid == 0) a.cnt[gridDim.x + 2 + g] = 0;  // re-arm the group's ticket
    __syncthreads();
    if (warp < 4) {
        const double a1 = mine ? s_res[7 * warp + c] : 0.0;
        const double j1 = mine ? s_res[7 * warp + 3 + c] : 0.0;
        correct_lanes_pre(a.s, i, k, c, 0, mine, tn, q, a1, j1, a.prm, a.sd, a.err,
                          a.dtmin_hits);
    }
}

template <bool DS>
__device__ __forceinline__ void small_item(const FusedArgs &a, int na, int n, int g, int c,
                                           int nchunk, int jc, double tn, float2 (*s_red)[SMALL_Q],
                                           float *s_fin, int *s_last)
{
    constexpr int G = 4, NW = FUSED_THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float eps2f = a.eps2f;
    float xh[G], yh[G], zh[G], xl[G], yl[G], zl[G], vx[G], vy[G], vz[G];
    int iid[G];
#pragma unroll
    for (int p = 0; p < G; ++p) {
        const int slot = min(4 * g + p, na - 1);
        const float4 *r = a.irec + (size_t)DS_REC * slot;
        const float4 A = __ldcg(r), B = __ldcg(r + 1), C = __ldcg(r + 2);
        xh[p] = A.x; yh[p] = A.y; zh[p] = A.z;
        xl[p] = B.x; yl[p] = B.y; zl[p] = B.z;
        vx[p] = C.x; vy[p] = C.y; vz[p] = C.z;
        iid[p] = __float_as_int(B.w);
    }
    // FP32 sums: per lane over its j (at most SMALL_CHUNK_MAX_J / 256 = 8), then a
    // fixed xor tree over the warp's 32 lanes (at most 256 terms per sum, fewer
    // than the 128-term sequential sums of the tile kernels' folds in error);
    // double-single from the sum over the warps on
    float S[G][7];
#pragma unroll
    for (int p = 0; p < G; ++p)
#pragma unroll
        for (int q = 0; q < 7; ++q) S[p][q] = 0.f;
    const int j0 = c * jc, j1 = min(n, j0 + jc);
    const int per_w = (((j1 - j0) + NW - 1) / NW + 31) & ~31;
    const int wj0 = j0 + warp * per_w, wj1 = min(j1, wj0 + per_w);
    const float4 *jr = a.s.rec;
    for (int jb = wj0; jb < wj1; jb += 32 * SMALL_JPL) {
        float4 A[SMALL_JPL], B[SMALL_JPL], C[SMALL_JPL];
        int jj[SMALL_JPL];
#pragma unroll
        for (int u = 0; u < SMALL_JPL; ++u) {
            const int j = jb + lane + 32 * u;
            jj[u] = j < wj1 ? j : -2;
            if (j < wj1) {
                A[u] = __ldcg(jr + (size_t)DS_REC * j);
                C[u] = __ldcg(jr + (size_t)DS_REC * j + 2);
                B[u] = DS ? __ldcg(jr + (size_t)DS_REC * j + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                A[u] = B[u] = C[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int p = 0; p < G; ++p) {
            float ta0 = 0.f, ta1 = 0.f, ta2 = 0.f, tj0 = 0.f, tj1 = 0.f, tj2 = 0.f, tp = 0.f;
#pragma unroll
            for (int u = 0; u < SMALL_JPL; ++u) {
                float dx, dy, dz;
                if (DS) {
                    dx = (A[u].x - xh[p]) + (B[u].x - xl[p]);
                    dy = (A[u].y - yh[p]) + (B[u].y - yl[p]);
                    dz = (A[u].z - zh[p]) + (B[u].z - zl[p]);
                } else {
                    dx = A[u].x - xh[p];
                    dy = A[u].y - yh[p];
                    dz = A[u].z - zh[p];
                }
                const float dvx = C[u].x - vx[p], dvy = C[u].y - vy[p], dvz = C[u].z - vz[p];
                float r2 = fmaf(dx, dx, eps2f);
                r2 = fmaf(dy, dy, r2);
                r2 = fmaf(dz, dz, r2);
                float rv = dx * dvx;
                rv = fmaf(dy, dvy, rv);
                rv = fmaf(dz, dvz, rv);
                float rinv = rsqrtf(r2);
                // the self pair and the padding slots (jj -2) contribute nothing
                rinv = (jj[u] == iid[p] || jj[u] < 0) ? 0.f : rinv;
                const float rinv2 = rinv * rinv;
                const float mrinv = A[u].w * rinv;
                const float mr3 = mrinv * rinv2;
                const float beta = -3.f * ((mr3 * rinv2) * rv);
                tp += mrinv;
                ta0 = fmaf(mr3, dx, ta0);
                ta1 = fmaf(mr3, dy, ta1);
                ta2 = fmaf(mr3, dz, ta2);
                tj0 = fmaf(beta, dx, fmaf(mr3, dvx, tj0));
                tj1 = fmaf(beta, dy, fmaf(mr3, dvy, tj1));
                tj2 = fmaf(beta, dz, fmaf(mr3, dvz, tj2));
            }
            S[p][0] += ta0;
            S[p][1] += ta1;
            S[p][2] += ta2;
            S[p][3] += tj0;
            S[p][4] += tj1;
            S[p][5] += tj2;
            S[p][6] += tp;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int p = 0; p < G; ++p)
#pragma unroll
            for (int q = 0; q < 7; ++q) S[p][q] += __shfl_xor_sync(0xffffffffu, S[p][q], o);
    if (lane == 0) {
#pragma unroll
        for (int p = 0; p < G; ++p)
#pragma unroll
            for (int q = 0; q < 7; ++q) s_red[warp][p * 7 + q] = make_float2(S[p][q], 0.f);
    }
    __syncthreads();
    if (tid < SMALL_Q) {
        dsf v{s_red[0][tid].x, s_red[0][tid].y};
#pragma unroll
        for (int w = 1; w < NW; ++w) ds_acc(v, dsf{s_red[w][tid].x, s_red[w][tid].y});
        a.part[((size_t)g * nchunk + c) * SMALL_Q + tid] = make_float2(v.hi, v.lo);
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) *s_last = (atomicAdd(a.cnt + gridDim.x + 2 + g, 1) == nchunk - 1);
    __syncthreads();
    if (*s_last) small_finish(a, na, g, nchunk, tn, s_fin);
    __syncthreads();  // s_red, s_fin and s_last are free for the next item
}

// t_next = next multiple after t_cur of the smallest occupied step; the due
// particles are exactly those whose step divides t_next (every t_i is a
// multiple of dt_i and t_i <= t_cur < t_i + dt_i), so the due count is the
// level histogram's sum over the levels k >= k0. Warp 0 of the CTA; lane 0
// writes s_tn and s_na.
__device__ __forceinline__ void next_block_time(const FusedArgs &a, double t_cur, double &s_tn,
                                                int &s_na)
{
    static_assert(NLEVEL == 64, "two ballot words of levels");
    const int lane = threadIdx.x & 31;
    const int h0 = __ldcg(a.sd->hist + lane);
    const int h1 = __ldcg(a.sd->hist + 32 + lane);
    const unsigned b0 = __ballot_sync(0xffffffffu, h0 > 0);
    const unsigned b1 = __ballot_sync(0xffffffffu, h1 > 0);
    const int kmax = b1 ? 63 - __clz(b1) : (b0 ? 31 - __clz(b0) : 0);
    const double dm = ldexp(a.prm.dt_max, -kmax);
    const double q = floor(t_cur * (1.0 / dm)) + 1.0;
    const unsigned long long qi = q < 9.0e18 ? (unsigned long long)q : 0ull;
    const int k0 = qi ? max(0, kmax - (__ffsll((long long)qi) - 1)) : NLEVEL;
    int c = (lane >= k0 ? h0 : 0) + (lane + 32 >= k0 ? h1 : 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        s_tn = q * dm;
        s_na = c;
    }
}

// Publish the end of a launch: the block time reached and, for a step handed
// to the caller, (epoch, t_next, N_active) in the mailbox like K5 + K1.
__device__ __forceinline__ void publish(const FusedArgs &a, double t_cur, double tn, int na,
                                        unsigned long long epoch)
{
    a.sd->t_cur = t_cur;
    a.sd->n_active = na;
    a.mail->t_next = tn;
    a.mail->n_active = na;
    __threadfence_system();
    a.mail->seq = epoch;
    a.sd->seq = epoch + 1ull;
}

// ---- the hand-off step -----------------------------------------------------

// A step the fused kernel does not take (due set larger than na_max): predict
// every particle to tn (FP64 pos_p, vel_p (and acc_p at order 6) and records),
// then gather the due set in ascending index (act, and at order 4 irec),
// exactly as K5 + K1 would, for the planned kernels the caller runs next.
// Returns false when a grid barrier gave up.
template <int ORD>
__device__ __forceinline__ bool handoff_predict_gather(const FusedArgs &a, double tn, int p0,
                                                       int p1, int nwords, unsigned *s_flags,
                                                       int *s_woff, int *s_wsum, int &s_total,
                                                       int &s_base, unsigned &gen)
{
    constexpr int NT = FUSED_THREADS, NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, bid = blockIdx.x;
    const StateDev &s = a.s;
    for (int w0 = 0; w0 < nwords; w0 += NW) {
        const int i = p0 + w0 * 32 + tid;
        bool due = false;
        if (i < p1) {
            if (ORD == 6) {
                due = predict6_one<true>(s, i, tn);
            } else {
                float4 rec[DS_REC];
                due = predict_one<true>(s, i, tn, rec);
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, due);
        if (lane == 0 && w0 + warp < nwords) s_flags[w0 + warp] = b;
    }
    __syncthreads();
    // word offsets inside the CTA (exclusive scan of the popcounts)
    for (int w0 = 0; w0 < nwords; w0 += NT) {
        const int w = w0 + tid;
        const int v = w < nwords ? __popc(s_flags[w]) : 0;
        const int incl = warp_incl_scan(v);
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int x = lane < NW ? s_wsum[lane] : 0;
            const int xi = warp_incl_scan(x);
            if (lane < NW) s_wsum[lane] = xi - x;
            if (lane == NW - 1) s_total = xi;
        }
        __syncthreads();
        const int carry = (w0 == 0) ? 0 : s_base;  // total of the previous rounds
        if (w < nwords) s_woff[w] = carry + s_wsum[warp] + incl - v;
        __syncthreads();
        if (tid == 0) s_base = carry + s_total;
        __syncthreads();
    }
    if (tid == 0) a.cnt[bid] = nwords > 0 ? s_base : 0;
    if (!grid_barrier(a.bar, gen)) return false;
    // this CTA's offset; gather its due particles
    if (warp == 0) {
        int before = 0;
        for (int q = lane; q < bid; q += 32) before += __ldcg(a.cnt + q);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
        if (lane == 0) s_base = before;
    }
    __syncthreads();
    const int base = s_base;
    for (int w = warp; w < nwords; w += NW) {
        const unsigned b = s_flags[w];
        if (b & (1u << lane)) {
            const int i = p0 + w * 32 + lane;
            const int slot = base + s_woff[w] + __popc(b & ((1u << lane) - 1u));
            a.act[slot] = i;
            if (ORD == 4) {
                const float4 *r = s.rec + (size_t)DS_REC * i;
                float4 *g = a.irec + (size_t)DS_REC * slot;
                g[0] = __ldcg(r);
                g[1] = __ldcg(r + 1);
                g[2] = __ldcg(r + 2);
            }
        }
    }
    (void)G;
    return grid_barrier(a.bar, gen);
}

// ---- the kernel ------------------------------------------------------------

template <bool DS>
__global__ void __launch_bounds__(FUSED_THREADS)
    k_fused_steps(FusedArgs a)
{
    constexpr int NT = FUSED_THREADS, NW = NT / 32;
    __shared__ unsigned s_flags[FUSED_MAX_WORDS];
    __shared__ int s_woff[FUSED_MAX_WORDS];
    __shared__ int s_wsum[NW];
    __shared__ int s_total, s_base, s_na, s_last;
    __shared__ double s_tn;
    __shared__ unsigned long long s_hist[32], s_step_ns[32], s_phase[4];
    __shared__ __align__(16) float4 s_tile[2][DS_REC * FUSED_TILE];
    float2(*s_red)[SMALL_Q] = reinterpret_cast<float2(*)[SMALL_Q]>(&s_tile[0][0]);
    float *s_fin = reinterpret_cast<float *>(&s_tile[1][0]);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, bid = blockIdx.x;
    const StateDev &s = a.s;
    const int n = s.n;
    const int per = (n + G - 1) / G;
    const int p0 = min(n, bid * per), p1 = min(n, p0 + per);
    const int nwords = (p1 - p0 + 31) / 32;
    const int total_warps = G * NW;
    int *dcnt = a.cnt + G;  // two due-set counters, used in alternate steps
    unsigned gen = 0;
    int par = 0;
    bool ok = true;
    double t_cur = __ldcg(&a.sd->t_cur);
    const unsigned long long epoch = __ldcg(&a.sd->seq);
    unsigned long long steps = 0;
    double inter = 0.0;
    if (tid < 32) s_hist[tid] = s_step_ns[tid] = 0ull;
    if (tid < 4) s_phase[tid] = 0ull;
    unsigned long long t_mark = 0;  // CTA 0, thread 0: stage boundaries
    if (bid == 0 && tid == 0) t_mark = globaltimer_ns();
    unsigned long long t_step = t_mark;
    auto mark = [&](int ph) {
        if (bid == 0 && tid == 0) {
            const unsigned long long t = globaltimer_ns();
            s_phase[ph] += t - t_mark;
            t_mark = t;
        }
    };

    for (;;) {
        // the next block time and its due count
        if (warp == 0) next_block_time(a, t_cur, s_tn, s_na);
        __syncthreads();
        const double tn = s_tn;
        const int na = s_na;
        if (!(tn <= a.t_end) || na < 1 || na > a.na_max) {
            // hand the step to the caller exactly as the scheduler kernel would
            if (tn <= a.t_end && na >= 1) {
                ok = handoff_predict_gather<4>(a, tn, p0, p1, nwords, s_flags, s_woff, s_wsum,
                                               s_total, s_base, gen);
                mark(0);
                if (!ok) break;
            }
            if (bid == 0 && tid == 0) publish(a, t_cur, tn, na, epoch);
            break;
        }

        // predict every particle of this CTA's range to tn (records only: the
        // corrector recomputes the FP64 prediction of the due ones); the due
        // ones take slots of the due set (in no particular order: each
        // particle's forces do not depend on its slot) with their records
        for (int w0 = 0; w0 < nwords; w0 += 2 * NW) {
            // two particles per thread, both states loaded before any arithmetic
            const int i0 = p0 + w0 * 32 + tid, i1 = i0 + NT;
            PState q0, q1;
            if (i0 < p1) pstate_load(s, i0, q0);
            if (i1 < p1) pstate_load(s, i1, q1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = h ? i1 : i0;
                float4 rec[DS_REC];
                const bool due = i < p1 && predict_rec_from(s, h ? q1 : q0, i, tn, rec);
                const unsigned b = __ballot_sync(0xffffffffu, due);
                if (b) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(dcnt + par, __popc(b));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (due) {
                        const int slot = base + __popc(b & ((1u << lane) - 1u));
                        a.act[slot] = i;
                        float4 *g = a.irec + (size_t)DS_REC * slot;
                        g[0] = rec[0];
                        g[1] = rec[1];
                        g[2] = rec[2];
                    }
                }
            }
        }
        if (!(ok = grid_barrier(a.bar, gen))) break;
        mark(0);
        if (__ldcg(dcnt + par) != na) {  // the histogram and the states disagree
            if (bid == 0 && tid == 0) atomicOr(a.err, DERR_SCHED);
            break;
        }
        if (bid == 0 && tid == 0) dcnt[par ^ 1] = 0;  // the next step's counter

        if (na <= FUSED_SMALL_NA) {
            // force, then (by the CTA that completes a group) reduction + corrector
            int nchunk, jc;
            small_chunking(na, n, G, nchunk, jc);
            const int ng = (na + 3) / 4;
            for (int it = bid; it < ng * nchunk; it += G) {
                const int g = it / nchunk, c = it - g * nchunk;
                small_item<DS>(a, na, n, g, c, nchunk, jc, tn, s_red, s_fin, &s_last);
            }
            mark(1);
        } else {
            // C: pair force, tile items (32 or 64 due slots x one j-chunk)
            const bool two = na >= FUSED_IPT2_NA;
            const int IB = two ? 64 : 32;
            int nchunk, jc;
            tile_chunking(na, n, G, IB, nchunk, jc);
            const int nib = (na + IB - 1) / IB;
            for (int it = bid; it < nib * nchunk; it += G) {
                const int ib = it / nchunk, c = it - ib * nchunk;
                const int j0 = c * jc;
                if (two)
                    tile_item<DS, 2>(a, na, IB * ib, j0, min(n, j0 + jc), c, s_tile);
                else
                    tile_item<DS, 1>(a, na, IB * ib, j0, min(n, j0 + jc), c, s_tile);
            }
            if (!(ok = grid_barrier(a.bar, gen))) break;
            mark(1);
            // D: chunk partials -> acc, jerk, pot (fixed order), then the corrector
            // particle k on CTA k % G, warp k / G: the due set spreads over the SMs
            // (and over each SM's four schedulers) before any SM takes a second
            // particle, so the FP64 correctors do not queue on one SM's FP64 pipes
            for (int k = bid + G * warp; k < na; k += total_warps) {
                // lanes 0..2: the particle's start-of-step state (component = lane),
                // requested with the chunk partials
                const bool mine = lane < 3;
                CState cs{};
                int i = 0;
                if (mine) {
                    i = __ldcg(a.act + k);
                    cstate_load(s, i, lane, cs);
                }
                // lane l holds chunks l, l + 32, l + 64, l + 96, all loaded at once
                constexpr int CPL = FUSED_MAX_CHUNKS / 32;
                float2 x[CPL][7];
#pragma unroll
                for (int u = 0; u < CPL; ++u)
#pragma unroll
                    for (int q = 0; q < 7; ++q) {
                        const int c = lane + 32 * u;
                        x[u][q] = c < nchunk ? __ldcg(a.part + ((size_t)c * 7 + q) * na + k)
                                             : make_float2(0.f, 0.f);
                    }
                dsf v[7];
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    v[q] = dsf{x[0][q].x, x[0][q].y};
#pragma unroll
                    for (int u = 1; u < CPL; ++u) ds_acc(v[q], dsf{x[u][q].x, x[u][q].y});
                }
#pragma unroll
                for (int q = 0; q < 7; ++q)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) ds_acc(v[q], ds_shfl_xor(v[q], o));
                // every lane holds the totals now; lane c takes component c
                double a1 = 0.0, j1 = 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (lane == c) {
                        a1 = ds_to_double(v[c]);
                        j1 = ds_to_double(v[3 + c]);
                    }
                if (lane == 0) {
                    bool fin = true;
#pragma unroll
                    for (int q = 0; q < 7; ++q) fin = fin && isfinite(ds_to_double(v[q]));
                    if (!fin) atomicOr(a.err, DERR_NONFINITE);
                }
                correct_lanes_pre(s, i, k, lane, 0, mine, tn, cs, a1, j1, a.prm, a.sd, a.err,
                                  a.dtmin_hits);
            }
            mark(2);
        }
        if (bid == 0 && tid == 0) {
            ++steps;
            inter += (double)na * (double)n;
            int lg = 0;
            while ((2LL << lg) <= na && lg < 31) ++lg;
            s_hist[lg] += 1ull;
        }
        t_cur = tn;
        par ^= 1;
        if (!(ok = grid_barrier(a.bar, gen))) break;
        if (bid == 0 && tid == 0) {
            const unsigned long long t = globaltimer_ns();
            s_phase[3] += t - t_mark;
            t_mark = t;
            int lg = 0;
            while ((2LL << lg) <= na && lg < 31) ++lg;
            s_step_ns[lg] += t - t_step;
            t_step = t;
        }
    }
    if (!ok && tid == 0) atomicOr(a.err, DERR_TIMEOUT);
    if (bid == 0) {
        __syncthreads();
        if (tid == 0) {
            a.stats->steps += steps;
            a.stats->interactions += inter;
        }
        if (tid < 32) {
            a.stats->active_hist[tid] += s_hist[tid];
            a.stats->step_ns_hist[tid] += s_step_ns[tid];
        }
        if (tid < 4) a.stats->phase_ns[tid] += s_phase[tid];
    }
}

// ---- the 6th-order scheme -----------------------------------------------------

// Small due sets of the 6th-order scheme take the same steps as the 4th-order
// small path: every CTA predicts its particle range (64-byte records: the
// double-single record plus the FP32 predicted acceleration), the due ones
// take slots; groups of four due slots meet j-chunks in items, and the CTA
// that completes a group's last chunk (its ticket) sums the group's partials
// in a fixed order and runs the order-6 corrector. Ten outputs per slot (acc,
// jerk, snap, P); larger due sets are handed to the caller's planned kernels.
constexpr int F6_Q = 40;                          // outputs of a group: 4 slots x 10
constexpr int F6_SUBS = FUSED_THREADS / F6_Q;     // 6 ranges per output
constexpr int F6_JPL = 2;                         // j-records per lane and batch
constexpr int F6_BATCH = 26;  // partial loads in flight: 6 x 26 = 156 chunks in one round trip
constexpr int F6_CHUNK_MAX_J = 8192;              // j per chunk: 32 per lane

// The j-chunks of an order-6 small due set (a function of (na, n, grid) only):
// at most one item per CTA while the chunks hold at most F6_CHUNK_MAX_J j, at
// least 32 j per chunk.
__device__ __forceinline__ void small6_chunking(int na, int n, int grid, int &nchunk, int &jc)
{
    const int ng = (na + 3) / 4;
    int nc = max(grid / ng, (n + F6_CHUNK_MAX_J - 1) / F6_CHUNK_MAX_J);
    nc = max(1, min(nc, (n + 31) / 32));
    jc = (n + nc - 1) / nc;
    jc = (jc + 31) & ~31;
    nchunk = (n + jc - 1) / jc;
}

__device__ __forceinline__ void small6_finish(const FusedArgs &a, int na, int g, int nchunk,
                                              double tn, float *s_fin)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __threadfence();
    // warps 0..3, lanes 0..2: the start-of-step state of slot 4 g + warp, component
    // lane, requested before the partial sums
    const int k = 4 * g + warp, c = lane;
    const bool mine = warp < 4 && lane < 3 && k < na;
    C6State q{};
    int i = 0;
    if (mine) {
        i = __ldcg(a.act + k);
        c6state_load(a.s, i, c, q);
    }
    if (tid < F6_SUBS * F6_Q) {
        const int o = tid % F6_Q, sub = tid / F6_Q;
        const int len = (nchunk + F6_SUBS - 1) / F6_SUBS;
        const int c0 = sub * len, c1 = min(nchunk, c0 + len);
        const float2 *base = a.part + (size_t)g * nchunk * F6_Q + o;
        dsf acc{0.f, 0.f};
        for (int cb = c0; cb < c1; cb += F6_BATCH) {
            float2 x[F6_BATCH];
#pragma unroll
            for (int u = 0; u < F6_BATCH; ++u)
                x[u] = cb + u < c1 ? __ldcg(base + (size_t)(cb + u) * F6_Q)
                                   : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < F6_BATCH; ++u) ds_acc(acc, dsf{x[u].x, x[u].y});
        }
        s_fin[2 * tid] = acc.hi;
        s_fin[2 * tid + 1] = acc.lo;
    }
    __syncthreads();
    double *s_res = reinterpret_cast<double *>(s_fin + 2 * F6_SUBS * F6_Q);  // [40]
    if (tid < F6_Q) {
        dsf v{s_fin[2 * tid], s_fin[2 * tid + 1]};
#pragma unroll
        for (int sub = 1; sub < F6_SUBS; ++sub) {
            const int r = sub * F6_Q + tid;
            ds_acc(v, dsf{s_fin[2 * r], s_fin[2 * r + 1]});
        }
        const double x = ds_to_double(v);
        s_res[tid] = x;
        if (4 * g + tid / 10 < na && !isfinite(x)) atomicOr(a.err, DERR_NONFINITE);
    }
    if (tid == 0) a.cnt[gridDim.x + 2 + g] = 0;  // re-arm the group's ticket
    __syncthreads();
    if (warp < 4) {
        const double a1 = mine ? s_res[10 * warp + c] : 0.0;
        const double j1 = mine ? s_res[10 * warp + 3 + c] : 0.0;
        const double s1 = mine ? s_res[10 * warp + 6 + c] : 0.0;
        correct6_lanes_pre(a.s, i, k, c, 0, mine, tn, q, a1, j1, s1, a.prm, a.sd, a.err,
                           a.dtmin_hits);
    }
}

// One item: group g (slots 4 g .. 4 g + 3; idle slots repeat the last due one)
// against j-chunk c. The eight warps split the chunk; every lane loads up to
// F6_JPL records before any arithmetic and sums its (at most 32) j in FP32; the
// lanes' sums meet in a fixed FP32 xor tree per warp and the warps' sums in a
// fixed-order double-single sum: one double-single partial per (group, chunk) and output
// q = 10 p + component (component 9: the positive potential sum).
template <bool DS>
__device__ __forceinline__ void small6_item(const FusedArgs &a, int na, int n, int g, int c,
                                            int nchunk, int jc, double tn,
                                            float2 (*s_red)[F6_Q], float4 (*s_i)[DS6_REC],
                                            float *s_fin, int *s_last)
{
    constexpr int G = 4, NW = FUSED_THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float eps2f = a.eps2f;
    // the group's four i-records in shared memory (read back as broadcasts, which
    // keeps the kernel within the registers of two CTAs per SM)
    if (tid < G * DS6_REC) {
        const int i = __ldcg(a.act + min(4 * g + tid / DS6_REC, na - 1));
        s_i[tid / DS6_REC][tid % DS6_REC] = __ldcg(a.s.rec6 + (size_t)DS6_REC * i + tid % DS6_REC);
    }
    __syncthreads();
    int iid[G];
#pragma unroll
    for (int p = 0; p < G; ++p) iid[p] = __float_as_int(s_i[p][1].w);
    // FP32 sums per lane (at most F6_CHUNK_MAX_J / 256 = 32 terms each)
    float t[G][10];
#pragma unroll
    for (int p = 0; p < G; ++p)
#pragma unroll
        for (int q = 0; q < 10; ++q) t[p][q] = 0.f;
    const int j0 = c * jc, j1 = min(n, j0 + jc);
    const int per_w = (((j1 - j0) + NW - 1) / NW + 31) & ~31;
    const int wj0 = j0 + warp * per_w, wj1 = min(j1, wj0 + per_w);
    const float4 *jr = a.s.rec6;
    for (int jb = wj0; jb < wj1; jb += 32 * F6_JPL) {
        float4 A[F6_JPL], B[F6_JPL], C[F6_JPL], D[F6_JPL];
        int jj[F6_JPL];
#pragma unroll
        for (int u = 0; u < F6_JPL; ++u) {
            const int j = jb + lane + 32 * u;
            jj[u] = j < wj1 ? j : -2;
            if (j < wj1) {
                const float4 *r = jr + (size_t)DS6_REC * j;
                A[u] = __ldcg(r);
                C[u] = __ldcg(r + 2);
                D[u] = __ldcg(r + 3);
                B[u] = DS ? __ldcg(r + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                A[u] = B[u] = C[u] = D[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int p = 0; p < G; ++p) {
            const float4 I0 = s_i[p][0], I1 = s_i[p][1], I2 = s_i[p][2], I3 = s_i[p][3];
#pragma unroll
            for (int u = 0; u < F6_JPL; ++u) {
                float dx, dy, dz;
                if (DS) {
                    dx = (A[u].x - I0.x) + (B[u].x - I1.x);
                    dy = (A[u].y - I0.y) + (B[u].y - I1.y);
                    dz = (A[u].z - I0.z) + (B[u].z - I1.z);
                } else {
                    dx = A[u].x - I0.x;
                    dy = A[u].y - I0.y;
                    dz = A[u].z - I0.z;
                }
                const float dvx = C[u].x - I2.x, dvy = C[u].y - I2.y, dvz = C[u].z - I2.z;
                const float dax = D[u].x - I3.x, day = D[u].y - I3.y, daz = D[u].z - I3.z;
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
                // the self pair and the padding slots (jj -2) contribute nothing
                rinv = (jj[u] == iid[p] || jj[u] < 0) ? 0.f : rinv;
                // the order-6 tile kernel's expansion: every term one FMA into its sum
                const float rinv2 = rinv * rinv;
                const float mrinv = A[u].w * rinv;
                const float mr3 = mrinv * rinv2;
                const float r3 = rinv2 * -3.f;
                const float m3a = rv * r3;  // -3 alpha
                const float m3u = w2 * r3;  // -3 (|v|^2 + r.a) / r^2
                const float k1 = m3a * mr3;
                const float c1 = k1 + k1;
                const float c2 = fmaf(m3a, m3a * (5.f / 3.f), m3u) * mr3;
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
        }
    }
    // the lanes' sums in a fixed FP32 xor tree (at most 1024 terms per sum per
    // warp), one slot at a time; double-single from the sum over the warps on
#pragma unroll
    for (int p = 0; p < G; ++p) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 10; ++q) t[p][q] += __shfl_xor_sync(0xffffffffu, t[p][q], o);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 10; ++q) s_red[warp][p * 10 + q] = make_float2(t[p][q], 0.f);
        }
    }
    __syncthreads();
    if (tid < F6_Q) {
        dsf v{s_red[0][tid].x, s_red[0][tid].y};
#pragma unroll
        for (int w = 1; w < NW; ++w) ds_acc(v, dsf{s_red[w][tid].x, s_red[w][tid].y});
        a.part[((size_t)g * nchunk + c) * F6_Q + tid] = make_float2(v.hi, v.lo);
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) *s_last = (atomicAdd(a.cnt + gridDim.x + 2 + g, 1) == nchunk - 1);
    __syncthreads();
    if (*s_last) small6_finish(a, na, g, nchunk, tn, s_fin);
    __syncthreads();  // s_red, s_fin and s_last are free for the next item
}

// The 6th-order fused kernel: the 4th-order kernel's loop with the small path
// only (due sets of up to FUSED6_MAX_NA particles).
template <bool DS>
__global__ void __launch_bounds__(FUSED_THREADS, 1)
    k_fused_steps6(FusedArgs a)
{
    constexpr int NT = FUSED_THREADS, NW = NT / 32;
    __shared__ unsigned s_flags[FUSED_MAX_WORDS];
    __shared__ int s_woff[FUSED_MAX_WORDS];
    __shared__ int s_wsum[NW];
    __shared__ int s_total, s_base, s_na, s_last;
    __shared__ double s_tn;
    __shared__ unsigned long long s_hist[32], s_step_ns[32], s_phase[4];
    __shared__ float2 s_red[NW][F6_Q];
    __shared__ float4 s_i[4][DS6_REC];
    __shared__ __align__(8) float s_fin[2 * F6_SUBS * F6_Q + 2 * F6_Q];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, bid = blockIdx.x;
    const StateDev &s = a.s;
    const int n = s.n;
    const int per = (n + G - 1) / G;
    const int p0 = min(n, bid * per), p1 = min(n, p0 + per);
    const int nwords = (p1 - p0 + 31) / 32;
    int *dcnt = a.cnt + G;  // two due-set counters, used in alternate steps
    unsigned gen = 0;
    int par = 0;
    bool ok = true;
    double t_cur = __ldcg(&a.sd->t_cur);
    const unsigned long long epoch = __ldcg(&a.sd->seq);
    unsigned long long steps = 0;
    double inter = 0.0;
    if (tid < 32) s_hist[tid] = s_step_ns[tid] = 0ull;
    if (tid < 4) s_phase[tid] = 0ull;
    unsigned long long t_mark = 0;  // CTA 0, thread 0: stage boundaries
    if (bid == 0 && tid == 0) t_mark = globaltimer_ns();
    unsigned long long t_step = t_mark;
    auto mark = [&](int ph) {
        if (bid == 0 && tid == 0) {
            const unsigned long long t = globaltimer_ns();
            s_phase[ph] += t - t_mark;
            t_mark = t;
        }
    };

    for (;;) {
        if (warp == 0) next_block_time(a, t_cur, s_tn, s_na);
        __syncthreads();
        const double tn = s_tn;
        const int na = s_na;
        if (!(tn <= a.t_end) || na < 1 || na > a.na_max) {
            if (tn <= a.t_end && na >= 1) {
                ok = handoff_predict_gather<6>(a, tn, p0, p1, nwords, s_flags, s_woff, s_wsum,
                                               s_total, s_base, gen);
                mark(0);
                if (!ok) break;
            }
            if (bid == 0 && tid == 0) publish(a, t_cur, tn, na, epoch);
            break;
        }

        // predict this CTA's range to tn (records only); the due particles take
        // slots of the due set in no particular order
        for (int w0 = 0; w0 < nwords; w0 += 2 * NW) {
            const int i0 = p0 + w0 * 32 + tid, i1 = i0 + NT;
            // two particles per thread, both states loaded before any arithmetic
            PState6 q0, q1;
            if (i0 < p1) pstate6_load(s, i0, q0);
            if (i1 < p1) pstate6_load(s, i1, q1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = h ? i1 : i0;
                const bool due = i < p1 && predict6_rec_from(s, h ? q1 : q0, i, tn);
                const unsigned b = __ballot_sync(0xffffffffu, due);
                if (b) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(dcnt + par, __popc(b));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (due) a.act[base + __popc(b & ((1u << lane) - 1u))] = i;
                }
            }
        }
        if (!(ok = grid_barrier(a.bar, gen))) break;
        mark(0);
        if (__ldcg(dcnt + par) != na) {  // the histogram and the states disagree
            if (bid == 0 && tid == 0) atomicOr(a.err, DERR_SCHED);
            break;
        }
        if (bid == 0 && tid == 0) dcnt[par ^ 1] = 0;  // the next step's counter

        {
            int nchunk, jc;
            small6_chunking(na, n, G, nchunk, jc);
            const int ng = (na + 3) / 4;
            for (int it = bid; it < ng * nchunk; it += G) {
                const int g = it / nchunk, c = it - g * nchunk;
                small6_item<DS>(a, na, n, g, c, nchunk, jc, tn, s_red, s_i, s_fin, &s_last);
            }
            mark(1);
        }
        if (bid == 0 && tid == 0) {
            ++steps;
            inter += (double)na * (double)n;
            int lg = 0;
            while ((2LL << lg) <= na && lg < 31) ++lg;
            s_hist[lg] += 1ull;
        }
        t_cur = tn;
        par ^= 1;
        if (!(ok = grid_barrier(a.bar, gen))) break;
        if (bid == 0 && tid == 0) {
            const unsigned long long t = globaltimer_ns();
            s_phase[3] += t - t_mark;
            t_mark = t;
            int lg = 0;
            while ((2LL << lg) <= na && lg < 31) ++lg;
            s_step_ns[lg] += t - t_step;
            t_step = t;
        }
    }
    if (!ok && tid == 0) atomicOr(a.err, DERR_TIMEOUT);
    if (bid == 0) {
        __syncthreads();
        if (tid == 0) {
            a.stats->steps += steps;
            a.stats->interactions += inter;
        }
        if (tid < 32) {
            a.stats->active_hist[tid] += s_hist[tid];
            a.stats->step_ns_hist[tid] += s_step_ns[tid];
        }
        if (tid < 4) a.stats->phase_ns[tid] += s_phase[tid];
    }
}

// Self-check of the bounded grid barrier: CTA 0 never arrives, the others give
// up after limit_ns, raise the abort flag and report DERR_TIMEOUT.
__global__ void k_selftest_barrier(unsigned *bar, unsigned *err, unsigned long long limit_ns)
{
    unsigned gen = 0;
    if (blockIdx.x == 0) return;
    if (!grid_barrier(bar, gen, limit_ns) && threadIdx.x == 0) atomicOr(err, DERR_TIMEOUT);
}

cudaError_t launch_selftest_barrier(unsigned *bar, unsigned *err, unsigned long long limit_ns,
                                    cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&bar, &err, &limit_ns};
    return cudaLaunchCooperativeKernel((const void *)k_selftest_barrier, 4, 64, args, 0, st);
}

int fused_grid(int device, int order)
{
    int coop = 0, sms = 0, per = 0;
    const void *fn = order == 6 ? (const void *)k_fused_steps6<true>
                                : (const void *)k_fused_steps<true>;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, FUSED_THREADS, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (!coop || per < 1) return 0;
    return sms * (per >= 2 ? 2 : 1);
}

size_t fused_part_float2s(int grid, int na_max, int order)
{
    if (order == 6) {
        // groups <= FUSED6_MAX_NA / 4, chunks <= max(G, n / 8192 + 1) <= 4 G + 1
        return (size_t)(FUSED6_MAX_NA / 4) * (4 * (size_t)grid + 2) * F6_Q;
    }
    // tile items: nchunk * na <= FUSED_MAX_CHUNKS * FUSED_IB for one i-block, else
    // (G / nib) * na <= G * FUSED_IB; small sets: ng * nchunk * 28 with ng <= 4 and
    // nchunk <= max(G, n / 2048 + 1) <= 4 G + 1 (n <= 8192 G)
    const size_t g = (size_t)grid;
    size_t need = 7 * (g * FUSED_IB + (size_t)FUSED_MAX_CHUNKS * FUSED_IB + 64);
    const size_t small = (size_t)(FUSED_SMALL_NA / 4) * (4 * g + 2) * SMALL_Q;
    if (small > need) need = small;
    (void)na_max;
    return need;
}

cudaError_t launch_fused_steps(const FusedArgs &a, int grid, bool ds, int order, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(a.bar, 0, 3 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    // the due-set counters and the group tickets
    e = cudaMemsetAsync(a.cnt + grid, 0, (fused_cnt_ints(grid) - grid) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    FusedArgs copy = a;
    void *args[] = {&copy};
    const void *fn;
    if (order == 6)
        fn = ds ? (const void *)k_fused_steps6<true> : (const void *)k_fused_steps6<false>;
    else
        fn = ds ? (const void *)k_fused_steps<true> : (const void *)k_fused_steps<false>;
    return cudaLaunchCooperativeKernel(fn, grid, FUSED_THREADS, args, 0, st);
}

}  // namespace nb
