// qbf_batched.cu -- many independent QUBOs of uneven n in one persistent pass.
//
// Work split (Section 3.1, applied across instances).  Instance i is walked
// with ns_i suffix bits per lane and 2^(n_i - ns_i) prefixes; prefixes are
// grouped into work items of 32 (one warp), and the items of all instances form
// one global queue.  A persistent grid of 4-warp CTAs pulls items with an
// atomic counter; each warp keeps the current instance's int32 image (S, lin)
// and its in-block corrections in its own slice of shared memory and reloads
// them only when it moves to another instance.  ns_i is the same for all large
// instances, so items cost about the same and the tail is one item.  An item
// of an instance whose fixed-point image fits 2^23 runs the deferred-correction
// walk (qbf_walk_defer_core.cuh; AUTO) or the two-pipe walk, the others the
// int32 walk.
//
// Certification per instance is the single-instance rule (qbf_select.cu):
// every item whose minimum is within W_i of instance i's minimum is re-walked,
// its states <= gmin_i + W_i become candidates (instance, natural index), each
// candidate is rescored in FP64 canonical order (float Q) or exact int64, and
// the per-instance lexicographic minimum (value, index) is found with two
// order-preserving 64-bit atomicMin passes (value first, then index among the
// states with that value), so the answer does not depend on emission order.
//
// The whole sequence -- descriptor upload, reset, prepare, tables, MIN walk,
// flags, EMIT walk, rescoring, argmin, result download -- is captured once in a
// CUDA graph per batch layout and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "qbf.h"
#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"
#include "qbf_walk_core.cuh"
#include "qbf_walk_defer_core.cuh"
#include "qbf_walk_mix_core.cuh"

namespace qbf {

namespace {

constexpr int kBatchThreads = 128;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchR = kRMax;
// the table-driven deferred walk's block: 2^7 = 128 steps (its seventh field
// from the lane's shared memory, as in the single-solve kernel)
constexpr int kBatchDeferR = 7;
constexpr int kBatchMaxNS = 18;
constexpr int kBatchDefaultNS = 18;  // suffix bits per lane when nothing is tuned
constexpr double kTuneMargin = 0.02; // a tuned choice must beat the default by 2%
constexpr int kBatchMinN = 11;  // smallest walk dimension: ns >= R and 32 prefixes per item
// per warp: a 16-byte aligned head -- the correction records of the two-pipe
// walk (128 x int4), or for the table-driven deferred walk the double buffer
// of F values (2 x 128 floats), the group terms of the mid variables (at most
// (kBatchMaxNS - 3 - kBatchDeferR) x 16 floats) and the lanes' seventh field
// (32 lanes x 2 x 16 bytes) -- then S, lin, K and the lane parts of the fields
constexpr int kWarpHeadInts = 640;
static_assert(2 * (1 << kBatchDeferR) + (kBatchMaxNS - 3 - kBatchDeferR) * 16 + 32 * 8 <=
                  kWarpHeadInts,
              "deferred-walk head of the warp slice");
constexpr int kWarpSmemInts =
    (kWarpHeadInts + QBF_BATCH_MAX_N * QBF_BATCH_MAX_N + QBF_BATCH_MAX_N + 128 +
     2 * (kBatchMaxNS - kBatchR) * 32 + 3) & ~3;
constexpr unsigned long long kBatchCandCap = 1ull << 20;
// resident CTAs per SM asked of the table-driven deferred MIN kernel (bounded
// by the 43.6 KB of shared memory per CTA: five fit in 228 KB)
constexpr int kBatchDeferCtas = 5;

// per-instance certification details, filled on the device (qbf_batch_info)
struct BatchInfoDev {
    double error_bound;
    unsigned long long ncand;
    int sigma;
    int walk;
};

struct BatchArgs {
    const BatchDesc *desc;
    int count;
    const Plan *plans;
    const Rec *recs;
    const int *K;
    unsigned long long total_items;
    int *item_min;
    unsigned *item_mask;  // per item: lanes whose minimum is within the window
                          // of the item's minimum (the only ones EMIT walks)
    int *gmin;
    const unsigned *flagged;
    Counters *ctr;
    unsigned long long *cand_idx;
    unsigned *cand_inst;
    unsigned long long cap;
    const float *ftab;  // suffix tables of the table-driven deferred walk
    const volatile int *cancel;  // nullptr, or the cancellation word
    int mix;  // MIN walk for instances whose image fits 2^23: 0 none (int32),
              // 1 the two-pipe walk, 2 the deferred-correction walk
};



__device__ __forceinline__ void emit_candidate(const BatchArgs &a, unsigned long long idx, int inst)
{
    const unsigned long long pos = atomicAdd(&a.ctr->cand, 1ull);
    if (pos < a.cap) {
        a.cand_idx[pos] = idx;
        a.cand_inst[pos] = (unsigned)inst;
    }
}

__device__ __forceinline__ int find_instance(const BatchDesc *d, int count, unsigned long long g)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].item_off <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// MIXK: the MIN walk of instances whose image fits 2^23 (a.mix): 0 none
// (int32 throughout; also the EMIT pass), 1 the two-pipe walk, 2 the
// table-driven deferred walk.  One instantiation per form keeps the register
// count of each to what its own paths need.
template <int MODE, int MIXK>
__global__ void __launch_bounds__(kBatchThreads, (MODE == kModeMin && MIXK == 2) ? kBatchDeferCtas : 1)
    batched_walk_kernel(BatchArgs a)
{
    __shared__ __align__(16) int sm[kBatchWarps][kWarpSmemInts];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int4 *sKx = reinterpret_cast<int4 *>(sm[w]);
    int *sS = sm[w] + kWarpHeadInts;
    int *sLin = sS, *sK = sS, *sC = sS;
    int cur = -1, n = 0, ns = 0, tau = 0, ok = 0, exact = 0, use_mix = 0;
    long long win = 0;
    unsigned long long nprefix = 0, item_off = 0;
    const int4 *rec4 = nullptr;
    const float *ftab_i = nullptr;
    // EMIT: each flagged item is 2^sx work units, so that a few flagged items
    // still spread over the grid (at least four units per resident warp,
    // while an item's prefixes split into at most 2^10 sub-walks)
    int sx = 0;
    if (MODE == kModeEmit) {
        const unsigned long long fl = a.ctr->flagged;
        const unsigned long long want = 4ull * gridDim.x * kBatchWarps;
        while (sx < 5 && (fl << sx) < want)
            ++sx;
    }
    const unsigned long long total =
        (MODE == kModeMin) ? a.total_items : ((unsigned long long)a.ctr->flagged << sx);

    while (true) {
        unsigned long long g = 0;
        if (lane == 0) {
            g = atomicAdd(&a.ctr->items[MODE], 1ull);
            if (cancelled(a.cancel))  // qbf_cancel: take no more items
                g = total;
        }
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= total)
            break;
        const unsigned long long gi =
            (MODE == kModeMin) ? g : (unsigned long long)a.flagged[g >> sx];
        const int inst = find_instance(a.desc, a.count, gi);
        if (inst != cur) {
            __syncwarp();
            const BatchDesc d = a.desc[inst];
            const Plan *plan = a.plans + inst;
            n = d.n;
            ns = d.ns;
            nprefix = d.nprefix;
            item_off = d.item_off;
            rec4 = reinterpret_cast<const int4 *>(a.recs + d.rec_off);
            ftab_i = (MIXK == 2 && d.ftab_off != ~0ull) ? a.ftab + d.ftab_off : nullptr;
            ok = (plan->status == QBF_OK);
            sLin = sS + n * n;
            sK = sLin + n;
            sC = sK + 128;
            for (int e = lane; e < n * n; e += 32)
                sS[e] = plan->S[e];
            for (int e = lane; e < n; e += 32)
                sLin[e] = plan->lin[e];
            for (int e = lane; e < 128; e += 32) {
                const int k = a.K[inst * 128 + e];
                const int kf = __float_as_int((float)k);  // exact when the image fits 2^23
                sK[e] = k;
                if (MIXK == 1)
                    sKx[e] = make_int4(kf, kf, k, 0);
            }
            if (MODE == kModeMin && MIXK == 2 && ftab_i) {
                // the table-driven deferred walk: the head of the slice holds
                // the warp's double buffer of F values, then the group terms
                // of every mid variable, both directions
                __syncwarp();
                const int nsw = ns - 3;
                float4 *sE = reinterpret_cast<float4 *>(sm[w] + 2 * (1 << kBatchDeferR));
                for (int e = lane; e < (nsw - kBatchDeferR) * 2; e += 32) {
                    const int i = kBatchDeferR + (e >> 1);
                    const float sg = (e & 1) ? 1.f : -1.f;
                    const float s0 = (float)sS[i * n + nsw], s1 = (float)sS[i * n + nsw + 1];
                    const float s2 = (float)sS[i * n + nsw + 2];
                    sE[e * 2] = make_float4(0.f, sg * s0, sg * s1, sg * (s1 + s0));
                    sE[e * 2 + 1] =
                        make_float4(sg * s2, sg * (s2 + s0), sg * (s1 + s2), sg * (s0 + s1 + s2));
                }
            }
            // eight-prefix walks: every partial sum must be exact in FP32, and
            // the lane needs R walked bits below its three group bits
            use_mix = (MODE == kModeMin) && MIXK && ok &&
                      ns >= (MIXK == 2 ? kBatchDeferR : kBatchR) + 3 &&
                      plan->vhat <= (long long)kF32Vmax && (MIXK != 2 || ftab_i);
            win = plan->window;
            if (MODE == kModeEmit && ok) {
                const long long t = (long long)a.gmin[inst] + plan->window;
                tau = (int)(t > (long long)INT_MAX ? (long long)INT_MAX : t);
                exact = (plan->window == 0);
            }
            cur = inst;
            __syncwarp();
        }
        if (!ok)
            continue;
        const unsigned long long pl = (gi - item_off) * 32 + lane;
        const bool active = pl < nprefix;
        const unsigned long long p = active ? pl : 0;
        if constexpr (MODE == kModeMin) {
            int m;
            if (MIXK == 2 && use_mix) {
                constexpr int RD = kBatchDeferR;
                constexpr int kE = 2 * (1 << RD);                     // group terms
                constexpr int kG = kE + (kBatchMaxNS - 3 - RD) * 16;  // seventh fields
                dfr2::Lane<RD> L;
                float *sCf = reinterpret_cast<float *>(sC);
                ulonglong2 *sGFx = reinterpret_cast<ulonglong2 *>(sm[w] + kG);
                dfr2::setup<RD>(L, p, n, ns, sS, sLin, sCf, 32, lane, sGFx);
                m = dfr2::walk_min<RD>(L, ns - 3, ftab_i, reinterpret_cast<float *>(sm[w]), lane,
                                       sCf, 32, lane, reinterpret_cast<const float4 *>(sm[w] + kE),
                                       sGFx);
            } else if (MIXK == 1 && use_mix) {
                mix::Lane<kBatchR> L;
                mix::setup<kBatchR>(L, p, n, ns, sS, sLin, sC, 32, lane);
                m = mix::walk_min_rt<kBatchR>(L, n, ns, rec4, sC, sS, 32, lane, sKx);
            } else {
                unsigned GL[kBatchR];
                const unsigned v = lane_setup<kBatchR>(p, n, ns, sS, sLin, sC, 32, lane, GL);
                m = walk_suffix_min<kBatchR>(v, GL, ns, rec4, sC, 32, lane, SmemK{sK});
            }
            int wm = active ? m : INT_MAX;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                wm = min(wm, __shfl_xor_sync(0xffffffffu, wm, o));
            // tau = gmin + W <= wm + W: only lanes within the window of the
            // item's own minimum can hold a state <= tau
            const unsigned mask =
                __ballot_sync(0xffffffffu, active && (long long)m <= (long long)wm + win);
            if (lane == 0) {
                a.item_min[gi] = wm;
                a.item_mask[gi] = mask;
                atomicMin(&a.gmin[inst], wm);
            }
        } else {
            // EMIT: re-walk only the item's lanes in its mask, each prefix's
            // 2^ns suffix states split into 2^j sub-walks of ns - j bits (its
            // top j suffix variables fixed per sub-walk): the same states,
            // 2^j times shorter per lane.  Unit g takes sub-walks 32 (g mod
            // 2^sx) .. + 31 of every masked prefix, one per lane.  The block
            // records of the ns-bit walk serve the shorter one (its first
            // blocks flip the same variables), and the lane set-up takes the
            // j fixed variables as prefix variables.
            const unsigned mask = a.item_mask[gi];
            const int j = min(5 + sx, ns - kBatchR);
            const int nse = ns - j;
            const unsigned sub = ((unsigned)(g & ((1ull << sx) - 1)) << 5) + (unsigned)lane;
            const bool sub_on = sub < (1u << j);
            if (!__any_sync(0xffffffffu, sub_on))
                continue;  // a short walk has fewer sub-walks than units
            unsigned long long best = ~0ull;
            for (unsigned mm = mask; mm; mm &= mm - 1) {
                const unsigned long long pl = (gi - item_off) * 32 + (unsigned)(__ffs(mm) - 1);
                const unsigned long long ps = (pl << j) | (unsigned long long)(sub_on ? sub : 0);
                unsigned GL[kBatchR];
                const unsigned v = lane_setup<kBatchR>(ps, n, nse, sS, sLin, sC, 32, lane, GL);
                const unsigned long long pbase = ps << nse;
                walk_suffix_visit<kBatchR>(
                    v, GL, nse, rec4, sC, 32, lane, SmemK{sK}, [&](unsigned val, unsigned t) {
                        if ((int)val <= tau && sub_on) {
                            const unsigned long long x =
                                pbase | (unsigned long long)(t ^ (t >> 1));
                            if (exact)
                                best = x < best ? x : best;  // W = 0: the lowest tie wins
                            else
                                emit_candidate(a, x, inst);
                        }
                    });
            }
            if (exact) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
                    best = y < best ? y : best;
                }
                if (lane == 0 && best != ~0ull)
                    emit_candidate(a, best, inst);
            }
        }
    }
}

__global__ void batched_reset_kernel(int count, int *gmin, unsigned long long *best_key,
                                     unsigned long long *best_idx, unsigned *lowest, Counters *ctr,
                                     BatchInfoDev *info)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        info[i].ncand = 0;
        gmin[i] = INT_MAX;
        lowest[i] = 0xFFFFFFFFu;
        best_key[i] = ~0ull;
        best_idx[i] = ~0ull;
    }
    if (i == 0) {
        ctr->gmin = INT_MAX;
        ctr->tau = 0;
        ctr->flagged = 0;
        ctr->lowest = 0xFFFFFFFFu;
        for (int j = 0; j < 4; ++j)
            ctr->items[j] = 0;
        ctr->cand = 0;
        ctr->status = QBF_OK;
    }
}

// Items that can hold a winning state.  With W = 0 (exact values) only the
// lowest such item of an instance is kept: its lowest tied state has the
// lowest natural index of the instance.
__global__ void batched_flag_kernel(const BatchDesc *desc, int count, const Plan *plans,
                                    const int *item_min, const int *gmin,
                                    unsigned long long total_items, unsigned *flagged,
                                    unsigned *lowest, Counters *ctr)
{
    for (unsigned long long g = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         g < total_items; g += (unsigned long long)gridDim.x * blockDim.x) {
        const int inst = find_instance(desc, count, g);
        const Plan *plan = plans + inst;
        if (plan->status != QBF_OK)
            continue;
        const long long tau = (long long)gmin[inst] + plan->window;
        if ((long long)item_min[g] <= tau) {
            if (plan->window == 0)
                atomicMin(&lowest[inst], (unsigned)g);
            else
                flagged[atomicAdd(&ctr->flagged, 1u)] = (unsigned)g;
        }
    }
}

__global__ void batched_lowest_kernel(int count, const unsigned *lowest, unsigned *flagged,
                                      Counters *ctr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count && lowest[i] != 0xFFFFFFFFu)
        flagged[atomicAdd(&ctr->flagged, 1u)] = lowest[i];
}

// order-preserving 64-bit keys
__device__ __forceinline__ unsigned long long key_of_double(double v)
{
    if (v == 0.0)
        v = 0.0;  // -0 and +0 compare equal
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ unsigned long long key_of_int(long long v)
{
    return (unsigned long long)v ^ 0x8000000000000000ull;
}

__device__ __forceinline__ double q_at_b(const void *Q, int dtype, int e)
{
    switch (dtype) {
    case QBF_F64: return static_cast<const double *>(Q)[e];
    case QBF_F32: return (double)static_cast<const float *>(Q)[e];
    case QBF_I32: return (double)static_cast<const int32_t *>(Q)[e];
    default: return (double)static_cast<const int16_t *>(Q)[e];
    }
}

// FP64 canonical order (float Q) or exact int64 (integer Q) over the caller's
// n_src variables; padded variables contribute exact zeros.
// One warp per candidate: lane i forms row i of the canonical sum (Q_ii +
// sum_{j>i, x_j} (Q_ij + Q_ji) in ascending j, as the oracle does), so the
// rows' loads overlap, and lane 0 adds the rows in ascending i: the same
// operations in the same order as a single thread, bit for bit.
__global__ void batched_rescore_kernel(const BatchDesc *desc, const unsigned long long *cand_idx,
                                       const unsigned *cand_inst, const Counters *ctr,
                                       unsigned long long cap, unsigned long long *keys,
                                       unsigned long long *best_key, BatchInfoDev *info)
{
    const unsigned long long count = ctr->cand < cap ? ctr->cand : cap;
    const int lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long e = blockIdx.x * (unsigned long long)(blockDim.x >> 5) +
                                (threadIdx.x >> 5);
         e < count; e += warps) {
        const unsigned inst = cand_inst[e];
        const BatchDesc d = desc[inst];
        const unsigned long long x = cand_idx[e];
        const int n = d.n_src;  // <= 34: rows i = lane and lane + 32
        unsigned long long key;
        if (d.dtype == QBF_I32 || d.dtype == QBF_I16) {
            long long rw[2] = {0, 0};
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                if (i >= n || !((x >> i) & 1ull))
                    continue;
                long long row = (long long)q_at_b(d.Q, d.dtype, i * n + i);
                for (int j = i + 1; j < n; ++j) {
                    const long long a = (long long)q_at_b(d.Q, d.dtype, i * n + j) +
                                        (long long)q_at_b(d.Q, d.dtype, j * n + i);
                    if ((x >> j) & 1ull)
                        row += a;
                }
                rw[h] = row;
            }
            long long acc = 0;
            for (int i = 0; i < n; ++i) {
                const long long r = __shfl_sync(0xffffffffu, (i >> 5) ? rw[1] : rw[0], i & 31);
                if ((x >> i) & 1ull)
                    acc += r;
            }
            key = key_of_int(acc);
        } else {
            double rw[2] = {0.0, 0.0};
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                if (i >= n || !((x >> i) & 1ull))
                    continue;
                double row = q_at_b(d.Q, d.dtype, i * n + i);
                for (int j = i + 1; j < n; ++j) {
                    const double a =
                        __dadd_rn(q_at_b(d.Q, d.dtype, i * n + j), q_at_b(d.Q, d.dtype, j * n + i));
                    if ((x >> j) & 1ull)
                        row = __dadd_rn(row, a);
                }
                rw[h] = row;
            }
            double acc = 0.0;
            for (int i = 0; i < n; ++i) {
                const double r = __shfl_sync(0xffffffffu, (i >> 5) ? rw[1] : rw[0], i & 31);
                if ((x >> i) & 1ull)
                    acc = __dadd_rn(acc, r);
            }
            key = key_of_double(acc);
        }
        if (lane == 0) {
            keys[e] = key;
            atomicMin(&best_key[inst], key);
            atomicAdd(&info[inst].ncand, 1ull);
        }
    }
}


// Suffix tables of the table-driven deferred walk: F(gray(t)) for t <
// 2^(ns - 3) on the instance's image (int64 sums, exact in FP32 since the
// image fits 2^23 whenever the walk uses them).  kFtabSplit CTAs per
// instance, each taking every kFtabSplit-th run of blockDim.x entries.
constexpr int kFtabSplit = 8;
__global__ void batched_ftab_kernel(const BatchDesc *desc, const Plan *plans, float *ftab)
{
    const int inst = blockIdx.x / kFtabSplit, part = blockIdx.x % kFtabSplit;
    const BatchDesc d = desc[inst];
    if (d.ftab_off == ~0ull)
        return;
    const Plan *plan = plans + inst;
    const int n = d.n;
    const unsigned N = 1u << (d.ns - 3);
    float *out = ftab + d.ftab_off;
    for (unsigned t = part * blockDim.x + threadIdx.x; t < N; t += kFtabSplit * blockDim.x) {
        const unsigned x = t ^ (t >> 1);
        long long f = 0;
        for (unsigned r = x; r; r &= r - 1) {
            const int i = __ffs(r) - 1;
            f += plan->lin[i];
            for (unsigned q = r & (r - 1); q; q &= q - 1)
                f += plan->S[i * n + (__ffs(q) - 1)];
        }
        out[t] = (float)f;
    }
}

// sigma, window and MIN walk form of every instance (the walk choice repeats
// the MIN kernel's eligibility test)
__global__ void batched_info_kernel(const BatchDesc *desc, int count, const Plan *plans, int mix,
                                    BatchInfoDev *info)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count)
        return;
    const Plan *plan = plans + i;
    const bool is_int = (desc[i].dtype == QBF_I32 || desc[i].dtype == QBF_I16);
    info[i].sigma = plan->sigma;
    info[i].error_bound = is_int ? 0.0 : plan->error_bound;
    const bool eight = mix && plan->status == QBF_OK &&
                       desc[i].ns >= (mix == 2 ? kBatchDeferR : kBatchR) + 3 &&
                       plan->vhat <= (long long)kF32Vmax;
    info[i].walk = eight ? (mix == 2 ? QBF_VARIANT_SPLIT_DEFER : QBF_VARIANT_SPLIT_MIX)
                         : QBF_VARIANT_SPLIT;
}

__global__ void batched_argmin_kernel(const unsigned long long *cand_idx,
                                      const unsigned *cand_inst, const Counters *ctr,
                                      unsigned long long cap, const unsigned long long *keys,
                                      const unsigned long long *best_key,
                                      unsigned long long *best_idx)
{
    const unsigned long long count = ctr->cand < cap ? ctr->cand : cap;
    for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         e < count; e += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned inst = cand_inst[e];
        if (keys[e] == best_key[inst])
            atomicMin(&best_idx[inst], cand_idx[e]);
    }
}

// ------------------------------------------------------------------------
// host side

struct BLayout {
    size_t desc, plans, K, recs, item_min, item_mask, flagged, gmin, best_key, best_idx, status, lowest,
        ctr, cand_idx, cand_inst, keys, info, ftab, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

BLayout blayout(int count, unsigned long long nrec, unsigned long long items,
                unsigned long long nftab)
{
    BLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = a256(o + bytes);
        return at;
    };
    L.desc = take(sizeof(BatchDesc) * count);
    L.plans = take(sizeof(Plan) * count);
    L.K = take(sizeof(int) * 128 * count);
    L.recs = take(sizeof(Rec) * nrec);
    L.item_min = take(sizeof(int) * items);
    L.item_mask = take(sizeof(unsigned) * items);
    L.flagged = take(sizeof(unsigned) * items);
    L.gmin = take(sizeof(int) * count);
    L.best_key = take(sizeof(unsigned long long) * count);
    L.best_idx = take(sizeof(unsigned long long) * count);
    L.status = take(sizeof(int) * count);
    L.lowest = take(sizeof(unsigned) * count);
    L.ctr = take(sizeof(Counters));
    L.cand_idx = take(sizeof(unsigned long long) * kBatchCandCap);
    L.cand_inst = take(sizeof(unsigned) * kBatchCandCap);
    L.keys = take(sizeof(unsigned long long) * kBatchCandCap);
    L.info = take(sizeof(BatchInfoDev) * count);
    L.ftab = take(sizeof(float) * nftab);
    L.total = o;
    return L;
}

// host staging (pinned): descriptors in, results out
struct BStage {
    size_t desc, best_key, best_idx, status, ctr, info, total;
};

BStage bstage(int count)
{
    BStage S;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = a256(o + bytes);
        return at;
    };
    S.desc = take(sizeof(BatchDesc) * count);
    S.best_key = take(sizeof(unsigned long long) * count);
    S.best_idx = take(sizeof(unsigned long long) * count);
    S.status = take(sizeof(int) * count);
    S.ctr = take(sizeof(Counters));
    S.info = take(sizeof(BatchInfoDev) * count);
    S.total = o;
    return S;
}

struct GraphKey {
    int count;
    int ns_max;
    int mix;
    unsigned long long nrec, items;
    void *dev, *host;
    int grid_min, grid_emit;
    bool operator==(const GraphKey &o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

struct BatchState {
    void *dev = nullptr;
    size_t dev_bytes = 0;
    void *host = nullptr;
    size_t host_bytes = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    GraphKey key;
    bool have_key = false;
    int tuned_ns = 0;
    // qbf_tune's choices per element class (0 float, 1 integer) and n; 0 = none
    int tab_ns[2][QBF_BATCH_MAX_N + 1] = {};
    int tab_ctas[2][QBF_BATCH_MAX_N + 1] = {};
    bool cache_loaded = false;
};

std::mutex g_bmu;
std::vector<BatchState> g_bstate;

// resident CTAs per SM of the MIN kernel of walk form `mix`, or of the EMIT kernel
int walk_bps(int mode, int mix = 0)
{
    int b = 0;
    cudaError_t e;
    if (mode != kModeMin)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batched_walk_kernel<kModeEmit, 0>,
                                                          kBatchThreads, 0);
    else if (mix == 2)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batched_walk_kernel<kModeMin, 2>,
                                                          kBatchThreads, 0);
    else if (mix == 1)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batched_walk_kernel<kModeMin, 1>,
                                                          kBatchThreads, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batched_walk_kernel<kModeMin, 0>,
                                                          kBatchThreads, 0);
    return (e != cudaSuccess || b < 1) ? 1 : b;
}

std::string default_tune_cache()
{
    if (const char *p = getenv("QBF_TUNE_CACHE"))
        if (*p)
            return p;
    if (const char *h = getenv("HOME"))
        if (*h)
            return std::string(h) + "/.cache/qbf_tune.txt";
    return std::string();
}

// device name with spaces replaced by '_' and its SM count
void device_tag(int dev, std::string *name, int *nsm)
{
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, dev);
    for (char *c = prop.name; *c; ++c)
        if (*c == ' ')
            *c = '_';
    *name = prop.name;
    *nsm = prop.multiProcessorCount;
}

// Read the lines of the default tuning cache that match this device; later
// lines win.  A missing or unreadable file leaves the tables empty.
void load_tune_cache(BatchState &B, int dev)
{
    B.cache_loaded = true;
    const std::string path = default_tune_cache();
    if (path.empty())
        return;
    FILE *f = fopen(path.c_str(), "r");
    if (!f)
        return;
    std::string name;
    int nsm = 0;
    device_tag(dev, &name, &nsm);
    char tag[32], dname[256];
    int fnsm, cls, n, ns, ctas;
    double sec;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        if (sscanf(line, "%31s %255s %d %d %d %d %d %lf", tag, dname, &fnsm, &cls, &n, &ns, &ctas,
                   &sec) != 8)
            continue;
        if (strcmp(tag, "qbf-tune-v1") != 0 || name != dname || fnsm != nsm)
            continue;
        if (cls < 0 || cls > 1 || n < 1 || n > QBF_BATCH_MAX_N || ns < kBatchR ||
            ns > kBatchMaxNS || ctas < 1 || ctas > 64)
            continue;
        B.tab_ns[cls][n] = ns;
        B.tab_ctas[cls][n] = ctas;
    }
    fclose(f);
}

#define B_CUDA(call, where)                                                                      \
    do {                                                                                         \
        cudaError_t b_e_ = (call);                                                               \
        if (b_e_ != cudaSuccess)                                                                 \
            return record_error(QBF_ECUDA, (std::string(where) + ": " + cudaGetErrorString(b_e_)).c_str()); \
    } while (0)

int enqueue_batch(BatchState &B, const BLayout &L, const BStage &S, int count,
                  unsigned long long items, int grid_min, int grid_emit, int mix, cudaStream_t s)
{
    char *d = (char *)B.dev;
    char *h = (char *)B.host;
    const BatchDesc *desc = (const BatchDesc *)(d + L.desc);
    Plan *plans = (Plan *)(d + L.plans);
    int *K = (int *)(d + L.K);
    Rec *recs = (Rec *)(d + L.recs);
    Counters *ctr = (Counters *)(d + L.ctr);
    int *gmin = (int *)(d + L.gmin);
    unsigned long long *best_key = (unsigned long long *)(d + L.best_key);
    unsigned long long *best_idx = (unsigned long long *)(d + L.best_idx);

    B_CUDA(cancel_reset_async(s), "clear the cancellation word");
    B_CUDA(cudaMemcpyAsync(d + L.desc, h + S.desc, sizeof(BatchDesc) * count,
                           cudaMemcpyHostToDevice, s),
           "batch descriptors");
    unsigned *lowest = (unsigned *)(d + L.lowest);
    BatchInfoDev *info = (BatchInfoDev *)(d + L.info);
    batched_reset_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, gmin, best_key, best_idx,
                                                             lowest, ctr, info);
    batched_prepare_kernel<<<count, 256, 0, s>>>(desc, plans, (int *)(d + L.status),
                                                 mix ? kF32Vmax : (long long)INT_MAX);
    batched_tables_kernel<<<count, 256, 0, s>>>(desc, plans, recs, K);
    if (mix == 2)
        batched_ftab_kernel<<<count * kFtabSplit, 256, 0, s>>>(desc, plans, (float *)(d + L.ftab));
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.desc = desc;
    a.count = count;
    a.plans = plans;
    a.recs = recs;
    a.K = K;
    a.total_items = items;
    a.item_min = (int *)(d + L.item_min);
    a.item_mask = (unsigned *)(d + L.item_mask);
    a.gmin = gmin;
    a.flagged = (const unsigned *)(d + L.flagged);
    a.ctr = ctr;
    a.cand_idx = (unsigned long long *)(d + L.cand_idx);
    a.cand_inst = (unsigned *)(d + L.cand_inst);
    a.cap = kBatchCandCap;
    a.mix = mix;
    a.ftab = (const float *)(d + L.ftab);
    a.cancel = cancel_word_dev();
    if (mix == 2)
        batched_walk_kernel<kModeMin, 2><<<grid_min, kBatchThreads, 0, s>>>(a);
    else if (mix == 1)
        batched_walk_kernel<kModeMin, 1><<<grid_min, kBatchThreads, 0, s>>>(a);
    else
        batched_walk_kernel<kModeMin, 0><<<grid_min, kBatchThreads, 0, s>>>(a);
    const int fb = (int)std::min<unsigned long long>((items + 255) / 256, 8192);
    batched_flag_kernel<<<fb, 256, 0, s>>>(desc, count, plans, a.item_min, gmin, items,
                                           (unsigned *)(d + L.flagged), lowest, ctr);
    batched_lowest_kernel<<<(count + 255) / 256, 256, 0, s>>>(count, lowest,
                                                              (unsigned *)(d + L.flagged), ctr);
    batched_walk_kernel<kModeEmit, 0><<<grid_emit, kBatchThreads, 0, s>>>(a);
    unsigned long long *keys = (unsigned long long *)(d + L.keys);
    batched_rescore_kernel<<<512, 256, 0, s>>>(desc, a.cand_idx, a.cand_inst, ctr, kBatchCandCap,
                                               keys, best_key, info);
    batched_info_kernel<<<(count + 255) / 256, 256, 0, s>>>(desc, count, plans, mix, info);
    batched_argmin_kernel<<<512, 256, 0, s>>>(a.cand_idx, a.cand_inst, ctr, kBatchCandCap, keys,
                                              best_key, best_idx);
    B_CUDA(cudaGetLastError(), "batched kernels");
    B_CUDA(cudaMemcpyAsync(h + S.best_key, best_key, sizeof(unsigned long long) * count,
                           cudaMemcpyDeviceToHost, s),
           "batch results");
    B_CUDA(cudaMemcpyAsync(h + S.best_idx, best_idx, sizeof(unsigned long long) * count,
                           cudaMemcpyDeviceToHost, s),
           "batch results");
    B_CUDA(cudaMemcpyAsync(h + S.status, d + L.status, sizeof(int) * count, cudaMemcpyDeviceToHost,
                           s),
           "batch status");
    B_CUDA(cudaMemcpyAsync(h + S.ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s),
           "batch counters");
    B_CUDA(cudaMemcpyAsync(h + S.info, info, sizeof(BatchInfoDev) * count, cudaMemcpyDeviceToHost,
                           s),
           "batch info");
    return QBF_OK;
}

int dtsize(int dt)
{
    return dt == QBF_F64 ? 8 : (dt == QBF_F32 || dt == QBF_I32) ? 4 : dt == QBF_I16 ? 2 : 0;
}

}  // namespace

// One batched pass; mix = 1 or 2: float instances take the 2^23 image and every
// instance whose image fits it takes the two-pipe (1) or the
// deferred-correction (2) MIN walk; mix = 0: the int32 walk throughout.
int solve_batched_mode(const void *const *Q, const int *n, const int *dtype, int count,
                       const qbf_options *opt_in, double *min_value, uint64_t *argmin,
                       cudaStream_t s, int *kernel_launches, int mix, qbf_batch_info *info_out,
                       int ctas_override, const BatchItemsOut *items_out)
{
    const NvtxRange range("qbf_solve_batched");
    if (!Q || !n || !dtype || !min_value || !argmin)
        return record_error(QBF_EINVAL, "null pointer argument");
    if (count < 1 || count > QBF_BATCH_MAX_COUNT)
        return record_error(QBF_EINVAL, "count must be in [1, 65536]");
    qbf_options o;
    qbf_default_options(&o);
    if (opt_in)
        o = *opt_in;
    if (o.top_k != 0 && o.top_k != 1)
        return record_error(QBF_ENOTIMPL, "qbf_solve_batched returns the minimum only (top_k = 1)");
    if (o.fix_bits != 0)
        return record_error(QBF_ENOTIMPL, "qbf_solve_batched does not restrict the space");
    if (items_out && (items_out->inst < 0 || items_out->inst >= count || !items_out->n_items ||
                      (items_out->max_items > 0 && !items_out->item_min)))
        return record_error(QBF_EINVAL, "item minima: inst must be in [0, count) and the "
                                        "output pointers non-null");
    std::lock_guard<std::mutex> lk(g_bmu);
    int dev = 0;
    B_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if ((int)g_bstate.size() <= dev)
        g_bstate.resize(dev + 1);
    BatchState &B = g_bstate[dev];
    if (!B.cache_loaded)
        load_tune_cache(B, dev);
    if (o.batch_suffix_bits != 0 &&
        (o.batch_suffix_bits < kBatchR || o.batch_suffix_bits > kBatchMaxNS))
        return record_error(QBF_EINVAL, "batch_suffix_bits must be in [6, 18]");
    const int NS_default = B.tuned_ns > 0 ? B.tuned_ns : kBatchDefaultNS;
    // states per (class, n): the n holding the most states picks the CTAs per SM
    double states_cn[2][QBF_BATCH_MAX_N + 1] = {};

    // plan every instance
    std::vector<BatchDesc> desc(count);
    unsigned long long items = 0, nrec = 0, nftab = 0;
    int ns_max = 0;
    for (int i = 0; i < count; ++i) {
        if (!Q[i])
            return record_error(QBF_EINVAL, ("null Q for instance " + std::to_string(i)).c_str());
        if (n[i] < 1 || n[i] > QBF_BATCH_MAX_N)
            return record_error(QBF_EINVAL,
                                ("instance " + std::to_string(i) + ": n must be in [1, 34]").c_str());
        if (dtsize(dtype[i]) == 0)
            return record_error(QBF_EDTYPE, ("instance " + std::to_string(i) + ": unknown dtype").c_str());
        BatchDesc &d = desc[i];
        d.Q = Q[i];
        d.n_src = n[i];
        d.n = std::max(n[i], kBatchMinN);
        d.dtype = dtype[i];
        const int cls = (dtype[i] == QBF_I32 || dtype[i] == QBF_I16) ? 1 : 0;
        const int NS = o.batch_suffix_bits > 0
                           ? o.batch_suffix_bits
                           : (B.tab_ns[cls][n[i]] > 0 ? B.tab_ns[cls][n[i]] : NS_default);
        states_cn[cls][n[i]] += (double)(1ull << n[i]);
        d.ns = std::max(kBatchR, std::min(NS, d.n - 5));
        d.nprefix = 1ull << (d.n - d.ns);
        d.item_off = items;
        d.rec_off = nrec;
        d.ftab_off = ~0ull;
        items += (d.nprefix + 31) / 32;
        nrec += 1ull << (d.ns - kBatchR);
        if (mix == 2 && d.ns >= kBatchDeferR + 3) {
            // suffix table of the table-driven deferred walk: 2^(ns - 3) floats,
            // a multiple of 64, so every block of it starts 256-byte aligned
            d.ftab_off = nftab;
            nftab += 1ull << (d.ns - 3);
        }
        ns_max = std::max(ns_max, d.ns);
    }
    const BLayout L = blayout(count, nrec, items, nftab);
    const BStage S = bstage(count);
    bool relayout = false;
    if (B.dev_bytes < L.total) {
        if (inject_alloc_failure())
            return record_error(QBF_ECUDA, "cudaMalloc(batch scratch): failure injected by "
                                           "QBF_INJECT_ALLOC_FAILURE");
        B_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
        if (B.dev)
            cudaFree(B.dev);
        B.dev = nullptr;
        B.dev_bytes = 0;
        B_CUDA(cudaMalloc(&B.dev, L.total), "cudaMalloc(batch scratch)");
        B.dev_bytes = L.total;
        relayout = true;
    }
    if (B.host_bytes < S.total) {
        B_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
        if (B.host)
            cudaFreeHost(B.host);
        B.host = nullptr;
        B.host_bytes = 0;
        B_CUDA(cudaMallocHost(&B.host, S.total), "cudaMallocHost(batch staging)");
        B.host_bytes = S.total;
        relayout = true;
    }
    if (!B.cap_stream)
        B_CUDA(cudaStreamCreateWithFlags(&B.cap_stream, cudaStreamNonBlocking), "capture stream");

    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int ctas = ctas_override;
    if (ctas <= 0) {
        int bc = 0, bn = 1;
        for (int c = 0; c < 2; ++c)
            for (int m = 1; m <= QBF_BATCH_MAX_N; ++m)
                if (states_cn[c][m] > states_cn[bc][bn]) {
                    bc = c;
                    bn = m;
                }
        ctas = B.tab_ctas[bc][bn];
    }
    const int bps = walk_bps(kModeMin, mix);
    const int cps = (ctas > 0 && ctas < bps) ? ctas : bps;
    const int grid_min = (int)std::max<unsigned long long>(
        1, std::min<unsigned long long>((unsigned long long)nsm * cps,
                                        (items + kBatchWarps - 1) / kBatchWarps));
    const int grid_emit = nsm * walk_bps(kModeEmit);

    char *h = (char *)B.host;
    // the previous replay may still read the staging buffer: wait for it
    B_CUDA(cudaStreamSynchronize(s), "batch stream");
    cancel_clear();
    memcpy(h + S.desc, desc.data(), sizeof(BatchDesc) * count);

    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.count = count;
    key.ns_max = ns_max;
    key.mix = mix;
    key.nrec = nrec;
    key.items = items;
    key.dev = B.dev;
    key.host = B.host;
    key.grid_min = grid_min;
    key.grid_emit = grid_emit;
    if (relayout || !B.have_key || !(B.key == key) || !B.exec) {
        if (B.exec) {
            cudaGraphExecDestroy(B.exec);
            B.exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        B_CUDA(cudaStreamBeginCapture(B.cap_stream, cudaStreamCaptureModeThreadLocal),
               "begin capture");
        int rc = enqueue_batch(B, L, S, count, items, grid_min, grid_emit, mix, B.cap_stream);
        cudaError_t ce = cudaStreamEndCapture(B.cap_stream, &graph);
        if (rc)
            return rc;
        B_CUDA(ce, "end capture");
        B_CUDA(cudaGraphInstantiate(&B.exec, graph, 0), "graph instantiate");
        cudaGraphDestroy(graph);
        B.key = key;
        B.have_key = true;
    }
    B_CUDA(cudaGraphLaunch(B.exec, s), "graph launch");
    B_CUDA(cudaStreamSynchronize(s), "batched solve");
    if (cancel_requested())
        return record_error(QBF_ECANCELED, "cancelled by qbf_cancel");
    if (kernel_launches)
        *kernel_launches = (mix == 2) ? 12 : 11;

    const unsigned long long *bk = (const unsigned long long *)(h + S.best_key);
    const unsigned long long *bi = (const unsigned long long *)(h + S.best_idx);
    const int *st = (const int *)(h + S.status);
    const Counters *ctr = (const Counters *)(h + S.ctr);
    for (int i = 0; i < count; ++i) {
        if (st[i] != QBF_OK)
            return record_error(st[i], ("instance " + std::to_string(i) +
                                        (st[i] == QBF_ENONFINITE ? ": Q holds NaN or Inf"
                                                                 : ": integer Q too large"))
                                           .c_str());
    }
    if (ctr->cand > kBatchCandCap)
        return record_error(QBF_EOVERFLOW, "more than 2^20 candidate states in the batch");
    for (int i = 0; i < count; ++i) {
        const bool is_int = (dtype[i] == QBF_I32 || dtype[i] == QBF_I16);
        const unsigned long long k = bk[i];
        if (k == ~0ull || bi[i] == ~0ull)
            return record_error(QBF_ECUDA, ("instance " + std::to_string(i) +
                                            ": internal error, no candidate").c_str());
        if (is_int) {
            min_value[i] = (double)(long long)(k ^ 0x8000000000000000ull);
        } else {
            const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
            double v;
            memcpy(&v, &b, sizeof(v));
            min_value[i] = v;
        }
        argmin[i] = bi[i];
    }
    if (info_out) {
        const BatchInfoDev *inf = (const BatchInfoDev *)(h + S.info);
        for (int i = 0; i < count; ++i) {
            info_out[i].error_bound = inf[i].error_bound;
            info_out[i].n_candidates = inf[i].ncand;
            info_out[i].scale_bits = inf[i].sigma;
            info_out[i].suffix_bits = desc[i].ns;
            info_out[i].prefix_bits = desc[i].n - desc[i].ns;
            info_out[i].walk = inf[i].walk;
        }
    }
    if (items_out) {
        const BatchDesc &d = desc[items_out->inst];
        const unsigned long long ni = (d.nprefix + 31) / 32;
        *items_out->n_items = ni;
        const unsigned long long c = std::min(ni, items_out->max_items);
        if (c > 0)
            B_CUDA(cudaMemcpy(items_out->item_min, (const char *)B.dev + L.item_min +
                                                       sizeof(int) * d.item_off,
                              sizeof(int) * c, cudaMemcpyDeviceToHost),
                   "item minima");
    }
    return QBF_OK;
}

// QBF_VARIANT_AUTO / SPLIT_DEFER: the deferred-correction pass, SPLIT_MIX: the
// two-pipe pass; AUTO repeats the batch on the int32 walk (2^31 images) if the
// wider windows of the FP32 images flag more candidates than the buffer holds.
// QBF_VARIANT_SPLIT: the int32 pass.
int solve_batched(const void *const *Q, const int *n, const int *dtype, int count,
                  const qbf_options *opt_in, double *min_value, uint64_t *argmin,
                  cudaStream_t s, int *kernel_launches, qbf_batch_info *info, int ctas_override,
                  const BatchItemsOut *items_out)
{
    const int variant = opt_in ? opt_in->variant : QBF_VARIANT_AUTO;
    if (variant != QBF_VARIANT_AUTO && variant != QBF_VARIANT_SPLIT &&
        variant != QBF_VARIANT_SPLIT_MIX && variant != QBF_VARIANT_SPLIT_DEFER)
        return record_error(QBF_ENOTIMPL,
                            "qbf_solve_batched runs the int32, two-pipe or deferred-correction walk");
    if (variant == QBF_VARIANT_SPLIT)
        return solve_batched_mode(Q, n, dtype, count, opt_in, min_value, argmin, s,
                                  kernel_launches, 0, info, ctas_override, items_out);
    const int rc = solve_batched_mode(Q, n, dtype, count, opt_in, min_value, argmin, s,
                                      kernel_launches, variant == QBF_VARIANT_SPLIT_MIX ? 1 : 2,
                                      info, ctas_override, items_out);
    if (rc == QBF_EOVERFLOW && variant == QBF_VARIANT_AUTO)
        return solve_batched_mode(Q, n, dtype, count, opt_in, min_value, argmin, s,
                                  kernel_launches, 0, info, ctas_override, items_out);
    return rc;
}

int set_tuned_batch_ns(int ns)
{
    std::lock_guard<std::mutex> lk(g_bmu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return record_error(QBF_ECUDA, "cudaGetDevice");
    if ((int)g_bstate.size() <= dev)
        g_bstate.resize(dev + 1);
    g_bstate[dev].tuned_ns = ns;
    return QBF_OK;
}

int release_batched()
{
    std::lock_guard<std::mutex> lk(g_bmu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_bstate.size(); ++d) {
        BatchState &B = g_bstate[d];
        if (!B.dev && !B.host && !B.exec && !B.cap_stream)
            continue;
        cudaSetDevice((int)d);
        cudaDeviceSynchronize();
        if (B.exec)
            cudaGraphExecDestroy(B.exec);
        if (B.cap_stream)
            cudaStreamDestroy(B.cap_stream);
        if (B.dev)
            cudaFree(B.dev);
        if (B.host)
            cudaFreeHost(B.host);
        BatchState keep = BatchState();
        keep.tuned_ns = B.tuned_ns;
        memcpy(keep.tab_ns, B.tab_ns, sizeof(B.tab_ns));
        memcpy(keep.tab_ctas, B.tab_ctas, sizeof(B.tab_ctas));
        keep.cache_loaded = B.cache_loaded;
        B = keep;
    }
    cudaSetDevice(cur);
    return QBF_OK;
}


namespace {

// Synthetic tuning instances: upper triangular, entries from a counter hash
// (splitmix64 finaliser) -- uniform in [-1, 1] for float dtypes, integers in
// [-50, 50] for integer dtypes.  Only the timing depends on them.
__global__ void tune_fill_kernel(void *buf, int n, int dtype, unsigned long long total,
                                 unsigned long long seed)
{
    for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         e < total; e += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long w = e % ((unsigned long long)n * n);
        const int i = (int)(w / n), j = (int)(w % n);
        unsigned long long z = seed + e * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const bool keep = (j >= i);
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
        const int iv = keep ? (int)(z % 101ull) - 50 : 0;
        const double fv = keep ? 2.0 * u - 1.0 : 0.0;
        switch (dtype) {
        case QBF_F64: static_cast<double *>(buf)[e] = fv; break;
        case QBF_F32: static_cast<float *>(buf)[e] = (float)fv; break;
        case QBF_I32: static_cast<int *>(buf)[e] = iv; break;
        default: static_cast<short *>(buf)[e] = (short)iv; break;
        }
    }
}

}  // namespace

// One n of qbf_tune.  A configuration is scored by the time difference between
// a synthetic batch of 2c instances and one of c instances (c = 2^36 / 2^n,
// at least 8 and at most 2048): the difference is the steady-state cost of c
// instances, free of the last partial wave of work items, which in a single
// small launch favours short walks but vanishes in a large mixed batch.  The
// default configuration (kBatchDefaultNS suffix bits, the most CTAs per SM) is
// scored first and kept unless another beats it by kTuneMargin: differences
// below that are within the run-to-run spread of the scores, and a choice
// made on noise alone measured slower in mixed batches.  The suffix widths
// searched are the five widest the instance allows (narrower ones only add
// per-prefix set-up), at the most CTAs per SM; then every CTA count at the
// best width.
static int tune_one_n(int n, int dtype, cudaStream_t s, int *best_ns, int *best_ctas,
                      double *best_sec)
{
    const int esz = dtsize(dtype);
    const unsigned long long c =
        std::max<unsigned long long>(8, std::min<unsigned long long>(2048, (1ull << 36) >> n));
    const unsigned long long count = 2 * c;
    const unsigned long long per = (unsigned long long)n * n;
    void *buf = nullptr;
    B_CUDA(cudaMalloc(&buf, per * count * esz), "cudaMalloc(tuning batch)");
    tune_fill_kernel<<<256, 256, 0, s>>>(buf, n, dtype, per * count, 0x5EEDull + n);
    cudaError_t fe = cudaStreamSynchronize(s);
    if (fe != cudaSuccess) {
        cudaFree(buf);
        return record_error(QBF_ECUDA, "tuning batch fill");
    }
    std::vector<const void *> ptr(count);
    std::vector<int> nn(count, n), dt(count, dtype);
    for (unsigned long long i = 0; i < count; ++i)
        ptr[i] = static_cast<const char *>(buf) + i * per * esz;
    std::vector<double> vmin(count);
    std::vector<uint64_t> am(count);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // best of two timed solves of the first `m` instances (after one that
    // builds the graph of this layout)
    auto time_m = [&](int ns, int ctas, unsigned long long m, double *sec) -> int {
        qbf_options o;
        qbf_default_options(&o);
        o.batch_suffix_bits = ns;
        int r = solve_batched(ptr.data(), nn.data(), dt.data(), (int)m, &o, vmin.data(),
                              am.data(), s, nullptr, nullptr, ctas);
        if (r)
            return r;
        float best = 1e30f;
        for (int k = 0; k < 2; ++k) {
            cudaEventRecord(e0, s);
            r = solve_batched(ptr.data(), nn.data(), dt.data(), (int)m, &o, vmin.data(),
                              am.data(), s, nullptr, nullptr, ctas);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            if (r)
                return r;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, t);
        }
        *sec = best * 1e-3;
        return QBF_OK;
    };
    auto score = [&](int ns, int ctas, double *sec) -> int {
        double t1 = 0, t2 = 0;
        int r = time_m(ns, ctas, c, &t1);
        if (r == QBF_OK)
            r = time_m(ns, ctas, count, &t2);
        *sec = t2 - t1;
        return r;
    };
    int rc = QBF_OK;
    const int bps = walk_bps(kModeMin, 2);  // the AUTO form the tuned solves run
    const int nw = std::max(n, kBatchMinN);
    const int ns_hi = std::max(kBatchR, std::min(kBatchMaxNS, nw - 5));
    const int ns_lo = std::max(kBatchR, ns_hi - 4);
    const int ns_def = std::max(kBatchR, std::min(kBatchDefaultNS, nw - 5));
    double bsec = 1e300;
    int bns = ns_def, bct = bps;
    rc = score(ns_def, bps, &bsec);
    for (int ns = ns_lo; ns <= ns_hi && rc == QBF_OK; ++ns) {
        if (ns == ns_def)
            continue;
        double t = 0;
        rc = score(ns, bps, &t);
        if (rc == QBF_OK && t < bsec * (1.0 - kTuneMargin)) {
            bsec = t;
            bns = ns;
        }
    }
    for (int cc = 1; cc < bps && rc == QBF_OK; ++cc) {
        double t = 0;
        rc = score(bns, cc, &t);
        if (rc == QBF_OK && t < bsec * (1.0 - kTuneMargin)) {
            bsec = t;
            bct = cc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc)
        return rc;
    *best_ns = bns;
    *best_ctas = bct;
    *best_sec = bsec;
    return QBF_OK;
}

int tune_batched_table(int n_min, int n_max, int dtype, const char *cache_path)
{
    if (n_min < 1 || n_max > QBF_BATCH_MAX_N || n_min > n_max)
        return record_error(QBF_EINVAL, "qbf_tune: need 1 <= n_min <= n_max <= 34");
    if (dtsize(dtype) == 0)
        return record_error(QBF_EDTYPE, "qbf_tune: unknown dtype");
    int dev = 0;
    B_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    {
        std::lock_guard<std::mutex> lk(g_bmu);
        if ((int)g_bstate.size() <= dev)
            g_bstate.resize(dev + 1);
        if (!g_bstate[dev].cache_loaded)
            load_tune_cache(g_bstate[dev], dev);
    }
    cudaStream_t s = nullptr;
    B_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "tuning stream");
    const int cls = (dtype == QBF_I32 || dtype == QBF_I16) ? 1 : 0;
    std::string name;
    int nsm = 0;
    device_tag(dev, &name, &nsm);
    std::string lines;
    int rc = QBF_OK;
    for (int n = n_min; n <= n_max && rc == QBF_OK; ++n) {
        int ns = 0, ctas = 0;
        double sec = 0;
        rc = tune_one_n(n, dtype, s, &ns, &ctas, &sec);
        if (rc)
            break;
        {
            std::lock_guard<std::mutex> lk(g_bmu);
            g_bstate[dev].tab_ns[cls][n] = ns;
            g_bstate[dev].tab_ctas[cls][n] = ctas;
        }
        char buf[512];
        snprintf(buf, sizeof(buf), "qbf-tune-v1 %s %d %d %d %d %d %.9f\n", name.c_str(), nsm, cls,
                 n, ns, ctas, sec);
        lines += buf;
    }
    cudaStreamDestroy(s);
    if (rc)
        return rc;
    const std::string path = cache_path ? std::string(cache_path) : default_tune_cache();
    if (!path.empty()) {
        FILE *f = fopen(path.c_str(), "a");
        if (!f)
            return record_error(QBF_EINVAL, ("qbf_tune: cannot write the cache " + path).c_str());
        fputs(lines.c_str(), f);
        fclose(f);
    }
    return QBF_OK;
}

int tuned_params(int n, int dtype, int *suffix_bits, int *ctas_per_sm)
{
    if (!suffix_bits || !ctas_per_sm)
        return record_error(QBF_EINVAL, "null pointer argument");
    if (n < 1 || n > QBF_BATCH_MAX_N || dtsize(dtype) == 0)
        return record_error(QBF_EINVAL, "qbf_tuned_params: n in [1, 34] and a known dtype");
    int dev = 0;
    B_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_bmu);
    if ((int)g_bstate.size() <= dev)
        g_bstate.resize(dev + 1);
    BatchState &B = g_bstate[dev];
    if (!B.cache_loaded)
        load_tune_cache(B, dev);
    const int cls = (dtype == QBF_I32 || dtype == QBF_I16) ? 1 : 0;
    *suffix_bits = B.tab_ns[cls][n];
    *ctas_per_sm = B.tab_ctas[cls][n];
    return QBF_OK;
}

}  // namespace qbf
