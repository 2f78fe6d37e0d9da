// qbf_select.cu -- steps A5-A7: reductions, certification window, rescoring, top-k.
//
// After the MIN walk every prefix p has its exact fixed-point minimum pmin[p]
// and Counters::gmin holds the global one.
//
//   threshold_kernel  tau = (k-th smallest prefix minimum) + W, where W is the
//                     certification window of the Plan (0 for integer Q).
//                     With k = 1 this is gmin + W.  Every state of the FP64
//                     top-k then has a fixed-point value <= tau: the k
//                     smallest prefix minima are k distinct states whose
//                     fixed-point values are <= tau - W.
//   flag_kernel       lists the prefixes with pmin <= tau (or, for a top-1
//                     solve with exact values, W = 0, only the lowest such
//                     prefix: its lowest tied state has the lowest index),
//                     numbered from p_lo.
//   rescore_kernel    evaluates every emitted candidate state from the
//                     caller's Q: the FP64 canonical sum for float Q (the
//                     order every FP64 value in this project uses), the exact
//                     int64 sum for integer Q.
//   select_kernel     the top_k smallest (value, natural index) pairs,
//                     lexicographic, so ties go to the lowest index.
// None of these uses floating-point atomics; the result does not depend on
// the order in which candidates were emitted.
#include <cfloat>
#include <climits>

#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"

namespace qbf {

__global__ void reset_counters_kernel(Counters *c)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->gmin = INT_MAX;
        c->tau = INT_MIN;
        c->flagged = 0;
        c->lowest = 0xFFFFFFFFu;
        for (int i = 0; i < 4; ++i)
            c->items[i] = 0;
        c->cand = 0;
        c->status = QBF_OK;
    }
}


__global__ void __launch_bounds__(1024) threshold_kernel(const Plan *plan, const int *pmin,
                                                         unsigned long long npref, int top_k,
                                                         Counters *c)
{
    if (plan->status != QBF_OK)
        return;
    long long base;
    if (top_k <= 1) {
        base = c->gmin;
    } else if (npref < (unsigned long long)top_k) {
        if (threadIdx.x == 0)
            c->tau = INT_MAX;
        return;
    } else {
        // smallest b with #{p : pmin[p] <= b} >= top_k: the top_k-th smallest
        // prefix minimum, by a radix select on order-preserving keys (the
        // sign bit flipped), 8 bits per pass from the top.  Each pass counts
        // the keys that match the digits chosen so far by their next digit
        // (a warp's equal digits in one shared add); the digit at which the
        // running count reaches the remaining rank is kept.
        __shared__ unsigned hist[256];
        __shared__ unsigned sel[2];  // chosen digit, keys of the group below it
        const int lane = threadIdx.x & 31;
        unsigned prefix = 0, pmask = 0;
        unsigned krem = (unsigned)top_k;  // rank within the matching group, 1-based
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int d = threadIdx.x; d < 256; d += blockDim.x)
                hist[d] = 0;
            __syncthreads();
            for (unsigned long long e0 = 0; e0 < npref; e0 += blockDim.x) {
                const unsigned long long e = e0 + threadIdx.x;
                const unsigned key = e < npref ? ((unsigned)pmin[e] ^ 0x80000000u) : 0u;
                const bool take = e < npref && (key & pmask) == prefix;
                const unsigned m = __ballot_sync(0xffffffffu, take);
                if (take) {
                    const unsigned d = (key >> shift) & 255u;
                    const unsigned peers = __match_any_sync(m, d);
                    if (lane == __ffs(peers) - 1)
                        atomicAdd(&hist[d], (unsigned)__popc(peers));
                }
            }
            __syncthreads();
            if (threadIdx.x < 32) {
                // lane L holds bins 8L .. 8L + 7; an inclusive scan of the lane
                // totals finds the lane, then the lane its bin
                unsigned b8[8], tot = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    b8[q] = hist[lane * 8 + q];
                    tot += b8[q];
                }
                unsigned inc = tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o)
                        inc += y;
                }
                const unsigned below = inc - tot;
                const unsigned hit = __ballot_sync(0xffffffffu, below < krem && inc >= krem);
                if (lane == __ffs(hit) - 1) {
                    unsigned c = below;
                    int q = 0;
                    while (c + b8[q] < krem) {
                        c += b8[q];
                        ++q;
                    }
                    sel[0] = (unsigned)(lane * 8 + q);
                    sel[1] = c;
                }
            }
            __syncthreads();
            prefix |= sel[0] << shift;
            pmask |= 255u << shift;
            krem -= sel[1];
            __syncthreads();  // every thread has read sel before the next pass
        }
        base = (long long)(int)(prefix ^ 0x80000000u);
    }
    if (threadIdx.x == 0) {
        long long t = base + plan->window;
        c->tau = (int)(t > (long long)INT_MAX ? (long long)INT_MAX : t);
    }
}

__global__ void flag_kernel(const Plan *plan, const int *pmin, unsigned long long npref,
                            int top_k, unsigned int *flagged, Counters *c)
{
    if (plan->status != QBF_OK)
        return;
    const int lowest_mode = (top_k == 1 && plan->window == 0);
    const int tau = c->tau;
    for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         e < npref; e += (unsigned long long)gridDim.x * blockDim.x) {
        if (pmin[e] <= tau) {
            // relative to p_lo (e < npref <= 2^28): fixed sub-spaces may sit
            // above 2^32 in absolute prefix numbers
            const unsigned p = (unsigned)e;
            if (lowest_mode)
                atomicMin(&c->lowest, p);
            else
                flagged[atomicAdd(&c->flagged, 1u)] = p;
        }
    }
}

namespace {

__device__ __forceinline__ double q_at(const void *Q, int dtype, int e)
{
    switch (dtype) {
    case QBF_F64: return static_cast<const double *>(Q)[e];
    case QBF_F32: return (double)static_cast<const float *>(Q)[e];
    case QBF_I32: return (double)static_cast<const int32_t *>(Q)[e];
    default: return (double)static_cast<const int16_t *>(Q)[e];
    }
}

__device__ __forceinline__ long long qi_at(const void *Q, int dtype, int e)
{
    return dtype == QBF_I32 ? (long long)static_cast<const int32_t *>(Q)[e]
                            : (long long)static_cast<const int16_t *>(Q)[e];
}

}  // namespace

// FP64 canonical order: acc = 0; for each set i ascending: row = Q_ii, then
// row = row + (Q_ij + Q_ji) for each set j > i ascending; acc = acc + row.
// Every add is an explicit round-to-nearest FP64 add.  The pair sums
// Q_ij + Q_ji (rounded once, as in that order) and the diagonal are staged in
// shared memory per block, so a candidate costs one add per set pair.
__global__ void __launch_bounds__(256) rescore_kernel(const Plan *plan, const void *Q, int n,
                                                      int dtype, const unsigned long long *cand,
                                                      const Counters *c, unsigned long long cap,
                                                      long long *vals)
{
    __shared__ long long sP[kMaxN * kMaxN];  // doubles' bits (float Q) or int64 (integer Q)
    if (plan->status != QBF_OK)
        return;
    const unsigned long long count = c->cand < cap ? c->cand : cap;
    if ((unsigned long long)blockIdx.x * (blockDim.x >> 5) >= count)
        return;  // no candidate for this block (uniform over the block)
    const bool is_int = (dtype == QBF_I32 || dtype == QBF_I16);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        if (j < i)
            continue;
        if (is_int)
            sP[e] = (i == j) ? qi_at(Q, dtype, e) : qi_at(Q, dtype, e) + qi_at(Q, dtype, j * n + i);
        else
            sP[e] = __double_as_longlong(
                (i == j) ? q_at(Q, dtype, e) : __dadd_rn(q_at(Q, dtype, e), q_at(Q, dtype, j * n + i)));
    }
    __syncthreads();
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    if (count > warps) {
        // many candidates: one thread each (throughput)
        for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
             e < count; e += (unsigned long long)gridDim.x * blockDim.x) {
            const unsigned long long x = cand[e];
            if (is_int) {
                long long acc = 0;
                for (int i = 0; i < n; ++i) {
                    if (!((x >> i) & 1ull))
                        continue;
                    long long row = sP[i * n + i];
                    for (int j = i + 1; j < n; ++j)
                        if ((x >> j) & 1ull)
                            row += sP[i * n + j];
                    acc += row;
                }
                vals[e] = acc;
            } else {
                double acc = 0.0;
                for (int i = 0; i < n; ++i) {
                    if (!((x >> i) & 1ull))
                        continue;
                    double row = __longlong_as_double(sP[i * n + i]);
                    for (int j = i + 1; j < n; ++j)
                        if ((x >> j) & 1ull)
                            row = __dadd_rn(row, __longlong_as_double(sP[i * n + j]));
                    acc = __dadd_rn(acc, row);
                }
                vals[e] = __double_as_longlong(acc);
            }
        }
        return;
    }
    // few candidates: one warp each (latency).  Lane i forms rows i and
    // i + 32 of the canonical sum (ascending j), and the rows are added in
    // ascending i: the same operations in the same order as one thread
    const int lane = threadIdx.x & 31;
    for (unsigned long long e = blockIdx.x * (unsigned long long)(blockDim.x >> 5) +
                                (threadIdx.x >> 5);
         e < count; e += warps) {
        const unsigned long long x = cand[e];
        if (is_int) {
            long long rw[2] = {0, 0};
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                if (i >= n || !((x >> i) & 1ull))
                    continue;
                long long row = sP[i * n + i];
                for (int j = i + 1; j < n; ++j)
                    if ((x >> j) & 1ull)
                        row += sP[i * n + j];
                rw[h] = row;
            }
            long long acc = 0;
            for (int i = 0; i < n; ++i) {
                const long long r = __shfl_sync(0xffffffffu, (i >> 5) ? rw[1] : rw[0], i & 31);
                if ((x >> i) & 1ull)
                    acc += r;
            }
            if (lane == 0)
                vals[e] = acc;
        } else {
            double rw[2] = {0.0, 0.0};
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                if (i >= n || !((x >> i) & 1ull))
                    continue;
                double row = __longlong_as_double(sP[i * n + i]);
                for (int j = i + 1; j < n; ++j)
                    if ((x >> j) & 1ull)
                        row = __dadd_rn(row, __longlong_as_double(sP[i * n + j]));
                rw[h] = row;
            }
            double acc = 0.0;
            for (int i = 0; i < n; ++i) {
                const double r = __shfl_sync(0xffffffffu, (i >> 5) ? rw[1] : rw[0], i & 31);
                if ((x >> i) & 1ull)
                    acc = __dadd_rn(acc, r);
            }
            if (lane == 0)
                vals[e] = __double_as_longlong(acc);
        }
    }
}

namespace {

struct Key {
    long long v;  // int64 value, or the bits of a double
    unsigned long long i;
    int ok;
};

__device__ __forceinline__ bool key_less(const Key &a, const Key &b, bool is_int)
{
    if (!a.ok)
        return false;
    if (!b.ok)
        return true;
    if (is_int) {
        if (a.v != b.v)
            return a.v < b.v;
    } else {
        const double x = __longlong_as_double(a.v), y = __longlong_as_double(b.v);
        if (x != y)
            return x < y;
    }
    return a.i < b.i;
}

// warp-wide minimum of keys (a total order: value, then index)
__device__ __forceinline__ Key warp_min_key(Key k, bool is_int)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Key other;
        other.v = __shfl_xor_sync(0xffffffffu, k.v, o);
        other.i = __shfl_xor_sync(0xffffffffu, k.i, o);
        other.ok = __shfl_xor_sync(0xffffffffu, k.ok, o);
        if (key_less(other, k, is_int))
            k = other;
    }
    return k;
}

}  // namespace

constexpr int kSelWarpK = 16;  // top_k up to this: per-warp lists, then one merge

__global__ void __launch_bounds__(1024) select_kernel(const Plan *plan,
                                                      const unsigned long long *cand,
                                                      const long long *vals, const Counters *c,
                                                      unsigned long long cap, int top_k,
                                                      DevResult *res)
{
    __shared__ Key sk[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    if (plan->status != QBF_OK) {
        if (t == 0) {
            res->status = plan->status;
            res->count = 0;
            res->n_candidates = 0;
        }
        return;
    }
    const bool is_int = (plan->dtype == QBF_I32 || plan->dtype == QBF_I16);
    const unsigned long long count = c->cand < cap ? c->cand : cap;
    int r = 0;
    if (top_k <= kSelWarpK) {
        // Each warp takes the top_k smallest of its share of the candidates
        // (lane-strided), one warp-wide minimum per rank, with no block
        // barrier; warp 0 then merges the warps' ascending lists, one head
        // per lane.  The same keys in the same order as the block-wide rounds
        // below, with one barrier instead of three per rank.
        __shared__ Key wl[32][kSelWarpK];
        Key prev;
        prev.ok = 0;
        int got = 0;
        for (; got < top_k; ++got) {
            Key best;
            best.v = 0;
            best.i = 0;
            best.ok = 0;
            for (unsigned long long e = (unsigned long long)wid * 32 + lane; e < count;
                 e += blockDim.x) {
                Key k;
                k.v = vals[e];
                k.i = cand[e];
                k.ok = 1;
                if (prev.ok && !key_less(prev, k, is_int))
                    continue;
                if (key_less(k, best, is_int))
                    best = k;
            }
            best = warp_min_key(best, is_int);
            if (!best.ok)
                break;
            if (lane == 0)
                wl[wid][got] = best;
            prev = best;
        }
        for (int q = got + lane; q < kSelWarpK; q += 32)
            wl[wid][q].ok = 0;  // past the end of this warp's list
        __syncthreads();
        if (wid == 0) {
            int head = 0;  // lane L reads warp L's list
            for (; r < top_k; ++r) {
                Key k;
                k.v = 0;
                k.i = 0;
                k.ok = 0;
                if (lane < nw && head < top_k)
                    k = wl[lane][head];
                const Key w = warp_min_key(k, is_int);
                if (!w.ok)
                    break;
                if (k.ok && k.i == w.i)
                    ++head;  // candidates are distinct states: one lane holds w
                if (lane == 0) {
                    res->topk_value[r] = is_int ? (double)w.v : __longlong_as_double(w.v);
                    res->topk_index[r] = w.i;
                }
            }
            if (lane == 0) {
                res->count = r;
                res->n_candidates = c->cand;
                res->status = (c->cand > cap) ? QBF_EOVERFLOW : QBF_OK;
            }
        }
        return;
    }
    Key prev;
    prev.ok = 0;
    for (; r < top_k; ++r) {
        // the smallest key above the previous winner: per thread, per warp
        // (shuffles), then over the warps (warp 0)
        Key best;
        best.v = 0;
        best.i = 0;
        best.ok = 0;
        for (unsigned long long e = t; e < count; e += blockDim.x) {
            Key k;
            k.v = vals[e];
            k.i = cand[e];
            k.ok = 1;
            if (prev.ok && !key_less(prev, k, is_int))
                continue;
            if (key_less(k, best, is_int))
                best = k;
        }
        best = warp_min_key(best, is_int);
        if (lane == 0)
            sk[wid] = best;
        __syncthreads();
        if (wid == 0) {
            Key k;
            k.v = 0;
            k.i = 0;
            k.ok = 0;
            if (lane < nw)
                k = sk[lane];
            k = warp_min_key(k, is_int);
            if (lane == 0)
                sk[0] = k;
        }
        __syncthreads();
        const Key w = sk[0];
        __syncthreads();
        if (!w.ok)
            break;
        if (t == 0) {
            res->topk_value[r] = is_int ? (double)w.v : __longlong_as_double(w.v);
            res->topk_index[r] = w.i;
        }
        prev = w;
    }
    if (t == 0) {
        res->count = r;
        res->n_candidates = c->cand;
        res->status = (c->cand > cap) ? QBF_EOVERFLOW : QBF_OK;
    }
}

}  // namespace qbf
