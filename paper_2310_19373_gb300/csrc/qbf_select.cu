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
//                     prefix: its lowest tied state has the lowest index).
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

namespace {

// Block-wide sum of a 64-bit count (blockDim.x multiple of 32, <= 1024).
__device__ unsigned long long block_sum_u64(unsigned long long x, unsigned long long *sh)
{
    for (int o = 16; o > 0; o >>= 1)
        x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
        sh[w] = x;
    __syncthreads();
    unsigned long long r = 0;
    for (int i = 0; i < nw; ++i)
        r += sh[i];
    __syncthreads();
    return r;
}

}  // namespace

__global__ void __launch_bounds__(1024) threshold_kernel(const Plan *plan, const int *pmin,
                                                         unsigned long long npref, int top_k,
                                                         Counters *c)
{
    __shared__ unsigned long long sh[32];
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
        // smallest b with #{p : pmin[p] <= b} >= top_k
        long long lo = c->gmin, hi = INT_MAX;
        while (lo < hi) {
            const long long mid = lo + ((hi - lo) >> 1);
            unsigned long long cnt = 0;
            for (unsigned long long e = threadIdx.x; e < npref; e += blockDim.x)
                cnt += ((long long)pmin[e] <= mid) ? 1ull : 0ull;
            cnt = block_sum_u64(cnt, sh);
            if (cnt >= (unsigned long long)top_k)
                hi = mid;
            else
                lo = mid + 1;
        }
        base = lo;
    }
    if (threadIdx.x == 0) {
        long long t = base + plan->window;
        c->tau = (int)(t > (long long)INT_MAX ? (long long)INT_MAX : t);
    }
}

__global__ void flag_kernel(const Plan *plan, const int *pmin, unsigned long long npref,
                            unsigned long long p_lo, int top_k, unsigned int *flagged, Counters *c)
{
    if (plan->status != QBF_OK)
        return;
    const int lowest_mode = (top_k == 1 && plan->window == 0);
    const int tau = c->tau;
    for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         e < npref; e += (unsigned long long)gridDim.x * blockDim.x) {
        if (pmin[e] <= tau) {
            const unsigned p = (unsigned)(p_lo + e);
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
// Every add is an explicit round-to-nearest FP64 add.
__global__ void rescore_kernel(const Plan *plan, const void *Q, int n, int dtype,
                               const unsigned long long *cand, const Counters *c,
                               unsigned long long cap, long long *vals)
{
    if (plan->status != QBF_OK)
        return;
    const unsigned long long count = c->cand < cap ? c->cand : cap;
    const bool is_int = (dtype == QBF_I32 || dtype == QBF_I16);
    for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         e < count; e += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long x = cand[e];
        if (is_int) {
            long long acc = 0;
            for (int i = 0; i < n; ++i) {
                if (!((x >> i) & 1ull))
                    continue;
                long long row = qi_at(Q, dtype, i * n + i);
                for (int j = i + 1; j < n; ++j)
                    if ((x >> j) & 1ull)
                        row += qi_at(Q, dtype, i * n + j) + qi_at(Q, dtype, j * n + i);
                acc += row;
            }
            vals[e] = acc;
        } else {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) {
                if (!((x >> i) & 1ull))
                    continue;
                double row = q_at(Q, dtype, i * n + i);
                for (int j = i + 1; j < n; ++j)
                    if ((x >> j) & 1ull)
                        row = __dadd_rn(row, __dadd_rn(q_at(Q, dtype, i * n + j),
                                                       q_at(Q, dtype, j * n + i)));
                acc = __dadd_rn(acc, row);
            }
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

}  // namespace

__global__ void __launch_bounds__(1024) select_kernel(const Plan *plan,
                                                      const unsigned long long *cand,
                                                      const long long *vals, const Counters *c,
                                                      unsigned long long cap, int top_k,
                                                      DevResult *res)
{
    __shared__ Key sk[1024];
    const int t = threadIdx.x;
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
    Key prev;
    prev.ok = 0;
    int r = 0;
    for (; r < top_k; ++r) {
        Key best;
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
        sk[t] = best;
        __syncthreads();
        for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
            if (t < s && key_less(sk[t + s], sk[t], is_int))
                sk[t] = sk[t + s];
            __syncthreads();
        }
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
