// qbf_walk_plain.cu -- the two reference forms of the MIN kernel on the GPU:
//
//   QBF_VARIANT_FIELD: the Gray-code walk as the paper states it (Section 3,
//     Eq. 2, Algorithm 1): each thread keeps the local field g_i of every
//     suffix variable in registers; flipping bit l = CTZ(t) changes the value
//     by +-g_l and every other field by +-S_il, so a state costs n_s + 1 adds
//     and one min.  The flipped bit and its direction are warp-uniform (all
//     lanes walk the same suffix), so the update is a switch over l with the
//     S column l as constant-bank operands.
//   QBF_VARIANT_NAIVE: every state evaluated from scratch in natural order,
//     f(x) = sum_i x_i (lin_i + sum_{j>i} x_j S_ij), O(n^2) per state -- the
//     naive brute force the paper improves on.
//
// Both walk the int32 fixed-point image of qbf_walk.cu (exact) and write the
// same per-prefix minima, so qbf_solve's certification applies unchanged.
// They exist to measure the paper's naive-vs-Gray comparison on this GPU next
// to the split walks, not to be fast.
#include <climits>
#include <cstddef>

#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"

namespace qbf {

constexpr int kFieldMaxNs = 20;
__constant__ int c_Sf[kFieldMaxNs][kFieldMaxNs];  // S among the suffix variables

namespace {

// flip suffix bit L (x_L: 0 -> 1 if up)
template <int NS, int L>
__device__ __forceinline__ void flip(int up, int &v, int (&g)[NS])
{
    if (up) {
        v += g[L];
#pragma unroll
        for (int i = 0; i < NS; ++i)
            if (i != L)
                g[i] += c_Sf[i][L];
    } else {
        v -= g[L];
#pragma unroll
        for (int i = 0; i < NS; ++i)
            if (i != L)
                g[i] -= c_Sf[i][L];
    }
}

#define QBF_FLIP_CASE(L)                 \
    case L:                              \
        if constexpr (L < NS)            \
            flip<NS, L>(up, v, g);       \
        break;

template <int NS>
__device__ __forceinline__ void flip_any(int l, int up, int &v, int (&g)[NS])
{
    switch (l) {
        QBF_FLIP_CASE(0) QBF_FLIP_CASE(1) QBF_FLIP_CASE(2) QBF_FLIP_CASE(3) QBF_FLIP_CASE(4)
        QBF_FLIP_CASE(5) QBF_FLIP_CASE(6) QBF_FLIP_CASE(7) QBF_FLIP_CASE(8) QBF_FLIP_CASE(9)
        QBF_FLIP_CASE(10) QBF_FLIP_CASE(11) QBF_FLIP_CASE(12) QBF_FLIP_CASE(13) QBF_FLIP_CASE(14)
        QBF_FLIP_CASE(15) QBF_FLIP_CASE(16) QBF_FLIP_CASE(17) QBF_FLIP_CASE(18) QBF_FLIP_CASE(19)
    default: break;
    }
}
#undef QBF_FLIP_CASE

// value of (prefix p, suffix 0) over the prefix variables ns..n-1
__device__ int prefix_value(unsigned long long p, int n, int ns, const int *sS, const int *sLin)
{
    const int kp = n - ns;
    int v = 0;
    for (int j = 0; j < kp; ++j) {
        if (!((p >> j) & 1))
            continue;
        const int i = ns + j;
        int row = sLin[i];
        for (int jj = j + 1; jj < kp; ++jj)
            if ((p >> jj) & 1)
                row += sS[i * n + ns + jj];
        v += row;
    }
    return v;
}

__device__ __forceinline__ bool next_item(const WalkArgs &a, int lane, unsigned long long &p,
                                          bool &active)
{
    unsigned long long item = 0;
    if (lane == 0) {
        item = atomicAdd(&a.ctr->items[kModeMin], 1ull);
        if (cancelled(a.cancel))  // qbf_cancel: take no more items
            item = a.nitems;
    }
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.nitems)
        return false;
    const unsigned long long i = a.p_lo + item * 32 + lane;
    active = i < a.p_hi;
    p = active ? i : a.p_lo;
    return true;
}

__device__ __forceinline__ void finish_prefix(const WalkArgs &a, int lane, unsigned long long p,
                                              bool active, int m)
{
    if (active)
        a.pmin[p - a.p_lo] = m;
    int wm = active ? m : INT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        wm = min(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    if (lane == 0)
        atomicMin(&a.ctr->gmin, wm);
}

}  // namespace

template <int NS>
__global__ void __launch_bounds__(kWalkThreads) field_min_kernel(const Plan *__restrict__ plan,
                                                                 WalkArgs a)
{
    extern __shared__ int smem[];
    const int n = a.n;
    int *sS = smem;
    int *sLin = sS + n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        sS[e] = plan->S[e];
    for (int e = threadIdx.x; e < n; e += blockDim.x)
        sLin[e] = plan->lin[e];
    __syncthreads();
    if (plan->status != QBF_OK)
        return;
    const int lane = threadIdx.x & 31;
    const int kp = n - NS;
    unsigned long long p;
    bool active;
    while (next_item(a, lane, p, active)) {
        int v = prefix_value(p, n, NS, sS, sLin);
        int g[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            int c = sLin[i];
            for (int j = 0; j < kp; ++j)
                if ((p >> j) & 1)
                    c += sS[i * n + NS + j];
            g[i] = c;
        }
        int m = v;
        for (unsigned t = 1; t < (1u << NS); ++t) {
            const int l = __ffs((int)t) - 1;
            const int up = ((t ^ (t >> 1)) >> l) & 1;
            flip_any<NS>(l, up, v, g);
            m = min(m, v);
        }
        finish_prefix(a, lane, p, active, m);
    }
}

__global__ void __launch_bounds__(kWalkThreads) naive_min_kernel(const Plan *__restrict__ plan,
                                                                 WalkArgs a)
{
    extern __shared__ int smem[];
    const int n = a.n;
    const int ns = a.ns;
    int *sS = smem;
    int *sLin = sS + n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        sS[e] = plan->S[e];
    for (int e = threadIdx.x; e < n; e += blockDim.x)
        sLin[e] = plan->lin[e];
    __syncthreads();
    if (plan->status != QBF_OK)
        return;
    const int lane = threadIdx.x & 31;
    unsigned long long p;
    bool active;
    while (next_item(a, lane, p, active)) {
        int m = INT_MAX;
        for (unsigned long long t = 0; t < (1ull << ns); ++t) {
            const unsigned long long x = (p << ns) | t;
            int f = 0;
            for (int i = 0; i < n; ++i) {
                int row = sLin[i];
                for (int j = i + 1; j < n; ++j)
                    row += ((x >> j) & 1ull) ? sS[i * n + j] : 0;
                f += ((x >> i) & 1ull) ? row : 0;
            }
            m = min(m, f);
        }
        finish_prefix(a, lane, p, active, m);
    }
}

size_t plain_smem_bytes(int n) { return (size_t)(n * n + n) * sizeof(int); }

template <class K>
static cudaError_t launch_plain(K k, const Plan *plan, const WalkArgs &a, int num_sms,
                                cudaStream_t s)
{
    const size_t smem = plain_smem_bytes(a.n);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kWalkThreads, smem);
    if (e != cudaSuccess)
        return e;
    if (bps < 1)
        bps = 1;
    const unsigned long long need = (a.nitems + (kWalkThreads / 32) - 1) / (kWalkThreads / 32);
    unsigned long long grid = (unsigned long long)num_sms * bps;
    if (grid > need)
        grid = need;
    if (grid < 1)
        grid = 1;
    k<<<(unsigned)grid, kWalkThreads, smem, s>>>(plan, a);
    return cudaGetLastError();
}

cudaError_t launch_walk_field(const Plan *plan, const WalkArgs &a, int num_sms, cudaStream_t s)
{
    const int ns = a.ns;
    if (ns < 1 || ns > kFieldMaxNs)
        return cudaErrorInvalidValue;
    // the suffix block of S (rows and columns 0..ns-1) into the constant bank
    int *cS = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&cS, c_Sf);
    if (e != cudaSuccess)
        return e;
    const char *S_dev = reinterpret_cast<const char *>(plan) + offsetof(Plan, S);
    e = cudaMemcpy2DAsync(cS, kFieldMaxNs * sizeof(int), S_dev, a.n * sizeof(int),
                          ns * sizeof(int), ns, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return e;
    switch (ns) {
#define QBF_FIELD_NS(NS) \
    case NS: return launch_plain(field_min_kernel<NS>, plan, a, num_sms, s);
        QBF_FIELD_NS(1) QBF_FIELD_NS(2) QBF_FIELD_NS(3) QBF_FIELD_NS(4) QBF_FIELD_NS(5)
        QBF_FIELD_NS(6) QBF_FIELD_NS(7) QBF_FIELD_NS(8) QBF_FIELD_NS(9) QBF_FIELD_NS(10)
        QBF_FIELD_NS(11) QBF_FIELD_NS(12) QBF_FIELD_NS(13) QBF_FIELD_NS(14) QBF_FIELD_NS(15)
        QBF_FIELD_NS(16) QBF_FIELD_NS(17) QBF_FIELD_NS(18) QBF_FIELD_NS(19) QBF_FIELD_NS(20)
#undef QBF_FIELD_NS
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_walk_naive(const Plan *plan, const WalkArgs &a, int num_sms, cudaStream_t s)
{
    return launch_plain(naive_min_kernel, plan, a, num_sms, s);
}

}  // namespace qbf
