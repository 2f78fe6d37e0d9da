// qbf_walk_defer.cu -- the MIN walk with the static correction deferred past
// the minimum (QBF_VARIANT_SPLIT_DEFER).
//
// Same split walk as qbf_walk.cu: R low bits unrolled, lane-invariant block
// records for the mid bits.  At in-block step u the value of every walked
// prefix moves by the lane part of the flipped variable's field (+-GF_l, a
// register) and by the static correction K[pi][u] (the cross terms among the
// R low bits, lane- and prefix-invariant).  The two-pipe walk pays that second
// add once per value.  Here a thread walks eight prefixes that differ in the
// three lowest prefix variables (group bits nsw..nsw+2), all as four f32x2
// pairs, and keeps each value without its in-block correction:
//     w_b(u) = v_b(u) - C[pi][u],   C[pi][u] = K[pi][1] + ... + K[pi][u],
// so a step is one packed add per pair (w_b(u) = w_b(u-1) +- GF_l).  Since
// C[pi][u] is the same for all eight values,
//     min_b v_b(u) = (min_b w_b(u)) + C[pi][u]:
// three three-input mins and one min reduce the eight values, then one scalar
// add (its operand straight from the constant bank) restores the correction
// and one min folds the step into the running minimum.  Per step and thread:
// 4 packed adds on the FP32 heavy pipe, 1 FP32 add, 5 mins on the ALU pipe --
// 10 instructions for 8 states, against 12 for the two-pipe walk.  At the
// block transition the values take C[pi][2^R - 1] back before the record's
// delta, so w = v again at every block start.
//
// Exactness: the image is bounded by 2^23 (sum |image| < 2^23 - 2^12, as for
// the other FP32-pipe walks), so |v| < 2^23 and |C| < 2^23, hence |w| < 2^24
// and every add, min and conversion here is exact.
//
// The minimum over the eight prefixes is the per-prefix minimum of a walk with
// nsw + 3 suffix bits, so certification (flag, re-walk, rescore, select) is
// unchanged.
#include <climits>

#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"
#include "qbf_walk_defer_core.cuh"

namespace qbf {

__constant__ float c_Cd[2][64];  // C[pi][u], C[pi][0] = 0
__constant__ float c_Ce[2];      // C[pi][2^R - 1]: a whole block's correction

namespace {

// sums from the constant bank (one instance per launch)
struct ConstC {
    __device__ __forceinline__ float c(int pi, int u) const { return c_Cd[pi][u]; }
    __device__ __forceinline__ float ce(int pi) const { return c_Ce[pi]; }
};

}  // namespace

// a.ns is the suffix width of the certification geometry (nsw + 3); the lane
// walks the nsw bits below the three group bits for all eight groups.
// three CTAs of 256 threads per SM (at most 80 registers): measured at n = 40,
// 57.8 ms against 59.3 ms for the same code at two CTAs (96 registers)
template <int R>
__global__ void __launch_bounds__(kWalkThreads, 3)
    walk_defer_min_kernel(const Plan *__restrict__ plan, const Rec *__restrict__ recs, WalkArgs a)
{
    extern __shared__ int smem[];
    const int n = a.n;
    const int nsg = a.ns;  // suffix bits incl. the group bits
    int *sS = smem;
    int *sLin = sS + n * n;
    int *sC = sLin + n;  // lane parts of the mid-bit fields, (nsw - R) x blockDim
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        sS[e] = plan->S[e];
    for (int e = threadIdx.x; e < n; e += blockDim.x)
        sLin[e] = plan->lin[e];
    __syncthreads();
    if (plan->status != QBF_OK)
        return;
    const int lane = threadIdx.x & 31;
    const int4 *rec4 = reinterpret_cast<const int4 *>(recs);
    const int stride = blockDim.x, slot = threadIdx.x;

    while (true) {
        unsigned long long item = 0;
        if (lane == 0) {
            item = atomicAdd(&a.ctr->items[kModeMin], 1ull);
            if (cancelled(a.cancel))  // qbf_cancel: take no more items
                item = a.nitems;
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.nitems)
            break;
        const unsigned long long i = a.p_lo + item * 32 + lane;
        const bool active = i < a.p_hi;
        const unsigned long long p = active ? i : a.p_lo;
        dfr::Lane<R> L;
        dfr::setup<R>(L, p, n, nsg, sS, sLin, sC, stride, slot);
        const int mi = dfr::walk_min<R>(L, n, nsg, rec4, sC, sS, stride, slot, ConstC{});
        if (active)
            a.pmin[p - a.p_lo] = mi;
        int wm = active ? mi : INT_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            wm = min(wm, __shfl_xor_sync(0xffffffffu, wm, o));
        if (lane == 0)
            atomicMin(&a.ctr->gmin, wm);
    }
}

// ---------------------------------------------------------------------------
// The table-driven form of the deferred walk (used when the suffix table
// fits, see launch_walk_defer).  The value of group b of a lane at suffix
// state s splits exactly (Eq. 1 over the fixed-point image) as
//     v_b(s) = F(s) + w_b(s),
// F(s)   = sum_{i in s} lin_i + sum_{i<j in s} S_ij   (suffix only: the same
//          for every lane and every group),
// w_b(s) = H_b(p) + sum_{i in s} c_i(b, p),  c_i(b, p) = sum of S_ij over the
//          set group and prefix variables j        (the lane part).
// Flipping suffix variable i moves w_b by +-c_i(b, p), a constant of the walk,
// so the low-bit fields never change and a block transition only adds the
// mid bit's +-c_i(b, p) to the eight values.  min_b v_b(s) = min_b w_b(s) +
// F(s): the lane-invariant F(gray(t)) of every suffix step t is a table built
// once per solve (2^nsw floats, exact: |F| < 2^23), which each warp stages
// block by block into shared memory with cp.async.  Per step and lane: 4 packed
// adds, three three-input mins and one min for the eight values, and per pair
// of steps one packed add of (F(t-1), F(t)) and one three-input min into the
// running minimum.  |w| and |F| stay below 2^23, so every operation is exact.
// ---------------------------------------------------------------------------

// Low bits per block (unrolled steps 2^R): 7 for long lane walks, where
// 128-step blocks halve the transition cost per state (n = 40: 53.0 against
// 54.5 ms), 6 for short ones, where the shorter code and set-up win (n = 32,
// 2^10 steps per lane: 0.297 against 0.311 ms).
constexpr int kDefer2LongR = 7;
constexpr int kDefer2LongNsw = 14;  // lane walks of at least 2^14 steps take R = 7
constexpr int kDefer2MaxM = 14;     // largest 2^M blocks of 2^R states per lane (table <= 8 MB)
constexpr int kDefer2Threads = 256;
constexpr int kDefer2CtasPerSm = 3;  // at most 80 registers


// F(gray(t)) for t < 2^nsw on the image of the plan (int64 sums, then FP32)
__global__ void defer2_ftab_kernel(const Plan *__restrict__ plan, int nsw, float *ftab)
{
    const int n = plan->n;
    const unsigned N = 1u << nsw;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) {
        const unsigned x = t ^ (t >> 1);
        long long f = 0;
        for (unsigned r = x; r; r &= r - 1) {
            const int i = __ffs(r) - 1;
            f += plan->lin[i];
            for (unsigned q = r & (r - 1); q; q &= q - 1)
                f += plan->S[i * n + (__ffs(q) - 1)];
        }
        ftab[t] = (float)f;
    }
}


// The table-driven MIN walk: same geometry, groups and output as
// walk_defer_min_kernel (a.ns = nsw + 3), with blocks of 2^R states
// (one more unrolled bit than the record-driven walk: the block transitions
// cost half as much per state, and the table needs no records).
template <int R>
__global__ void __launch_bounds__(kDefer2Threads, kDefer2CtasPerSm)
    walk_defer2_min_kernel(const Plan *__restrict__ plan, const float *__restrict__ ftab, WalkArgs a)
{
    extern __shared__ __align__(16) int smem[];
    const int n = a.n;
    const int nsg = a.ns;
    const int nsw = nsg - 3;
    const int nmid = nsw - R;
    float *fbufs = reinterpret_cast<float *>(smem);  // per warp: two blocks of 2^R F values
    ulonglong2 *sGFx = reinterpret_cast<ulonglong2 *>(fbufs + (kDefer2Threads / 32) * (2 << R));
    float4 *sE = reinterpret_cast<float4 *>(sGFx + (R - kDefer2RegBits) * 2 * kDefer2Threads);
    float *sCf = reinterpret_cast<float *>(sE + nmid * 4);
    int *sS = reinterpret_cast<int *>(sCf + nmid * kDefer2Threads);
    int *sLin = sS + n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        sS[e] = plan->S[e];
    for (int e = threadIdx.x; e < n; e += blockDim.x)
        sLin[e] = plan->lin[e];
    __syncthreads();
    // group terms of every mid variable i, both directions: sign * (b0 S_i,nsw +
    // b1 S_i,nsw+1 + b2 S_i,nsw+2) for the eight groups b
    for (int e = threadIdx.x; e < nmid * 2; e += blockDim.x) {
        const int i = R + (e >> 1);
        const float sg = (e & 1) ? 1.f : -1.f;
        const float s0 = (float)sS[i * n + nsw], s1 = (float)sS[i * n + nsw + 1];
        const float s2 = (float)sS[i * n + nsw + 2];
        sE[e * 2] = make_float4(0.f, sg * s0, sg * s1, sg * (s1 + s0));
        sE[e * 2 + 1] = make_float4(sg * s2, sg * (s2 + s0), sg * (s1 + s2), sg * (s0 + s1 + s2));
    }
    __syncthreads();
    if (plan->status != QBF_OK)
        return;
    const int lane = threadIdx.x & 31;
    float *fbuf = fbufs + (threadIdx.x >> 5) * (2 << R);
    const int stride = blockDim.x, slot = threadIdx.x;
    while (true) {
        unsigned long long item = 0;
        if (lane == 0) {
            item = atomicAdd(&a.ctr->items[kModeMin], 1ull);
            if (cancelled(a.cancel))  // qbf_cancel: take no more items
                item = a.nitems;
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.nitems)
            break;
        const unsigned long long i = a.p_lo + item * 32 + lane;
        const bool active = i < a.p_hi;
        const unsigned long long p = active ? i : a.p_lo;
        dfr2::Lane<R> L;
        dfr2::setup<R>(L, p, n, nsg, sS, sLin, sCf, stride, slot, sGFx);
        const int mi = dfr2::walk_min<R>(L, nsw, ftab, fbuf, lane, sCf, stride, slot, sE, sGFx);
        if (active)
            a.pmin[p - a.p_lo] = mi;
        int wm = active ? mi : INT_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            wm = min(wm, __shfl_xor_sync(0xffffffffu, wm, o));
        if (lane == 0)
            atomicMin(&a.ctr->gmin, wm);
    }
}

size_t walk_defer_table_floats(int R, int nsw)
{
    if (R != kRMax || nsw < kRMax || nsw - (nsw >= kDefer2LongNsw ? kDefer2LongR : kRMax) > kDefer2MaxM)
        return 0;
    return (size_t)1 << nsw;
}

template <int R>
static cudaError_t launch_defer2(const Plan *plan, float *ftab, const WalkArgs &a, int num_sms,
                                 cudaStream_t s)
{
    const int nsw = a.ns - 3;
    const unsigned N = 1u << nsw;
    defer2_ftab_kernel<<<(N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096, 256, 0, s>>>(plan, nsw,
                                                                                      ftab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const int nmid = nsw - R;
    const size_t smem = sizeof(float) * (kDefer2Threads / 32) * (2 << R) +
                        sizeof(ulonglong2) * (R - kDefer2RegBits) * 2 * kDefer2Threads +
                        sizeof(float4) * nmid * 4 +
                        sizeof(float) * nmid * kDefer2Threads + sizeof(int) * (a.n * a.n + a.n);
    auto k = walk_defer2_min_kernel<R>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kDefer2Threads, smem);
    if (e != cudaSuccess)
        return e;
    if (bps < 1)
        bps = 1;
    const unsigned long long need = (a.nitems + (kDefer2Threads / 32) - 1) / (kDefer2Threads / 32);
    unsigned long long grid = (unsigned long long)num_sms * bps;
    if (grid > need)
        grid = need;
    if (grid < 1)
        grid = 1;
    k<<<(unsigned)grid, kDefer2Threads, smem, s>>>(plan, ftab, a);
    return cudaGetLastError();
}

namespace {

// C[pi][u] = K[pi][1] + ... + K[pi][u] (exact in int32: |C| < 2^23) and the
// block totals C[pi][2^R - 1], as FP32: out[pi * 64 + u], out[128 + pi]
__global__ void k_defer_tables_kernel(const int *Kbuf, int R, float *out)
{
    const int pi = threadIdx.x;
    if (pi < 2) {
        int c = 0;
        out[pi * 64] = 0.f;
        for (int u = 1; u < 64; ++u) {
            c += Kbuf[pi * 64 + u];  // zero for u >= 2^R
            out[pi * 64 + u] = (float)c;
        }
        out[128 + pi] = out[pi * 64 + (1 << R) - 1];
    }
}

}  // namespace

size_t walk_defer_smem_bytes(int n, int nsg, int R)
{
    const int nsw = nsg - 3;
    return (size_t)(n * n + n) * sizeof(int) + (size_t)(nsw - R) * kWalkThreads * sizeof(int);
}

template <int R>
static cudaError_t launch_defer_r(const Plan *plan, const Rec *recs, const WalkArgs &a,
                                  int num_sms, cudaStream_t s)
{
    const size_t smem = walk_defer_smem_bytes(a.n, a.ns, R);
    auto k = walk_defer_min_kernel<R>;
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
    k<<<(unsigned)grid, kWalkThreads, smem, s>>>(plan, recs, a);
    return cudaGetLastError();
}

cudaError_t launch_walk_defer(int R, const Plan *plan, const Rec *recs, const WalkArgs &a,
                              const int *Kbuf_dev, void *scratch_dev, int num_sms, cudaStream_t s,
                              float *ftab_dev)
{
    if (R < 1 || R > kRMax)
        return cudaErrorInvalidValue;
    if (ftab_dev && walk_defer_table_floats(R, a.ns - 3) > 0)
        return a.ns - 3 >= kDefer2LongNsw
                   ? launch_defer2<kDefer2LongR>(plan, ftab_dev, a, num_sms, s)
                   : launch_defer2<kRMax>(plan, ftab_dev, a, num_sms, s);
    float *tab = static_cast<float *>(scratch_dev);  // 130 floats
    k_defer_tables_kernel<<<1, 32, 0, s>>>(Kbuf_dev, R, tab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    e = cudaMemcpyToSymbolAsync(c_Cd, tab, sizeof(float) * 128, 0, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return e;
    e = cudaMemcpyToSymbolAsync(c_Ce, tab + 128, sizeof(float) * 2, 0, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return e;
    switch (R) {
    case 1: return launch_defer_r<1>(plan, recs, a, num_sms, s);
    case 2: return launch_defer_r<2>(plan, recs, a, num_sms, s);
    case 3: return launch_defer_r<3>(plan, recs, a, num_sms, s);
    case 4: return launch_defer_r<4>(plan, recs, a, num_sms, s);
    case 5: return launch_defer_r<5>(plan, recs, a, num_sms, s);
    default: return launch_defer_r<6>(plan, recs, a, num_sms, s);
    }
}

}  // namespace qbf
