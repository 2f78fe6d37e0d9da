// qbf_walk_mix.cu -- the MIN walk on both arithmetic pipes (QBF_VARIANT_SPLIT_MIX).
//
// Same split walk as qbf_walk.cu (R low bits unrolled with static corrections,
// lane-invariant block records).  Every state costs two adds (the lane part of
// the flipped variable's field and the static correction) and one min input.
// The int32 walk runs all three on the ALU pipe, the packed-FP32 walk runs the
// adds on the FP32 pipe and the mins on the ALU pipe; each pipe retires about
// 128 values per clock per SM, so neither keeps both busy.  Here every thread
// walks eight prefixes that differ in the three lowest prefix variables
// (group bits g0, g1, g2 = variables nsw, nsw+1, nsw+2):
//   - six of them as three f32x2 pairs (g2 g1 g0 = 00x, 01x, 10x): per step
//     two packed adds on the FP32 pipe and one three-input min on the ALU
//     pipe per pair;
//   - two of them as int32 values (110, 111): per step one three-input add
//     each and one three-input min for both, all on the ALU pipe.
// Per step and thread: 6 packed adds (FP32 pipe) and 3 + 2 + 1 half-rate ALU
// instructions: both pipes carry the same load.  The fixed-point image is
// bounded by 2^23 (every partial sum exact in FP32), as for the packed walk.
//
// The minimum over the eight prefixes is the per-prefix minimum of a walk with
// nsw + 3 suffix bits, so certification (flag, re-walk, rescore, select) is
// unchanged.
#include <climits>

#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"
#include "qbf_walk_mix_core.cuh"

namespace qbf {

__constant__ int c_Km[2][64];                  // K[parity][u] (int32 groups)
__constant__ unsigned long long c_K2m[2][64];  // (K, K) as FP32 pairs (packed groups)

namespace {

// corrections from the constant bank (one instance per launch)
struct ConstKm {
    __device__ __forceinline__ int k(int pi, int u) const { return c_Km[pi][u]; }
    __device__ __forceinline__ unsigned long long k2(int pi, int u) const { return c_K2m[pi][u]; }
};

}  // namespace

// a.ns is the suffix width of the certification geometry (nsw + 3); the lane
// walks the nsw bits below the three group bits for all eight groups.
template <int R>
__global__ void __launch_bounds__(kWalkThreads) walk_mix_min_kernel(const Plan *__restrict__ plan,
                                                                    const Rec *__restrict__ recs,
                                                                    WalkArgs a)
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
        mix::Lane<R> L;
        mix::setup<R>(L, p, n, nsg, sS, sLin, sC, stride, slot);
        const int mi = mix::walk_min<R>(L, n, nsg, rec4, sC, sS, stride, slot, ConstKm{});
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

namespace {

__global__ void k_mix_pairs_kernel(const int *Kbuf, unsigned long long *Kf2)
{
    const int e = threadIdx.x;
    if (e < 128) {
        const float k = (float)Kbuf[e];  // exact: |K| < 2^23
        Kf2[e] = ((unsigned long long)__float_as_uint(k) << 32) | __float_as_uint(k);
    }
}

}  // namespace

size_t walk_mix_smem_bytes(int n, int nsg, int R)
{
    const int nsw = nsg - 3;
    return (size_t)(n * n + n) * sizeof(int) + (size_t)(nsw - R) * kWalkThreads * sizeof(int);
}

template <int R>
static cudaError_t launch_mix_r(const Plan *plan, const Rec *recs, const WalkArgs &a, int num_sms,
                                cudaStream_t s)
{
    const size_t smem = walk_mix_smem_bytes(a.n, a.ns, R);
    auto k = walk_mix_min_kernel<R>;
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

cudaError_t launch_walk_mix(int R, const Plan *plan, const Rec *recs, const WalkArgs &a,
                            const int *Kbuf_dev, unsigned long long *Kf2_dev, int num_sms,
                            cudaStream_t s)
{
    k_mix_pairs_kernel<<<1, 128, 0, s>>>(Kbuf_dev, Kf2_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    e = cudaMemcpyToSymbolAsync(c_K2m, Kf2_dev, sizeof(unsigned long long) * 128, 0,
                                cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return e;
    e = cudaMemcpyToSymbolAsync(c_Km, Kbuf_dev, sizeof(int) * 128, 0, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return e;
    switch (R) {
    case 1: return launch_mix_r<1>(plan, recs, a, num_sms, s);
    case 2: return launch_mix_r<2>(plan, recs, a, num_sms, s);
    case 3: return launch_mix_r<3>(plan, recs, a, num_sms, s);
    case 4: return launch_mix_r<4>(plan, recs, a, num_sms, s);
    case 5: return launch_mix_r<5>(plan, recs, a, num_sms, s);
    default: return launch_mix_r<6>(plan, recs, a, num_sms, s);
    }
}

}  // namespace qbf
