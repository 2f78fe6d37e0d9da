// qbf_walk_f32.cu -- the MIN walk in packed FP32 (QBF_VARIANT_SPLIT_F32).
//
// Same walk as qbf_walk.cu (split field, R low bits unrolled, lane-invariant
// block records), with two changes that move the value updates from the
// integer pipe to the FP32 pipe:
//   - every value is an integer below 2^23 (the fixed-point image is built with
//     sum |image| < 2^23), so FP32 adds are exact: each intermediate of
//     v + (+-GL) + K is bounded by 2 * 2^23;
//   - each lane walks a pair of prefixes that differ only in the lowest prefix
//     variable (the "pair bit", variable nsw), packed as (a, b) into one 64-bit
//     register: one add.rn.f32x2 moves both.  The pair bit adds S[i][nsw] to
//     the b half of every field and lin + its prefix field to the b value.
// Per step: two packed adds (the signed low-bit field pair, then the static
// correction pair from the constant bank) and one three-input min over both
// halves.  The minimum is
// recorded per pair, i.e. per prefix of a walk with nsw + 1 suffix bits.
#include <climits>

#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"
#include "qbf_walk_core.cuh"
#include "qbf_f32x2.cuh"

namespace qbf {

__constant__ unsigned long long c_K2[2][64];  // (K, K): the static corrections as FP32 pairs

namespace {

using f32x2::u64;

template <int R, int PI>
__device__ __forceinline__ void block_f2(u64 &v, float &m, const u64 (&GL)[R])
{
#pragma unroll
    for (int u = 1; u < (1 << R); ++u) {
        const int l = ctz_c(u);
        const int g = u ^ (u >> 1);
        const int nb = ((g >> l) & 1) ^ ((l == R - 1) ? PI : 0);
        v = nb ? f32x2::add(v, GL[l]) : f32x2::sub(v, GL[l]);
        v = f32x2::add(v, c_K2[PI][u]);
        float lo, hi;
        f32x2::unpack(v, lo, hi);
        m = f32x2::min3(m, lo, hi);
    }
}

template <int R>
__device__ __forceinline__ void trans_f2(u64 &v, float &m, u64 (&GL)[R], const int4 ra,
                                         const int4 rb, const u64 *sC2, int stride, int slot)
{
    const float T = (float)ra.x;
    v = f32x2::add(v, f32x2::pack(T, T));
    v = f32x2::add(v, sC2[ra.y * stride + slot]);
    float lo, hi;
    f32x2::unpack(v, lo, hi);
    m = f32x2::min3(m, lo, hi);
    const int W[6] = {ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const float w = (float)W[i];
        GL[i] = f32x2::add(GL[i], f32x2::pack(w, w));
    }
}

}  // namespace

// a.ns is the suffix width of the pair geometry (nsw + 1); the lane walks the
// nsw bits below the pair bit for both of its halves.
template <int R>
__global__ void __launch_bounds__(kWalkThreads) walk_f32x2_min_kernel(const Plan *__restrict__ plan,
                                                                      const Rec *__restrict__ recs,
                                                                      WalkArgs a)
{
    extern __shared__ int smem[];
    const int n = a.n;
    const int nsp = a.ns;        // suffix bits incl. the pair bit
    const int nsw = nsp - 1;     // walked bits
    const int kp = n - nsp;      // prefix bits of a lane
    int *sS = smem;
    int *sLin = sS + n * n;
    // 8-byte aligned start of the packed lane parts
    u64 *sC2 = reinterpret_cast<u64 *>(smem + ((n * n + n + 1) & ~1));
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        sS[e] = plan->S[e];
    for (int e = threadIdx.x; e < n; e += blockDim.x)
        sLin[e] = plan->lin[e];
    __syncthreads();
    if (plan->status != QBF_OK)
        return;
    const int lane = threadIdx.x & 31;
    const int4 *rec4 = reinterpret_cast<const int4 *>(recs);
    const int M = nsw - R;
    const unsigned nblocks = 1u << M;
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

        // value of (prefix, pair bit 0, suffix 0) and the prefix part of every field
        int va = 0;
        for (int j = 0; j < kp; ++j) {
            if (!((p >> j) & 1))
                continue;
            const int vj = nsp + j;
            int row = sLin[vj];
            for (int jj = j + 1; jj < kp; ++jj)
                if ((p >> jj) & 1)
                    row += sS[vj * n + nsp + jj];
            va += row;
        }
        int fpair = sLin[nsw];  // field of the pair bit from the prefix
        for (int j = 0; j < kp; ++j)
            if ((p >> j) & 1)
                fpair += sS[nsw * n + nsp + j];
        const int vb = va + fpair;
        u64 GL[R];
#pragma unroll
        for (int ii = 0; ii < R; ++ii) {
            int c = sLin[ii];
            for (int j = 0; j < kp; ++j)
                if ((p >> j) & 1)
                    c += sS[ii * n + nsp + j];
            GL[ii] = f32x2::pack((float)c, (float)(c + sS[ii * n + nsw]));
        }
        for (int ii = R; ii < nsw; ++ii) {
            int c = 0;
            for (int j = 0; j < kp; ++j)
                if ((p >> j) & 1)
                    c += sS[ii * n + nsp + j];
            const int cb = c + sS[ii * n + nsw];
            sC2[(2 * (ii - R) + 1) * stride + slot] = f32x2::pack((float)c, (float)cb);
            sC2[(2 * (ii - R)) * stride + slot] = f32x2::pack((float)-c, (float)-cb);
        }
        u64 v = f32x2::pack((float)va, (float)vb);
        float m = fminf((float)va, (float)vb);
        if (M == 0) {
            block_f2<R, 0>(v, m, GL);
        } else {
            for (unsigned B = 0; B < nblocks; B += 2) {
                const int4 r1a = __ldg(rec4 + 2 * (B + 1));
                const int4 r1b = __ldg(rec4 + 2 * (B + 1) + 1);
                const unsigned B2 = (B + 2 < nblocks) ? B + 2 : B + 1;
                const int4 r2a = __ldg(rec4 + 2 * B2);
                const int4 r2b = __ldg(rec4 + 2 * B2 + 1);
                block_f2<R, 0>(v, m, GL);
                trans_f2<R>(v, m, GL, r1a, r1b, sC2, stride, slot);
                block_f2<R, 1>(v, m, GL);
                if (B + 2 < nblocks)
                    trans_f2<R>(v, m, GL, r2a, r2b, sC2, stride, slot);
            }
        }
        const int mi = (int)m;  // exact: an integer below 2^23
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

__global__ void k_pairs_kernel(const int *Kbuf, unsigned long long *Kf2)
{
    const int e = threadIdx.x;
    if (e < 128) {
        const float k = (float)Kbuf[e];  // exact: |K| < 2^23
        Kf2[e] = ((unsigned long long)__float_as_uint(k) << 32) | __float_as_uint(k);
    }
}

size_t walk_f32_smem_bytes(int n, int nsp, int R)
{
    const int nsw = nsp - 1;
    return (size_t)((n * n + n + 1) & ~1) * sizeof(int) +
           (size_t)2 * (nsw - R) * kWalkThreads * sizeof(unsigned long long);
}

template <int R>
static cudaError_t launch_f32_r(const Plan *plan, const Rec *recs, const WalkArgs &a, int num_sms,
                                cudaStream_t s)
{
    const size_t smem = walk_f32_smem_bytes(a.n, a.ns, R);
    auto k = walk_f32x2_min_kernel<R>;
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

cudaError_t launch_walk_f32(int R, const Plan *plan, const Rec *recs, const WalkArgs &a,
                            const int *Kbuf_dev, unsigned long long *Kf2_dev, int num_sms,
                            cudaStream_t s)
{
    k_pairs_kernel<<<1, 128, 0, s>>>(Kbuf_dev, Kf2_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    e = cudaMemcpyToSymbolAsync(c_K2, Kf2_dev, sizeof(unsigned long long) * 128, 0,
                                cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return e;
    switch (R) {
    case 1: return launch_f32_r<1>(plan, recs, a, num_sms, s);
    case 2: return launch_f32_r<2>(plan, recs, a, num_sms, s);
    case 3: return launch_f32_r<3>(plan, recs, a, num_sms, s);
    case 4: return launch_f32_r<4>(plan, recs, a, num_sms, s);
    case 5: return launch_f32_r<5>(plan, recs, a, num_sms, s);
    default: return launch_f32_r<6>(plan, recs, a, num_sms, s);
    }
}

}  // namespace qbf
