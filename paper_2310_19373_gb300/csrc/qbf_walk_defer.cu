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

#include "qbf_f32x2.cuh"
#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"
#include "qbf_walk_core.cuh"

namespace qbf {

__constant__ float c_Cd[2][64];  // C[pi][u], C[pi][0] = 0
__constant__ float c_Ce[2];      // C[pi][2^R - 1]: a whole block's correction

namespace dfr {

using f32x2::u64;

template <int R>
struct Lane {
    u64 v[4];      // (b2 b1 b0) = (00x, 01x, 10x, 11x) as (lo, hi) = (b0 = 0, b0 = 1)
    u64 GF[4][R];  // lane parts of the low-bit fields, per pair
    float m[2];    // running minima (two chains)
};

__device__ __forceinline__ float min8(const float (&x)[8])
{
    const float a = f32x2::min3(x[0], x[1], x[2]);
    const float b = f32x2::min3(x[3], x[4], x[5]);
    const float c = f32x2::min3(x[6], x[7], a);
    return fminf(b, c);
}

// one block of 2^R - 1 in-block steps of parity PI
template <int R, int PI>
__device__ __forceinline__ void block(Lane<R> &L)
{
#pragma unroll
    for (int u = 1; u < (1 << R); ++u) {
        const int l = ctz_c(u);
        const int g = u ^ (u >> 1);
        const int nb = ((g >> l) & 1) ^ ((l == R - 1) ? PI : 0);
        float x[8];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            L.v[s] = nb ? f32x2::add(L.v[s], L.GF[s][l]) : f32x2::sub(L.v[s], L.GF[s][l]);
            f32x2::unpack(L.v[s], x[2 * s], x[2 * s + 1]);
        }
        L.m[u & 1] = fminf(L.m[u & 1], min8(x) + c_Cd[PI][u]);
    }
}

// Block transition after a block of parity PI: record (ra, rb) = (T, code,
// W0..W5) as in the two-pipe walk; the values first take the block's
// correction back (w -> v), then the mid-bit flip.
template <int R, int PI>
__device__ __forceinline__ void trans(Lane<R> &L, const int4 ra, const int4 rb, const int *sC,
                                      const int *sS, int n, int nsw, int stride, int slot)
{
    const int rel = ra.y >> 1;
    const bool plus = ra.y & 1;
    const int *Si = sS + (R + rel) * n + nsw;
    const int c = sC[rel * stride + slot];
    const int cs = plus ? c : -c;
    const int t0 = plus ? Si[0] : -Si[0];
    const int t1 = plus ? Si[1] : -Si[1];
    const int t2 = plus ? Si[2] : -Si[2];
    const int base = ra.x + cs;
    const u64 ce = f32x2::splat(c_Ce[PI]);
    const int d[8] = {base,      base + t0,      base + t1,      base + t1 + t0,
                      base + t2, base + t2 + t0, base + t1 + t2, base + t0 + t1 + t2};
    float x[8];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        L.v[s] = f32x2::add(f32x2::add(L.v[s], ce),
                            f32x2::pack((float)d[2 * s], (float)d[2 * s + 1]));
        f32x2::unpack(L.v[s], x[2 * s], x[2 * s + 1]);
    }
    L.m[0] = fminf(L.m[0], min8(x));
    const int W[6] = {ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const u64 w2 = f32x2::splat((float)W[i]);
#pragma unroll
        for (int s = 0; s < 4; ++s)
            L.GF[s][i] = f32x2::add(L.GF[s][i], w2);
    }
}

// Lane set-up for prefix p (variables nsg..n-1, nsg = nsw + 3): the eight
// start values, the low-bit fields of every group and the lane parts of the
// mid-bit fields (sC[(i - R) * stride + slot]).
template <int R>
__device__ __forceinline__ void setup(Lane<R> &L, unsigned long long p, int n, int nsg,
                                      const int *sS, const int *sLin, int *sC, int stride, int slot)
{
    const int nsw = nsg - 3;
    const int kp = n - nsg;
    int va = 0;
    for (int j = 0; j < kp; ++j) {
        if (!((p >> j) & 1))
            continue;
        const int vj = nsg + j;
        int row = sLin[vj];
        for (int jj = j + 1; jj < kp; ++jj)
            if ((p >> jj) & 1)
                row += sS[vj * n + nsg + jj];
        va += row;
    }
    int gf[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        int f = sLin[nsw + t];
        for (int j = 0; j < kp; ++j)
            if ((p >> j) & 1)
                f += sS[(nsw + t) * n + nsg + j];
        gf[t] = f;
    }
    const int s01 = sS[nsw * n + nsw + 1], s02 = sS[nsw * n + nsw + 2];
    const int s12 = sS[(nsw + 1) * n + nsw + 2];
    // v(b) = va + sum_t b_t gf_t + sum_{t<t'} b_t b_t' S_tt'
    const int v000 = va, v001 = va + gf[0];
    const int v010 = va + gf[1], v011 = v010 + gf[0] + s01;
    const int v100 = va + gf[2], v101 = v100 + gf[0] + s02;
    const int v110 = v010 + gf[2] + s12, v111 = v011 + gf[2] + s02 + s12;
    L.v[0] = f32x2::pack((float)v000, (float)v001);
    L.v[1] = f32x2::pack((float)v010, (float)v011);
    L.v[2] = f32x2::pack((float)v100, (float)v101);
    L.v[3] = f32x2::pack((float)v110, (float)v111);
#pragma unroll
    for (int ii = 0; ii < R; ++ii) {
        int c = sLin[ii];
        for (int j = 0; j < kp; ++j)
            if ((p >> j) & 1)
                c += sS[ii * n + nsg + j];
        const int s0 = sS[ii * n + nsw], s1 = sS[ii * n + nsw + 1], s2 = sS[ii * n + nsw + 2];
        L.GF[0][ii] = f32x2::pack((float)c, (float)(c + s0));
        L.GF[1][ii] = f32x2::pack((float)(c + s1), (float)(c + s1 + s0));
        L.GF[2][ii] = f32x2::pack((float)(c + s2), (float)(c + s2 + s0));
        L.GF[3][ii] = f32x2::pack((float)(c + s1 + s2), (float)(c + s0 + s1 + s2));
    }
    for (int ii = R; ii < nsw; ++ii) {
        int c = 0;
        for (int j = 0; j < kp; ++j)
            if ((p >> j) & 1)
                c += sS[ii * n + nsg + j];
        sC[(ii - R) * stride + slot] = c;
    }
    L.m[0] = fminf(fminf(fminf((float)v000, (float)v001), fminf((float)v010, (float)v011)),
                   fminf(fminf((float)v100, (float)v101), fminf((float)v110, (float)v111)));
    L.m[1] = L.m[0];
}

// the whole walk of one lane; returns the lane's minimum (an exact integer)
template <int R>
__device__ __forceinline__ int walk_min(Lane<R> &L, int n, int nsg, const int4 *rec4,
                                        const int *sC, const int *sS, int stride, int slot)
{
    const int nsw = nsg - 3;
    const int M = nsw - R;
    const unsigned nblocks = 1u << M;
    if (M == 0) {
        block<R, 0>(L);
    } else {
        for (unsigned B = 0; B < nblocks; B += 2) {
            const int4 r1a = __ldg(rec4 + 2 * (B + 1));
            const int4 r1b = __ldg(rec4 + 2 * (B + 1) + 1);
            const unsigned B2 = (B + 2 < nblocks) ? B + 2 : B + 1;
            const int4 r2a = __ldg(rec4 + 2 * B2);
            const int4 r2b = __ldg(rec4 + 2 * B2 + 1);
            block<R, 0>(L);
            trans<R, 0>(L, r1a, r1b, sC, sS, n, nsw, stride, slot);
            block<R, 1>(L);
            if (B + 2 < nblocks)
                trans<R, 1>(L, r2a, r2b, sC, sS, n, nsw, stride, slot);
        }
    }
    return (int)fminf(L.m[0], L.m[1]);
}

}  // namespace dfr

// a.ns is the suffix width of the certification geometry (nsw + 3); the lane
// walks the nsw bits below the three group bits for all eight groups.
template <int R>
__global__ void __launch_bounds__(kWalkThreads)
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
        if (lane == 0)
            item = atomicAdd(&a.ctr->items[kModeMin], 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.nitems)
            break;
        const unsigned long long i = a.p_lo + item * 32 + lane;
        const bool active = i < a.p_hi;
        const unsigned long long p = active ? i : a.p_lo;
        dfr::Lane<R> L;
        dfr::setup<R>(L, p, n, nsg, sS, sLin, sC, stride, slot);
        const int mi = dfr::walk_min<R>(L, n, nsg, rec4, sC, sS, stride, slot);
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
                              const int *Kbuf_dev, void *scratch_dev, int num_sms, cudaStream_t s)
{
    if (R < 1 || R > kRMax)
        return cudaErrorInvalidValue;
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
