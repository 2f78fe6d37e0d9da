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

#include "qbf_f32x2.cuh"
#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"
#include "qbf_walk_core.cuh"

namespace qbf {

__constant__ int c_Km[2][64];                  // K[parity][u] (int32 streams)
__constant__ unsigned long long c_K2m[2][64];  // (K, K) as FP32 pairs (packed streams)

namespace {

using f32x2::u64;

// one block of 2^R - 1 in-block steps of parity PI
template <int R, int PI>
__device__ __forceinline__ void mix_block(u64 (&vF)[3], float (&mF)[3], unsigned (&vI)[2], int &mI,
                                          const u64 (&GF)[3][R], const unsigned (&GI)[2][R])
{
#pragma unroll
    for (int u = 1; u < (1 << R); ++u) {
        const int l = ctz_c(u);
        const int g = u ^ (u >> 1);
        const int nb = ((g >> l) & 1) ^ ((l == R - 1) ? PI : 0);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            u64 v = nb ? f32x2::add(vF[s], GF[s][l]) : f32x2::sub(vF[s], GF[s][l]);
            v = f32x2::add(v, c_K2m[PI][u]);
            float lo, hi;
            f32x2::unpack(v, lo, hi);
            mF[s] = f32x2::min3(mF[s], lo, hi);
            vF[s] = v;
        }
        const unsigned k = (unsigned)c_Km[PI][u];
        vI[0] = vI[0] + (nb ? GI[0][l] : 0u - GI[0][l]) + k;
        vI[1] = vI[1] + (nb ? GI[1][l] : 0u - GI[1][l]) + k;
        mI = __vimin3_s32(mI, (int)vI[0], (int)vI[1]);
    }
}

// Block transition: record (ra, rb) = (T, code, W0..W5).  The flipped mid bit
// is i = R + (code >> 1), entered with sign + if code is odd; its field for
// group b is T (signed, lane-invariant) + sign * (c_i + b0 s0 + b1 s1 + b2 s2)
// with c_i the lane part from the prefix and s_t = S[i][nsw + t].
template <int R>
__device__ __forceinline__ void mix_trans(u64 (&vF)[3], float (&mF)[3], unsigned (&vI)[2], int &mI,
                                          u64 (&GF)[3][R], unsigned (&GI)[2][R], const int4 ra,
                                          const int4 rb, const int *sC, const int *sS, int n,
                                          int nsw, int stride, int slot)
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
    vF[0] = f32x2::add(vF[0], f32x2::pack((float)base, (float)(base + t0)));
    vF[1] = f32x2::add(vF[1], f32x2::pack((float)(base + t1), (float)(base + t1 + t0)));
    vF[2] = f32x2::add(vF[2], f32x2::pack((float)(base + t2), (float)(base + t2 + t0)));
    vI[0] += (unsigned)(base + t1 + t2);
    vI[1] += (unsigned)(base + t0 + t1 + t2);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        float lo, hi;
        f32x2::unpack(vF[s], lo, hi);
        mF[s] = f32x2::min3(mF[s], lo, hi);
    }
    mI = __vimin3_s32(mI, (int)vI[0], (int)vI[1]);
    const int W[6] = {ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const u64 w2 = f32x2::splat((float)W[i]);
#pragma unroll
        for (int s = 0; s < 3; ++s)
            GF[s][i] = f32x2::add(GF[s][i], w2);
        GI[0][i] += (unsigned)W[i];
        GI[1][i] += (unsigned)W[i];
    }
}

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
    const int nsg = a.ns;     // suffix bits incl. the group bits
    const int nsw = nsg - 3;  // walked bits
    const int kp = n - nsg;   // prefix bits of a lane
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
    const int M = nsw - R;
    const unsigned nblocks = 1u << M;
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

        // value of (prefix, group 0, suffix 0) and the group bits' fields
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
        u64 vF[3] = {f32x2::pack((float)v000, (float)v001), f32x2::pack((float)v010, (float)v011),
                     f32x2::pack((float)v100, (float)v101)};
        unsigned vI[2] = {(unsigned)v110, (unsigned)v111};
        u64 GF[3][R];
        unsigned GI[2][R];
#pragma unroll
        for (int ii = 0; ii < R; ++ii) {
            int c = sLin[ii];
            for (int j = 0; j < kp; ++j)
                if ((p >> j) & 1)
                    c += sS[ii * n + nsg + j];
            const int s0 = sS[ii * n + nsw], s1 = sS[ii * n + nsw + 1], s2 = sS[ii * n + nsw + 2];
            GF[0][ii] = f32x2::pack((float)c, (float)(c + s0));
            GF[1][ii] = f32x2::pack((float)(c + s1), (float)(c + s1 + s0));
            GF[2][ii] = f32x2::pack((float)(c + s2), (float)(c + s2 + s0));
            GI[0][ii] = (unsigned)(c + s1 + s2);
            GI[1][ii] = (unsigned)(c + s0 + s1 + s2);
        }
        for (int ii = R; ii < nsw; ++ii) {
            int c = 0;
            for (int j = 0; j < kp; ++j)
                if ((p >> j) & 1)
                    c += sS[ii * n + nsg + j];
            sC[(ii - R) * stride + slot] = c;
        }
        float mF[3] = {fminf((float)v000, (float)v001), fminf((float)v010, (float)v011),
                       fminf((float)v100, (float)v101)};
        int mI = min(v110, v111);
        if (M == 0) {
            mix_block<R, 0>(vF, mF, vI, mI, GF, GI);
        } else {
            for (unsigned B = 0; B < nblocks; B += 2) {
                const int4 r1a = __ldg(rec4 + 2 * (B + 1));
                const int4 r1b = __ldg(rec4 + 2 * (B + 1) + 1);
                const unsigned B2 = (B + 2 < nblocks) ? B + 2 : B + 1;
                const int4 r2a = __ldg(rec4 + 2 * B2);
                const int4 r2b = __ldg(rec4 + 2 * B2 + 1);
                mix_block<R, 0>(vF, mF, vI, mI, GF, GI);
                mix_trans<R>(vF, mF, vI, mI, GF, GI, r1a, r1b, sC, sS, n, nsw, stride, slot);
                mix_block<R, 1>(vF, mF, vI, mI, GF, GI);
                if (B + 2 < nblocks)
                    mix_trans<R>(vF, mF, vI, mI, GF, GI, r2a, r2b, sC, sS, n, nsw, stride, slot);
            }
        }
        // exact: integers below 2^23
        const int mi = min(min((int)mF[0], (int)mF[1]), min((int)mF[2], mI));
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
