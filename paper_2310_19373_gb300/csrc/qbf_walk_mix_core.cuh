// qbf_walk_mix_core.cuh -- device building blocks of the two-pipe walk, shared
// by the single-instance kernel (qbf_walk_mix.cu) and the batched persistent
// kernel (qbf_batched.cu).  The derivation is in qbf_walk_mix.cu.
//
// A lane walks nsw suffix bits for the eight values b = (b2 b1 b0) of its
// three group bits (variables nsw, nsw+1, nsw+2): groups 00x, 01x, 10x as
// three f32x2 pairs (vF), groups 110 and 111 as int32 values (vI).  KS gives
// the static in-block corrections: k(pi, u) as int32 and k2(pi, u) as an
// FP32 pair (K, K).
#pragma once

#include <climits>

#include "qbf_f32x2.cuh"
#include "qbf_internal.cuh"
#include "qbf_walk_core.cuh"

namespace qbf {
namespace mix {

using f32x2::u64;

template <int R>
struct Lane {
    u64 vF[3];
    unsigned vI[2];
    float mF[3];
    int mI;
    u64 GF[3][R];
    unsigned GI[2][R];
};

// one block of 2^R - 1 in-block steps of parity PI
template <int R, int PI, class KS>
__device__ __forceinline__ void block(Lane<R> &L, const KS &ks)
{
#pragma unroll
    for (int u = 1; u < (1 << R); ++u) {
        const int l = ctz_c(u);
        const int g = u ^ (u >> 1);
        const int nb = ((g >> l) & 1) ^ ((l == R - 1) ? PI : 0);
        const u64 k2 = ks.k2(PI, u);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            u64 v = nb ? f32x2::add(L.vF[s], L.GF[s][l]) : f32x2::sub(L.vF[s], L.GF[s][l]);
            v = f32x2::add(v, k2);
            float lo, hi;
            f32x2::unpack(v, lo, hi);
            L.mF[s] = f32x2::min3(L.mF[s], lo, hi);
            L.vF[s] = v;
        }
        const unsigned k = (unsigned)ks.k(PI, u);
        L.vI[0] = L.vI[0] + (nb ? L.GI[0][l] : 0u - L.GI[0][l]) + k;
        L.vI[1] = L.vI[1] + (nb ? L.GI[1][l] : 0u - L.GI[1][l]) + k;
        L.mI = __vimin3_s32(L.mI, (int)L.vI[0], (int)L.vI[1]);
    }
}

// Block transition: record (ra, rb) = (T, code, W0..W5).  The flipped mid bit
// is i = R + (code >> 1), entered with sign + if code is odd; its field for
// group b is T (signed, lane-invariant) + sign * (c_i + b0 s0 + b1 s1 + b2 s2)
// with c_i the lane part from the prefix (sC) and s_t = S[i][nsw + t].
template <int R>
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
    L.vF[0] = f32x2::add(L.vF[0], f32x2::pack((float)base, (float)(base + t0)));
    L.vF[1] = f32x2::add(L.vF[1], f32x2::pack((float)(base + t1), (float)(base + t1 + t0)));
    L.vF[2] = f32x2::add(L.vF[2], f32x2::pack((float)(base + t2), (float)(base + t2 + t0)));
    L.vI[0] += (unsigned)(base + t1 + t2);
    L.vI[1] += (unsigned)(base + t0 + t1 + t2);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        float lo, hi;
        f32x2::unpack(L.vF[s], lo, hi);
        L.mF[s] = f32x2::min3(L.mF[s], lo, hi);
    }
    L.mI = __vimin3_s32(L.mI, (int)L.vI[0], (int)L.vI[1]);
    const int W[6] = {ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const u64 w2 = f32x2::splat((float)W[i]);
#pragma unroll
        for (int s = 0; s < 3; ++s)
            L.GF[s][i] = f32x2::add(L.GF[s][i], w2);
        L.GI[0][i] += (unsigned)W[i];
        L.GI[1][i] += (unsigned)W[i];
    }
}

// Lane set-up for prefix p (variables nsg..n-1, nsg = nsw + 3): the eight
// start values, the low-bit fields of every group and the lane parts of the
// mid-bit fields (sC[(i - R) * stride + slot], unsigned: the sign is applied
// at the transition).
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
    L.vF[0] = f32x2::pack((float)v000, (float)v001);
    L.vF[1] = f32x2::pack((float)v010, (float)v011);
    L.vF[2] = f32x2::pack((float)v100, (float)v101);
    L.vI[0] = (unsigned)v110;
    L.vI[1] = (unsigned)v111;
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
        L.GI[0][ii] = (unsigned)(c + s1 + s2);
        L.GI[1][ii] = (unsigned)(c + s0 + s1 + s2);
    }
    for (int ii = R; ii < nsw; ++ii) {
        int c = 0;
        for (int j = 0; j < kp; ++j)
            if ((p >> j) & 1)
                c += sS[ii * n + nsg + j];
        sC[(ii - R) * stride + slot] = c;
    }
    L.mF[0] = fminf((float)v000, (float)v001);
    L.mF[1] = fminf((float)v010, (float)v011);
    L.mF[2] = fminf((float)v100, (float)v101);
    L.mI = min(v110, v111);
}

// The whole walk of one lane (nsw = nsg - 3 bits, eight groups); returns the
// lane's minimum, an integer below 2^23.
template <int R, class KS>
__device__ __forceinline__ int walk_min(Lane<R> &L, int n, int nsg, const int4 *rec4,
                                        const int *sC, const int *sS, int stride, int slot,
                                        const KS &ks)
{
    const int nsw = nsg - 3;
    const int M = nsw - R;
    const unsigned nblocks = 1u << M;
    if (M == 0) {
        block<R, 0>(L, ks);
    } else {
        for (unsigned B = 0; B < nblocks; B += 2) {
            const int4 r1a = __ldg(rec4 + 2 * (B + 1));
            const int4 r1b = __ldg(rec4 + 2 * (B + 1) + 1);
            const unsigned B2 = (B + 2 < nblocks) ? B + 2 : B + 1;
            const int4 r2a = __ldg(rec4 + 2 * B2);
            const int4 r2b = __ldg(rec4 + 2 * B2 + 1);
            block<R, 0>(L, ks);
            trans<R>(L, r1a, r1b, sC, sS, n, nsw, stride, slot);
            block<R, 1>(L, ks);
            if (B + 2 < nblocks)
                trans<R>(L, r2a, r2b, sC, sS, n, nsw, stride, slot);
        }
    }
    return min(min((int)L.mF[0], (int)L.mF[1]), min((int)L.mF[2], L.mI));
}

// Compact form for kernels where code size matters more than a constant-bank
// operand (the batched kernel, which also holds the int32 walk): one copy of
// the block with the parity pi a runtime value (it only changes the sign of
// the step that flips bit R - 1 and which correction row is read), and the
// corrections of step u as one 16-byte shared-memory record
// kx[pi * 64 + u] = (K as FP32 pair, K as int32, unused).
template <int R>
__device__ __forceinline__ void block_rt(Lane<R> &L, const int4 *kx, int pi)
{
    const int4 *row = kx + pi * 64;
#pragma unroll
    for (int u = 1; u < (1 << R); ++u) {
        const int l = ctz_c(u);
        const int g = u ^ (u >> 1);
        const int4 kk = row[u];
        const u64 k2 = ((u64)(unsigned)kk.y << 32) | (unsigned)kk.x;
        const bool top = (l == R - 1);
        const int nb = ((g >> l) & 1) ^ (top ? pi : 0);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            u64 v = nb ? f32x2::add(L.vF[s], L.GF[s][l]) : f32x2::sub(L.vF[s], L.GF[s][l]);
            v = f32x2::add(v, k2);
            float lo, hi;
            f32x2::unpack(v, lo, hi);
            L.mF[s] = f32x2::min3(L.mF[s], lo, hi);
            L.vF[s] = v;
        }
        L.vI[0] = L.vI[0] + (nb ? L.GI[0][l] : 0u - L.GI[0][l]) + (unsigned)kk.z;
        L.vI[1] = L.vI[1] + (nb ? L.GI[1][l] : 0u - L.GI[1][l]) + (unsigned)kk.z;
        L.mI = __vimin3_s32(L.mI, (int)L.vI[0], (int)L.vI[1]);
    }
}

template <int R>
__device__ __forceinline__ int walk_min_rt(Lane<R> &L, int n, int nsg, const int4 *rec4,
                                           const int *sC, const int *sS, int stride, int slot,
                                           const int4 *kx)
{
    const int nsw = nsg - 3;
    const unsigned nblocks = 1u << (nsw - R);
    for (unsigned B = 0;; ++B) {
        int4 ra, rb;
        const bool more = B + 1 < nblocks;
        if (more) {
            ra = __ldg(rec4 + 2 * (B + 1));
            rb = __ldg(rec4 + 2 * (B + 1) + 1);
        }
        block_rt<R>(L, kx, (int)(B & 1));
        if (!more)
            break;
        trans<R>(L, ra, rb, sC, sS, n, nsw, stride, slot);
    }
    return min(min((int)L.mF[0], (int)L.mF[1]), min((int)L.mF[2], L.mI));
}

}  // namespace mix
}  // namespace qbf
