// qbf_walk_defer_core.cuh -- device building blocks of the deferred-correction
// walk, shared by the single-instance kernel (qbf_walk_defer.cu, where the
// derivation is) and the batched persistent kernel (qbf_batched.cu).
//
// A lane walks nsw suffix bits for the eight values b = (b2 b1 b0) of its
// three group bits (variables nsw, nsw+1, nsw+2) as four f32x2 pairs, each
// value kept without its in-block correction C[pi][u].  CS gives the sums:
// cs.c(pi, u) = C[pi][u] and cs.ce(pi) = C[pi][2^R - 1].
#pragma once

#include "qbf_f32x2.cuh"
#include "qbf_internal.cuh"
#include "qbf_walk_core.cuh"

namespace qbf {
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
template <int R, int PI, class CS>
__device__ __forceinline__ void block(Lane<R> &L, const CS &cs)
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
        L.m[u & 1] = fminf(L.m[u & 1], min8(x) + cs.c(PI, u));
    }
}

// Block transition: record (ra, rb) = (T, code, W0..W5) as in the two-pipe
// walk; the values first take the finished block's whole correction ce back
// (w -> v), then the mid-bit flip.
template <int R>
__device__ __forceinline__ void trans(Lane<R> &L, const int4 ra, const int4 rb, const int *sC,
                                      const int *sS, int n, int nsw, int stride, int slot, float ce_)
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
    const u64 ce = f32x2::splat(ce_);
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
template <int R, class CS>
__device__ __forceinline__ int walk_min(Lane<R> &L, int n, int nsg, const int4 *rec4,
                                        const int *sC, const int *sS, int stride, int slot,
                                        const CS &cs)
{
    const int nsw = nsg - 3;
    const int M = nsw - R;
    const unsigned nblocks = 1u << M;
    if (M == 0) {
        block<R, 0>(L, cs);
    } else {
        // records are read at the transition, not prefetched a block pair
        // ahead: the 16 registers a prefetch holds keep the kernel at 96
        // registers and two CTAs per SM; without them it runs three
        for (unsigned B = 0; B < nblocks; B += 2) {
            block<R, 0>(L, cs);
            {
                const int4 ra = __ldg(rec4 + 2 * (B + 1));
                const int4 rb = __ldg(rec4 + 2 * (B + 1) + 1);
                trans<R>(L, ra, rb, sC, sS, n, nsw, stride, slot, cs.ce(0));
            }
            block<R, 1>(L, cs);
            if (B + 2 < nblocks) {
                const int4 ra = __ldg(rec4 + 2 * (B + 2));
                const int4 rb = __ldg(rec4 + 2 * (B + 2) + 1);
                trans<R>(L, ra, rb, sC, sS, n, nsw, stride, slot, cs.ce(1));
            }
        }
    }
    return (int)fminf(L.m[0], L.m[1]);
}

// Compact form for the batched kernel, where code size matters more than a
// constant-bank operand: one copy of the block with the parity pi a runtime
// value, the sums C from shared memory: cd[pi * 64 + u], the block totals at
// u = 2^R - 1.
template <int R>
__device__ __forceinline__ void block_rt(Lane<R> &L, const float *cd, int pi)
{
    const float *row = cd + pi * 64;
#pragma unroll
    for (int u = 1; u < (1 << R); ++u) {
        const int l = ctz_c(u);
        const int g = u ^ (u >> 1);
        const bool top = (l == R - 1);
        const int nb = ((g >> l) & 1) ^ (top ? pi : 0);
        float x[8];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            L.v[s] = nb ? f32x2::add(L.v[s], L.GF[s][l]) : f32x2::sub(L.v[s], L.GF[s][l]);
            f32x2::unpack(L.v[s], x[2 * s], x[2 * s + 1]);
        }
        L.m[u & 1] = fminf(L.m[u & 1], min8(x) + row[u]);
    }
}

template <int R>
__device__ __forceinline__ int walk_min_rt(Lane<R> &L, int n, int nsg, const int4 *rec4,
                                           const int *sC, const int *sS, int stride, int slot,
                                           const float *cd)
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
        const int pi = (int)(B & 1);
        block_rt<R>(L, cd, pi);
        if (!more)
            break;
        trans<R>(L, ra, rb, sC, sS, n, nsw, stride, slot, cd[pi * 64 + (1 << R) - 1]);
    }
    return (int)fminf(L.m[0], L.m[1]);
}

}  // namespace dfr
}  // namespace qbf
