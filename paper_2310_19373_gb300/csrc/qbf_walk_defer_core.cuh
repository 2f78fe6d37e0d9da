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
// ---------------------------------------------------------------------------
// Table-driven form (qbf_walk_defer.cu has the derivation): the lane keeps
// only the lane parts w_b of its eight values, its low-bit fields are
// constants of the walk, and the lane-invariant suffix energy F(gray(t)) of
// every step comes from a table staged per warp into shared memory.
// ---------------------------------------------------------------------------

// low-bit fields kept in registers; those of variables kDefer2RegBits..R-1
// (flipped 2^(R-1-l) times per block) are read from the lane's shared memory.
// Measured at n = 40 with 64-step blocks: all six in registers 54.5 ms; five
// 57.2 ms; four 57.1 ms (three CTAs per SM), 58.6 ms (four CTAs per SM, 64
// registers with spills).  With 128-step blocks the seventh (flipped once per
// block) comes from shared memory: 53.0 ms.
constexpr int kDefer2RegBits = 6;

namespace dfr2 {

using f32x2::u64;

template <int R>
struct Lane {
    u64 w[4];      // lane parts of the eight values, pairs (b0 = 0, b0 = 1) of (b2 b1)
    u64 GF[4][R];  // lane parts c_l(b, p) of the low-bit fields (constant; only
                   // l < kDefer2RegBits live here, the rest in shared memory)
    float m[2];    // running minima (two chains)
};

// cp.async of 16 bytes, global -> shared
__device__ __forceinline__ void cp16(void *dst_smem, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One block of 2^R states, parity pi (a runtime value: it only reverses the
// flip of variable R - 1 at u = 2^(R-1), so one unrolled copy serves both).
// State u = 0 is the block's first state; Fs holds its 2^R table values.
template <int R>
__device__ __forceinline__ void block(Lane<R> &L, const float *Fs, int pi,
                                      const ulonglong2 *sGFx, int stride, int slot)
{
    float tp = 0.f;
    float4 f4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < (1 << R); ++u) {
        if (u > 0) {
            const int l = ctz_c(u);
            const int nb = ((u ^ (u >> 1)) >> l) & 1;
            u64 g[4];
            if (l < kDefer2RegBits) {
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    g[s] = L.GF[s][l];
            } else {
                const ulonglong2 g01 = sGFx[((l - kDefer2RegBits) * 2) * stride + slot];
                const ulonglong2 g23 = sGFx[((l - kDefer2RegBits) * 2 + 1) * stride + slot];
                g[0] = g01.x;
                g[1] = g01.y;
                g[2] = g23.x;
                g[3] = g23.y;
            }
            if (l == R - 1) {
                if (nb ^ pi) {
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        L.w[s] = f32x2::add(L.w[s], g[s]);
                } else {
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        L.w[s] = f32x2::sub(L.w[s], g[s]);
                }
            } else {
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    L.w[s] = nb ? f32x2::add(L.w[s], g[s]) : f32x2::sub(L.w[s], g[s]);
            }
        }
        float x[8];
#pragma unroll
        for (int s = 0; s < 4; ++s)
            f32x2::unpack(L.w[s], x[2 * s], x[2 * s + 1]);
        const float t = dfr::min8(x);
        if ((u & 3) == 0)
            f4 = *reinterpret_cast<const float4 *>(Fs + u);
        if (u & 1) {
            // states u - 1 and u: one packed add of their F, one three-input min
            const float fa = (u & 2) ? f4.z : f4.x;
            const float fb = (u & 2) ? f4.w : f4.y;
            const u64 y = f32x2::add(f32x2::pack(tp, t), f32x2::pack(fa, fb));
            float lo, hi;
            f32x2::unpack(y, lo, hi);
            L.m[(u >> 1) & 1] = f32x2::min3(L.m[(u >> 1) & 1], lo, hi);
        } else {
            tp = t;
        }
    }
}

// Transition into block B >= 1: mid variable R + j, j = CTZ(B), takes bit j of
// gray(B); the eight values move by +-c_{R+j}(b, p): the lane part (sCf) plus
// the lane-invariant group terms (sE: per mid variable and direction, the
// eight signed values as two float4).
template <int R>
__device__ __forceinline__ void mid_flip(Lane<R> &L, unsigned B, const float *sCf, int stride,
                                         int slot, const float4 *sE)
{
    const int j = __ffs(B) - 1;
    const int up = ((B ^ (B >> 1)) >> j) & 1;
    const float c = sCf[j * stride + slot];
    const float sc = up ? c : -c;
    const u64 y = f32x2::pack(sc, sc);
    const float4 e01 = sE[(j * 2 + up) * 2];
    const float4 e23 = sE[(j * 2 + up) * 2 + 1];
    L.w[0] = f32x2::add(L.w[0], f32x2::add(y, f32x2::pack(e01.x, e01.y)));
    L.w[1] = f32x2::add(L.w[1], f32x2::add(y, f32x2::pack(e01.z, e01.w)));
    L.w[2] = f32x2::add(L.w[2], f32x2::add(y, f32x2::pack(e23.x, e23.y)));
    L.w[3] = f32x2::add(L.w[3], f32x2::add(y, f32x2::pack(e23.z, e23.w)));
}

// Lane set-up for prefix p (variables nsg..n-1): the eight start values (F of
// the empty suffix is 0, so they are the values themselves), the lane parts
// of the low-bit fields, and those of the mid-bit fields (sCf).
template <int R>
__device__ __forceinline__ void setup(Lane<R> &L, unsigned long long p, int n, int nsg,
                                      const int *sS, const int *sLin, float *sCf, int stride,
                                      int slot, ulonglong2 *sGFx)
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
    const int v000 = va, v001 = va + gf[0];
    const int v010 = va + gf[1], v011 = v010 + gf[0] + s01;
    const int v100 = va + gf[2], v101 = v100 + gf[0] + s02;
    const int v110 = v010 + gf[2] + s12, v111 = v011 + gf[2] + s02 + s12;
    L.w[0] = f32x2::pack((float)v000, (float)v001);
    L.w[1] = f32x2::pack((float)v010, (float)v011);
    L.w[2] = f32x2::pack((float)v100, (float)v101);
    L.w[3] = f32x2::pack((float)v110, (float)v111);
#pragma unroll
    for (int ii = 0; ii < R; ++ii) {
        int c = 0;
        for (int j = 0; j < kp; ++j)
            if ((p >> j) & 1)
                c += sS[ii * n + nsg + j];
        const int s0 = sS[ii * n + nsw], s1 = sS[ii * n + nsw + 1], s2 = sS[ii * n + nsw + 2];
        const u64 g0 = f32x2::pack((float)c, (float)(c + s0));
        const u64 g1 = f32x2::pack((float)(c + s1), (float)(c + s1 + s0));
        const u64 g2 = f32x2::pack((float)(c + s2), (float)(c + s2 + s0));
        const u64 g3 = f32x2::pack((float)(c + s1 + s2), (float)(c + s0 + s1 + s2));
        if (ii < kDefer2RegBits) {
            L.GF[0][ii] = g0;
            L.GF[1][ii] = g1;
            L.GF[2][ii] = g2;
            L.GF[3][ii] = g3;
        } else {
            sGFx[((ii - kDefer2RegBits) * 2) * stride + slot] = make_ulonglong2(g0, g1);
            sGFx[((ii - kDefer2RegBits) * 2 + 1) * stride + slot] = make_ulonglong2(g2, g3);
        }
    }
    for (int ii = R; ii < nsw; ++ii) {
        int c = 0;
        for (int j = 0; j < kp; ++j)
            if ((p >> j) & 1)
                c += sS[ii * n + nsg + j];
        sCf[(ii - R) * stride + slot] = (float)c;
    }
    L.m[0] = L.m[1] = __int_as_float(0x7f800000);  // +inf: every state is compared
}

// The whole walk of one lane: blocks in Gray order of the mid bits, each
// block's F staged by the warp into its double buffer one block ahead.
template <int R>
__device__ __forceinline__ int walk_min(Lane<R> &L, int nsw, const float *ftab, float *fbuf,
                                        int lane, const float *sCf, int stride, int slot,
                                        const float4 *sE, const ulonglong2 *sGFx)
{
    constexpr int BS = 1 << R;  // F values per block; a multiple of 4 (R >= 2)
    const unsigned nblocks = 1u << (nsw - R);
    if (lane < BS / 4)
        cp16(fbuf + 4 * lane, ftab + 4 * lane);
    cp_commit();
    for (unsigned B = 0; B < nblocks; ++B) {
        const float *cur = fbuf + (B & 1) * BS;
        if (B + 1 < nblocks) {
            if (lane < BS / 4)
                cp16(fbuf + ((B + 1) & 1) * BS + 4 * lane, ftab + (size_t)(B + 1) * BS + 4 * lane);
            cp_commit();
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncwarp();
        if (B > 0)
            mid_flip<R>(L, B, sCf, stride, slot, sE);
        block<R>(L, cur, (int)(B & 1), sGFx, stride, slot);
        __syncwarp();  // every lane is done with cur before it is refilled
    }
    return (int)fminf(L.m[0], L.m[1]);
}

}  // namespace dfr2

}  // namespace qbf
