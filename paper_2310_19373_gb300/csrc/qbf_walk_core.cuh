// qbf_walk_core.cuh -- device building blocks of the split-field Gray walk,
// shared by the single-instance kernel (qbf_walk.cu) and the batched
// persistent kernel (qbf_batched.cu).  The derivation is in qbf_walk.cu.
#pragma once

#include <climits>

#include "qbf_internal.cuh"

namespace qbf {

__host__ __device__ constexpr int ctz_c(int u)
{
    int l = 0;
    while (!((u >> l) & 1))
        ++l;
    return l;
}

// Corrections K[parity][u] read from shared memory (batched kernel: one
// instance per warp, so the constant bank cannot hold them).
struct SmemK {
    const int *p;
    __device__ __forceinline__ int get(int pi, int u) const { return p[pi * 64 + u]; }
};

// Steps u = 1 .. 2^R - 1 of one block of parity PI (MIN mode).  Two
// consecutive states share one three-input min, so a state costs one
// three-input add plus half a min.
template <int R, int PI, class KS>
__device__ __forceinline__ void walk_block_min(unsigned &v, int &m, const unsigned (&GL)[R],
                                               const KS &ks)
{
#pragma unroll
    for (int u = 1; u < (1 << R); u += 2) {
        const int l1 = ctz_c(u);
        const int g1 = u ^ (u >> 1);
        const int nb1 = ((g1 >> l1) & 1) ^ ((l1 == R - 1) ? PI : 0);
        const unsigned va = v + (nb1 ? GL[l1] : 0u - GL[l1]) + (unsigned)ks.get(PI, u);
        if (u + 1 < (1 << R)) {
            const int u2 = u + 1;
            const int l2 = ctz_c(u2);
            const int g2 = u2 ^ (u2 >> 1);
            const int nb2 = ((g2 >> l2) & 1) ^ ((l2 == R - 1) ? PI : 0);
            const unsigned vb = va + (nb2 ? GL[l2] : 0u - GL[l2]) + (unsigned)ks.get(PI, u2);
            m = __vimin3_s32(m, (int)va, (int)vb);
            v = vb;
        } else {
            m = min(m, (int)va);
            v = va;
        }
    }
}

// Block transition (MIN mode): record (ra, rb) = (T, code, W0..W5); the
// signed lane part of the flipped mid bit is sC[code * stride + slot].
template <int R>
__device__ __forceinline__ void block_transition_min(unsigned &v, int &m, unsigned (&GL)[R],
                                                     const int4 ra, const int4 rb, const int *sC,
                                                     int stride, int slot)
{
    const int c = sC[ra.y * stride + slot];
    v = v + (unsigned)ra.x + (unsigned)c;
    m = min(m, (int)v);
    const int W[6] = {ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
    for (int i = 0; i < R; ++i)
        GL[i] += (unsigned)W[i];
}

// Lane set-up for prefix p (variables ns..n-1): value of (p, suffix 0), the
// low-bit fields GL and the signed lane parts of the mid-bit fields.
template <int R>
__device__ __forceinline__ unsigned lane_setup(unsigned long long p, int n, int ns, const int *sS,
                                               const int *sLin, int *sC, int stride, int slot,
                                               unsigned (&GL)[R])
{
    const int kp = n - ns;
    unsigned v = 0;
    for (int j = 0; j < kp; ++j) {
        if (!((p >> j) & 1))
            continue;
        const int i = ns + j;
        unsigned row = (unsigned)sLin[i];
        for (int jj = j + 1; jj < kp; ++jj)
            if ((p >> jj) & 1)
                row += (unsigned)sS[i * n + ns + jj];
        v += row;
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        unsigned c = (unsigned)sLin[i];
        for (int j = 0; j < kp; ++j)
            if ((p >> j) & 1)
                c += (unsigned)sS[i * n + ns + j];
        GL[i] = c;
    }
    for (int i = R; i < ns; ++i) {
        unsigned c = 0;
        for (int j = 0; j < kp; ++j)
            if ((p >> j) & 1)
                c += (unsigned)sS[i * n + ns + j];
        sC[(2 * (i - R) + 1) * stride + slot] = (int)c;
        sC[(2 * (i - R)) * stride + slot] = (int)(0u - c);
    }
    return v;
}

// The whole suffix walk of one lane in MIN mode; returns the lane's minimum.
template <int R, class KS>
__device__ __forceinline__ int walk_suffix_min(unsigned v, unsigned (&GL)[R], int ns,
                                               const int4 *rec4, const int *sC, int stride,
                                               int slot, const KS &ks)
{
    int m = (int)v;
    const int M = ns - R;
    const unsigned nblocks = 1u << M;
    if (M == 0) {
        walk_block_min<R, 0>(v, m, GL, ks);
        return m;
    }
    for (unsigned B = 0; B < nblocks; B += 2) {
        const int4 r1a = __ldg(rec4 + 2 * (B + 1));
        const int4 r1b = __ldg(rec4 + 2 * (B + 1) + 1);
        const unsigned B2 = (B + 2 < nblocks) ? B + 2 : B + 1;
        const int4 r2a = __ldg(rec4 + 2 * B2);
        const int4 r2b = __ldg(rec4 + 2 * B2 + 1);
        walk_block_min<R, 0>(v, m, GL, ks);
        block_transition_min<R>(v, m, GL, r1a, r1b, sC, stride, slot);
        walk_block_min<R, 1>(v, m, GL, ks);
        if (B + 2 < nblocks)
            block_transition_min<R>(v, m, GL, r2a, r2b, sC, stride, slot);
    }
    return m;
}

// The whole suffix walk of one lane calling visit(value, t) at every state t
// (t = step counter; the suffix state is gray(t) = t ^ (t >> 1)).  Used by
// the EMIT and TRACE modes, which are not on the timed path.
template <int R, class KS, class F>
__device__ __forceinline__ void walk_suffix_visit(unsigned v, unsigned (&GL)[R], int ns,
                                                  const int4 *rec4, const int *sC, int stride,
                                                  int slot, const KS &ks, F &&visit)
{
    const int M = ns - R;
    const unsigned nblocks = 1u << M;
    visit(v, 0u);
    for (unsigned B = 0; B < nblocks; ++B) {
        const int pi = B & 1;
        if (B > 0) {
            const int4 ra = __ldg(rec4 + 2 * B);
            const int4 rb = __ldg(rec4 + 2 * B + 1);
            const int c = sC[ra.y * stride + slot];
            v = v + (unsigned)ra.x + (unsigned)c;
            visit(v, B << R);
            const int W[6] = {ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
            for (int i = 0; i < R; ++i)
                GL[i] += (unsigned)W[i];
        }
#pragma unroll
        for (int u = 1; u < (1 << R); ++u) {
            const int l = ctz_c(u);
            const int g = u ^ (u >> 1);
            const int nb = ((g >> l) & 1) ^ ((l == R - 1) ? pi : 0);
            v = v + (nb ? GL[l] : 0u - GL[l]) + (unsigned)ks.get(pi, u);
            visit(v, (B << R) | (unsigned)u);
        }
    }
}

}  // namespace qbf
