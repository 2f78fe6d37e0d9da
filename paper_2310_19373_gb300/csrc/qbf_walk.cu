// qbf_walk.cu -- the Gray-code walk (steps A2-A4 of a solve).
//
// Work split (Section 3.1).  The top kp = n - ns variables of x are fixed per
// GPU thread ("prefix" p, variables ns..n-1); every thread walks the 2^ns
// suffix states of variables 0..ns-1 in reflected Gray order, so step t >= 1
// flips bit CTZ(t) (Section 2.2) and moves the objective by the one-bit
// delta of Eq. 2.  All lanes of a warp walk the same suffix at the same step:
// the flipped bit, its sign and every Q entry the step touches are uniform
// across the warp, and nothing diverges.
//
// Field split.  The local field of suffix bit l,
//     g_l = lin_l + sum_{j != l} S_lj x_j,
// is a lane part c_l(p) = sum_{j in prefix} S_lj p_j, constant over the whole
// walk, plus a lane-invariant part that depends only on the suffix state,
// which is the same for every lane.  The walk keeps only what differs per
// lane in registers:
//   - the fields GL_i of the R low bits (i < R) at the start of each block of
//     2^R steps;
//   - the lane parts c_l of the mid bits (R <= l < ns) in shared memory.
// Inside a block (steps u = 1 .. 2^R - 1, flipped bit l = CTZ(u) < R) the
// low-bit state relative to the block start is a compile-time function of u
// and of the block's parity, so
//     delta_u = s_u * GL_l + K[parity][u]
// with s_u = +-1 and the correction K static per (parity, u) (constant bank).
// At block transitions (u = 0, B >= 1, l = R + CTZ(B)) the delta is
//     s_B * c_l(p) + T_B,
// T_B lane-invariant, and the block-start fields move by lane-invariant W_B.
// Records (T_B, code, W_B) come from tables_kernel.  Per visited state a lane
// therefore spends one three-input integer add and one min.
//
// All arithmetic is int32 on the fixed-point image of Q (qbf_prepare.cu):
// exact for every state, so there is no drift to re-anchor.
//
// Modes: MIN records each prefix's minimum and the global minimum; EMIT
// re-walks flagged prefixes (split into 2^q sub-prefixes) and emits every
// state whose value is <= tau; TRACE writes every visited state (tests).
#include <climits>

#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"
#include "qbf_walk_core.cuh"

namespace qbf {

__constant__ int c_K[2][64];

namespace {

// corrections from the constant bank (one instance per launch)
struct ConstK {
    __device__ __forceinline__ int get(int pi, int u) const { return c_K[pi][u]; }
};

}  // namespace

template <int R, int MODE>
__global__ void __launch_bounds__(kWalkThreads) walk_split_kernel(const Plan *__restrict__ plan,
                                                                  const Rec *__restrict__ recs,
                                                                  WalkArgs a)
{
    extern __shared__ int smem[];
    const int n = a.n;
    const int ns = a.ns;
    int *sS = smem;
    int *sLin = sS + n * n;
    int *sC = sLin + n;
    if (plan->status != QBF_OK)
        return;

    unsigned long long nitems;
    unsigned long long total = 0;
    unsigned long long nflag = 0;
    const int lowest_mode = (MODE == kModeEmit) && a.top_k == 1 && plan->window == 0;
    if constexpr (MODE == kModeEmit) {
        nflag = lowest_mode ? 1ull : (unsigned long long)a.ctr->flagged;
        if (lowest_mode && a.ctr->lowest == 0xFFFFFFFFu)
            nflag = 0;
        total = nflag << a.q;
        nitems = (total + 31) >> 5;
    } else {
        nitems = a.nitems;
    }
    // the EMIT grid is sized before the flagged count is known: blocks past
    // the work leave before staging the image (the others drain every item)
    if ((unsigned long long)blockIdx.x * (blockDim.x >> 5) >= nitems)
        return;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        sS[e] = plan->S[e];
    for (int e = threadIdx.x; e < n; e += blockDim.x)
        sLin[e] = plan->lin[e];
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int4 *rec4 = reinterpret_cast<const int4 *>(recs);

    const int tau = (MODE == kModeEmit) ? a.ctr->tau : 0;

    while (true) {
        unsigned long long item = 0;
        if (lane == 0) {
            item = atomicAdd(&a.ctr->items[MODE], 1ull);
            if (cancelled(a.cancel))  // qbf_cancel: take no more items
                item = nitems;
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems)
            break;

        // ---- A2: the lane's prefix ------------------------------------
        unsigned long long p;
        bool active;
        if constexpr (MODE == kModeEmit) {
            unsigned long long i = item * 32 + lane;
            active = i < total;
            unsigned long long ic = active ? i : total - 1;
            // flagged prefixes are numbered from p_lo (the MIN walk's range)
            unsigned long long fp = a.p_lo + (lowest_mode ? (unsigned long long)a.ctr->lowest
                                                          : (unsigned long long)a.flagged[ic >> a.q]);
            p = (fp << a.q) | (ic & ((1ull << a.q) - 1));
        } else {
            unsigned long long i = a.p_lo + item * 32 + lane;
            active = i < a.p_hi;
            p = active ? i : a.p_lo;
        }
        const unsigned long long pbase = p << ns;
        const unsigned long long slot0 = (p - a.p_lo) << ns;

        // value of (prefix, suffix = 0) and the lane parts of the suffix fields
        unsigned GL[R];
        unsigned v = lane_setup<R>(p, n, ns, sS, sLin, sC, blockDim.x, threadIdx.x, GL);

        // ---- A3/A4: the walk -------------------------------------------
        int m = (int)v;
        if constexpr (MODE == kModeMin) {
            m = walk_suffix_min<R>(v, GL, ns, rec4, sC, blockDim.x, threadIdx.x, ConstK());
        } else if (MODE == kModeEmit && lowest_mode) {
            // exact values (W = 0), top-1: only the lowest tied index of each
            // lane can win, so each lane emits that one state
            unsigned long long best = ~0ull;
            walk_suffix_visit<R>(v, GL, ns, rec4, sC, blockDim.x, threadIdx.x, ConstK(),
                                 [&](unsigned val, unsigned t) {
                                     if ((int)val <= tau) {
                                         const unsigned long long x =
                                             pbase | (unsigned long long)(t ^ (t >> 1));
                                         best = x < best ? x : best;
                                     }
                                 });
            if (active && best != ~0ull) {
                unsigned long long pos = atomicAdd(&a.ctr->cand, 1ull);
                if (pos < a.cand_cap)
                    a.cand[pos] = best;
            }
        } else if constexpr (MODE == kModeEmit) {
            walk_suffix_visit<R>(v, GL, ns, rec4, sC, blockDim.x, threadIdx.x, ConstK(),
                                 [&](unsigned val, unsigned t) {
                                     if ((int)val <= tau && active) {
                                         unsigned long long pos = atomicAdd(&a.ctr->cand, 1ull);
                                         if (pos < a.cand_cap)
                                             a.cand[pos] = pbase | (unsigned long long)(t ^ (t >> 1));
                                     }
                                 });
        } else {
            walk_suffix_visit<R>(v, GL, ns, rec4, sC, blockDim.x, threadIdx.x, ConstK(),
                                 [&](unsigned val, unsigned t) {
                                     if (active) {
                                         a.trace_idx[slot0 + t] =
                                             pbase | (unsigned long long)(t ^ (t >> 1));
                                         a.trace_val[slot0 + t] = (long long)(int)val;
                                     }
                                 });
        }

        if constexpr (MODE == kModeMin) {
            if (active)
                a.pmin[p - a.p_lo] = m;
            int wm = active ? m : INT_MAX;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                wm = min(wm, __shfl_xor_sync(0xffffffffu, wm, o));
            if (lane == 0)
                atomicMin(&a.ctr->gmin, wm);
        }
    }
}

// ---------------------------------------------------------------------------
// launch helpers

template <int R, int MODE>
static cudaError_t launch_walk_r(const Plan *plan, const Rec *recs, const WalkArgs &a, int grid,
                                 size_t smem, cudaStream_t s)
{
    auto k = walk_split_kernel<R, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    k<<<grid, kWalkThreads, smem, s>>>(plan, recs, a);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_walk_m(int R, const Plan *plan, const Rec *recs, const WalkArgs &a,
                                 int grid, size_t smem, cudaStream_t s)
{
    switch (R) {
    case 1: return launch_walk_r<1, MODE>(plan, recs, a, grid, smem, s);
    case 2: return launch_walk_r<2, MODE>(plan, recs, a, grid, smem, s);
    case 3: return launch_walk_r<3, MODE>(plan, recs, a, grid, smem, s);
    case 4: return launch_walk_r<4, MODE>(plan, recs, a, grid, smem, s);
    case 5: return launch_walk_r<5, MODE>(plan, recs, a, grid, smem, s);
    default: return launch_walk_r<6, MODE>(plan, recs, a, grid, smem, s);
    }
}

size_t walk_smem_bytes(int n, int ns, int R)
{
    return (size_t)(n * n + n + 2 * (ns - R) * kWalkThreads) * sizeof(int);
}

template <int R, int MODE>
static int occ_r(size_t smem)
{
    int b = 0;
    auto k = walk_split_kernel<R, MODE>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kWalkThreads, smem) != cudaSuccess)
        return 1;
    return b < 1 ? 1 : b;
}

int walk_blocks_per_sm(int R, int mode, size_t smem)
{
#define QBF_OCC(RR)                                                                              \
    case RR:                                                                                     \
        return mode == kModeMin ? occ_r<RR, kModeMin>(smem)                                      \
                                : (mode == kModeEmit ? occ_r<RR, kModeEmit>(smem)                \
                                                     : occ_r<RR, kModeTrace>(smem));
    switch (R) {
        QBF_OCC(1)
        QBF_OCC(2)
        QBF_OCC(3)
        QBF_OCC(4)
        QBF_OCC(5)
    default:
        QBF_OCC(6)
    }
#undef QBF_OCC
}

cudaError_t launch_walk(int mode, int R, const Plan *plan, const Rec *recs, const WalkArgs &a,
                        int grid, cudaStream_t s)
{
    const size_t smem = walk_smem_bytes(a.n, a.ns, R);
    switch (mode) {
    case kModeMin: return launch_walk_m<kModeMin>(R, plan, recs, a, grid, smem, s);
    case kModeEmit: return launch_walk_m<kModeEmit>(R, plan, recs, a, grid, smem, s);
    default: return launch_walk_m<kModeTrace>(R, plan, recs, a, grid, smem, s);
    }
}

cudaError_t copy_corrections(const int *Kbuf_dev, cudaStream_t s)
{
    return cudaMemcpyToSymbolAsync(c_K, Kbuf_dev, sizeof(int) * 128, 0, cudaMemcpyDeviceToDevice, s);
}

}  // namespace qbf
