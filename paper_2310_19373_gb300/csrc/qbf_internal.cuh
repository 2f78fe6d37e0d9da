// qbf_internal.cuh -- device-side data layout shared by the libqubobf kernels.
//
// Notation (arXiv 2310.19373):
//   f(x) = x^T Q x (Eq. 1).  With lin_i = Q_ii and S_ij = Q_ij + Q_ji (i != j,
//   the symmetrised off-diagonal of Section 3), f(x) = sum_i lin_i x_i +
//   sum_{i<j} S_ij x_i x_j, and flipping bit l changes f by
//   s_l * g_l with g_l = lin_l + sum_{j != l} S_lj x_j (Eq. 2),
//   s_l = +1 if bit l becomes 1, else -1.
//
// The walk kernels run on an int32 fixed-point image of Q:
//   lin^_i = round(lin_i * 2^sigma), S^_ij = round(S_ij * 2^sigma)
// with sigma chosen so that sum |lin^| + sum_{i<j} |S^| < 2^31.  Every
// objective value and every field g^ of every state is then bounded by that
// sum, so int32 adds (wrapping, two's complement) give the exact fixed-point
// value of every state.
#pragma once

#include <cstdint>

#include "qbf.h"

namespace qbf {

constexpr int kMaxN = QBF_MAX_N;
constexpr int kRMax = 6;  // low bits whose walk is unrolled at compile time

// Two-limb images of the log Z walks (qbf_prepare.cu): each limb's sum of
// |entries| is at most kLzLimbMax = 2^22, so the walks run exactly in FP32;
// the lo limb carries logz_lo_bits(n) more bits: its entries are at most
// 2^(L-1) in magnitude over n(n+1)/2 of them, L = 23 - ceil(log2(n(n+1)/2)),
// at most 16.
constexpr long long kLzLimbMax = 1ll << 22;
__host__ __device__ constexpr int logz_lo_bits(int n)
{
    int c = 0;
    while ((1ll << c) < (long long)n * (n + 1) / 2)
        ++c;
    return 23 - c < 16 ? 23 - c : 16;
}

// Cancellation: a flag word in device memory (qbf_cancel writes it with the
// copy engine while a solve runs).  A warp's lane 0 reads it whenever it takes
// a work item; once it is set the warp takes no more, so every persistent walk
// ends at its current items.
__device__ __forceinline__ bool cancelled(const volatile int *cancel)
{
    return cancel != nullptr && *cancel != 0;
}

// Written by the prepare kernel, read by every later kernel of a solve.
struct Plan {
    int n;
    int status;       // QBF_OK or the error found while preparing
    int sigma;        // fixed-point scale exponent
    int dtype;
    long long window; // certification window W, in fixed-point quanta
    long long vhat;   // sum |lin^| + sum_{i<j} |S^|
    double error_bound;  // W / 2 in units of f
    double eq_quanta;    // quantisation error bound, quanta
    int lin[kMaxN];
    int S[kMaxN * kMaxN];  // symmetric, zero diagonal
};

// Lane-invariant data of the block transition B (see qbf_walk.cu).
struct Rec {
    int T;          // s_B * (lane-invariant part of the field of the flipped bit)
    int code;       // 2 * (l - R) + (new value of bit l); selects the signed lane field
    int W[kRMax];   // change of the low-bit block-start fields
};

// Flags and counters of one solve (device memory, zeroed per solve).
struct Counters {
    int gmin;                 // global fixed-point minimum (atomicMin)
    int tau;                  // candidate threshold
    unsigned int flagged;     // number of flagged prefixes
    unsigned int lowest;      // lowest flagged prefix (exact top-1 mode)
    unsigned long long items[4];  // work-queue heads, one per walk mode
    unsigned long long cand;  // number of emitted candidates (may exceed capacity)
    int status;
    int pad1;
};

// Final answer written by the select kernel, copied to the host.
struct DevResult {
    double topk_value[QBF_MAX_TOPK];
    unsigned long long topk_index[QBF_MAX_TOPK];
    int count;
    int status;
    unsigned long long n_candidates;
};

// One instance of a batched solve (written by the host, read by the kernels).
struct BatchDesc {
    const void *Q;                 // caller's matrix, n_src x n_src, row-major
    int n_src;                     // caller's n
    int n;                         // walk dimension (>= n_src; extra variables are zero)
    int dtype;
    int ns;                        // suffix bits walked per lane
    unsigned long long nprefix;    // 2^(n - ns)
    unsigned long long item_off;   // first global work item (32 prefixes each)
    unsigned long long rec_off;    // first walk record
    unsigned long long ftab_off;   // first suffix-table entry (table-driven deferred
                                   // walk), or ~0 when the instance has none
};

}  // namespace qbf
