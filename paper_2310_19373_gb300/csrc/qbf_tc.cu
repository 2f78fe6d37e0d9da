// qbf_tc.cu -- the blocked tensor-core form of the minimum walk (row A8).
//
// x is split into s (variables 0..6, 128 values: the rows of a tile), c
// (variables 7..13, 128 values: the columns) and T (variables 14..n-1, fixed
// per tile).  With lin/S the fixed-point image of Q (qbf_prepare.cu, built with
// sum |image| < 2^22 for this kernel):
//     f(T, c, s) = f_ss(s) + D[s, c],
//     D[s, c]    = sum_{i<7} s_i h_i(c, T) + F(c, T),
//     h_i(c, T)  = sum_{j in c, T} S_ij x_j        (cross field of row bit i)
//     F(c, T)    = f restricted to the (c, T) variables.
// (the tensor core computes the parts of D that depend on c; see below)
// D for the whole 128 x 128 tile is one tcgen05.mma (kind::f16, M = N = 128,
// K = 16): A[s, 2i] = 2048 s_i, A[s, 2i+1] = s_i, A[s, 14] = 2048, A[s, 15] = 1
// and B[2i, c] / B[2i+1, c] the high / low limbs of h_i (h = 2048 hi + lo,
// |hi| <= 2048, |lo| <= 1024), B[14..15, c] the limbs of F.  Every operand is an
// integer exactly representable in FP16, every product and partial sum is an
// integer below 2^23, so the FP32 accumulator in tensor memory holds D exactly.
// f_ss(s) is constant along a row, so it is added once after the row minimum.
// The epilogue per state is therefore half of a three-input min.
//
// Only the column part of h_i goes through the MMA: T's part,
// sum_i s_i HT_i(T), is constant along a row, like f_ss(s) and f_TT(T), and is
// added after the row minimum.  So the 14 cross-field rows of B depend only on
// the column and are written once; per tile each column rewrites just the two
// limbs of F'(c, T) = F_cc(c) + sum_j c_j G_j(T) (G_j: field of column bit j
// from T's variables).
//
// Output: the minimum over each tile's 2^14 states, i.e. the per-prefix minima
// of a walk with 14 suffix bits, so the certification step of qbf_solve (flag,
// re-walk, rescore, select) applies unchanged.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"

namespace qbf {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcRowBits = 7;  // s: M = 128
constexpr int kTcColBits = 7;  // c: N = 128
constexpr int kTcTileBits = kTcRowBits + kTcColBits;
constexpr uint32_t kTcCols = 128;  // TMEM columns (one 128 x 128 FP32 accumulator)
constexpr unsigned long long kTcSpinLimit = 1ull << 20;  // waits of <= 1 us each
constexpr uint32_t kTcSuspendNs = 1000;

// ---- inline PTX wrappers ---------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void mma_f16_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// the waiting thread may be suspended for up to kTcSuspendNs instead of spinning
__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity), "r"(kTcSuspendNs)
        : "memory");
    return ok;
}

// bounded wait: returns false if the barrier did not complete
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity)
{
    for (unsigned long long it = 0; it < kTcSpinLimit; ++it)
        if (mbar_try_wait(mbar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]), "=f"(r[16]), "=f"(r[17]), "=f"(r[18]), "=f"(r[19]), "=f"(r[20]), "=f"(r[21]), "=f"(r[22]), "=f"(r[23]), "=f"(r[24]), "=f"(r[25]), "=f"(r[26]), "=f"(r[27]), "=f"(r[28]), "=f"(r[29]), "=f"(r[30]), "=f"(r[31])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Shared-memory matrix descriptor, no swizzle, K-major: core matrices of 8 rows
// x 16 bytes; lbo = byte distance between K-adjacent core matrices, sbo =
// between M/N-adjacent 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for this architecture
    return d;                // base offset 0, absolute LBO mode, layout type 0 (no swizzle)
}

// kind::f16 instruction descriptor: D F32, A/B F16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t M, uint32_t N)
{
    return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// byte offset of element (row, k) of a K-major 16-bit matrix with K = 16:
// 8-row groups 256 B apart, the two 8-element K halves 128 B apart
__host__ __device__ constexpr uint32_t kmajor_off(uint32_t row, uint32_t k)
{
    return (row >> 3) * 256u + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

constexpr uint32_t kLbo = 128, kSbo = 256;

// split v (|v| < 2^22) into hi * 2048 + lo with |lo| <= 1024
__device__ __forceinline__ void limbs(int v, int &hi, int &lo)
{
    hi = (v + 1024) >> 11;
    lo = v - hi * 2048;
}

struct TcShared {
    alignas(1024) unsigned char A[128 * 32];   // 128 x 16 FP16, K-major
    alignas(1024) unsigned char Bm[128 * 32];  // 128 x 16 FP16, K-major
    alignas(8) unsigned long long mbar;
    uint32_t tmem_base;
    int err;
    int uni[2][16];        // per tile (double-buffered): HT_0..6, G_0..6, f_TT
    __half2 uniL[2][8];    // limbs of HT_i (hi, lo)
    int wmin[kTcThreads / 32];
    int S[kMaxN * kMaxN];
    int lin[kMaxN];
};

// Warp 0 keeps the per-tile uniform values of the current tile prefix T in
// registers and publishes them to buffer buf:
//   HT_i = sum_{j in T} S[i][14+j]      (lane i, i < 7)
//   G_j  = sum_{j' in T} S[7+j][14+j']   (lane 7 + j, j < 7)
//   f_TT = f restricted to T's variables (lane 0)
//   g_j  = lin + sum_{j' in T, j' != j} S  -- field of tile bit j (lanes j, j+32)
// Tiles are visited in Gray order inside aligned chunks, so consecutive tiles
// differ in one tile bit b and every value moves by one signed S entry.
struct TileTracker {
    int u;       // HT / G value of lanes 0..13
    int ft;      // f_TT (lane 0)
    int g0, g1;  // fields of tile bits lane and lane + 32

    __device__ __forceinline__ void from_scratch(const int *S, const int *lin, int n, int nT,
                                                 unsigned long long T, int lane)
    {
        const int row = lane < 7 ? lane : kTcRowBits + (lane - 7);
        u = 0;
        if (lane < 14)
            for (int j = 0; j < nT; ++j)
                if ((T >> j) & 1ull)
                    u += S[row * n + kTcTileBits + j];
        g0 = g1 = 0;
        int part = 0;
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            if (j >= nT)
                continue;
            const int vj = kTcTileBits + j;
            int g = lin[vj];
            for (int j2 = 0; j2 < nT; ++j2)
                if (j2 != j && ((T >> j2) & 1ull))
                    g += S[vj * n + kTcTileBits + j2];
            if (h == 0)
                g0 = g;
            else
                g1 = g;
            // f_TT = sum over set bits j of (lin_j + sum_{j2 > j set} S_j,j2)
            if ((T >> j) & 1ull) {
                int rw = lin[vj];
                for (int j2 = j + 1; j2 < nT; ++j2)
                    if ((T >> j2) & 1ull)
                        rw += S[vj * n + kTcTileBits + j2];
                part += rw;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            part += __shfl_xor_sync(0xffffffffu, part, o);
        ft = part;
    }

    // flip tile bit b to value nb
    __device__ __forceinline__ void flip(const int *S, int n, int nT, int b, int nb, int lane)
    {
        const int vb = kTcTileBits + b;
        const int gb = __shfl_sync(0xffffffffu, b < 32 ? g0 : g1, b & 31);
        ft += nb ? gb : -gb;
        if (lane < 14) {
            const int row = lane < 7 ? lane : kTcRowBits + (lane - 7);
            const int sv = S[row * n + vb];
            u += nb ? sv : -sv;
        }
        if (lane < nT && lane != b) {
            const int sv = S[(kTcTileBits + lane) * n + vb];
            g0 += nb ? sv : -sv;
        }
        if (lane + 32 < nT && lane + 32 != b) {
            const int sv = S[(kTcTileBits + lane + 32) * n + vb];
            g1 += nb ? sv : -sv;
        }
    }

    __device__ __forceinline__ void publish(int *uni, int lane) const
    {
        if (lane < 14)
            uni[lane] = u;
        if (lane == 0)
            uni[14] = ft;
    }

    // field of tile bit b (unchanged by flipping b itself)
    __device__ __forceinline__ int field(int b) const
    {
        return __shfl_sync(0xffffffffu, b < 32 ? g0 : g1, b & 31);
    }
};

// Shared memory of the MIN kernel: one CTA per SM runs kTcGroups independent
// 128-thread pipelines (one per 128 TMEM columns).
constexpr int kTcGroups = 4;

constexpr int kTcMaxTileBits = 28;  // n <= 42

struct TcGroupShared {
    alignas(1024) unsigned char A[128 * 32];               // static operand, shared
    alignas(1024) unsigned char Bm[kTcGroups][128 * 32];   // per-group tile operand
    alignas(8) unsigned long long mbar[kTcGroups];
    uint32_t tmem_base;
    int err;
    int uni[kTcGroups][2][16];  // chunk start: HT_0..6, G_0..6, f_TT; else [15] = g_b
    int wmin[kTcGroups][4];
    int Kc[kTcMaxTileBits][128];  // K_b(c) = sum_{j in c} S[7+j][14+b]
    int Rr[kTcMaxTileBits][128];  // R_b(s) = sum_{i in s} S[i][14+b]
    int S[kMaxN * kMaxN];
    int lin[kMaxN];
};

__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kTcThreads) : "memory");
}


}  // namespace

// ---------------------------------------------------------------------------
// self-test: D = A * B for given FP16 A (128 x 16) and B (16 x 128), one CTA.
__global__ void __launch_bounds__(kTcThreads) tc_selftest_kernel(const __half *A, const __half *B,
                                                                 float *D, int *err)
{
    __shared__ TcShared sh;
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    // A[r][k] row-major input -> K-major core-matrix layout
    for (int e = t; e < 128 * 16; e += blockDim.x) {
        const int r = e / 16, k = e % 16;
        *(__half *)(sh.A + kmajor_off(r, k)) = A[e];
        // B[k][c] (K x N row-major) -> column c, K-major
        const int kk = e / 128, c = e % 128;
        *(__half *)(sh.Bm + kmajor_off(c, kk)) = B[e];
    }
    if (w == 0)
        tmem_alloc(smem_u32(&sh.tmem_base), kTcCols);
    if (t == 0)
        mbar_init(smem_u32(&sh.mbar), 1);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sh.tmem_base;
    if (t == 0) {
        const uint64_t ad = smem_desc(smem_u32(sh.A), kLbo, kSbo);
        const uint64_t bd = smem_desc(smem_u32(sh.Bm), kLbo, kSbo);
        mma_f16_ss(tbase, ad, bd, idesc_f16(128, 128), 0);
        mma_commit(smem_u32(&sh.mbar));
    }
    const bool ok = mbar_wait_bounded(smem_u32(&sh.mbar), 0);
    tc_fence_after();
    if (ok) {
        for (int cb = 0; cb < 128; cb += 32) {
            float r[32];
            tmem_ld32(tbase + ((uint32_t)(32 * w) << 16) + (uint32_t)cb, r);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j)
                D[(32 * w + l) * 128 + cb + j] = r[j];
        }
    } else if (l == 0) {
        atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0)
        tmem_dealloc(tbase, kTcCols);
}

// ---------------------------------------------------------------------------
// MIN: per-tile minima of the fixed-point objective (tiles = prefixes of a walk
// with 14 suffix bits).  One CTA of kTcGroups x 128 threads per SM; group g owns
// TMEM columns [128 g, 128 g + 128), its own B buffer, mbarrier and named
// barrier, and walks the chunks g, g + G, ... of its CTA's share in a fixed
// stride (every tile costs the same).
__global__ void __launch_bounds__(kTcThreads * kTcGroups, 1)
    tc_min_kernel(const Plan *__restrict__ plan, int n, unsigned long long p_lo,
                  unsigned long long p_hi, int *pmin, Counters *ctr)
{
    extern __shared__ unsigned char tc_dyn[];
    TcGroupShared &sh = *reinterpret_cast<TcGroupShared *>(
        (reinterpret_cast<uintptr_t>(tc_dyn) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x;
    const int g = tid / kTcThreads, t = tid % kTcThreads;
    const int w = t >> 5, l = t & 31;
    for (int e = tid; e < n * n; e += blockDim.x)
        sh.S[e] = plan->S[e];
    for (int e = tid; e < n; e += blockDim.x)
        sh.lin[e] = plan->lin[e];
    if (tid == 0)
        sh.err = 0;
    if (t == 0)
        mbar_init(smem_u32(&sh.mbar[g]), 1);
    __syncthreads();
    if (plan->status != QBF_OK)
        return;
    const int nT = n - kTcTileBits;  // tile (prefix) bits

    // static A: rows s = 0..127 (group 0 writes it)
    if (g == 0) {
        const int srow = t;
        for (int k = 0; k < 16; ++k) {
            float a;
            if (k < 14)
                a = ((srow >> (k >> 1)) & 1) ? ((k & 1) ? 1.f : 2048.f) : 0.f;
            else
                a = (k == 14) ? 2048.f : 1.f;
            *(__half *)(sh.A + kmajor_off(srow, k)) = __float2half_rn(a);
        }
    }
    // row constant f_ss(s) for this thread's epilogue row r = t
    int fss = 0;
    for (int i = 0; i < kTcRowBits; ++i) {
        if (!((t >> i) & 1))
            continue;
        fss += sh.lin[i];
        for (int i2 = i + 1; i2 < kTcRowBits; ++i2)
            if ((t >> i2) & 1)
                fss += sh.S[i * n + i2];
    }
    // column c = t: the 14 cross-field rows of B (limbs of c's part of h_i)
    // are the same for every tile, so they are written once; F_cc(c) is kept
    int fcc = 0;
    {
        const int c = t;
        alignas(16) __half2 col[8];
        for (int i = 0; i < kTcRowBits; ++i) {
            int v = 0;
            for (int j = 0; j < kTcColBits; ++j)
                if ((c >> j) & 1)
                    v += sh.S[i * n + kTcRowBits + j];
            int hi, lo;
            limbs(v, hi, lo);
            col[i] = __halves2half2(__int2half_rn(hi), __int2half_rn(lo));
        }
        col[7] = __halves2half2(__int2half_rn(0), __int2half_rn(0));
        const uint32_t off = kmajor_off(c, 0);
        *reinterpret_cast<uint4 *>(sh.Bm[g] + off) = *reinterpret_cast<const uint4 *>(&col[0]);
        *reinterpret_cast<uint4 *>(sh.Bm[g] + off + 128) = *reinterpret_cast<const uint4 *>(&col[4]);
        for (int j = 0; j < kTcColBits; ++j) {
            if (!((c >> j) & 1))
                continue;
            const int vj = kTcRowBits + j;
            fcc += sh.lin[vj];
            for (int j2 = j + 1; j2 < kTcColBits; ++j2)
                if ((c >> j2) & 1)
                    fcc += sh.S[vj * n + kTcRowBits + j2];
        }
    }
    uint32_t *fslot = reinterpret_cast<uint32_t *>(sh.Bm[g] + kmajor_off(t, 14));
    // per tile bit b: how F'(c) (column t) and the row term (row t) move when b flips
    if (g == 0) {
        for (int b = 0; b < nT; ++b) {
            int kc = 0, rr = 0;
            for (int j = 0; j < kTcColBits; ++j)
                if ((t >> j) & 1)
                    kc += sh.S[(kTcRowBits + j) * n + kTcTileBits + b];
            for (int i = 0; i < kTcRowBits; ++i)
                if ((t >> i) & 1)
                    rr += sh.S[i * n + kTcTileBits + b];
            sh.Kc[b][t] = kc;
            sh.Rr[b][t] = rr;
        }
    }
    if (tid < 32)
        tmem_alloc(smem_u32(&sh.tmem_base), kTcCols * kTcGroups);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sh.tmem_base + (uint32_t)(kTcCols * g);
    if (tid < 32)
        tmem_relinquish();
    const uint64_t adesc = smem_desc(smem_u32(sh.A), kLbo, kSbo);
    const uint64_t bdesc = smem_desc(smem_u32(sh.Bm[g]), kLbo, kSbo);
    const uint32_t idesc = idesc_f16(128, 128);
    const uint32_t mbar = smem_u32(&sh.mbar[g]);
    const unsigned long long ntiles = p_hi - p_lo;  // a power of two
    uint32_t phase = 0;
    // tiles in Gray order inside aligned chunks of 2^r
    int lg = 0;
    while ((1ull << (lg + 1)) <= ntiles)
        ++lg;
    const int r = lg < 8 ? lg : 8;
    const unsigned long long nchunks = ntiles >> r;
    const unsigned long long per_chunk = 1ull << r;
    const unsigned long long cstride = (unsigned long long)gridDim.x * kTcGroups;
    unsigned long long ch = (unsigned long long)blockIdx.x * kTcGroups + g, jt = 0;
    TileTracker tr;
    if (w == 0 && ch < nchunks) {
        tr.from_scratch(sh.S, sh.lin, n, nT, p_lo + (ch << r), l);
        tr.publish(&sh.uni[g][0][0], l);
    }
    group_sync(g);

    int Fp = 0, rowT = 0;  // F'(column t) and row t's constant for the current tile
    int gm = INT_MAX;      // this group's minimum over its tiles (thread 0)
    for (int it = 0; ch < nchunks; ++it) {
        const unsigned long long ti = (ch << r) + (jt ^ (jt >> 1));
        unsigned long long nch = ch, njt = jt + 1;
        if (njt == per_chunk) {
            nch = ch + cstride;
            njt = 0;
        }
        const int buf = it & 1;
        const int *uni = &sh.uni[g][buf][0];
        if (jt == 0) {
            // chunk start: from the tracker's full values
            Fp = fcc;
            rowT = uni[14];
#pragma unroll
            for (int j = 0; j < kTcColBits; ++j) {
                if ((t >> j) & 1) {
                    Fp += uni[7 + j];
                    rowT += uni[j];
                }
            }
        } else {
            // one tile bit b flipped to nb since the previous tile
            const int b = __ffsll((long long)jt) - 1;
            const int nb = (int)(((jt ^ (jt >> 1)) >> b) & 1ull);
            const int dF = sh.Kc[b][t], dR = uni[15] + sh.Rr[b][t];
            Fp += nb ? dF : -dF;
            rowT += nb ? dR : -dR;
        }
        {
            int hi, lo;
            limbs(Fp, hi, lo);
            const __half2 fl = __halves2half2(__int2half_rn(hi), __int2half_rn(lo));
            *fslot = *reinterpret_cast<const uint32_t *>(&fl);
        }
        fence_async_smem();
        group_sync(g);
        if (t == 0) {
            tc_fence_after();
            mma_f16_ss(tbase, adesc, bdesc, idesc, 0);
            mma_commit(mbar);
        }
        if (w == 0 && nch < nchunks) {
            if (njt == 0) {
                tr.from_scratch(sh.S, sh.lin, n, nT, p_lo + (nch << r), l);
                tr.publish(&sh.uni[g][buf ^ 1][0], l);
            } else {
                const int b = __ffsll((long long)njt) - 1;
                const int nb = (int)(((njt ^ (njt >> 1)) >> b) & 1ull);
                const int gb = tr.field(b);
                if (l == 0)
                    sh.uni[g][buf ^ 1][15] = gb;
                tr.flip(sh.S, n, nT, b, nb, l);
            }
        }
        const bool ok = mbar_wait_bounded(mbar, phase);
        phase ^= 1u;
        tc_fence_after();
        float m = INFINITY;
        if (ok) {
            float m0 = INFINITY, m1 = INFINITY, m2 = INFINITY, m3 = INFINITY;
#pragma unroll
            for (int cb = 0; cb < 128; cb += 32) {
                float ra[16], rb[16];
                const uint32_t ta = tbase + ((uint32_t)(32 * w) << 16) + (uint32_t)cb;
                tmem_ld16(ta, ra);
                tmem_ld16(ta + 16, rb);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    m0 = fmin3(m0, ra[j], ra[j + 1]);
                    m1 = fmin3(m1, ra[j + 2], ra[j + 3]);
                    m2 = fmin3(m2, rb[j], rb[j + 1]);
                    m3 = fmin3(m3, rb[j + 2], rb[j + 3]);
                }
            }
            m = fminf(fmin3(m0, m1, m2), m3);
        } else if (l == 0) {
            sh.err = 1;
            atomicExch(&ctr->status, QBF_ECUDA);
        }
        // row minimum + f_ss(row) + the tile's row constant; exact integers
        int rm = (int)m + fss + rowT;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            rm = min(rm, __shfl_xor_sync(0xffffffffu, rm, o));
        if (l == 0)
            sh.wmin[g][w] = rm;
        tc_fence_before();
        group_sync(g);
        if (sh.err)
            break;
        if (t == 0) {
            int tm = sh.wmin[g][0];
            for (int i = 1; i < 4; ++i)
                tm = min(tm, sh.wmin[g][i]);
            pmin[ti] = tm;
            gm = min(gm, tm);
        }
        ch = nch;
        jt = njt;
    }
    if (t == 0 && gm != INT_MAX)
        atomicMin(&ctr->gmin, gm);
    tc_fence_before();
    __syncthreads();
    if (tid < 32)
        tmem_dealloc(sh.tmem_base, kTcCols * kTcGroups);
}

size_t tc_smem_bytes() { return sizeof(TcGroupShared) + 1024; }

cudaError_t launch_tc_min(const Plan *plan, int n, unsigned long long p_lo,
                          unsigned long long p_hi, int *pmin, Counters *ctr, int num_sms,
                          cudaStream_t s)
{
    const size_t smem = tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(tc_min_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, tc_min_kernel, kTcThreads * kTcGroups,
                                                      smem);
    if (e != cudaSuccess)
        return e;
    if (bps < 1)
        return cudaErrorInvalidConfiguration;
    // one CTA per SM: it holds all 512 TMEM columns (four groups of 128)
    const unsigned long long tiles = p_hi - p_lo;
    unsigned long long chunks = tiles;
    while (chunks > 1 && tiles / chunks < 256)
        chunks >>= 1;
    unsigned long long grid = (chunks + kTcGroups - 1) / kTcGroups;
    if (grid > (unsigned long long)num_sms)
        grid = num_sms;
    tc_min_kernel<<<(unsigned)grid, kTcThreads * kTcGroups, smem, s>>>(plan, n, p_lo, p_hi, pmin,
                                                                       ctr);
    return cudaGetLastError();
}

cudaError_t run_tc_selftest(const void *A_host, const void *B_host, float *D_host, int *err_host)
{
    __half *dA = nullptr, *dB = nullptr;
    float *dD = nullptr;
    int *dErr = nullptr;
    cudaError_t e = cudaMalloc(&dA, 128 * 16 * sizeof(__half));
    if (e == cudaSuccess)
        e = cudaMalloc(&dB, 16 * 128 * sizeof(__half));
    if (e == cudaSuccess)
        e = cudaMalloc(&dD, 128 * 128 * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&dErr, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(dA, A_host, 128 * 16 * sizeof(__half), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(dB, B_host, 16 * 128 * sizeof(__half), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(dErr, 0, sizeof(int));
    if (e == cudaSuccess) {
        tc_selftest_kernel<<<1, kTcThreads>>>(dA, dB, dD, dErr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(D_host, dD, 128 * 128 * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(err_host, dErr, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dErr);
    return e;
}

}  // namespace qbf
