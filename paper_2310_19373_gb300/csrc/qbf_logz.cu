// qbf_logz.cu -- exact Boltzmann log-partition and its gradient by the same
// Gray-code walk (rows A10, A11).
//
//   log Z(Q, beta) = log sum_x exp(-beta f(x)),      f(x) = x^T Q x (Eq. 1)
//   d log Z / d Q_ij = -beta E_beta[x_i x_j]         (f is linear in every Q_ij)
//   d min f / d Q_ij = x*_i x*_j                     (Danskin, x* = lowest argmin)
//
// Energies.  Each instance is walked on a two-limb fixed-point image
// (qbf_prepare.cu: hi = round(y 2^s), lo = L more bits of the residual, L =
// logz_lo_bits(n), 14 at n = 28), i.e. f at scale 2^(s+L) = hi_value * 2^L +
// lo_value.  Each limb's sum of |entries| is at most 2^22, so both limbs walk
// exactly in FP32, in lockstep as one packed pair: one packed add per field
// and per correction, and no integer-to-float conversion per state (those
// share the exponential unit with ex2, which bounds this walk).  The shift m
// is the image value of the certified argmin (from the batched minimiser), so
// every weight w = exp(-beta (f - m)) is <= ~1.  w = ex2(c (d_hi + d_lo 2^-L))
// with d the limb differences to m and c = -beta log2(e) 2^-s (the FP32
// argument keeps 24 bits either way: the lo limb matters only where d_hi is
// small).  Weights are summed in FP32 per block of
// 2^R states, blocks are added with Kahan compensation per lane, lanes in FP64
// in a fixed order.
//
// Second moment without O(n^2) work per state.  Walk A fixes the top kA
// variables per lane (prefix p) and walks the bottom nsA: per lane it keeps
// Z_p = sum_s w and M1_p[j] = sum_s w s_j.  Then
//   top x top:     sum_p Z_p p_i p_j
//   top x bottom:  sum_p p_i M1_p[j]
// Walk B runs on the variables rotated by nsA, so the bottom nsA variables
// become its prefix, and gives bottom x bottom = sum_p' Z_p' p'_i p'_j from its
// per-lane Z alone.  Dividing by Z gives E[x_i x_j] for every pair.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "qbf.h"
#include "qbf_internal.cuh"
#include "qbf_f32x2.cuh"
#include "qbf_kernels.cuh"
#include "qbf_walk_core.cuh"

namespace qbf {

namespace {

constexpr int kLzThreads = 128;
constexpr int kLzMaxBeta = 8;

struct LzArgs {
    int n, ns, kp, nbeta, R;
    int batch;                  // instances in this launch
    unsigned long long lanes;   // 2^kp prefixes per instance
    const Plan *plans;          // (b * 2 + w) * 2 + limb
    int walk;                   // 0: A, 1: B
    const Rec *recs;
    unsigned rec_stride;
    const int *K;
    const int *shift;           // per instance and walk: (hi, lo) value of the argmin
    const float2 *cc;           // [b][kLzMaxBeta]: (c_hi, c_lo) of each beta
    float lo_scale;             // 2^-L: weight of the lo limb
    const volatile int *cancel; // nullptr, or the cancellation word
    int beta0;                  // first beta of this launch
    double *laneZ;              // MODE Z:  [b][lane][beta]
    double *laneM1;             // MODE M1: [b][lane][ns]
};

constexpr int kModeZ = 0;   // Z for every beta
constexpr int kModeM1 = 1;  // Z and M1 for up to kLzM1Beta betas
constexpr int kLzM1Beta = 3;

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// Two FP32-exact walks (hi and lo limb) over the same suffix in lockstep, as
// one packed pair v = (hi, lo).  The block records and the in-block
// corrections hold FP32 bits (logz_tables_kernel), the lane parts of the mid
// fields sCh / sCl are FP32.  visit(v, U, pi) is called at every state, with
// U the compile-time step in the block (0 for the block's first state) and pi
// the block parity; the low R bits of the state's Gray code are then gray(U),
// except bit R - 1, which is gray(U)'s bit R - 1 xor pi.  flush(B) follows
// every block B.
template <int R, class F, class G>
__device__ __forceinline__ void walk2(f32x2::u64 v, f32x2::u64 (&GL)[R], int ns, const int4 *rh,
                                      const int4 *rl, const float *sCh, const float *sCl,
                                      int stride, int slot, const f32x2::u64 *K2, F &&visit,
                                      G &&flush)
{
    const int M = ns - R;
    const unsigned nblocks = 1u << M;
    for (unsigned B = 0; B < nblocks; ++B) {
        const int pi = B & 1;
        if (B > 0) {
            const int4 ah = __ldg(rh + 2 * B), bh = __ldg(rh + 2 * B + 1);
            const int4 al = __ldg(rl + 2 * B), bl = __ldg(rl + 2 * B + 1);
            const f32x2::u64 t = f32x2::pack(__int_as_float(ah.x), __int_as_float(al.x));
            const f32x2::u64 c =
                f32x2::pack(sCh[ah.y * stride + slot], sCl[al.y * stride + slot]);
            v = f32x2::add(v, f32x2::add(t, c));
            const int Wh[6] = {ah.z, ah.w, bh.x, bh.y, bh.z, bh.w};
            const int Wl[6] = {al.z, al.w, bl.x, bl.y, bl.z, bl.w};
#pragma unroll
            for (int i = 0; i < R; ++i)
                GL[i] = f32x2::add(GL[i],
                                   f32x2::pack(__int_as_float(Wh[i]), __int_as_float(Wl[i])));
        }
        visit(v, std::integral_constant<int, 0>{}, pi);
        static_for<1, (1 << R)>([&](auto U) {
            constexpr int u = decltype(U)::value;
            constexpr int l = ctz_c(u);
            constexpr int g = u ^ (u >> 1);
            const int nb = ((g >> l) & 1) ^ ((l == R - 1) ? pi : 0);
            // the step's field and correction are added to each other off the
            // chain of states, so the state chain is one packed add (every
            // sum is an integer below 2^24 in magnitude: exact)
            const f32x2::u64 k = K2[pi * 64 + u];  // both limbs' corrections, one load
            v = f32x2::add(v, nb ? f32x2::add(k, GL[l]) : f32x2::sub(k, GL[l]));
            visit(v, U, pi);
        });
        flush(B);
    }
}

template <int R, int MODE, int NB>
__global__ void __launch_bounds__(kLzThreads) logz_walk_kernel(LzArgs a)
{
    extern __shared__ int sm[];
    const int n = a.n, ns = a.ns;
    const unsigned long long blocks_per_inst = (a.lanes + kLzThreads - 1) / kLzThreads;
    const int b = (int)(blockIdx.x / blocks_per_inst);
    const unsigned long long p0 = (blockIdx.x % blocks_per_inst) * kLzThreads;
    const Plan *ph = a.plans + (size_t)(b * 2 + a.walk) * 2;
    const Plan *pl = ph + 1;
    int *sSh = sm, *sSl = sSh + n * n, *sLh = sSl + n * n, *sLl = sLh + n;
    // (2n^2 + 2n ints before it: 8-byte aligned)
    int2 *sK2 = reinterpret_cast<int2 *>(sLl + n);
    int *sCh = reinterpret_cast<int *>(sK2 + 128), *sCl = sCh + 2 * (ns - R) * kLzThreads;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        sSh[e] = ph->S[e];
        sSl[e] = pl->S[e];
    }
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        sLh[e] = ph->lin[e];
        sLl[e] = pl->lin[e];
    }
    const int pidx = (b * 2 + a.walk) * 2;
    for (int e = threadIdx.x; e < 128; e += blockDim.x) {
        sK2[e] = make_int2(a.K[pidx * 128 + e], a.K[(pidx + 1) * 128 + e]);
    }
    __shared__ int s_stop;  // read once per block, so the block leaves as one
    if (threadIdx.x == 0)
        s_stop = cancelled(a.cancel);
    __syncthreads();
    if (ph->status != QBF_OK || s_stop)
        return;
    const unsigned long long p = p0 + threadIdx.x;
    const bool active = p < a.lanes;
    const unsigned long long pp = active ? p : 0;
    unsigned GLh[R], GLl[R];
    // the limbs are walked relative to the argmin's image (the walk is linear
    // in its start value), so a state's offset to m needs no subtraction
    const unsigned mh = (unsigned)a.shift[(b * 2 + a.walk) * 2];
    const unsigned ml = (unsigned)a.shift[(b * 2 + a.walk) * 2 + 1];
    const unsigned vh =
        lane_setup<R>(pp, n, ns, sSh, sLh, sCh, kLzThreads, threadIdx.x, GLh) - mh;
    const unsigned vl =
        lane_setup<R>(pp, n, ns, sSl, sLl, sCl, kLzThreads, threadIdx.x, GLl) - ml;
    const int4 *rh = reinterpret_cast<const int4 *>(a.recs + (size_t)pidx * a.rec_stride);
    const int4 *rl = reinterpret_cast<const int4 *>(a.recs + (size_t)(pidx + 1) * a.rec_stride);
    // to FP32 (exact: every limb value is below 2^23 in magnitude): the start
    // pair, the low-bit fields and this lane's parts of the mid-bit fields
    const f32x2::u64 v0 = f32x2::pack((float)(int)vh, (float)(int)vl);
    f32x2::u64 GL[R];
#pragma unroll
    for (int i = 0; i < R; ++i)
        GL[i] = f32x2::pack((float)(int)GLh[i], (float)(int)GLl[i]);
    for (int e = 0; e < 2 * (ns - R); ++e) {
        int *ch = sCh + e * kLzThreads + threadIdx.x, *cl = sCl + e * kLzThreads + threadIdx.x;
        *ch = __float_as_int((float)*ch);
        *cl = __float_as_int((float)*cl);
    }
    const float *sChf = reinterpret_cast<const float *>(sCh);
    const float *sClf = reinterpret_cast<const float *>(sCl);
    const f32x2::u64 *sKf = reinterpret_cast<const f32x2::u64 *>(sK2);
    const float lsc = a.lo_scale;

    if constexpr (MODE == kModeZ) {
        // NB betas (exactly a.nbeta for NB <= 4; up to NB = 8 with the rest
        // predicated off), each an FP32 block sum flushed into a Kahan sum
        constexpr bool exact_nb = NB <= 4;
        float acc[NB], sum[NB], comp[NB], ch[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            acc[j] = sum[j] = comp[j] = 0.f;
            const float2 c2 = a.cc[(size_t)b * kLzMaxBeta + a.beta0 + j];
            ch[j] = c2.x;
        }
        walk2<R>(v0, GL, ns, rh, rl, sChf, sClf, kLzThreads, threadIdx.x, sKf,
                 [&](f32x2::u64 v, auto, int) {
                     // c_lo = c_hi 2^-L exactly, so c_hi dh + c_lo dl =
                     // c_hi (dh + dl 2^-L): one FFMA per state, one FMUL per beta
                     float xh, xl;
                     f32x2::unpack(v, xh, xl);
                     const float d = fmaf(xl, lsc, xh);
#pragma unroll
                     for (int j = 0; j < NB; ++j)
                         if (exact_nb || j < a.nbeta)
                             acc[j] += ex2_approx(d * ch[j]);
                 },
                 [&](unsigned) {
#pragma unroll
                     for (int j = 0; j < NB; ++j) {
                         kahan_add(sum[j], comp[j], acc[j]);
                         acc[j] = 0.f;
                     }
                 });
        if (active) {
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (exact_nb || j < a.nbeta)
                    a.laneZ[((size_t)b * a.lanes + p) * a.nbeta + j] =
                        (double)sum[j] - (double)comp[j];
        }
    } else {
        // For each of the NB betas of this launch: Z and M1[j] = sum of w
        // over the states with suffix bit j set.  Bits below R - 1 are
        // compile-time per step, bit R - 1 depends on the block parity, bits
        // >= R are constant over a block: they take the block total at the
        // flush.  Z and the low R bits keep Kahan sums in registers, the mid
        // bits in this thread's column of shared memory (sMid).
        float acc0[NB], accTop[NB], accLo[NB][R > 1 ? R - 1 : 1], wq[NB][4];
        float sum0[NB], comp0[NB], sumLo[NB][R], compLo[NB][R], ch[NB];
        float *sMid = reinterpret_cast<float *>(sCl + 2 * (ns - R) * kLzThreads);
        const int nmid = ns - R;
#pragma unroll
        for (int bb = 0; bb < NB; ++bb) {
            const float2 c2 = a.cc[(size_t)b * kLzMaxBeta + a.beta0 + bb];
            ch[bb] = c2.x;
            acc0[bb] = accTop[bb] = sum0[bb] = comp0[bb] = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                wq[bb][q] = 0.f;
#pragma unroll
            for (int J = 0; J < (R > 1 ? R - 1 : 1); ++J)
                accLo[bb][J] = 0.f;
#pragma unroll
            for (int J = 0; J < R; ++J)
                sumLo[bb][J] = compLo[bb][J] = 0.f;
        }
        for (int e = 0; e < 2 * NB * nmid; ++e)
            sMid[e * kLzThreads + threadIdx.x] = 0.f;
        walk2<R>(v0, GL, ns, rh, rl, sChf, sClf, kLzThreads, threadIdx.x, sKf,
                 [&](f32x2::u64 v, auto U, int pi) {
                     constexpr int u = decltype(U)::value;
                     constexpr int g = u ^ (u >> 1);
                     float xh, xl;
                     f32x2::unpack(v, xh, xl);
                     const float d = fmaf(xl, lsc, xh);
#pragma unroll
                     for (int bb = 0; bb < NB; ++bb) {
                         const float w = ex2_approx(d * ch[bb]);
                         if constexpr (R >= 3) {
                             // aligned quads of steps: bits 2.. of the Gray code
                             // are constant over a quad, bit 0 is set at its
                             // steps 1 and 2, bit 1 at steps 0, 1 or 2, 3 (by
                             // bit 2 of u); sum the quad first, then add it
                             // once per set bit
                             wq[bb][u & 3] = w;
                             if constexpr ((u & 3) == 3) {
                                 const float p01 = wq[bb][0] + wq[bb][1];
                                 const float p23 = wq[bb][2] + wq[bb][3];
                                 const float q = p01 + p23;
                                 acc0[bb] += q;
                                 accLo[bb][0] += wq[bb][1] + wq[bb][2];
                                 accLo[bb][1] += ((u >> 2) & 1) ? p01 : p23;
                                 static_for<2, R - 1>([&](auto J) {
                                     if constexpr ((g >> decltype(J)::value) & 1)
                                         accLo[bb][decltype(J)::value] += q;
                                 });
                                 if (((g >> (R - 1)) & 1) ^ pi)
                                     accTop[bb] += q;
                             }
                         } else {
                             acc0[bb] += w;
                             static_for<0, R - 1>([&](auto J) {
                                 if constexpr ((g >> decltype(J)::value) & 1)
                                     accLo[bb][decltype(J)::value] += w;
                             });
                             if (((g >> (R - 1)) & 1) ^ pi)
                                 accTop[bb] += w;
                         }
                     }
                 },
                 [&](unsigned B) {
                     const unsigned gB = B ^ (B >> 1);
#pragma unroll
                     for (int bb = 0; bb < NB; ++bb) {
                         const float blk = acc0[bb];
                         kahan_add(sum0[bb], comp0[bb], acc0[bb]);
                         acc0[bb] = 0.f;
#pragma unroll
                         for (int J = 0; J < R - 1; ++J) {
                             kahan_add(sumLo[bb][J], compLo[bb][J], accLo[bb][J]);
                             accLo[bb][J] = 0.f;
                         }
                         kahan_add(sumLo[bb][R - 1], compLo[bb][R - 1], accTop[bb]);
                         accTop[bb] = 0.f;
                         for (int j = 0; j < nmid; ++j) {
                             if (!((gB >> j) & 1u))
                                 continue;
                             float *ps = sMid + (size_t)((j * NB + bb) * 2) * kLzThreads + threadIdx.x;
                             float sv = ps[0], cv = ps[kLzThreads];
                             kahan_add(sv, cv, blk);
                             ps[0] = sv;
                             ps[kLzThreads] = cv;
                         }
                     }
                 });
        if (active) {
#pragma unroll
            for (int bb = 0; bb < NB; ++bb) {
                // beta bb's Z and M1 go to its own slab: [bb][b][lane](...)
                const size_t slab = (size_t)bb * a.batch * a.lanes;
                a.laneZ[slab + (size_t)b * a.lanes + p] = (double)sum0[bb] - (double)comp0[bb];
                double *m1 = a.laneM1 + (slab + (size_t)b * a.lanes + p) * ns;
#pragma unroll
                for (int J = 0; J < R; ++J)
                    m1[J] = (double)sumLo[bb][J] - (double)compLo[bb][J];
                for (int j = 0; j < nmid; ++j) {
                    const float *ps = sMid + (size_t)((j * NB + bb) * 2) * kLzThreads + threadIdx.x;
                    m1[R + j] = (double)ps[0] - (double)ps[kLzThreads];
                }
            }
        }
    }
}

// Per instance b and beta j < nbeta: c = -beta log2(e) 2^-sigma_b for the hi
// limb and c 2^-L for the lo limb, rounded from FP64 (entries j >= nbeta are
// zero); st[b] = the instance's prepare status.
__global__ void logz_consts_kernel(const Plan *plans, const double *beta, int nbeta, int batch,
                                   float2 *cc, int *st)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch)
        return;
    const Plan *P = plans + (size_t)b * 4;
    st[b] = P->status;
    for (int j = 0; j < kLzMaxBeta; ++j) {
        float2 v = make_float2(0.f, 0.f);
        if (j < nbeta) {
            const double c = -beta[j] * 1.4426950408889634 * ldexp(1.0, -P->sigma);
            v = make_float2((float)c, (float)(c * ldexp(1.0, P->sigma - P[1].sigma)));
        }
        cc[(size_t)b * kLzMaxBeta + j] = v;
    }
}

// Image value (hi, lo limbs) of each instance's argmin under both walks' plans.
__global__ void logz_shift_kernel(const Plan *plans, const unsigned long long *argmin, int n,
                                  int rot, int *shift)
{
    const int b = blockIdx.x;
    const int w = threadIdx.x >> 1, limb = threadIdx.x & 1;
    if (threadIdx.x >= 4)
        return;
    const Plan *P = plans + (size_t)(b * 2 + w) * 2 + limb;
    const unsigned long long x = argmin[b];
    // walk variable v holds the caller's variable (v + rot) mod n in walk B
    unsigned long long xw = 0;
    for (int v = 0; v < n; ++v) {
        const int src = w ? (v + rot) % n : v;
        xw |= ((x >> src) & 1ull) << v;
    }
    unsigned acc = 0;
    for (int i = 0; i < n; ++i) {
        if (!((xw >> i) & 1ull))
            continue;
        acc += (unsigned)P->lin[i];
        for (int j = i + 1; j < n; ++j)
            if ((xw >> j) & 1ull)
                acc += (unsigned)P->S[i * n + j];
    }
    shift[(b * 2 + w) * 2 + limb] = (int)acc;
}

// deterministic FP64 sum over [0, count) with stride
__device__ double block_sum_fixed(const double *v, unsigned long long count, size_t stride,
                                  double *red)
{
    double s = 0.0;
    for (unsigned long long e = threadIdx.x; e < count; e += blockDim.x)
        s += v[e * stride];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// log Z per (instance, beta) from walk A's per-lane Z.
__global__ void __launch_bounds__(256) logz_reduce_kernel(const Plan *plans, const double *laneZ,
                                                          unsigned long long lanes, int nbeta,
                                                          const double *beta, const int *shift,
                                                          double *logz)
{
    __shared__ double red[256];
    const int b = blockIdx.x;
    const Plan *ph = plans + (size_t)(b * 2) * 2;
    for (int j = 0; j < nbeta; ++j) {
        const double Z = block_sum_fixed(laneZ + (size_t)b * lanes * nbeta + j, lanes, nbeta, red);
        if (threadIdx.x == 0) {
            if (ph->status != QBF_OK) {
                logz[b * nbeta + j] = NAN;
                continue;
            }
            const int L = ph[1].sigma - ph->sigma;
            const long long m = ((long long)shift[b * 4] << L) + (long long)shift[b * 4 + 1];
            const double mreal = ldexp((double)m, -ph[1].sigma);
            logz[b * nbeta + j] = -beta[j] * mreal + log(Z);
        }
    }
}

// Sums of a per-lane value v(p) over the 2^k lanes of a walk, split by the
// lane index p = r 2^l + c into rows r (the high h = k - l bits) and columns
// c (the low l = k / 2 <= 8 bits): rows[r] = sum_c v, cols[c] = sum_r v and,
// when y is given, y[r * 8 + t] = sum_c [bit t of c] v for t < l.  Each entry
// is summed by one thread in ascending order, so the sums do not depend on
// scheduling.  Every pair sum sum_p v(p) [p_s] [p_t] then follows from these
// tables in O(2^h + 2^l) adds instead of O(2^k) per pair.
template <class V>
__device__ void lz_rows_cols(const V &v, int k, double *rows, double *cols, double *y)
{
    const int l = k / 2, h = k - l;
    const unsigned C = 1u << l, Rn = 1u << h;
    for (unsigned r = threadIdx.x; r < Rn; r += blockDim.x) {
        double sr = 0.0, yy[8];
#pragma unroll
        for (int t = 0; t < 8; ++t)
            yy[t] = 0.0;
        for (unsigned c = 0; c < C; ++c) {
            const double x = v((unsigned long long)r * C + c);
            sr += x;
            if (y) {
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (t < l && ((c >> t) & 1u))  // c is the same in every lane
                        yy[t] += x;
            }
        }
        rows[r] = sr;
        if (y) {
#pragma unroll
            for (int t = 0; t < 8; ++t)
                y[r * 8 + t] = yy[t];
        }
    }
    for (unsigned c = threadIdx.x; c < C; c += blockDim.x) {
        double sc = 0.0;
        for (unsigned r = 0; r < Rn; ++r)
            sc += v((unsigned long long)r * C + c);
        cols[c] = sc;
    }
}

// sum_p v(p) [p_s] [p_t] (s <= t < k) from the tables of lz_rows_cols
__device__ double lz_pair_sum(int k, int s, int t, const double *rows, const double *cols,
                              const double *y)
{
    const int l = k / 2, h = k - l;
    double a = 0.0;
    if (t < l) {
        for (unsigned c = 0; c < (1u << l); ++c)
            if (((c >> s) & 1u) && ((c >> t) & 1u))
                a += cols[c];
    } else if (s >= l) {
        for (unsigned r = 0; r < (1u << h); ++r)
            if (((r >> (s - l)) & 1u) && ((r >> (t - l)) & 1u))
                a += rows[r];
    } else {
        for (unsigned r = 0; r < (1u << h); ++r)
            if ((r >> (t - l)) & 1u)
                a += y[r * 8 + s];
    }
    return a;
}

// sum_p v(p) [p_t] from the row and column sums
__device__ double lz_bit_sum(int k, int t, const double *rows, const double *cols)
{
    const int l = k / 2, h = k - l;
    double a = 0.0;
    if (t < l) {
        for (unsigned c = 0; c < (1u << l); ++c)
            if ((c >> t) & 1u)
                a += cols[c];
    } else {
        for (unsigned r = 0; r < (1u << h); ++r)
            if ((r >> (t - l)) & 1u)
                a += rows[r];
    }
    return a;
}

// E[x_i x_j] for one beta from walk A (Z, M1) and walk B (Z); adds
// up[b] * (-beta) * E into grad and optionally stores E.  Grid (instance b,
// part): part 0 takes the pairs of top variables (walk A's prefix bits, from
// its per-lane Z), part 1 the pairs of bottom variables (walk B's prefix bits,
// from its per-lane Z), part 2 + i the bottom variable i against every top
// variable (walk A's first moments of bit i).  Dynamic shared memory:
// lz_moments_smem(n) bytes.  Every sum has a fixed order.
__global__ void __launch_bounds__(256) logz_moments_kernel(
    int n, int nsA, unsigned long long lanesA, unsigned long long lanesB, const double *ZA,
    const double *M1A, const double *ZB, int zb_stride, int zb_off, double beta,
    const double *up, int up_stride, int up_off, double *grad, double *moment,
    int moment_stride, int moment_off)
{
    extern __shared__ double lzm[];
    const int b = blockIdx.x, part = blockIdx.y;
    const int kA = n - nsA, kB = nsA;
    const double *za = ZA + (size_t)b * lanesA;
    const double *m1 = M1A + (size_t)b * lanesA * nsA;
    const double *zb = ZB + (size_t)b * lanesB * zb_stride + zb_off;  // beta column
    const int k = (part == 1) ? kB : kA;
    const int hk = k - k / 2;
    double *rows = lzm, *cols = rows + (1u << hk), *y = cols + (1u << (k / 2));
    double *tot = y + (1u << hk) * 8;
    auto vA = [&](unsigned long long p) { return __ldg(za + p); };
    auto vB = [&](unsigned long long p) { return __ldg(zb + p * zb_stride); };
    if (part == 1)
        lz_rows_cols(vB, k, rows, cols, y);
    else
        lz_rows_cols(vA, k, rows, cols, part == 0 ? y : nullptr);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (unsigned r = 0; r < (1u << hk); ++r)
            t += rows[r];
        tot[0] = t;
    }
    __syncthreads();
    const double Zt = tot[0];  // walk B's total for part 1, walk A's otherwise
    const double u = up ? up[b * up_stride + up_off] : 1.0;
    auto emit = [&](int vi, int vj, double sum) {
        const double E = sum / Zt;
        const double gval = u * (-beta) * E;
        grad[(size_t)b * n * n + vi * n + vj] += gval;
        if (vi != vj)
            grad[(size_t)b * n * n + vj * n + vi] += gval;
        if (moment) {
            double *mm = moment + (size_t)b * moment_stride + moment_off;
            mm[vi * n + vj] = E;
            mm[vj * n + vi] = E;
        }
    };
    if (part <= 1) {
        // walk A's prefix bit t is variable nsA + t, walk B's is variable t
        const int off = (part == 0) ? nsA : 0;
        const int npairs = k * (k + 1) / 2;
        for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
            int s = 0, rem = q;
            while (rem >= k - s) {
                rem -= k - s;
                ++s;
            }
            const int t = s + rem;
            emit(off + s, off + t, lz_pair_sum(k, s, t, rows, cols, y));
        }
    } else {
        const int i = part - 2;
        auto vM = [&](unsigned long long p) { return __ldg(m1 + p * nsA + i); };
        lz_rows_cols(vM, kA, rows, cols, nullptr);  // Z's tables are no longer read
        __syncthreads();
        for (int t = threadIdx.x; t < kA; t += blockDim.x)
            emit(i, nsA + t, lz_bit_sum(kA, t, rows, cols));
    }
}

size_t lz_moments_smem(int n)
{
    int hmax = 0, lmax = 0;
    for (int k : {n - n / 2, n / 2}) {
        hmax = std::max(hmax, k - k / 2);
        lmax = std::max(lmax, k / 2);
    }
    return sizeof(double) * (((size_t)1 << hmax) * 9 + ((size_t)1 << lmax) + 1);
}

__global__ void danskin_kernel(const unsigned long long *argmin, int n, int batch,
                               const double *up, double *grad)
{
    const int b = blockIdx.x;
    if (b >= batch)
        return;
    const unsigned long long x = argmin[b];
    const double u = up ? up[b] : 1.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        grad[(size_t)b * n * n + e] = (((x >> i) & 1ull) && ((x >> j) & 1ull)) ? u : 0.0;
    }
}

// ------------------------------------------------------------------------
// host side

std::mutex g_lmu;

struct LzPool {
    void *dev = nullptr;
    size_t bytes = 0;
};
std::vector<LzPool> g_lpool;

#define L_CUDA(call, where)                                                                      \
    do {                                                                                         \
        cudaError_t l_e_ = (call);                                                               \
        if (l_e_ != cudaSuccess)                                                                 \
            return record_error(QBF_ECUDA,                                                       \
                                (std::string(where) + ": " + cudaGetErrorString(l_e_)).c_str()); \
    } while (0)

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct LzGeo {
    int n, nsA, kA, nsB, kB, RA, RB;
    unsigned long long lanesA, lanesB;
    unsigned rec_stride;
};

LzGeo lz_geo(int n)
{
    LzGeo g;
    g.n = n;
    g.nsA = n / 2;
    g.kA = n - g.nsA;
    g.nsB = g.kA;
    g.kB = g.nsA;
    g.RA = std::min(kRMax, g.nsA);
    g.RB = std::min(kRMax, g.nsB);
    g.lanesA = 1ull << g.kA;
    g.lanesB = 1ull << g.kB;
    g.rec_stride = 1u << std::max(g.nsA - g.RA, g.nsB - g.RB);
    return g;
}

struct LzLayout {
    size_t plans, recs, K, shift, argmin, laneZA, laneM1, laneZB, beta, cc, st, total;
};

LzLayout lz_layout(const LzGeo &g, int batch, int nbeta)
{
    LzLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = al(o + bytes);
        return at;
    };
    L.plans = take(sizeof(Plan) * batch * 4);
    L.recs = take(sizeof(Rec) * (size_t)g.rec_stride * batch * 4);
    L.K = take(sizeof(int) * 128 * batch * 4);
    L.shift = take(sizeof(int) * 4 * batch);
    L.argmin = take(sizeof(unsigned long long) * batch);
    L.laneZA = take(sizeof(double) * g.lanesA * batch * std::max(nbeta, 1));
    L.laneM1 = take(sizeof(double) * g.lanesA * batch * g.nsA * std::min(nbeta, kLzM1Beta));
    L.laneZB = take(sizeof(double) * g.lanesB * batch * std::max(nbeta, 1));
    L.beta = take(sizeof(double) * kLzMaxBeta);
    L.cc = take(sizeof(float2) * kLzMaxBeta * batch);
    L.st = take(sizeof(int) * batch);
    L.total = o;
    return L;
}

int lz_pool(size_t bytes, char **base)
{
    int dev = 0;
    L_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if ((int)g_lpool.size() <= dev)
        g_lpool.resize(dev + 1);
    LzPool &P = g_lpool[dev];
    if (P.bytes < bytes) {
        L_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
        if (P.dev)
            cudaFree(P.dev);
        P.dev = nullptr;
        P.bytes = 0;
        L_CUDA(cudaMalloc(&P.dev, bytes), "cudaMalloc(logz scratch)");
        P.bytes = bytes;
    }
    *base = (char *)P.dev;
    return QBF_OK;
}

template <int MODE, int NB>
cudaError_t launch_lz_nb(int R, const LzArgs &a_in, int batch, cudaStream_t s)
{
    LzArgs a = a_in;
    a.batch = batch;
    // + the moment walk's mid-bit Kahan sums: 2 floats per beta and mid bit
    const size_t smem =
        sizeof(int) * (2 * a.n * a.n + 2 * a.n + 256 + 2 * 2 * (a.ns - R) * kLzThreads +
                       (MODE == kModeM1 ? 2 * NB * (a.ns - R) * kLzThreads : 0));
    const unsigned long long bpi = (a.lanes + kLzThreads - 1) / kLzThreads;
    const unsigned grid = (unsigned)(bpi * batch);
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
        kern<<<grid, kLzThreads, smem, s>>>(a);
        return cudaGetLastError();
    };
    switch (R) {
    case 1: return go(logz_walk_kernel<1, MODE, NB>);
    case 2: return go(logz_walk_kernel<2, MODE, NB>);
    case 3: return go(logz_walk_kernel<3, MODE, NB>);
    case 4: return go(logz_walk_kernel<4, MODE, NB>);
    case 5: return go(logz_walk_kernel<5, MODE, NB>);
    default: return go(logz_walk_kernel<6, MODE, NB>);
    }
}

// the moment walk takes up to kLzM1Beta betas per launch; the Z walk is
// compiled per beta count
template <int MODE>
cudaError_t launch_lz(int R, const LzArgs &a, int batch, cudaStream_t s)
{
    if constexpr (MODE == kModeM1) {
        switch (a.nbeta) {
        case 1: return launch_lz_nb<MODE, 1>(R, a, batch, s);
        case 2: return launch_lz_nb<MODE, 2>(R, a, batch, s);
        case 3: return launch_lz_nb<MODE, 3>(R, a, batch, s);
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (a.nbeta) {
        case 1: return launch_lz_nb<MODE, 1>(R, a, batch, s);
        case 2: return launch_lz_nb<MODE, 2>(R, a, batch, s);
        case 3: return launch_lz_nb<MODE, 3>(R, a, batch, s);
        case 4: return launch_lz_nb<MODE, 4>(R, a, batch, s);
        default: return launch_lz_nb<MODE, kLzMaxBeta>(R, a, batch, s);  // 5..8, predicated
        }
    }
}

size_t dts(int dt) { return dt == QBF_F64 ? 8 : dt == QBF_I16 ? 2 : (dt == QBF_F32 || dt == QBF_I32) ? 4 : 0; }

int lz_check(const void *Q, int n, int dtype, int batch, const double *beta, int nbeta)
{
    if (!Q || !beta)
        return record_error(QBF_EINVAL, "null pointer argument");
    if (n < 2 || n > QBF_BATCH_MAX_N)
        return record_error(QBF_EINVAL, "log Z needs 2 <= n <= 34");
    if (batch < 1 || batch > 4096)
        return record_error(QBF_EINVAL, "batch must be in [1, 4096]");
    if (nbeta < 1 || nbeta > kLzMaxBeta)
        return record_error(QBF_EINVAL, "nbeta must be in [1, 8]");
    for (int j = 0; j < nbeta; ++j)
        if (!(beta[j] > 0.0) || !std::isfinite(beta[j]))
            return record_error(QBF_EINVAL, "every beta must be finite and > 0");
    if (dts(dtype) == 0)
        return record_error(QBF_EDTYPE, "unknown dtype");
    return QBF_OK;
}

// certified argmin of every instance (batched minimiser), then the images,
// tables and shifts shared by the forward and backward walks
int lz_setup(const void *Q, int n, int dtype, int batch, const LzGeo &g, char *base,
             const LzLayout &L, double *min_value, uint64_t *argmin, cudaStream_t s)
{
    std::vector<const void *> ptrs(batch);
    std::vector<int> ns(batch, n), dt(batch, dtype);
    for (int b = 0; b < batch; ++b)
        ptrs[b] = (const char *)Q + (size_t)b * n * n * dts(dtype);
    int rc = solve_batched(ptrs.data(), ns.data(), dt.data(), batch, nullptr, min_value, argmin, s,
                           nullptr);
    if (rc)
        return rc;
    Plan *plans = (Plan *)(base + L.plans);
    L_CUDA(cudaMemcpyAsync(base + L.argmin, argmin, sizeof(unsigned long long) * batch,
                           cudaMemcpyHostToDevice, s),
           "argmin upload");
    logz_prepare_kernel<<<batch * 2, 256, 0, s>>>(Q, n, dtype, g.nsA, plans);
    logz_tables_kernel<<<batch * 4, 256, 0, s>>>(plans, g.nsA, g.nsB, (Rec *)(base + L.recs),
                                                 g.rec_stride, (int *)(base + L.K));
    logz_shift_kernel<<<batch, 32, 0, s>>>(plans, (const unsigned long long *)(base + L.argmin), n,
                                           g.nsA, (int *)(base + L.shift));
    L_CUDA(cudaGetLastError(), "log Z set-up kernels");
    return QBF_OK;
}

LzArgs lz_args(const LzGeo &g, char *base, const LzLayout &L, int walk, int nbeta,
               const double *beta, int sigma_hint)
{
    (void)sigma_hint;
    LzArgs a;
    memset(&a, 0, sizeof(a));
    a.n = g.n;
    a.ns = walk ? g.nsB : g.nsA;
    a.kp = walk ? g.kB : g.kA;
    a.R = walk ? g.RB : g.RA;
    a.lanes = walk ? g.lanesB : g.lanesA;
    a.nbeta = nbeta;
    a.plans = (const Plan *)(base + L.plans);
    a.walk = walk;
    a.recs = (const Rec *)(base + L.recs);
    a.rec_stride = g.rec_stride;
    a.K = (const int *)(base + L.K);
    a.shift = (const int *)(base + L.shift);
    a.laneZ = (double *)(base + (walk ? L.laneZB : L.laneZA));
    a.laneM1 = (double *)(base + L.laneM1);
    a.cc = (const float2 *)(base + L.cc);
    a.lo_scale = (float)ldexp(1.0, -logz_lo_bits(g.n));
    a.cancel = cancel_word_dev();
    a.beta0 = 0;
    (void)beta;
    return a;
}

// Upload the betas, derive every instance's exp constants on the device and
// check that every instance prepared (one status download).
int lz_consts(const LzLayout &L, char *base, int batch, const double *beta, int nbeta,
              cudaStream_t s)
{
    L_CUDA(cudaMemcpyAsync(base + L.beta, beta, sizeof(double) * nbeta, cudaMemcpyHostToDevice, s),
           "beta upload");
    logz_consts_kernel<<<(batch + 127) / 128, 128, 0, s>>>(
        (const Plan *)(base + L.plans), (const double *)(base + L.beta), nbeta, batch,
        (float2 *)(base + L.cc), (int *)(base + L.st));
    L_CUDA(cudaGetLastError(), "log Z constants");
    std::vector<int> st(batch);
    L_CUDA(cudaMemcpyAsync(st.data(), base + L.st, sizeof(int) * batch, cudaMemcpyDeviceToHost, s),
           "status");
    L_CUDA(cudaStreamSynchronize(s), "log Z set-up");
    for (int b = 0; b < batch; ++b)
        if (st[b] != QBF_OK)
            return record_error(st[b], ("instance " + std::to_string(b) + ": prepare failed").c_str());
    return QBF_OK;
}

}  // namespace

int logz_forward(const void *Q, int n, int dtype, int batch, const double *beta, int nbeta,
                 double *logz, double *min_value, uint64_t *argmin, cudaStream_t s)
{
    const NvtxRange range("qbf_logz_forward");
    int rc = lz_check(Q, n, dtype, batch, beta, nbeta);
    if (rc)
        return rc;
    if (!logz || !min_value || !argmin)
        return record_error(QBF_EINVAL, "null pointer argument");
    std::lock_guard<std::mutex> lk(g_lmu);
    const LzGeo g = lz_geo(n);
    const LzLayout L = lz_layout(g, batch, nbeta);
    char *base = nullptr;
    if ((rc = lz_pool(L.total, &base)))
        return rc;
    if ((rc = lz_setup(Q, n, dtype, batch, g, base, L, min_value, argmin, s)))
        return rc;
    if ((rc = lz_consts(L, base, batch, beta, nbeta, s)))
        return rc;
    // walk A over every instance in one launch (each instance reads its own
    // scale-dependent constants)
    LzArgs a = lz_args(g, base, L, 0, nbeta, beta, 0);
    L_CUDA(launch_lz<kModeZ>(a.R, a, batch, s), "log Z walk");
    double *dlogz = (double *)(base + L.laneM1);  // reuse: batch * nbeta doubles
    logz_reduce_kernel<<<batch, 256, 0, s>>>((const Plan *)(base + L.plans),
                                             (const double *)(base + L.laneZA), g.lanesA, nbeta,
                                             (const double *)(base + L.beta),
                                             (const int *)(base + L.shift), dlogz);
    L_CUDA(cudaGetLastError(), "log Z reduce");
    L_CUDA(cudaMemcpyAsync(logz, dlogz, sizeof(double) * batch * nbeta, cudaMemcpyDeviceToHost, s),
           "log Z download");
    L_CUDA(cudaStreamSynchronize(s), "log Z");
    if (cancel_requested())
        return record_error(QBF_ECANCELED, "cancelled by qbf_cancel");
    return QBF_OK;
}

int logz_backward(const void *Q, int n, int dtype, int batch, const double *beta, int nbeta,
                  const double *upstream, double *grad, double *moment, cudaStream_t s)
{
    const NvtxRange range("qbf_logz_backward");
    int rc = lz_check(Q, n, dtype, batch, beta, nbeta);
    if (rc)
        return rc;
    if (!grad)
        return record_error(QBF_EINVAL, "null pointer argument");
    std::lock_guard<std::mutex> lk(g_lmu);
    const LzGeo g = lz_geo(n);
    const LzLayout L = lz_layout(g, batch, nbeta);
    char *base = nullptr;
    if ((rc = lz_pool(L.total, &base)))
        return rc;
    std::vector<double> vmin(batch);
    std::vector<uint64_t> am(batch);
    if ((rc = lz_setup(Q, n, dtype, batch, g, base, L, vmin.data(), am.data(), s)))
        return rc;
    if ((rc = lz_consts(L, base, batch, beta, nbeta, s)))
        return rc;
    L_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * batch * n * n, s), "grad clear");
    // walk B (rotated variables) needs only Z: one pass for every beta
    {
        LzArgs a = lz_args(g, base, L, 1, nbeta, beta, 0);
        L_CUDA(launch_lz<kModeZ>(a.R, a, batch, s), "log Z walk (rotated)");
    }
    // walk A with first moments, up to kLzM1Beta betas per launch; beta
    // j0 + jj leaves its Z and M1 in slab jj of laneZA / laneM1
    for (int j0 = 0; j0 < nbeta; j0 += kLzM1Beta) {
        const int nb = std::min(kLzM1Beta, nbeta - j0);
        LzArgs a = lz_args(g, base, L, 0, nb, beta, 0);
        a.beta0 = j0;
        L_CUDA(launch_lz<kModeM1>(a.R, a, batch, s), "log Z moment walk");
        for (int jj = 0; jj < nb; ++jj) {
            const int j = j0 + jj;
            const size_t slab = (size_t)jj * batch * g.lanesA;
            logz_moments_kernel<<<dim3(batch, 2 + g.nsA), 256, lz_moments_smem(n), s>>>(
                n, g.nsA, g.lanesA, g.lanesB, (const double *)(base + L.laneZA) + slab,
                (const double *)(base + L.laneM1) + slab * g.nsA,
                (const double *)(base + L.laneZB), nbeta, j, beta[j], upstream, nbeta, j, grad,
                moment, nbeta * n * n, j * n * n);
            L_CUDA(cudaGetLastError(), "log Z moments");
        }
    }
    L_CUDA(cudaStreamSynchronize(s), "log Z backward");
    if (cancel_requested())
        return record_error(QBF_ECANCELED, "cancelled by qbf_cancel");
    return QBF_OK;
}

int danskin(const uint64_t *argmin_host, int n, int batch, const double *upstream, double *grad,
            cudaStream_t s)
{
    if (!argmin_host || !grad)
        return record_error(QBF_EINVAL, "null pointer argument");
    if (n < 1 || n > 64 || batch < 1)
        return record_error(QBF_EINVAL, "need 1 <= n <= 64 and batch >= 1");
    std::lock_guard<std::mutex> lk(g_lmu);
    char *base = nullptr;
    int rc = lz_pool(al(sizeof(unsigned long long) * batch), &base);
    if (rc)
        return rc;
    L_CUDA(cudaMemcpyAsync(base, argmin_host, sizeof(unsigned long long) * batch,
                           cudaMemcpyHostToDevice, s),
           "argmin upload");
    danskin_kernel<<<batch, 256, 0, s>>>((const unsigned long long *)base, n, batch, upstream, grad);
    L_CUDA(cudaGetLastError(), "danskin");
    L_CUDA(cudaStreamSynchronize(s), "danskin");
    return QBF_OK;
}

int release_logz()
{
    std::lock_guard<std::mutex> lk(g_lmu);
    for (size_t d = 0; d < g_lpool.size(); ++d) {
        if (!g_lpool[d].dev)
            continue;
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice((int)d);
        cudaDeviceSynchronize();
        cudaFree(g_lpool[d].dev);
        g_lpool[d] = LzPool();
        cudaSetDevice(cur);
    }
    return QBF_OK;
}

}  // namespace qbf
