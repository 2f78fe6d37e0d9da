// qbf_prepare.cu -- step A1 of a solve: fixed-point image of Q and walk tables.
//
// prepare_kernel  (one CTA)
//   Reads the caller's Q (any dtype), rejects NaN/Inf, forms lin_i = Q_ii and
//   the symmetrised off-diagonal S_ij = Q_ij + Q_ji (Section 3's split of Q
//   into a linear part and a symmetric quadratic part), picks the largest
//   scale 2^sigma with sum |round(.)| < 2^31 and writes the int32 image, the
//   quantisation error bound and the certification window W to the Plan.
//
// tables_kernel
//   Builds, for a walk with suffix width ns and R unrolled low bits, the
//   lane-invariant record of every block transition B and the static
//   in-block corrections K[parity][u] (derivation in qbf_walk.cu).
#include <cfloat>
#include <climits>
#include <cmath>

#include "qbf_internal.cuh"

namespace qbf {

namespace {

__device__ double load_q(const void *Q, int dtype, int e)
{
    switch (dtype) {
    case QBF_F64: return static_cast<const double *>(Q)[e];
    case QBF_F32: return (double)static_cast<const float *>(Q)[e];
    case QBF_I32: return (double)static_cast<const int32_t *>(Q)[e];
    default: return (double)static_cast<const int16_t *>(Q)[e];
    }
}

// Deterministic block sum over a fixed tree, red[t] += red[t + s] for
// s = 128, 64, ..., 1; blockDim.x must be 256.  The levels s >= 32 go through
// shared memory, the last five through shuffles in warp 0 (the same pairs in
// the same order, so the same result).
template <class T>
__device__ T block_sum_tree(T x, T *red)
{
    const int t = threadIdx.x;
    red[t] = x;
    __syncthreads();
    for (int s = 128; s >= 32; s >>= 1) {
        if (t < s)
            red[t] = red[t] + red[t + s];
        __syncthreads();
    }
    if (t < 32) {
        T v = red[t];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1)
            v = v + __shfl_down_sync(0xffffffffu, v, s);
        if (t == 0)
            red[0] = v;
    }
    __syncthreads();
    const T r = red[0];
    __syncthreads();
    return r;
}

__device__ double block_sum_d(double x, double *red) { return block_sum_tree(x, red); }

__device__ long long block_sum_ll(long long x, long long *red) { return block_sum_tree(x, red); }

}  // namespace

// One CTA of 256 threads prepares one instance.  The walk dimension n may
// exceed the caller's n_src: the extra variables get zero rows and columns
// (used to give tiny instances of a batch the minimum walk width).
__device__ void prepare_body(const void *Q, int n_src, int n, int dtype, Plan *plan,
                             long long vmax)
{
    __shared__ double sQ[kMaxN * kMaxN];
    __shared__ double redd[256];
    __shared__ long long redl[256];
    const int t = threadIdx.x;
    const int nn = n * n;
    const bool is_int = (dtype == QBF_I32 || dtype == QBF_I16);

    int bad = 0;
    for (int e = t; e < nn; e += blockDim.x) {
        const int qi = e / n, qj = e % n;
        double q = (qi < n_src && qj < n_src) ? load_q(Q, dtype, qi * n_src + qj) : 0.0;
        if (!isfinite(q))
            bad = 1;
        sQ[e] = q;
    }
    bad = __syncthreads_or(bad);
    if (bad) {
        if (t == 0) {
            plan->n = n;
            plan->status = QBF_ENONFINITE;
        }
        return;
    }

    // V_all = sum |Q_ij| (bounds the FP64 canonical sum); V_sym = sum |lin| + sum_{i<j} |S_ij|.
    double va = 0.0, vs = 0.0;
    for (int e = t; e < nn; e += blockDim.x) {
        int i = e / n, j = e % n;
        va += fabs(sQ[e]);
        if (i == j)
            vs += fabs(sQ[e]);
        else if (i < j)
            vs += fabs(sQ[e] + sQ[j * n + i]);
    }
    const double V_all = block_sum_d(va, redd);
    const double V_sym = block_sum_d(vs, redd);

    int sigma = 0;
    if (!is_int && V_sym > 0.0) {
        double room = ((double)vmax - (double)nn) / V_sym;
        sigma = ilogb(room);  // floor(log2(room))
        if (sigma > 1000)
            sigma = 1000;
        if (sigma < -1000)
            sigma = -1000;
    }
    // Shrink sigma until the int32 image provably cannot overflow.
    long long vhat = 0;
    for (int iter = 0; iter < 64; ++iter) {
        long long part = 0;
        for (int e = t; e < nn; e += blockDim.x) {
            int i = e / n, j = e % n;
            if (i > j)
                continue;
            double x = (i == j) ? sQ[e] : sQ[e] + sQ[j * n + i];
            part += llabs(__double2ll_rn(ldexp(x, sigma)));
        }
        vhat = block_sum_ll(part, redl);
        if (vhat <= vmax || is_int)
            break;
        --sigma;
    }
    if (is_int && vhat > vmax) {
        if (t == 0) {
            plan->n = n;
            plan->status = QBF_ERANGE;
            plan->vhat = vhat;
        }
        return;
    }

    // int32 image and the quantisation error bound (quanta).
    double eq = 0.0;
    for (int e = t; e < nn; e += blockDim.x) {
        int i = e / n, j = e % n;
        if (i == j) {
            double y = ldexp(sQ[e], sigma);
            long long r = __double2ll_rn(y);
            plan->lin[i] = (int)r;
            plan->S[e] = 0;
            eq += fabs((double)r - y);
        } else {
            double y = ldexp(sQ[e] + sQ[j * n + i], sigma);
            long long r = __double2ll_rn(y);
            plan->S[e] = (int)r;
            if (i < j)
                eq += fabs((double)r - y);
        }
    }
    eq = block_sum_d(eq, redd);

    if (t == 0) {
        plan->n = n;
        plan->dtype = dtype;
        plan->sigma = sigma;
        plan->vhat = vhat;
        long long W = 0;
        double Eq = 0.0;
        if (!is_int) {
            const double u = 0x1p-53;
            // S_ij = Q_ij + Q_ji is itself rounded for FP64 input.
            Eq = eq * (1.0 + 0x1p-40) + (dtype == QBF_F64 ? ldexp(u * V_all, sigma) : 0.0);
            // |FP64 canonical sum - exact f| <= gamma_N * V_all, N = n^2 additions.
            const double N = (double)nn;
            const double e64 = (N * u / (1.0 - N * u)) * V_all;
            double w = 2.0 * (Eq + ldexp(e64, sigma)) * (1.0 + 0x1p-30);
            if (w > 0.0)
                W = (long long)ceil(w) + 1;
            if (W > (long long)INT_MAX)
                W = INT_MAX;
        }
        plan->eq_quanta = Eq;
        plan->window = W;
        plan->error_bound = ldexp((double)W * 0.5, -sigma);
        plan->status = QBF_OK;
    }
}

__global__ void __launch_bounds__(256) prepare_kernel(const void *Q, int n, int dtype, Plan *plan,
                                                      long long vmax)
{
    prepare_body(Q, n, n, dtype, plan, vmax);
}

// Records and in-block corrections for a walk over suffix bits 0..ns-1 with
// R low bits unrolled (M = ns - R mid bits, 2^M blocks).  Record B (1 <= B < 2^M)
// describes the flip at the start of block B; entry 0 is unused.  The thread
// with B < 128 also writes correction K[B / 64][B % 64], so callers visit
// every B below max(2^M, 128).
__device__ void tables_body(const Plan *__restrict__ plan, int ns, int R, Rec *recs,
                            unsigned nrec, int *Kbuf, unsigned B)
{
    const int n = plan->n;
    const int *S = plan->S;
    const int *lin = plan->lin;

    if (B < 128) {
        // K[pi][u]: static part of the delta at in-block step u of a block of parity pi.
        const int pi = (int)(B >> 6), u = (int)(B & 63);
        int val = 0;
        if (u >= 1 && u < (1 << R)) {
            int l = __ffs(u) - 1;
            int gprev = (u - 1) ^ ((u - 1) >> 1);
            int gnow = u ^ (u >> 1);
            int nb = ((gnow >> l) & 1) ^ ((l == R - 1) ? pi : 0);
            unsigned corr = 0;
            for (int j = 0; j < R; ++j) {
                if (j == l)
                    continue;
                int bit = (gprev >> j) & 1;
                int d = (j == R - 1 && pi) ? -bit : bit;
                corr += (unsigned)(d * S[l * n + j]);
            }
            val = (int)(nb ? corr : 0u - corr);
        }
        Kbuf[pi * 64 + u] = val;
    }
    if (B == 0 || B >= nrec)
        return;

    const int l = R + __ffs(B) - 1;        // flipped bit: R + CTZ(B)
    const unsigned g = B ^ (B >> 1);       // mid bits of the Gray state in block B
    const unsigned gprev = (B - 1) ^ ((B - 1) >> 1);
    const int nb = (g >> (l - R)) & 1;     // new value of bit l
    unsigned U = (unsigned)lin[l];
    for (int j = R; j < ns; ++j)
        if (j != l && ((gprev >> (j - R)) & 1))
            U += (unsigned)S[l * n + j];
    if (B & 1)  // the low bits end block B-1 at e_{R-1} when B-1 is even
        U += (unsigned)S[l * n + (R - 1)];
    Rec r;
    r.T = (int)(nb ? U : 0u - U);
    r.code = 2 * (l - R) + nb;
    for (int i = 0; i < kRMax; ++i) {
        unsigned w = 0;
        if (i < R) {
            unsigned s_il = (unsigned)S[i * n + l];
            w = nb ? s_il : 0u - s_il;
            if (i != R - 1) {
                unsigned s_ir = (unsigned)S[i * n + (R - 1)];
                w += (B & 1) ? s_ir : 0u - s_ir;
            }
        }
        r.W[i] = (int)w;
    }
    recs[B] = r;
}

__global__ void tables_kernel(const Plan *__restrict__ plan, int ns, int R, Rec *recs,
                              unsigned nrec, int *Kbuf)
{
    if (plan->status != QBF_OK)
        return;
    tables_body(plan, ns, R, recs, nrec, Kbuf, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---- batched: one CTA per instance ---------------------------------------

__global__ void __launch_bounds__(256) batched_prepare_kernel(const BatchDesc *desc, Plan *plans,
                                                              int *status, long long vmax_float)
{
    const BatchDesc d = desc[blockIdx.x];
    Plan *plan = plans + blockIdx.x;
    // integer instances keep their exact image (2^31 bound); float instances
    // are scaled into vmax_float
    const bool is_int = (d.dtype == QBF_I32 || d.dtype == QBF_I16);
    prepare_body(d.Q, d.n_src, d.n, d.dtype, plan, is_int ? (long long)INT_MAX : vmax_float);
    if (threadIdx.x == 0)
        status[blockIdx.x] = plan->status;
}

__global__ void __launch_bounds__(256) batched_tables_kernel(const BatchDesc *desc,
                                                             const Plan *plans, Rec *recs, int *K)
{
    const int i = blockIdx.x;
    const Plan *plan = plans + i;
    if (plan->status != QBF_OK)
        return;
    const BatchDesc d = desc[i];
    const unsigned nrec = 1u << (d.ns - kRMax);
    for (unsigned B = threadIdx.x; B < max(nrec, 128u); B += blockDim.x)
        tables_body(plan, d.ns, kRMax, recs + d.rec_off, nrec, K + i * 128, B);
}

// ---- Boltzmann log-partition: two-limb images ------------------------------
//
// For instance b and walk w (0: identity order, 1: variables rotated so that
// walk variable v is the caller's variable (v + rot) mod n), writes two Plans:
// hi = round(y * 2^sigma) and lo = round((y * 2^sigma - hi) * 2^L) for every
// lin / S entry y, L = logz_lo_bits(n).  sigma keeps sum |hi| <= 2^22, and
// |lo| <= 2^(L-1) over at most n(n+1)/2 entries keeps sum |lo| <= 2^22, so
// every value the walk forms (a state's value minus the shift, plus one field
// or correction) stays below 3 * 2^22 < 2^24 in each limb: both limbs walk
// exactly in FP32, as one packed pair.  hi * 2^L + lo is the fixed-point value
// at scale 2^(sigma + L).  sigma comes from the unrotated order so both walks
// share it.
__global__ void __launch_bounds__(256) logz_prepare_kernel(const void *Q, int n, int dtype,
                                                           int rot, Plan *plans)
{
    __shared__ double sQ[kMaxN * kMaxN];
    __shared__ double redd[256];
    __shared__ long long redl[256];
    const int b = blockIdx.x >> 1, w = blockIdx.x & 1;
    const int t = threadIdx.x;
    const int nn = n * n;
    const size_t esz = (dtype == QBF_F64) ? 8 : (dtype == QBF_I16 ? 2 : 4);
    const void *Qb = (const char *)Q + (size_t)b * nn * esz;
    Plan *hi = plans + (size_t)(b * 2 + w) * 2;
    Plan *lo = hi + 1;
    int bad = 0;
    double vs = 0.0;
    for (int e = t; e < nn; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const double q = load_q(Qb, dtype, e);
        if (!isfinite(q))
            bad = 1;
        if (i == j)
            vs += fabs(q);
        else if (i < j)
            vs += fabs(q + load_q(Qb, dtype, j * n + i));
        // rotated copy: walk variable (i', j') holds caller (i, j)
        const int ri = w ? (i - rot + n) % n : i, rj = w ? (j - rot + n) % n : j;
        sQ[ri * n + rj] = q;
    }
    bad = __syncthreads_or(bad);
    if (bad) {
        if (t == 0) {
            hi->n = lo->n = n;
            hi->status = lo->status = QBF_ENONFINITE;
        }
        return;
    }
    const double V_sym = block_sum_d(vs, redd);
    const double limb_max = (double)kLzLimbMax;
    int sigma = 0;
    if (V_sym > 0.0) {
        sigma = ilogb((limb_max - (double)nn) / V_sym);
        sigma = max(-1000, min(1000, sigma));
    }
    for (int iter = 0; iter < 64; ++iter) {
        long long part = 0;
        for (int e = t; e < nn; e += blockDim.x) {
            const int i = e / n, j = e % n;
            if (i > j)
                continue;
            const double y = (i == j) ? sQ[e] : sQ[e] + sQ[j * n + i];
            part += llabs(__double2ll_rn(ldexp(y, sigma)));
        }
        if (block_sum_ll(part, redl) <= kLzLimbMax)
            break;
        --sigma;
    }
    const int L = logz_lo_bits(n);
    for (int e = t; e < nn; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const double y = (i == j) ? ldexp(sQ[e], sigma) : ldexp(sQ[e] + sQ[j * n + i], sigma);
        const long long h = __double2ll_rn(y);
        const long long l = __double2ll_rn(ldexp(y - (double)h, L));
        if (i == j) {
            hi->lin[i] = (int)h;
            lo->lin[i] = (int)l;
            hi->S[e] = lo->S[e] = 0;
        } else {
            hi->S[e] = (int)h;
            lo->S[e] = (int)l;
        }
    }
    if (t == 0) {
        hi->n = lo->n = n;
        hi->dtype = lo->dtype = dtype;
        hi->sigma = sigma;
        lo->sigma = sigma + L;
        hi->window = lo->window = 0;
        hi->status = lo->status = QBF_OK;
    }
}

// Walk tables for every (instance, walk, limb) plan: block = plan index.
__global__ void __launch_bounds__(256) logz_tables_kernel(const Plan *plans, int nsA, int nsB,
                                                          Rec *recs, unsigned rec_stride, int *K)
{
    const int pi = blockIdx.x;           // (b * 2 + w) * 2 + limb
    const int w = (pi >> 1) & 1;
    const Plan *plan = plans + pi;
    if (plan->status != QBF_OK)
        return;
    const int ns = w ? nsB : nsA;
    const int R = min(kRMax, ns);
    const unsigned nrec = 1u << (ns - R);
    Rec *rp = recs + (size_t)pi * rec_stride;
    int *Kp = K + pi * 128;
    for (unsigned B = threadIdx.x; B < max(nrec, 128u); B += blockDim.x) {
        tables_body(plan, ns, R, rp, nrec, Kp, B);
        // the log Z walks add these in FP32 (exact: |value| <= 2 * 2^22); this
        // thread wrote exactly the entries of index B
        if (B < 128)
            Kp[B] = __float_as_int((float)Kp[B]);
        if (B > 0 && B < nrec) {
            rp[B].T = __float_as_int((float)rp[B].T);
            for (int i = 0; i < kRMax; ++i)
                rp[B].W[i] = __float_as_int((float)rp[B].W[i]);
        }
    }
}

}  // namespace qbf
