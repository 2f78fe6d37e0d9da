/*
 * qubo_oracle_blocked.c -- the blocked natural-order oracle for large n.
 *
 * TEST INFRASTRUCTURE ONLY, like qubo_oracle.c (same library, same rules:
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it; it shares nothing with the CUDA library and uses no Gray
 * code).  "parity unpinned" does not apply: every function here is pinned
 * against the literal oracle of qubo_oracle.c, bit for bit, on random
 * instances with many ties (tests/test_oracle_pins.py).
 *
 * What it computes: exactly what the literal oracle computes -- the k
 * smallest states of f(x) = x^T Q x (Eq. 1) by (value, natural index), with
 * float values in the canonical FP64 order (documented in qubo_oracle.c) and
 * integer values in exact int64 -- but fast enough for n = 40..44, where the
 * literal loop's O(n^2) additions per state would take days.
 *
 * Enumeration is still the naive method of Section 3: idx runs over
 * [lo, hi) in ascending natural order, x_i = bit i of idx.  Only the
 * arithmetic is blocked.  With L = min(n, 12) low variables a = idx mod 2^L
 * and the high part h = idx - a, Eq. 1 splits exactly as
 *     f(a + h) = f(a) + f(h) + sum_{i < L, x_i = 1} c_i(h),
 *     c_i(h)   = sum_{j >= L, x_j = 1} (Q_ij + Q_ji),
 * (the cross terms between the two parts).  f(a) is a table of 2^L
 * canonical values, f(h) and the c_i are formed once per block of 2^L
 * states, and the sums of c_i over the set bits of a come from two subset-sum
 * tables over a's low six and high L - 6 variables.  A state then costs two
 * additions and a comparison.
 *
 * Integer Q: all of that is exact in int64, so the blocked value IS the
 * value and the top-k is kept exactly by (value, idx).
 *
 * Float Q: the blocked value v~ is another rounding of the same real sum.
 * Each entry Q_ij of a state passes through at most d = 2n + 2 additions in
 * either evaluation order (one for the pair Q_ij + Q_ji, at most n - 1 along
 * a row or a c_i, at most n + 3 more), so by the standard bound for any
 * summation tree (|error| <= gamma_d * sum |terms|, gamma_d = d u / (1 - d u),
 * u = 2^-53; no multiplications, so no underflow loss) both v~ and the
 * canonical value lie within gamma_d * A of the exact f, A = sum |Q_ij|.  With
 * B = 2 gamma_d A (taken here with d = 2n + 16):
 *   tau = the k-th smallest v~ over the range.  There are k states with
 *   canonical value <= tau + B, so the k-th smallest canonical value T is
 *   <= tau + B, and every state with canonical value <= T has v~ <= T + B
 *   <= tau + 2B.
 * So every state with v~ <= tau + 2B is kept as a candidate (tau is the
 * running k-th smallest while walking, which only falls), re-evaluated with
 * orc_eval_f64 in canonical order, and the k smallest candidates by
 * (canonical value, idx) are the answer -- bit for bit the literal oracle's.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define BLK_LMAX 12         /* low variables per block: 2^12 doubles = 32 KB   */
#define BLK_LA 6            /* low variables of the first subset-sum table      */
#define BLK_MAX_THREADS 256
#define BLK_MAX_TOPK 1024
#define BLK_CAND_HARD (1u << 24) /* candidates one thread may hold after pruning */

double orc_eval_f64(const double *Q, int n, uint64_t idx);
int64_t orc_eval_i64(const int64_t *Q, int n, uint64_t idx);
int orc_default_threads(void);

typedef double vd4 __attribute__((vector_size(16)));
typedef int64_t vi4 __attribute__((vector_size(16)));

/* ------------------------------------------------------------------ */
/* the problem, tables shared by all threads (read only)                */
/* ------------------------------------------------------------------ */

typedef struct {
    int n, L, La, Lb;
    const double *Qd;    /* float Q (FP64), or NULL                        */
    const int64_t *Qi;   /* integer Q, or NULL                             */
    double *pair_d;      /* pair[i*n + j] = Q_ij + Q_ji (one rounding)     */
    int64_t *pair_i;
    double *fl_d;        /* f of the low-only state a, canonical, 2^L      */
    int64_t *fl_i;
    double B;            /* float: 2 gamma_d A; integer: 0                 */
    int zero;            /* float Q with every entry 0: f = 0 everywhere    */
} blk_ctx;

static int ctx_init(blk_ctx *C, const double *Qd, const int64_t *Qi, int n)
{
    memset(C, 0, sizeof(*C));
    C->n = n;
    C->L = n < BLK_LMAX ? n : BLK_LMAX;
    C->La = C->L < BLK_LA ? C->L : BLK_LA;
    C->Lb = C->L - C->La;
    C->Qd = Qd;
    C->Qi = Qi;
    const size_t nn = (size_t)n * n;
    const size_t nl = (size_t)1 << C->L;
    if (Qd) {
        double A = 0.0;
        for (size_t e = 0; e < nn; ++e) {
            if (!isfinite(Qd[e]))
                return -1;
            A += fabs(Qd[e]);
        }
        if (!(A < 1e300))
            return -1;
        C->zero = (A == 0.0);
        /* A itself was summed with rounding: inflate by (1 + 2 n^2 u) */
        const double u = ldexp(1.0, -53);
        const double Ain = A * (1.0 + 2.0 * (double)nn * u);
        const double d = 2.0 * n + 16.0;
        const double gam = d * u / (1.0 - d * u);
        C->B = 2.0 * gam * Ain;
        C->pair_d = (double *)malloc(nn * sizeof(double));
        C->fl_d = (double *)malloc(nl * sizeof(double));
        if (!C->pair_d || !C->fl_d)
            return -2;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                C->pair_d[(size_t)i * n + j] = Qd[(size_t)i * n + j] + Qd[(size_t)j * n + i];
        for (size_t a = 0; a < nl; ++a)
            C->fl_d[a] = orc_eval_f64(Qd, n, a);
    } else {
        /* exact int64 needs sum |Q_ij| < 2^62 */
        uint64_t A = 0;
        for (size_t e = 0; e < nn; ++e) {
            const int64_t q = Qi[e];
            if (q > ((int64_t)1 << 52) || q < -((int64_t)1 << 52))
                return -1;
            A += (uint64_t)(q < 0 ? -q : q);
            if (A >= ((uint64_t)1 << 62))
                return -1;
        }
        C->pair_i = (int64_t *)malloc(nn * sizeof(int64_t));
        C->fl_i = (int64_t *)malloc(nl * sizeof(int64_t));
        if (!C->pair_i || !C->fl_i)
            return -2;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                C->pair_i[(size_t)i * n + j] = Qi[(size_t)i * n + j] + Qi[(size_t)j * n + i];
        for (size_t a = 0; a < nl; ++a)
            C->fl_i[a] = orc_eval_i64(Qi, n, a);
    }
    return 0;
}

static void ctx_free(blk_ctx *C)
{
    free(C->pair_d);
    free(C->pair_i);
    free(C->fl_d);
    free(C->fl_i);
}

/* ------------------------------------------------------------------ */
/* per-block set-up: f(h) in canonical order and the cross sums           */
/* ------------------------------------------------------------------ */

/* Canonical f of the high-only state h (the low L bits are zero): visiting
 * only the set bits in ascending order performs exactly the additions of
 * orc_eval_f64, in the same order. */
static double high_value_d(const blk_ctx *C, uint64_t h)
{
    const int n = C->n;
    int bits[64], nb = 0;
    for (uint64_t m = h; m; m &= m - 1)
        bits[nb++] = __builtin_ctzll(m);
    double acc = 0.0;
    for (int s = 0; s < nb; ++s) {
        const int i = bits[s];
        double row = C->Qd[(size_t)i * n + i];
        for (int t = s + 1; t < nb; ++t)
            row = row + C->pair_d[(size_t)i * n + bits[t]];
        acc = acc + row;
    }
    return acc;
}

static int64_t high_value_i(const blk_ctx *C, uint64_t h)
{
    const int n = C->n;
    int bits[64], nb = 0;
    for (uint64_t m = h; m; m &= m - 1)
        bits[nb++] = __builtin_ctzll(m);
    int64_t acc = 0;
    for (int s = 0; s < nb; ++s) {
        const int i = bits[s];
        int64_t row = C->Qi[(size_t)i * n + i];
        for (int t = s + 1; t < nb; ++t)
            row += C->pair_i[(size_t)i * n + bits[t]];
        acc += row;
    }
    return acc;
}

/* cA[t] = sum of c_i over the set bits i of t (variables 0..La-1),
 * cB[t] = the same over variables La..L-1 (bit t_b = variable La + b). */
static void cross_tables_d(const blk_ctx *C, uint64_t h, double *cA, double *cB)
{
    const int n = C->n, L = C->L;
    double c[BLK_LMAX];
    for (int i = 0; i < L; ++i) {
        double s = 0.0;
        for (uint64_t m = h; m; m &= m - 1)
            s = s + C->pair_d[(size_t)i * n + __builtin_ctzll(m)];
        c[i] = s;
    }
    cA[0] = 0.0;
    for (int t = 1; t < (1 << C->La); ++t)
        cA[t] = cA[t & (t - 1)] + c[__builtin_ctz(t)];
    cB[0] = 0.0;
    for (int t = 1; t < (1 << C->Lb); ++t)
        cB[t] = cB[t & (t - 1)] + c[C->La + __builtin_ctz(t)];
}

static void cross_tables_i(const blk_ctx *C, uint64_t h, int64_t *cA, int64_t *cB)
{
    const int n = C->n, L = C->L;
    int64_t c[BLK_LMAX];
    for (int i = 0; i < L; ++i) {
        int64_t s = 0;
        for (uint64_t m = h; m; m &= m - 1)
            s += C->pair_i[(size_t)i * n + __builtin_ctzll(m)];
        c[i] = s;
    }
    cA[0] = 0;
    for (int t = 1; t < (1 << C->La); ++t)
        cA[t] = cA[t & (t - 1)] + c[__builtin_ctz(t)];
    cB[0] = 0;
    for (int t = 1; t < (1 << C->Lb); ++t)
        cB[t] = cB[t & (t - 1)] + c[C->La + __builtin_ctz(t)];
}

/* The blocked value of the state h + a.  The vector loops below form the
 * same two additions in the same order, so both give identical values. */
static inline double vblk_d(const blk_ctx *C, const double *cA, const double *cB, double K,
                            unsigned a)
{
    const unsigned am = (1u << C->La) - 1;
    return (C->fl_d[a] + cA[a & am]) + (K + cB[a >> C->La]);
}

static inline int64_t vblk_i(const blk_ctx *C, const int64_t *cA, const int64_t *cB, int64_t K,
                             unsigned a)
{
    const unsigned am = (1u << C->La) - 1;
    return (C->fl_i[a] + cA[a & am]) + (K + cB[a >> C->La]);
}

/* Does any state a in [a0, a1) have a blocked value <= thr (float)?  The
 * whole-block form tests 2^L values with compares OR-ed into masks, two
 * doubles per vector (the native width of SSE2 and of NEON). */
static int block_hit_d(const blk_ctx *C, const double *cA, const double *cB, double K,
                       unsigned a0, unsigned a1, double thr)
{
    if (a0 == 0 && a1 == (1u << C->L) && C->La == BLK_LA) {
        const vd4 vt = {thr, thr};
        vi4 h[8] = {{0, 0}};
        vd4 ca[32];
        memcpy(ca, cA, sizeof(ca));
        for (int b = 0; b < (1 << C->Lb); ++b) {
            const double base = K + cB[b];
            const vd4 vb = {base, base};
            vd4 r[32];
            memcpy(r, C->fl_d + ((size_t)b << BLK_LA), sizeof(r));
            for (int t = 0; t < 32; t += 8)
                for (int e = 0; e < 8; ++e)
                    h[e] |= ((r[t + e] + ca[t + e]) + vb) <= vt;
        }
        vi4 o = h[0] | h[1] | h[2] | h[3] | h[4] | h[5] | h[6] | h[7];
        return (o[0] | o[1]) != 0;
    }
    for (unsigned a = a0; a < a1; ++a)
        if (vblk_d(C, cA, cB, K, a) <= thr)
            return 1;
    return 0;
}

/* Integer form: any value < thr, or == thr when `eq` (exact int64). */
static int block_hit_i(const blk_ctx *C, const int64_t *cA, const int64_t *cB, int64_t K,
                       unsigned a0, unsigned a1, int64_t thr, int eq)
{
    /* v <= thr - 1 is v < thr; thr = INT64_MIN with eq = 0 admits nothing */
    if (!eq && thr == INT64_MIN)
        return 0;
    const int64_t t = eq ? thr : thr - 1;
    if (a0 == 0 && a1 == (1u << C->L) && C->La == BLK_LA) {
        const vi4 vt = {t, t};
        vi4 h[8] = {{0, 0}};
        vi4 ca[32];
        memcpy(ca, cA, sizeof(ca));
        for (int b = 0; b < (1 << C->Lb); ++b) {
            const int64_t base = K + cB[b];
            const vi4 vb = {base, base};
            vi4 r[32];
            memcpy(r, C->fl_i + ((size_t)b << BLK_LA), sizeof(r));
            for (int u = 0; u < 32; u += 8)
                for (int e = 0; e < 8; ++e)
                    h[e] |= ((r[u + e] + ca[u + e]) + vb) <= vt;
        }
        vi4 o = h[0] | h[1] | h[2] | h[3] | h[4] | h[5] | h[6] | h[7];
        return (o[0] | o[1]) != 0;
    }
    for (unsigned a = a0; a < a1; ++a)
        if (vblk_i(C, cA, cB, K, a) <= t)
            return 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* one thread's running state                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    double v;     /* blocked value (float) */
    uint64_t ix;
} cand_t;

typedef struct {
    int k, kc;
    /* float: the kc smallest blocked values seen, ascending; candidates */
    double kb[BLK_MAX_TOPK];
    cand_t *cand;
    size_t nc, cap;
    /* integer: the kc smallest (value, idx), lexicographic, exact */
    int64_t kv[BLK_MAX_TOPK];
    uint64_t ki[BLK_MAX_TOPK];
    int err;
} acc_t;

static int acc_init(acc_t *S, int k)
{
    memset(S, 0, sizeof(*S));
    S->k = k;
    S->cap = 1u << 12;
    S->cand = (cand_t *)malloc(S->cap * sizeof(cand_t));
    return S->cand ? 0 : -2;
}

/* margin added to the running k-th smallest value: 2B plus the rounding of
 * forming tau + 2B itself */
static inline double cand_threshold(const blk_ctx *C, const acc_t *S)
{
    if (S->kc < S->k)
        return INFINITY;
    const double tau = S->kb[S->k - 1];
    return tau + (2.0 * C->B + 4.0 * ldexp(1.0, -53) * fabs(tau) + 1e-300);
}

static void kb_insert(acc_t *S, double v)
{
    int pos = S->kc;
    if (pos == S->k) {
        if (!(v < S->kb[S->k - 1]))
            return;
        pos = S->k - 1;
    } else {
        S->kc++;
    }
    while (pos > 0 && v < S->kb[pos - 1]) {
        S->kb[pos] = S->kb[pos - 1];
        --pos;
    }
    S->kb[pos] = v;
}

static void cand_push(const blk_ctx *C, acc_t *S, double v, uint64_t ix)
{
    if (S->nc == S->cap) {
        const double thr = cand_threshold(C, S);
        size_t w = 0;
        for (size_t e = 0; e < S->nc; ++e)
            if (S->cand[e].v <= thr)
                S->cand[w++] = S->cand[e];
        S->nc = w;
        if (S->nc > S->cap / 2) {
            if (S->cap >= BLK_CAND_HARD) {
                S->err = -3;
                return;
            }
            cand_t *g = (cand_t *)realloc(S->cand, 2 * S->cap * sizeof(cand_t));
            if (!g) {
                S->err = -2;
                return;
            }
            S->cand = g;
            S->cap *= 2;
        }
    }
    S->cand[S->nc].v = v;
    S->cand[S->nc].ix = ix;
    S->nc++;
}

static inline int lexlt_i(int64_t a, uint64_t ia, int64_t b, uint64_t ib)
{
    return a < b || (a == b && ia < ib);
}

static void ki_insert(acc_t *S, int64_t v, uint64_t ix)
{
    int pos = S->kc;
    if (pos == S->k) {
        if (!lexlt_i(v, ix, S->kv[S->k - 1], S->ki[S->k - 1]))
            return;
        pos = S->k - 1;
    } else {
        S->kc++;
    }
    while (pos > 0 && lexlt_i(v, ix, S->kv[pos - 1], S->ki[pos - 1])) {
        S->kv[pos] = S->kv[pos - 1];
        S->ki[pos] = S->ki[pos - 1];
        --pos;
    }
    S->kv[pos] = v;
    S->ki[pos] = ix;
}

/* Walk idx in [lo, hi) (any bounds) into S, block by block, ascending. */
static void walk_range(const blk_ctx *C, acc_t *S, uint64_t lo, uint64_t hi)
{
    const int L = C->L;
    const uint64_t lmask = ((uint64_t)1 << L) - 1;
    double cAd[1 << BLK_LA], cBd[1 << (BLK_LMAX - BLK_LA)];
    int64_t cAi[1 << BLK_LA], cBi[1 << (BLK_LMAX - BLK_LA)];
    uint64_t idx = lo;
    while (idx < hi && !S->err) {
        const uint64_t h = idx & ~lmask;
        const unsigned a0 = (unsigned)(idx & lmask);
        const uint64_t nb = h + lmask + 1;
        const uint64_t end = nb < hi ? nb : hi;
        const unsigned a1 = (unsigned)(end - h);  /* 1 .. 2^L */
        if (C->Qd) {
            const double K = high_value_d(C, h);
            cross_tables_d(C, h, cAd, cBd);
            if (block_hit_d(C, cAd, cBd, K, a0, a1, cand_threshold(C, S))) {
                for (unsigned a = a0; a < a1 && !S->err; ++a) {
                    const double v = vblk_d(C, cAd, cBd, K, a);
                    if (S->kc < S->k || v < S->kb[S->k - 1])
                        kb_insert(S, v);
                    if (v <= cand_threshold(C, S))
                        cand_push(C, S, v, h + a);
                }
            }
        } else {
            const int64_t K = high_value_i(C, h);
            cross_tables_i(C, h, cAi, cBi);
            /* a state of this block can enter the exact top-k only with a value
             * below the k-th, or equal to it at a lower index */
            const int full = S->kc == S->k;
            if (!full || block_hit_i(C, cAi, cBi, K, a0, a1, S->kv[S->k - 1],
                                     h + a0 < S->ki[S->k - 1])) {
                for (unsigned a = a0; a < a1; ++a) {
                    const int64_t v = vblk_i(C, cAi, cBi, K, a);
                    if (S->kc < S->k || lexlt_i(v, h + a, S->kv[S->k - 1], S->ki[S->k - 1]))
                        ki_insert(S, v, h + a);
                }
            }
        }
        idx = end;
    }
}

/* ------------------------------------------------------------------ */
/* threads: blocks of the range taken from a shared counter             */
/* ------------------------------------------------------------------ */

typedef struct {
    const blk_ctx *C;
    acc_t S;
    uint64_t lo, hi, base, piece;
    uint64_t *next; /* shared: next piece number */
    uint64_t npieces;
} thr_job;

static void *thr_worker(void *arg)
{
    thr_job *J = (thr_job *)arg;
    for (;;) {
        const uint64_t p = __atomic_fetch_add(J->next, 1, __ATOMIC_RELAXED);
        if (p >= J->npieces || J->S.err)
            break;
        /* pieces are aligned to whole blocks from `base` (lo rounded down) */
        uint64_t a = J->base + p * J->piece, b = a + J->piece;
        if (a < J->lo)
            a = J->lo;
        if (b > J->hi)
            b = J->hi;
        walk_range(J->C, &J->S, a, b);
    }
    return NULL;
}

static int cmp_cand_canon(const void *x, const void *y)
{
    const cand_t *a = (const cand_t *)x, *b = (const cand_t *)y;
    if (a->v < b->v)
        return -1;
    if (a->v > b->v)
        return 1;
    return (a->ix > b->ix) - (a->ix < b->ix);
}

/* k smallest over [lo, hi) with T threads; returns the count written or < 0 */
static int blocked_topk(const double *Qd, const int64_t *Qi, int n, uint64_t lo, uint64_t hi,
                        int k, int threads, double *vd, int64_t *vi, uint64_t *ix,
                        uint64_t *n_candidates)
{
    if (n < 1 || n > 62 || lo >= hi || hi > ((uint64_t)1 << n) || k < 1 || k > BLK_MAX_TOPK)
        return -1;
    blk_ctx C;
    int rc = ctx_init(&C, Qd, Qi, n);
    if (rc) {
        ctx_free(&C);
        return rc;
    }
    if (C.zero) {
        /* float Q = 0: every state ties at 0, the lowest indices win */
        const uint64_t m = hi - lo < (uint64_t)k ? hi - lo : (uint64_t)k;
        for (uint64_t e = 0; e < m; ++e) {
            vd[e] = 0.0;
            ix[e] = lo + e;
        }
        if (n_candidates)
            *n_candidates = 0;
        ctx_free(&C);
        return (int)m;
    }
    int T = threads > 0 ? threads : orc_default_threads();
    if (T > BLK_MAX_THREADS)
        T = BLK_MAX_THREADS;
    /* pieces of whole blocks, about 64 per thread for balance */
    const uint64_t blk = (uint64_t)1 << C.L;
    uint64_t piece = (hi - lo) / ((uint64_t)T * 64);
    piece = ((piece + blk - 1) / blk) * blk;
    if (piece < blk)
        piece = blk;
    const uint64_t base = lo & ~(blk - 1);
    const uint64_t npieces = (hi - base + piece - 1) / piece;
    if ((uint64_t)T > npieces)
        T = (int)npieces;
    thr_job *jobs = (thr_job *)calloc((size_t)T, sizeof(thr_job));
    if (!jobs) {
        ctx_free(&C);
        return -2;
    }
    uint64_t next = 0;
    for (int t = 0; t < T; ++t) {
        jobs[t].C = &C;
        jobs[t].lo = lo;
        jobs[t].hi = hi;
        jobs[t].base = base;
        jobs[t].piece = piece;
        jobs[t].next = &next;
        jobs[t].npieces = npieces;
        if (acc_init(&jobs[t].S, k))
            rc = -2;
    }
    pthread_t tid[BLK_MAX_THREADS];
    if (!rc) {
        for (int t = 1; t < T; ++t)
            pthread_create(&tid[t], NULL, thr_worker, &jobs[t]);
        thr_worker(&jobs[0]);
        for (int t = 1; t < T; ++t)
            pthread_join(tid[t], NULL);
        for (int t = 0; t < T; ++t)
            if (jobs[t].S.err)
                rc = jobs[t].S.err;
    }
    int cnt = 0;
    if (!rc && Qi) {
        acc_t *all = &jobs[0].S;
        for (int t = 1; t < T; ++t)
            for (int e = 0; e < jobs[t].S.kc; ++e)
                ki_insert(all, jobs[t].S.kv[e], jobs[t].S.ki[e]);
        cnt = all->kc;
        for (int e = 0; e < cnt; ++e) {
            vi[e] = all->kv[e];
            ix[e] = all->ki[e];
        }
        if (n_candidates)
            *n_candidates = 0;
    } else if (!rc) {
        /* the global k-th smallest blocked value, then every candidate under it */
        acc_t *all = &jobs[0].S;
        for (int t = 1; t < T; ++t)
            for (int e = 0; e < jobs[t].S.kc; ++e)
                kb_insert(all, jobs[t].S.kb[e]);
        const double thr = cand_threshold(&C, all);
        size_t total = 0;
        for (int t = 0; t < T; ++t)
            for (size_t e = 0; e < jobs[t].S.nc; ++e)
                total += jobs[t].S.cand[e].v <= thr;
        cand_t *list = (cand_t *)malloc((total ? total : 1) * sizeof(cand_t));
        if (!list) {
            rc = -2;
        } else {
            size_t w = 0;
            for (int t = 0; t < T; ++t)
                for (size_t e = 0; e < jobs[t].S.nc; ++e)
                    if (jobs[t].S.cand[e].v <= thr) {
                        list[w].ix = jobs[t].S.cand[e].ix;
                        list[w].v = orc_eval_f64(Qd, n, list[w].ix); /* canonical */
                        ++w;
                    }
            qsort(list, w, sizeof(cand_t), cmp_cand_canon);
            cnt = (int)(w < (size_t)k ? w : (size_t)k);
            for (int e = 0; e < cnt; ++e) {
                vd[e] = list[e].v;
                ix[e] = list[e].ix;
            }
            if (n_candidates)
                *n_candidates = w;
            free(list);
        }
    }
    for (int t = 0; t < T; ++t)
        free(jobs[t].S.cand);
    free(jobs);
    ctx_free(&C);
    return rc ? rc : cnt;
}

/* ------------------------------------------------------------------ */
/* exported                                                             */
/* ------------------------------------------------------------------ */

/* k smallest states over idx in [lo, hi) by (canonical FP64 value, idx):
 * the same answer as orc_topk_f64.  Returns the count written (min(k, hi -
 * lo)), or < 0: -1 bad arguments / non-finite Q, -2 out of memory, -3 more
 * than 2^24 near-tied candidates in one thread.  *n_candidates (may be
 * NULL) receives the number of states re-evaluated canonically. */
int orc_topk_blocked_f64(const double *Q, int n, uint64_t lo, uint64_t hi, int k, int threads,
                         double *vals, uint64_t *idx, uint64_t *n_candidates)
{
    return blocked_topk(Q, NULL, n, lo, hi, k, threads, vals, NULL, idx, n_candidates);
}

/* The same in exact int64 (orc_topk_i64's answer); entries |Q_ij| <= 2^52
 * and sum |Q_ij| < 2^62, else -1. */
int orc_topk_blocked_i64(const int64_t *Q, int n, uint64_t lo, uint64_t hi, int k, int threads,
                         int64_t *vals, uint64_t *idx)
{
    return blocked_topk(NULL, Q, n, lo, hi, k, threads, NULL, vals, idx, NULL);
}

/* Minimum of every segment [lo + s*seg, lo + (s+1)*seg), s < nseg, with its
 * lowest argmin: one single-threaded blocked walk per segment, segments
 * shared among the threads.  Returns 0 or < 0 as above. */
typedef struct {
    const blk_ctx *C;
    uint64_t lo, seg, nseg;
    uint64_t *next;
    double *vd;
    int64_t *vi;
    uint64_t *ix;
    int err;
} seg_job;

static void *seg_worker(void *arg)
{
    seg_job *J = (seg_job *)arg;
    acc_t *S = (acc_t *)malloc(sizeof(acc_t));
    if (!S || acc_init(S, 1)) {
        J->err = -2;
        free(S);
        return NULL;
    }
    for (;;) {
        const uint64_t s = __atomic_fetch_add(J->next, 1, __ATOMIC_RELAXED);
        if (s >= J->nseg)
            break;
        S->kc = 0;
        S->nc = 0;
        const uint64_t a = J->lo + s * J->seg;
        walk_range(J->C, S, a, a + J->seg);
        if (S->err) {
            J->err = S->err;
            break;
        }
        if (J->C->Qi) {
            J->vi[s] = S->kv[0];
            J->ix[s] = S->ki[0];
        } else {
            const double thr = cand_threshold(J->C, S);
            double best = INFINITY;
            uint64_t bi = 0;
            int have = 0;
            for (size_t e = 0; e < S->nc; ++e) {
                if (!(S->cand[e].v <= thr))
                    continue;
                const uint64_t x = S->cand[e].ix;
                const double v = orc_eval_f64(J->C->Qd, J->C->n, x);
                if (!have || v < best || (v == best && x < bi)) {
                    best = v;
                    bi = x;
                    have = 1;
                }
            }
            J->vd[s] = best;
            J->ix[s] = bi;
        }
    }
    free(S->cand);
    free(S);
    return NULL;
}

static int blocked_segmin(const double *Qd, const int64_t *Qi, int n, uint64_t lo, uint64_t seg,
                          uint64_t nseg, int threads, double *vd, int64_t *vi, uint64_t *ix)
{
    if (n < 1 || n > 62 || seg < 1 || nseg < 1 || lo + seg * nseg > ((uint64_t)1 << n) ||
        seg > ((uint64_t)1 << n))
        return -1;
    blk_ctx C;
    int rc = ctx_init(&C, Qd, Qi, n);
    if (rc) {
        ctx_free(&C);
        return rc;
    }
    if (C.zero) {
        for (uint64_t e = 0; e < nseg; ++e) {
            vd[e] = 0.0;
            ix[e] = lo + e * seg;
        }
        ctx_free(&C);
        return 0;
    }
    int T = threads > 0 ? threads : orc_default_threads();
    if (T > BLK_MAX_THREADS)
        T = BLK_MAX_THREADS;
    if ((uint64_t)T > nseg)
        T = (int)nseg;
    seg_job jobs[BLK_MAX_THREADS];
    uint64_t next = 0;
    for (int t = 0; t < T; ++t) {
        jobs[t].C = &C;
        jobs[t].lo = lo;
        jobs[t].seg = seg;
        jobs[t].nseg = nseg;
        jobs[t].next = &next;
        jobs[t].vd = vd;
        jobs[t].vi = vi;
        jobs[t].ix = ix;
        jobs[t].err = 0;
    }
    pthread_t tid[BLK_MAX_THREADS];
    for (int t = 1; t < T; ++t)
        pthread_create(&tid[t], NULL, seg_worker, &jobs[t]);
    seg_worker(&jobs[0]);
    for (int t = 1; t < T; ++t)
        pthread_join(tid[t], NULL);
    for (int t = 0; t < T; ++t)
        if (jobs[t].err)
            rc = jobs[t].err;
    ctx_free(&C);
    return rc;
}

int orc_segmin_blocked_f64(const double *Q, int n, uint64_t lo, uint64_t seg, uint64_t nseg,
                           int threads, double *vals, uint64_t *idx)
{
    return blocked_segmin(Q, NULL, n, lo, seg, nseg, threads, vals, NULL, idx);
}

int orc_segmin_blocked_i64(const int64_t *Q, int n, uint64_t lo, uint64_t seg, uint64_t nseg,
                           int threads, int64_t *vals, uint64_t *idx)
{
    return blocked_segmin(NULL, Q, n, lo, seg, nseg, threads, NULL, vals, idx);
}
