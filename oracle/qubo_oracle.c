/*
 * qubo_oracle.c -- CPU oracle for exhaustive QUBO minimisation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * GPU path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library, and it does not use Gray code.
 *
 * What it computes (arXiv 2310.19373):
 *   f_Q(x) = x^T Q x = sum_{i,j} Q_ij x_i x_j   over x in {0,1}^n      (Eq. 1)
 * For the upper-triangular Q of Eq. 1 this is sum_{i<=j} Q_ij x_i x_j; for a
 * general dense Q the lower entries are folded in, which is still x^T Q x.
 *
 * Enumeration is the naive method of Section 3: the integer idx runs over
 * 0 .. 2^n - 1 in ascending ("natural") order and x_i = bit i of idx.  The
 * minimum starts from (f(0) = 0, idx 0) -- the all-zero vector always has
 * value 0 (Section 2.1) -- and a later state replaces it only when its value
 * is strictly smaller, so among equal values the lowest index is kept.
 *
 * Canonical floating-point order (the paper fixes none; this is the reading
 * the whole project uses so that FP64 values can be compared bit for bit):
 *     acc = 0
 *     for i = 0 .. n-1 with x_i = 1:
 *         row = Q_ii
 *         for j = i+1 .. n-1 with x_j = 1:  row = row + (Q_ij + Q_ji)
 *         acc = acc + row
 * every operation an IEEE binary64 round-to-nearest add (compiled with
 * -ffp-contract=off; there are no multiplies).  Integer matrices use the
 * same order in int64, which is exact.
 *
 * Also here, all by the same natural-order enumeration:
 *   - the k smallest states by (value, idx);
 *   - the Boltzmann log-partition log Z(beta) = log sum_x exp(-beta f(x)) and
 *     the second moment E_beta[x_i x_j], in FP64 with a max shift (pass 1
 *     finds m = min f, pass 2 sums exp(-beta (f - m)) with Kahan
 *     compensation).  The paper does not define these; they are the plain
 *     definitions of the quantities.
 *
 * Threads split the index range into contiguous chunks; each chunk keeps the
 * same strict-< rule and the chunk results are combined by (value, idx), so
 * the answer does not depend on the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_MAX_THREADS 256
#define ORC_MAX_TOPK 1024

/* ------------------------------------------------------------------ */
/* single-state evaluation (Eq. 1, canonical order)                     */
/* ------------------------------------------------------------------ */

double orc_eval_f64(const double *Q, int n, uint64_t idx)
{
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!((idx >> i) & 1u))
            continue;
        double row = Q[(size_t)i * n + i];
        for (int j = i + 1; j < n; ++j) {
            if ((idx >> j) & 1u) {
                double pair = Q[(size_t)i * n + j] + Q[(size_t)j * n + i];
                row = row + pair;
            }
        }
        acc = acc + row;
    }
    return acc;
}

int64_t orc_eval_i64(const int64_t *Q, int n, uint64_t idx)
{
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
        if (!((idx >> i) & 1u))
            continue;
        int64_t row = Q[(size_t)i * n + i];
        for (int j = i + 1; j < n; ++j)
            if ((idx >> j) & 1u)
                row += Q[(size_t)i * n + j] + Q[(size_t)j * n + i];
        acc += row;
    }
    return acc;
}

void orc_eval_many_f64(const double *Q, int n, const uint64_t *idx, int64_t count, double *out)
{
    for (int64_t c = 0; c < count; ++c)
        out[c] = orc_eval_f64(Q, n, idx[c]);
}

void orc_eval_many_i64(const int64_t *Q, int n, const uint64_t *idx, int64_t count, int64_t *out)
{
    for (int64_t c = 0; c < count; ++c)
        out[c] = orc_eval_i64(Q, n, idx[c]);
}

/* ------------------------------------------------------------------ */
/* thread helpers                                                       */
/* ------------------------------------------------------------------ */

int orc_default_threads(void)
{
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1)
        c = 1;
    if (c > ORC_MAX_THREADS)
        c = ORC_MAX_THREADS;
    return (int)c;
}

static int clamp_threads(int threads, uint64_t work)
{
    if (threads <= 0)
        threads = orc_default_threads();
    if (threads > ORC_MAX_THREADS)
        threads = ORC_MAX_THREADS;
    if ((uint64_t)threads > work)
        threads = work ? (int)work : 1;
    return threads;
}

/* chunk c of T over [lo, hi): contiguous, ascending */
static void chunk_range(uint64_t lo, uint64_t hi, int c, int T, uint64_t *a, uint64_t *b)
{
    uint64_t len = hi - lo;
    uint64_t q = len / (uint64_t)T, r = len % (uint64_t)T;
    uint64_t start = lo + q * (uint64_t)c + ((uint64_t)c < r ? (uint64_t)c : r);
    uint64_t size = q + ((uint64_t)c < r ? 1 : 0);
    *a = start;
    *b = start + size;
}

/* ------------------------------------------------------------------ */
/* minimum over an index range                                          */
/* ------------------------------------------------------------------ */

typedef struct {
    const double *Qd;
    const int64_t *Qi;
    int n;
    uint64_t lo, hi;
    double vmin_d;
    int64_t vmin_i;
    uint64_t argmin;
    int has;
} min_job;

static void *min_worker(void *arg)
{
    min_job *J = (min_job *)arg;
    J->has = 0;
    for (uint64_t idx = J->lo; idx < J->hi; ++idx) {
        if (J->Qd) {
            double v = orc_eval_f64(J->Qd, J->n, idx);
            if (!J->has || v < J->vmin_d) {
                J->vmin_d = v;
                J->argmin = idx;
                J->has = 1;
            }
        } else {
            int64_t v = orc_eval_i64(J->Qi, J->n, idx);
            if (!J->has || v < J->vmin_i) {
                J->vmin_i = v;
                J->argmin = idx;
                J->has = 1;
            }
        }
    }
    return NULL;
}

static int range_min(const double *Qd, const int64_t *Qi, int n, uint64_t lo, uint64_t hi,
                     int threads, double *vd, int64_t *vi, uint64_t *argmin)
{
    if (n < 1 || n > 63 || lo >= hi || hi > (1ull << n))
        return -1;
    int T = clamp_threads(threads, hi - lo);
    min_job jobs[ORC_MAX_THREADS];
    pthread_t tid[ORC_MAX_THREADS];
    for (int c = 0; c < T; ++c) {
        memset(&jobs[c], 0, sizeof(min_job));
        jobs[c].Qd = Qd;
        jobs[c].Qi = Qi;
        jobs[c].n = n;
        chunk_range(lo, hi, c, T, &jobs[c].lo, &jobs[c].hi);
    }
    for (int c = 1; c < T; ++c)
        pthread_create(&tid[c], NULL, min_worker, &jobs[c]);
    min_worker(&jobs[0]);
    for (int c = 1; c < T; ++c)
        pthread_join(tid[c], NULL);
    /* chunks are ascending in idx: strict < across them keeps the lowest idx */
    int have = 0;
    for (int c = 0; c < T; ++c) {
        if (!jobs[c].has)
            continue;
        if (Qd) {
            if (!have || jobs[c].vmin_d < *vd) {
                *vd = jobs[c].vmin_d;
                *argmin = jobs[c].argmin;
                have = 1;
            }
        } else {
            if (!have || jobs[c].vmin_i < *vi) {
                *vi = jobs[c].vmin_i;
                *argmin = jobs[c].argmin;
                have = 1;
            }
        }
    }
    return have ? 0 : -1;
}

/* Minimum of f over idx in [lo, hi), natural order, ties -> lowest idx.
 * With lo = 0 the first state is x = 0 with f = 0, the paper's start. */
int orc_min_f64(const double *Q, int n, uint64_t lo, uint64_t hi, int threads,
                double *vmin, uint64_t *argmin)
{
    int64_t dummy;
    return range_min(Q, NULL, n, lo, hi, threads, vmin, &dummy, argmin);
}

int orc_min_i64(const int64_t *Q, int n, uint64_t lo, uint64_t hi, int threads,
                int64_t *vmin, uint64_t *argmin)
{
    double dummy;
    return range_min(NULL, Q, n, lo, hi, threads, &dummy, vmin, argmin);
}

/* ------------------------------------------------------------------ */
/* k smallest by (value, idx)                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    const double *Qd;
    const int64_t *Qi;
    int n, k;
    uint64_t lo, hi;
    int count;
    double vd[ORC_MAX_TOPK];
    int64_t vi[ORC_MAX_TOPK];
    uint64_t ix[ORC_MAX_TOPK];
} topk_job;

/* (a, ia) < (b, ib) lexicographically */
static int lex_less_d(double a, uint64_t ia, double b, uint64_t ib)
{
    return a < b || (a == b && ia < ib);
}
static int lex_less_i(int64_t a, uint64_t ia, int64_t b, uint64_t ib)
{
    return a < b || (a == b && ia < ib);
}

static void topk_insert(topk_job *J, double vd, int64_t vi, uint64_t ix)
{
    int k = J->k;
    int pos = J->count;
    if (pos == k) {
        int worse = J->Qd ? lex_less_d(vd, ix, J->vd[k - 1], J->ix[k - 1])
                          : lex_less_i(vi, ix, J->vi[k - 1], J->ix[k - 1]);
        if (!worse)
            return;
        pos = k - 1;
    } else {
        J->count++;
    }
    while (pos > 0) {
        int less = J->Qd ? lex_less_d(vd, ix, J->vd[pos - 1], J->ix[pos - 1])
                         : lex_less_i(vi, ix, J->vi[pos - 1], J->ix[pos - 1]);
        if (!less)
            break;
        J->vd[pos] = J->vd[pos - 1];
        J->vi[pos] = J->vi[pos - 1];
        J->ix[pos] = J->ix[pos - 1];
        --pos;
    }
    J->vd[pos] = vd;
    J->vi[pos] = vi;
    J->ix[pos] = ix;
}

static void *topk_worker(void *arg)
{
    topk_job *J = (topk_job *)arg;
    for (uint64_t idx = J->lo; idx < J->hi; ++idx) {
        if (J->Qd)
            topk_insert(J, orc_eval_f64(J->Qd, J->n, idx), 0, idx);
        else
            topk_insert(J, 0.0, orc_eval_i64(J->Qi, J->n, idx), idx);
    }
    return NULL;
}

static int range_topk(const double *Qd, const int64_t *Qi, int n, uint64_t lo, uint64_t hi, int k,
                      int threads, double *vd, int64_t *vi, uint64_t *ix)
{
    if (n < 1 || n > 63 || lo >= hi || hi > (1ull << n) || k < 1 || k > ORC_MAX_TOPK)
        return -1;
    int T = clamp_threads(threads, hi - lo);
    topk_job *jobs = (topk_job *)calloc((size_t)T + 1, sizeof(topk_job));
    if (!jobs)
        return -2;
    pthread_t tid[ORC_MAX_THREADS];
    for (int c = 0; c < T; ++c) {
        jobs[c].Qd = Qd;
        jobs[c].Qi = Qi;
        jobs[c].n = n;
        jobs[c].k = k;
        chunk_range(lo, hi, c, T, &jobs[c].lo, &jobs[c].hi);
    }
    for (int c = 1; c < T; ++c)
        pthread_create(&tid[c], NULL, topk_worker, &jobs[c]);
    topk_worker(&jobs[0]);
    for (int c = 1; c < T; ++c)
        pthread_join(tid[c], NULL);
    topk_job *all = &jobs[T];
    all->Qd = Qd;
    all->Qi = Qi;
    all->k = k;
    for (int c = 0; c < T; ++c)
        for (int e = 0; e < jobs[c].count; ++e)
            topk_insert(all, jobs[c].vd[e], jobs[c].vi[e], jobs[c].ix[e]);
    int cnt = all->count;
    for (int e = 0; e < cnt; ++e) {
        if (vd)
            vd[e] = all->vd[e];
        if (vi)
            vi[e] = all->vi[e];
        ix[e] = all->ix[e];
    }
    free(jobs);
    return cnt;
}

/* Returns the number of entries written (min(k, hi - lo)), or < 0 on error. */
int orc_topk_f64(const double *Q, int n, uint64_t lo, uint64_t hi, int k, int threads,
                 double *vals, uint64_t *idx)
{
    return range_topk(Q, NULL, n, lo, hi, k, threads, vals, NULL, idx);
}

int orc_topk_i64(const int64_t *Q, int n, uint64_t lo, uint64_t hi, int k, int threads,
                 int64_t *vals, uint64_t *idx)
{
    return range_topk(NULL, Q, n, lo, hi, k, threads, NULL, vals, idx);
}

/* ------------------------------------------------------------------ */
/* Boltzmann log-partition and second moment                            */
/* ------------------------------------------------------------------ */

typedef struct {
    double s, c; /* Kahan sum and compensation */
} kahan;

static inline void kahan_add(kahan *k, double x)
{
    double y = x - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

typedef struct {
    const double *Q;
    int n;
    uint64_t lo, hi;
    double beta, m;
    int want_moment;
    kahan Z;
    kahan *S; /* n*n, upper triangle used */
} logz_job;

static void *logz_worker(void *arg)
{
    logz_job *J = (logz_job *)arg;
    int n = J->n;
    for (uint64_t idx = J->lo; idx < J->hi; ++idx) {
        double f = orc_eval_f64(J->Q, n, idx);
        double w = exp(-J->beta * (f - J->m));
        kahan_add(&J->Z, w);
        if (J->want_moment) {
            for (int i = 0; i < n; ++i) {
                if (!((idx >> i) & 1u))
                    continue;
                for (int j = i; j < n; ++j)
                    if ((idx >> j) & 1u)
                        kahan_add(&J->S[(size_t)i * n + j], w);
            }
        }
    }
    return NULL;
}

/* For each beta[b]: logz[b] = log sum_x exp(-beta f(x)), and, when
 * moment != NULL, moment[b*n*n + i*n + j] = E_beta[x_i x_j] (symmetric).
 * Also returns the exact FP64 minimum (natural order, lowest idx). */
int orc_logz_f64(const double *Q, int n, const double *beta, int nbeta, int threads,
                 double *logz, double *moment, double *vmin, uint64_t *argmin)
{
    if (n < 1 || n > 40 || nbeta < 1)
        return -1;
    uint64_t N = 1ull << n;
    double m;
    uint64_t am;
    if (orc_min_f64(Q, n, 0, N, threads, &m, &am) != 0)
        return -1;
    if (vmin)
        *vmin = m;
    if (argmin)
        *argmin = am;
    int T = clamp_threads(threads, N);
    logz_job *jobs = (logz_job *)calloc((size_t)T, sizeof(logz_job));
    if (!jobs)
        return -2;
    pthread_t tid[ORC_MAX_THREADS];
    for (int b = 0; b < nbeta; ++b) {
        for (int c = 0; c < T; ++c) {
            jobs[c].Q = Q;
            jobs[c].n = n;
            jobs[c].beta = beta[b];
            jobs[c].m = m;
            jobs[c].want_moment = moment != NULL;
            jobs[c].Z.s = jobs[c].Z.c = 0.0;
            jobs[c].S = moment ? (kahan *)calloc((size_t)n * n, sizeof(kahan)) : NULL;
            chunk_range(0, N, c, T, &jobs[c].lo, &jobs[c].hi);
        }
        for (int c = 1; c < T; ++c)
            pthread_create(&tid[c], NULL, logz_worker, &jobs[c]);
        logz_worker(&jobs[0]);
        for (int c = 1; c < T; ++c)
            pthread_join(tid[c], NULL);
        kahan Z = {0.0, 0.0};
        for (int c = 0; c < T; ++c)
            kahan_add(&Z, jobs[c].Z.s);
        logz[b] = -beta[b] * m + log(Z.s);
        if (moment) {
            double *E = moment + (size_t)b * n * n;
            for (int i = 0; i < n; ++i)
                for (int j = i; j < n; ++j) {
                    kahan S = {0.0, 0.0};
                    for (int c = 0; c < T; ++c)
                        kahan_add(&S, jobs[c].S[(size_t)i * n + j].s);
                    E[(size_t)i * n + j] = S.s / Z.s;
                    E[(size_t)j * n + i] = S.s / Z.s;
                }
            for (int c = 0; c < T; ++c)
                free(jobs[c].S);
        }
    }
    free(jobs);
    return 0;
}
