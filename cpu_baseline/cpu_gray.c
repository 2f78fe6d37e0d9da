/*
 * cpu_gray.c -- the paper's CPU design, written fresh, as a timing baseline.
 *
 * NOT a parity reference and not part of the GPU path: only bench.py's CPU
 * baseline leg loads it, to time the method as the paper runs it, on the
 * host cores of the machine that also holds the GPU.
 *
 * Algorithm 1 with the parallel split of Section 3.1:
 *   - the top m variables are fixed per work item (a prefix p), the other
 *     n_s = n - m are walked in reflected Gray order from x_suffix = 0, so
 *     step t flips variable l = CTZ(t) (Section 2.2);
 *   - each flip recomputes the delta of Eq. 2 from the row of Q through l
 *     and the current x (O(n) per state, the paper's update): with the
 *     symmetrised row S_lj = Q_lj + Q_jl (j != l) the delta is
 *     Q_ll + sum_j S_lj x_j, signed by the flip direction;
 *   - prefixes are handed to threads from a shared counter and the
 *     per-thread minima are combined by a minimum (the paper's combine).
 * FP64 throughout.  The walk value drifts by rounding, so the reported
 * minimum is approximate; ties go to the lower natural index among equal
 * walk values.  Threads: POSIX threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define CG_MAX_N 62
#define CG_MAX_THREADS 256

typedef struct {
    int n, m;
    const double *S;   /* n x n symmetrised off-diagonal, zero diagonal */
    const double *lin; /* Q_ii */
    const uint64_t *prefixes;
    uint64_t count;
    uint64_t *next;
    double best;
    uint64_t arg;
    int has;
} cg_job;

static double value_of(const cg_job *J, const double *x)
{
    double v = 0.0;
    for (int i = 0; i < J->n; ++i) {
        if (x[i] == 0.0)
            continue;
        double row = J->lin[i];
        for (int j = i + 1; j < J->n; ++j)
            row += J->S[(size_t)i * J->n + j] * x[j];
        v += row;
    }
    return v;
}

static void *cg_worker(void *arg)
{
    cg_job *J = (cg_job *)arg;
    const int n = J->n, ns = n - J->m;
    double x[CG_MAX_N];
    for (;;) {
        const uint64_t e = __atomic_fetch_add(J->next, 1, __ATOMIC_RELAXED);
        if (e >= J->count)
            break;
        const uint64_t p = J->prefixes[e];
        for (int i = 0; i < n; ++i)
            x[i] = (i >= ns && ((p >> (i - ns)) & 1)) ? 1.0 : 0.0;
        uint64_t idx = p << ns;
        double v = value_of(J, x);
        if (!J->has || v < J->best || (v == J->best && idx < J->arg)) {
            J->best = v;
            J->arg = idx;
            J->has = 1;
        }
        const uint64_t steps = (uint64_t)1 << ns;
        for (uint64_t t = 1; t < steps; ++t) {
            const int l = __builtin_ctzll(t);
            x[l] = 1.0 - x[l];
            const double *row = J->S + (size_t)l * n;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int j = 0;
            for (; j + 4 <= n; j += 4) {
                a0 += row[j] * x[j];
                a1 += row[j + 1] * x[j + 1];
                a2 += row[j + 2] * x[j + 2];
                a3 += row[j + 3] * x[j + 3];
            }
            for (; j < n; ++j)
                a0 += row[j] * x[j];
            const double delta = J->lin[l] + ((a0 + a1) + (a2 + a3));
            v += (x[l] != 0.0) ? delta : -delta;
            idx ^= (uint64_t)1 << l;
            if (v < J->best || (v == J->best && idx < J->arg)) {
                J->best = v;
                J->arg = idx;
            }
        }
    }
    return NULL;
}

/* Walk the listed prefixes (top m variables) of the n-variable problem Q
 * (dense row-major FP64) with `threads` threads (0 = all cores).  Writes the
 * smallest walk value and its natural index; returns the thread count used,
 * or < 0 for bad arguments. */
int cg_walk_prefixes(const double *Q, int n, int m, const uint64_t *prefixes, uint64_t count,
                     int threads, double *best, uint64_t *argmin)
{
    if (!Q || !prefixes || n < 2 || n > CG_MAX_N || m < 0 || m >= n || count == 0)
        return -1;
    double *S = (double *)calloc((size_t)n * n, sizeof(double));
    double *lin = (double *)malloc((size_t)n * sizeof(double));
    if (!S || !lin) {
        free(S);
        free(lin);
        return -2;
    }
    for (int i = 0; i < n; ++i) {
        lin[i] = Q[(size_t)i * n + i];
        for (int j = 0; j < n; ++j)
            if (j != i)
                S[(size_t)i * n + j] = Q[(size_t)i * n + j] + Q[(size_t)j * n + i];
    }
    long nc = sysconf(_SC_NPROCESSORS_ONLN);
    int T = threads > 0 ? threads : (int)(nc > 0 ? nc : 1);
    if (T > CG_MAX_THREADS)
        T = CG_MAX_THREADS;
    if ((uint64_t)T > count)
        T = (int)count;
    cg_job jobs[CG_MAX_THREADS];
    uint64_t next = 0;
    for (int t = 0; t < T; ++t) {
        memset(&jobs[t], 0, sizeof(cg_job));
        jobs[t].n = n;
        jobs[t].m = m;
        jobs[t].S = S;
        jobs[t].lin = lin;
        jobs[t].prefixes = prefixes;
        jobs[t].count = count;
        jobs[t].next = &next;
    }
    pthread_t tid[CG_MAX_THREADS];
    for (int t = 1; t < T; ++t)
        pthread_create(&tid[t], NULL, cg_worker, &jobs[t]);
    cg_worker(&jobs[0]);
    for (int t = 1; t < T; ++t)
        pthread_join(tid[t], NULL);
    int have = 0;
    for (int t = 0; t < T; ++t) {
        if (!jobs[t].has)
            continue;
        if (!have || jobs[t].best < *best || (jobs[t].best == *best && jobs[t].arg < *argmin)) {
            *best = jobs[t].best;
            *argmin = jobs[t].arg;
            have = 1;
        }
    }
    free(S);
    free(lin);
    return T;
}
