/*
 * qbf.h -- C ABI of libqubobf, exhaustive QUBO minimisation on one GB300.
 *
 * Method: arXiv 2310.19373, "Faster QUBO Brute-Force Solving using Gray Code".
 *   f_Q(x) = x^T Q x over x in {0,1}^n                              (Eq. 1)
 *   all 2^n vectors are visited in reflected Gray-code order, so step t
 *   flips bit CTZ(t) (Section 2.2) and the objective moves by the one-bit
 *   delta of Eq. 2 instead of being re-evaluated;                    (Alg. 1)
 *   the top bits of x are fixed per worker and the sub-walks are combined
 *   by a minimum (Section 3.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Q is dense, row-major, n x n.  f(x) = sum_{i,j} Q_ij x_i x_j uses every
 *    entry, which is Eq. 1 when Q is upper triangular.
 *  - A state is reported by its natural index idx(x) = sum_i x_i 2^i
 *    (x_i = bit i, as in the naive method of Section 3).
 *  - Ties go to the lowest natural index.  (Algorithm 1 keeps the first
 *    state met in Gray order; this library reports the unique answer that
 *    does not depend on the enumeration order.)
 *  - Every entry point returns an int status (QBF_OK = 0) and never aborts.
 *    On error, qbf_last_error_string() describes the failure (thread-local).
 *  - Pointers named *_dev must be device memory of the current device;
 *    pointers named *_host are host memory.  The caller owns all buffers;
 *    the library keeps no pointer after a call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls that fill a host struct wait
 *    for that stream before returning.
 *  - The library keeps a per-device scratch pool (grow-only, reused across
 *    calls, freed by qbf_release).  Calls are serialised by an internal lock.
 *  - qbf_solve of a device matrix with options and a pool seen before (the
 *    second and later identical calls) replays a CUDA graph of the solve
 *    captured at its second sighting; the kernels read Q when the graph runs,
 *    so new contents in the same buffer are solved afresh.  Eight such solves
 *    are remembered per device; setting the environment variable
 *    QBF_NO_SOLVE_GRAPHS=1 runs every solve directly.  Solves with
 *    opt->timing set, or with Q in host memory, always run directly.
 */
#ifndef QBF_H
#define QBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QBF_MAX_N 48    /* largest n for qbf_solve                        */
#define QBF_MAX_TOPK 64 /* largest top_k                                  */
#define QBF_BATCH_MAX_N 34          /* largest n of one batched instance  */
#define QBF_BATCH_MAX_COUNT 65536   /* most instances per batched call    */

/* element type of Q */
typedef enum {
    QBF_F64 = 0, /* double                                                 */
    QBF_F32 = 1, /* float                                                  */
    QBF_I32 = 2, /* int32_t                                                */
    QBF_I16 = 3  /* int16_t                                                */
} qbf_dtype;

/* status codes */
enum {
    QBF_OK = 0,
    QBF_EINVAL = 1,     /* bad argument (null pointer, n out of range ...)  */
    QBF_ENONFINITE = 2, /* Q holds NaN or Inf                               */
    QBF_EDTYPE = 3,     /* unknown dtype                                    */
    QBF_ECUDA = 4,      /* a CUDA call failed                               */
    QBF_EOVERFLOW = 5,  /* more candidate states than the scratch can hold  */
    QBF_ECANCELED = 6,  /* qbf_cancel() stopped the call; no result       */
    QBF_ENOTIMPL = 7,
    QBF_ERANGE = 8      /* integer Q whose sum |Q_ij| does not fit in int32 */
};

/* walk kernels */
enum {
    QBF_VARIANT_AUTO = 0,  /* n >= 24: SPLIT_DEFER, repeated on SPLIT if its
                              2^23 image bound does not hold (integer Q) or
                              its wider certification window overflows the
                              candidate buffer (float Q); n < 24: SPLIT     */
    QBF_VARIANT_FIELD = 1, /* the plain Gray walk: per-thread field vector g
                              in registers, n_s + 1 adds per state (suffix
                              n_s <= 20); a reference form, not fast        */
    QBF_VARIANT_SPLIT = 2, /* field split into lane-invariant + lane parts  */
    QBF_VARIANT_TC = 3,    /* blocked form: cross term on tcgen05 tensor
                              cores, tiles of 2^14 states (15 <= n <= 42)  */
    QBF_VARIANT_SPLIT_F32 = 4, /* split walk in packed FP32 on exact integers
                                  (image < 2^23), two prefixes per thread    */
    QBF_VARIANT_SPLIT_MIX = 5, /* split walk on both pipes: per thread three
                                  packed-FP32 pairs and two int32 prefixes
                                  (image < 2^23, n >= 4)                     */
    QBF_VARIANT_NAIVE = 6,     /* no Gray code: every state evaluated from
                                  scratch in natural order, O(n^2) per state;
                                  a reference form, not fast                 */
    QBF_VARIANT_SPLIT_DEFER = 7 /* split walk, eight prefixes per thread as
                                   four packed-FP32 pairs, the static in-block
                                   correction added once per step after the
                                   minimum over the eight (image < 2^23,
                                   n >= 4)                                   */
};

typedef struct {
    int top_k;          /* number of best states to return, 1..64 (0 -> 1)  */
    int variant;        /* QBF_VARIANT_*                                     */
    int prefix_bits;    /* bits fixed per GPU thread (Section 3.1's m);
                           -1 = chosen by the planner.  A thread walks at
                           most 2^20 blocks of 2^6 states: n - prefix_bits
                           <= 26 (29 for SPLIT_MIX / SPLIT_DEFER, whose
                           three group bits are not walked), else
                           QBF_EINVAL                                        */
    int fix_bits;       /* restrict the search to states whose top fix_bits
                           variables x_{n-fix_bits..n-1} equal fix_value;
                           0 = whole space                                   */
    uint64_t fix_value;
    int timing;         /* 1: time the main walk kernel with CUDA events on
                           `stream` and report it in qbf_result.walk_seconds */
    int batch_suffix_bits; /* qbf_solve_batched: suffix bits walked per lane,
                              6..18; 0 = the value qbf_tune chose for the
                              instance's n (cache), else 18                 */
    int reserved[6];
} qbf_options;

typedef struct {
    double min_value;   /* min f; FP64 canonical sum for float Q (rows i
                           ascending, row = Q_ii + sum_{j>i} (Q_ij + Q_ji)
                           in ascending j, rows added in order), exact for
                           integer Q                                        */
    uint64_t argmin;    /* lowest natural index attaining min_value         */
    int top_k;          /* entries filled in topk_* (<= requested)          */
    double topk_value[QBF_MAX_TOPK];   /* ascending by (value, index)       */
    uint64_t topk_index[QBF_MAX_TOPK];
    int scale_bits;     /* sigma: the walk runs on round(Q * 2^sigma)       */
    double error_bound; /* half-width of the certification window, in units
                           of f (0 for integer Q)                          */
    uint64_t n_candidates; /* states rescored in FP64 / int64               */
    int prefix_bits;    /* k actually used                                  */
    int suffix_bits;    /* n - k                                            */
    int variant;        /* walk kernel actually used                        */
    int walk_launches;  /* launches of the MIN walk kernel in this call     */
    double walk_seconds;/* device time of the main walk kernel(s) when
                           opt->timing was set, else 0                      */
    int kernel_launches;/* kernels this call launched                       */
    int reserved[3];
} qbf_result;

/* Fill *opt with defaults (top_k = 1, auto variant, auto prefix width). */
void qbf_default_options(qbf_options *opt);

/*
 * qbf_solve -- minimum, lowest-index argmin and optional top-k of x^T Q x.
 *
 * Q_dev : device pointer, n*n elements of `dtype`, row-major.  Read only.
 * n     : 1 .. QBF_MAX_N.
 * opt   : NULL for defaults.
 * out   : host struct, filled when the call returns QBF_OK.
 *
 * Float Q is walked exactly on a fixed-point image round(Q * 2^sigma) in
 * int32; every state whose fixed-point value lies within the rounding bound
 * of the best is rescored with the FP64 canonical sum, so the reported min
 * and argmin are those of the FP64 canonical objective.  Integer Q is walked
 * exactly (QBF_ERANGE when sum |Q_ij| >= 2^31).
 * A walk over more than 2^41 states (n > 41 without fix_bits) runs as several
 * MIN launches over consecutive prefix slices of at most 2^41 states, about
 * 0.1 s each, so no kernel runs for seconds; out->walk_launches reports how
 * many (the tensor-core form always uses one).
 * Errors: QBF_EINVAL, QBF_EDTYPE, QBF_ENONFINITE, QBF_ERANGE, QBF_EOVERFLOW
 * (the certification window holds more than 2^22 states, e.g. massive exact
 * ties with top_k > 1), QBF_ECANCELED (qbf_cancel), QBF_ECUDA.
 */
int qbf_solve(const void *Q_dev, int n, int dtype, const qbf_options *opt, qbf_result *out,
              void *stream);

/* Same as qbf_solve with Q in host memory: copies Q to the device on
 * `stream` first (the end-to-end path). */
int qbf_solve_host(const void *Q_host, int n, int dtype, const qbf_options *opt,
                   qbf_result *out, void *stream);

/*
 * Chunked, resumable enumeration (n up to QBF_MAX_N).
 *
 * The top `chunk_bits` variables index 2^chunk_bits chunks; each chunk is one
 * certified qbf_solve with fix_bits = chunk_bits, fix_value = the chunk
 * (Section 3.1's prefix split, one level up), and the chunks' top-k lists
 * merge into the global top-k by (value, index).  A qbf_checkpoint is plain
 * data (no pointers; 1104 bytes, fixed layout): a caller may copy it to a file
 * after any step and resume in another process, or run shards of the chunk
 * sequence on different GPUs or hosts and merge the finished checkpoints.
 * The paper has no counterpart; it follows from the disjoint prefix ranges.
 */
#define QBF_CKPT_VERSION 1u
typedef struct {
    uint32_t version;       /* QBF_CKPT_VERSION                                 */
    int32_t n, dtype;       /* the problem                                      */
    int32_t top_k;          /* length of the merged list, 1..64                 */
    int32_t chunk_bits;     /* chunks = values of the top chunk_bits variables  */
    int32_t shard, nshards; /* this sequence: chunks shard, shard + nshards, ...*/
    int32_t count;          /* valid entries of best_value / best_index         */
    uint64_t q_hash;        /* FNV-1a of Q's bytes: steps refuse another Q      */
    uint64_t next;          /* next position in this shard's chunk sequence     */
    uint64_t chunks_done;   /* chunks walked (summed over merged shards)        */
    uint64_t done_mask;     /* bit r: shard r has walked all of its chunks      */
    uint64_t n_candidates;  /* certification candidates, summed over chunks     */
    double error_bound;     /* largest per-chunk bound (0 for integer Q)        */
    double best_value[QBF_MAX_TOPK];    /* ascending by (value, index)          */
    uint64_t best_index[QBF_MAX_TOPK];
} qbf_checkpoint;

/* Start shard `shard` of `nshards` (1..64): 1 <= chunk_bits <= min(n - 1, 24),
 * top_k 1..64.  Q_dev: device pointer, as qbf_solve (read to fingerprint it;
 * synchronises `stream`). */
int qbf_chunked_init(qbf_checkpoint *ck, const void *Q_dev, int n, int dtype, int top_k,
                     int chunk_bits, int shard, int nshards, void *stream);

/* Walk up to max_chunks further chunks of the shard (each a qbf_solve with
 * `opt`, whose top_k, fix_bits and fix_value are replaced).  QBF_EINVAL if Q
 * does not match the checkpoint's fingerprint.  When the shard's sequence
 * ends, its bit is set in done_mask; further steps do nothing. */
int qbf_chunked_step(qbf_checkpoint *ck, const void *Q_dev, const qbf_options *opt,
                     uint64_t max_chunks, void *stream);

/* Host only, no GPU: fold the finished shards of `other` into `into`.  Both
 * must be finished (done_mask != 0), describe the same problem and split,
 * and cover disjoint shards; QBF_EINVAL otherwise. */
int qbf_chunked_merge(qbf_checkpoint *into, const qbf_checkpoint *other);

/* Host only, no GPU: the result once every shard is in done_mask (min,
 * argmin, top-k, error_bound, n_candidates; the other fields 0).  QBF_EINVAL
 * while chunks are missing. */
int qbf_chunked_result(const qbf_checkpoint *ck, qbf_result *out);

/*
 * qbf_solve_ising -- ground state of an Ising energy by the same solver.
 *
 * The introduction (Section 1) motivates QUBO by its equivalence with the
 * Ising model.  For spins s_i in {-1, +1} this call minimises
 *     E(s) = s^T J s + h^T s = sum_ij J_ij s_i s_j + sum_i h_i s_i
 * (every entry of J counts; the diagonal adds the constant sum_i J_ii).  With
 * s = 2x - 1, E(s) = x^T Q x + c for Q = 4J + diag(2h - 2R - 2C) (R, C: row
 * and column sums of J) and c = sum_ij J_ij - sum_i h_i; the call builds Q on
 * the device and runs qbf_solve on it.
 *
 * J_dev : device pointer, n*n elements of `dtype`, row-major.  Read only.
 * h_dev : device pointer, n elements of `dtype`.  Read only.
 * out   : as qbf_solve, with values E(s) (= f_Q + c) and indices whose bit i
 *         is 1 iff s_i = +1; ties go to the lowest such index.  Float J, h:
 *         Q is formed in FP64 (its diagonal with one rounding per term) and
 *         c is added in FP64, so the values carry those roundings on top of
 *         the certified f_Q.  Integer J, h: exact; QBF_ERANGE if an entry of
 *         Q leaves int32.
 * Uses a fixed device buffer of the library (no allocation beyond
 * qbf_solve's); synchronises `stream` before returning.
 */
int qbf_solve_ising(const void *J_dev, const void *h_dev, int n, int dtype,
                    const qbf_options *opt, qbf_result *out, void *stream);

/*
 * qubo_bf_solve -- the one-call form: minimum, lowest-index argmin and
 * optionally the top-k of x^T Q x (Eq. 1) for Q in HOST memory, n*n elements
 * of `dtype`, row-major.  Synchronous on the default stream, default options
 * (AUTO variant).  min_value and argmin receive the minimum and its natural
 * index (bit i = x_i).  top_k may be 0 (then topk_value / topk_index may be
 * NULL); otherwise up to 64 best states are written to the caller's arrays of
 * that length, and the number written is returned through *count (may be NULL).
 * Same status codes as qbf_solve.
 */
int qubo_bf_solve(const void *Q_host, int n, int dtype, double *min_value, uint64_t *argmin,
                  int top_k, double *topk_value, uint64_t *topk_index, int *count);

/*
 * qbf_solve_batched -- minimum and lowest-index argmin of many independent QUBOs.
 *
 * Section 3.1's prefix split applied across instances: the prefixes of all
 * instances form one queue of equal-cost work items that a single persistent
 * kernel drains; the whole pipeline (prepare, walk, certification, rescoring,
 * per-instance selection) is replayed as one CUDA graph, rebuilt only when the
 * batch layout changes.
 *
 * Q_dev     : host array of `count` device pointers; Q_dev[i] holds n[i]*n[i]
 *             elements of dtype[i], row-major.
 * n, dtype  : host arrays of `count` entries; 1 <= n[i] <= QBF_BATCH_MAX_N.
 * opt       : NULL or top_k = 1, fix_bits = 0; batch_suffix_bits selects the
 *             per-lane suffix width (0 = the qbf_tune choice for each
 *             instance's n, else 18; see qbf_tune and qbf_tune_batched);
 *             variant AUTO / SPLIT_DEFER (instances whose image fits 2^23
 *             walk in the deferred-correction form, the rest in int32; AUTO
 *             repeats the batch on the int32 walk after QBF_EOVERFLOW),
 *             SPLIT_MIX (the same with the two-pipe form), SPLIT (int32
 *             throughout); other variants give QBF_ENOTIMPL.
 * min_value, argmin : host arrays of `count` entries (same meaning as
 *             qbf_result.min_value / argmin).
 * 1 <= count <= QBF_BATCH_MAX_COUNT.  Errors name the first failing instance.
 * Certification is per instance, as in qbf_solve; QBF_EOVERFLOW if the whole
 * batch has more than 2^20 states inside its windows.
 */
int qbf_solve_batched(const void *const *Q_dev, const int *n, const int *dtype, int count,
                      const qbf_options *opt, double *min_value, uint64_t *argmin, void *stream);

/*
 * qbf_solve_batched_info -- qbf_solve_batched with per-instance certification
 * details.
 *
 * Same arguments, work and status codes as qbf_solve_batched (the result
 * struct of the paper's listing, per instance: the minimum and its vector,
 * Appendix A), plus `info`: NULL or a host array of `count` entries.  Entry i
 * describes how instance i was certified:
 */
typedef struct {
    double error_bound;    /* half-width of the certification window in units
                              of f (0 for integer Q), as qbf_result         */
    uint64_t n_candidates; /* states rescored for this instance            */
    int scale_bits;        /* sigma of the instance's fixed-point image     */
    int suffix_bits;       /* suffix bits walked per lane (n - prefix bits)  */
    int prefix_bits;       /* prefix bits (2^prefix_bits prefixes)          */
    int walk;              /* MIN walk the instance took: QBF_VARIANT_SPLIT_DEFER,
                              QBF_VARIANT_SPLIT_MIX or QBF_VARIANT_SPLIT    */
} qbf_batch_info;
/* Per-instance top-k is not offered (top_k > 1 gives QBF_ENOTIMPL): a
 * batched caller wanting the k best of one instance calls qbf_solve on it. */
int qbf_solve_batched_info(const void *const *Q_dev, const int *n, const int *dtype, int count,
                           const qbf_options *opt, double *min_value, uint64_t *argmin,
                           qbf_batch_info *info, void *stream);

/*
 * qbf_solve_batched_item_minima -- the batched MIN walk's per-item minima of
 * one instance, for checking the walk against a reference at its own depth.
 *
 * Runs the same work as qbf_solve_batched_info (same arguments; `info` may be
 * NULL) and then copies out what the MIN pass wrote for instance `inst`
 * (0 <= inst < count).  The batch walks Section 3.1's split: instance i has
 * 2^p prefixes, p = info[i].prefix_bits, each walked over its 2^s suffix
 * states, s = info[i].suffix_bits.  The work items are runs of 32 prefixes,
 * and item j of the instance covers the natural indices
 * [32 j 2^s, (32 j + 32) 2^s) ∩ [0, 2^n).  item_min[j] is the minimum over
 * those states of f on the walk's fixed-point image:
 *   - the diagonal is round(Q_ii 2^sigma);
 *   - each pair i < j adds round((Q_ij + Q_ji) 2^sigma);
 *   - sigma = info[inst].scale_bits, and rounding is half to even;
 *   - the value is an int32.
 * Instances with n below 11 are walked padded to n = 11 with zero rows, so
 * their items cover the padded space.
 *
 * item_min : host array of max_items entries (may be NULL if max_items = 0);
 *            the first min(max_items, count of items) are written.
 * n_items  : receives the instance's item count, ceil(2^p / 32).
 * With QBF_VARIANT_AUTO the minima are those of the pass that answered: the
 * int32 pass when the FP32 windows overflowed.  Errors as qbf_solve_batched,
 * plus QBF_EINVAL for inst out of range or a null n_items.
 */
int qbf_solve_batched_item_minima(const void *const *Q_dev, const int *n, const int *dtype,
                                  int count, const qbf_options *opt, int inst, int32_t *item_min,
                                  uint64_t max_items, uint64_t *n_items, qbf_batch_info *info,
                                  void *stream);

/*
 * qbf_tune -- autotuner of the batched solver, per n and element class.
 *
 * For every n in [n_min, n_max] (1 <= n_min <= n_max <= QBF_BATCH_MAX_N) it
 * builds synthetic batches of that n on the current device (upper-triangular
 * instances, uniform in [-1, 1] for float dtypes, integers in [-50, 50] for
 * integer dtypes; c and 2c instances, c = 2^36 / 2^n, at least 8 and at
 * most 2048) and scores each configuration by the difference of their
 * qbf_solve_batched times: the steady-state cost of c instances, as in a large
 * mixed batch, without the last partial wave of one small launch.  It searches
 * the suffix width walked per lane (the five widest the instance allows; it
 * fixes the prefix width k = n - suffix bits, Section 3.1's split) and then
 * the number of resident 128-thread CTAs per SM of the walk kernel.  It keeps
 * the default pair (18 suffix bits or the widest allowed, the most CTAs per
 * SM) unless another is faster by more than 2%, the run-to-run spread of the
 * scores.  The choices
 * take effect at once in this process for the current device, and one line
 * per n is appended to `cache_path`:
 *     qbf-tune-v1 <device name> <SM count> <class> <n> <suffix bits> <CTAs/SM> <seconds>
 * (class 0 = float, 1 = integer; spaces in the name become '_').  NULL uses the
 * default cache: the file named by the environment variable QBF_TUNE_CACHE,
 * else $HOME/.cache/qbf_tune.txt.  qbf_solve_batched reads the default cache
 * once per device on its first call (later lines win) and uses, for each
 * instance, the tuned suffix width of its n and class, and for the walk grid
 * the CTAs per SM of the n that holds the most states of the batch; an
 * explicit batch_suffix_bits in the options overrides the suffix width.
 * Allocates its synthetic batch with cudaMalloc and frees it; synchronises the
 * device.  Errors: QBF_EINVAL (range, dtype), QBF_ECUDA, and QBF_EINVAL when
 * the cache file cannot be written (the in-process choices are kept).
 */
int qbf_tune(int n_min, int n_max, int dtype, const char *cache_path);

/* The batched solver's current choices for instances of n variables and
 * `dtype` on the current device (after qbf_tune or a loaded cache): suffix
 * bits walked per lane and CTAs per SM, 0 where nothing is tuned (then the
 * defaults apply: 18 suffix bits, as many CTAs as fit). */
int qbf_tuned_params(int n, int dtype, int *suffix_bits, int *ctas_per_sm);

/*
 * qbf_tune_batched -- picks the per-lane suffix width of qbf_solve_batched.
 *
 * Times qbf_solve_batched on the given batch for every suffix width in
 * [6, 18] between lo_bits and hi_bits, keeps the fastest as this process's
 * default for the current device and returns it in *best_bits (and its time
 * in *best_seconds).  If the environment variable QBF_TUNE_CACHE names a file,
 * a line "<device name> <SM count> <bits> <seconds>" is appended to it.
 */
int qbf_tune_batched(const void *const *Q_dev, const int *n, const int *dtype, int count,
                     int lo_bits, int hi_bits, int *best_bits, double *best_seconds,
                     void *stream);

/*
 * qbf_logz -- exact Boltzmann log-partition log Z(Q, beta) = log sum_x
 * exp(-beta x^T Q x) of `batch` instances, by the same Gray-code walk.
 *
 * Q_dev   : device, batch * n * n elements of dtype, instance b at offset b*n*n.
 * n       : 2 .. QBF_BATCH_MAX_N.  batch: 1 .. 4096.  beta: host, nbeta (1..8)
 *           values, each finite and > 0.
 * logz    : host, batch * nbeta (logz[b * nbeta + j]).
 * min_value, argmin : host, batch entries; the certified minimum and lowest
 *           argmin (as qbf_solve_batched), which also fix the shift m.
 * Energies come from an exact two-limb fixed-point image of Q.  Each limb's
 * entries sum to at most 2^22 in magnitude, so both limbs walk exactly in
 * FP32.  The resolution is 2^-(sigma+L) of f, where sigma is the hi limb's
 * scale and L = 23 - ceil(log2(n(n+1)/2)), at most 16 (14 at n = 28).  The
 * weights exp(-beta (f - m)) are FP32, summed in FP32 per block,
 * Kahan-compensated per thread, and summed in FP64 across threads.
 */
int qbf_logz(const void *Q_dev, int n, int dtype, int batch, const double *beta, int nbeta,
             double *logz, double *min_value, uint64_t *argmin, void *stream);

/*
 * qbf_logz_backward -- gradient of sum_{b,j} upstream[b,j] * log Z(Q_b, beta_j).
 *
 * d log Z / d Q_ij = -beta E_beta[x_i x_j] for every entry (f uses every Q_ij).
 * upstream_dev : device, batch * nbeta doubles, or NULL for all ones.
 * grad_dev     : device, batch * n * n doubles (overwritten).
 * moment_dev   : device, batch * nbeta * n * n doubles receiving E_beta[x x^T],
 *                or NULL.
 * Re-walks the enumeration: a walk with the top ceil(n/2) variables fixed per
 * thread gives per-thread sums of w and w * x_j, a second walk on the rotated
 * variable order gives the remaining block.
 */
int qbf_logz_backward(const void *Q_dev, int n, int dtype, int batch, const double *beta,
                      int nbeta, const double *upstream_dev, double *grad_dev, double *moment_dev,
                      void *stream);

/*
 * qbf_danskin -- subgradient of min_x x^T Q x: grad[b] = upstream[b] x* x*^T
 * with x* the lowest-index argmin (argmin_host from qbf_solve_batched or
 * qbf_logz).  upstream_dev: device, batch doubles or NULL (ones);
 * grad_dev: device, batch * n * n doubles.
 */
int qbf_danskin(const uint64_t *argmin_host, int n, int batch, const double *upstream_dev,
                double *grad_dev, void *stream);

/*
 * qbf_solve_noalloc -- qbf_solve without any memory allocation by the call.
 *
 * The paper has no counterpart: this is a deployment variant of qbf_solve for
 * callers that cannot allocate GPU memory -- processes that reserve the whole
 * device up front and hand memory out only through their own pool, plug-ins
 * whose host application owns the GPU memory budget, and services that cannot
 * accept the device-wide synchronisation cudaMalloc/cudaFree can cause.  The
 * caller passes Q and the result struct; all scratch lives in one array of
 * QBF_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library holds until the process exits.  No cudaMalloc, cudaFree
 * or other allocating routine is called.
 *
 * Same arguments as qbf_solve.  The answer (min_value, argmin, the top-k list)
 * is qbf_solve's, whatever variant qbf_solve runs; this call always walks the
 * int32 image, so scale_bits, error_bound and n_candidates are those of
 * qbf_solve with variant = QBF_VARIANT_SPLIT.  opt->variant and opt->timing
 * are ignored (walk_seconds stays 0).  Limits: n <= QBF_NOALLOC_MAX_N, at most
 * 2^16 prefixes (prefix_bits <= 16) and 2^20 suffix states per thread, at
 * most 2^16 states in the certification window (else QBF_EOVERFLOW, e.g. an
 * exact top-k > 1 with massive ties, which qbf_solve's 2^22-state window
 * still takes).  Larger problems are rejected with QBF_EINVAL and a message
 * naming the limit.  The first call on a device looks up the scratch array's
 * device address (cudaGetSymbolAddress) with that device current, and, under
 * lazy module loading (the CUDA default), that lookup and the first kernel
 * launches load the library's kernels and the array onto the device, which
 * sets memory aside there; make that first call during set-up, before any
 * stream capture (CUDA_MODULE_LOADING=EAGER moves the loading to process
 * start).  Later calls set nothing aside.  All calls share the array and
 * each leaves its contents behind (every call resets what must start at zero);
 * calls whose GPU work overlaps race -- including with a concurrent qbf_solve --
 * so issue them from one thread at a time.  The call waits for `stream`.
 */
#define QBF_NOALLOC_SCRATCH_BYTES (3u << 20) /* 3 MiB per device */
#define QBF_NOALLOC_MAX_N 36
int qbf_solve_noalloc(const void *Q_dev, int n, int dtype, const qbf_options *opt,
                      qbf_result *out, void *stream);

/*
 * qbf_walk_trace -- debug walk that records every visited state.
 *
 * Runs the split walk with 2^prefix_bits threads over the whole space
 * (n <= 24) and writes, for visit slot s = p * 2^(n-k) + t (thread p, step
 * t), the natural index of the state it visits to idx_dev[s] and its
 * fixed-point objective round(Q * 2^sigma) evaluated by the walk to
 * val_dev[s].  *sigma_out receives sigma.  idx_dev and val_dev hold 2^n
 * entries each.  Used to check Eq. 2's incremental update and the Gray
 * enumeration state by state.
 */
int qbf_walk_trace(const void *Q_dev, int n, int dtype, int prefix_bits, uint64_t *idx_dev,
                   int64_t *val_dev, int *sigma_out, void *stream);

/*
 * qbf_prefix_minima -- the MIN kernel alone, exposing its per-prefix minima.
 *
 * Runs the production MIN kernel of `variant` over the whole space:
 * QBF_VARIANT_SPLIT / AUTO the int32 Gray walk with 2^prefix_bits threads;
 * SPLIT_F32, SPLIT_MIX, SPLIT_DEFER the FP32-image walks (a thread walks 2 or
 * 8 values at once: its pair or group bits are the top suffix bits); FIELD and NAIVE
 * the reference forms; TC the tensor-core blocked form, which requires
 * prefix_bits = n - 14.  For every prefix p (the top prefix_bits variables) it
 * writes the minimum over its 2^(n - prefix_bits) suffix states of the
 * fixed-point objective round(Q * 2^sigma) to pmin_dev[p] (int32,
 * 2^prefix_bits entries, caller-owned device memory).  *sigma_out receives
 * sigma.  1 <= n <= 48, 0 <= prefix_bits <= min(n-1, 28), plus each variant's
 * limits (QBF_EINVAL otherwise).  Used to test the kernels prefix by prefix
 * against the oracle.
 */
int qbf_prefix_minima(const void *Q_dev, int n, int dtype, int prefix_bits, int variant,
                      int32_t *pmin_dev, int *sigma_out, void *stream);

/*
 * qbf_prefix_minima_fixed -- qbf_prefix_minima over a window of prefixes.
 *
 * Section 3.1's split with its top fix_bits prefix variables fixed: the MIN
 * kernel of `variant` runs in the geometry a solve with prefix_bits prefix
 * variables uses (same suffix width, block records and in-block unrolling),
 * but only over the 2^(prefix_bits - fix_bits) prefixes p whose top fix_bits
 * bits equal fix_value, i.e. the natural indices
 *     [fix_value * 2^(n - fix_bits), (fix_value + 1) * 2^(n - fix_bits)).
 * pmin_dev[j] (int32, 2^(prefix_bits - fix_bits) entries, caller-owned device
 * memory) receives the minimum of round(Q * 2^sigma) over prefix
 * p = fix_value * 2^(prefix_bits - fix_bits) + j, whose states are the natural
 * indices [p * 2^(n - prefix_bits), (p + 1) * 2^(n - prefix_bits)).  sigma is
 * that of the whole problem (the same image as a full solve).  Requires
 * 0 <= fix_bits <= prefix_bits and fix_value < 2^fix_bits, plus
 * qbf_prefix_minima's limits (QBF_EINVAL otherwise).  Lets a test check the
 * kernels prefix by prefix at the full walk depth of a large solve without
 * walking all of its prefixes.
 */
int qbf_prefix_minima_fixed(const void *Q_dev, int n, int dtype, int prefix_bits, int variant,
                            int fix_bits, uint64_t fix_value, int32_t *pmin_dev, int *sigma_out,
                            void *stream);

/*
 * qbf_tc_selftest -- one tcgen05 MMA on given operands: D = A * B with A
 * 128 x 16 and B 16 x 128 (row-major FP16 bit patterns, host memory) and D
 * 128 x 128 FP32 (host).  Checks the shared-memory operand layout and the
 * instruction descriptor the blocked form uses.  Allocates small device
 * buffers and synchronises the device.
 */
int qbf_tc_selftest(const uint16_t *A_host, const uint16_t *B_host, float *D_host);

/*
 * qbf_alu_microbench -- measures one ALU instruction class on every SM.
 *
 * op: 0 IADD3, 1 IMNMX, 2 3-input integer min, 3 FADD, 4 FFMA, 5 FMNMX,
 *     6 3-input FMNMX, 7 packed FADD (f32x2), 8 IADD3+IMNMX pair,
 *     9 FADD+FMNMX pair, 10 ex2.approx (exponential unit), 11 FP64 add,
 *     12 integer multiply-add, 13 int32 -> FP32 -> int32 conversion pair
 *     (each conversion counts one), 14 the step mix of the table-driven
 *     deferred walk without memory traffic (value-ops: 2 per state, at the
 *     walk's launch shape; the ceiling of that instruction mix).
 *     Operations are counted as written in PTX:
 *     the assembler may merge consecutive dependent two-input mins.
 * Writes scalar lane operations per SM clock per SM to *ops_per_clk_sm (a
 * packed f32x2 add counts two, each instruction of a pair counts one), the
 * SM clock seen during the run to *sm_mhz and the elapsed device time to
 * *seconds.  Allocates and frees its own small buffers.  Used for the
 * roofline denominator of the walk.
 */
int qbf_alu_microbench(int op, double *ops_per_clk_sm, double *sm_mhz, double *seconds,
                       void *stream);

/* Human-readable description of the last error on this thread. */
const char *qbf_last_error_string(void);

/*
 * qbf_cancel -- stop the solve that is running, from any host thread.
 *
 * Sets a host flag and, with the copy engine on a stream of its own, a flag
 * word in the memory of every device that has run a solve, so the write
 * lands while a solve's kernels run.  The walks read the word each time a
 * warp takes a work item, so they stop within one item's time: about 3 ms
 * at n = 40 at the automatic prefix width.  The log Z walks read it when a
 * block starts.  The running qbf_solve, qbf_solve_host, qubo_bf_solve,
 * qbf_chunked_step, qbf_solve_batched(_info) or qbf_logz(_backward) then
 * returns QBF_ECANCELED, with no result and its outputs unspecified.  A
 * chunked run stays at its last completed step.  Every such call clears the
 * flags when it starts, so a qbf_cancel with no call running has no effect.
 * A solve in the tensor-core form (QBF_VARIANT_TC) does not stop early: it
 * runs to its end and then reports QBF_ECANCELED.  qbf_solve_noalloc and the
 * prefix-minima and trace entry points ignore the flags.  Returns QBF_OK
 * (a failed device write only delays the stop to the end of the call).
 */
int qbf_cancel(void);

/* Free the library's scratch pools, captured solve graphs and cancellation
 * words on every device it touched (the next call allocates afresh).  Call
 * it before resetting a device with cudaDeviceReset. */
int qbf_release(void);

/* Library version as an integer (major*10000 + minor*100 + patch). */
int qbf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QBF_H */
