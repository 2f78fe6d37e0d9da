// qbf_kernels.cuh -- launch interfaces between the host runtime and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdlib>

#include "qbf_internal.cuh"

namespace qbf {

constexpr int kWalkThreads = 256;
constexpr int kModeMin = 0;
constexpr int kModeEmit = 1;
constexpr int kModeTrace = 2;
constexpr unsigned long long kCandCap = 1ull << 22;  // candidate states per solve
// tables_kernel output: K[2][64] in-block corrections
constexpr int kKbufInts = 128;

struct WalkArgs {
    int n;                          // variables
    int ns;                         // suffix bits walked per thread
    unsigned long long p_lo, p_hi;  // MIN/TRACE: prefixes [p_lo, p_hi)
    unsigned long long nitems;      // MIN/TRACE: warp items = ceil((p_hi - p_lo) / 32)
    int q;                          // EMIT: sub-prefix bits per flagged prefix
    int top_k;                      // EMIT: with top_k = 1 and an exact plan (W = 0)
                                    // only the lowest flagged prefix is re-walked
    const unsigned int *flagged;    // EMIT: flagged prefixes (absolute, n - ns - q bits)
    Counters *ctr;
    int *pmin;                      // MIN: per-prefix minimum, index p - p_lo
    unsigned long long *cand;       // EMIT: candidate natural indices
    unsigned long long cand_cap;
    unsigned long long *trace_idx;  // TRACE
    long long *trace_val;
    const volatile int *cancel;     // nullptr, or the cancellation word
};

// qbf_prepare.cu
__global__ void prepare_kernel(const void *Q, int n, int dtype, Plan *plan, long long vmax);
__global__ void batched_prepare_kernel(const BatchDesc *desc, Plan *plans, int *status,
                                       long long vmax_float);
__global__ void batched_tables_kernel(const BatchDesc *desc, const Plan *plans, Rec *recs, int *K);
__global__ void logz_prepare_kernel(const void *Q, int n, int dtype, int rot, Plan *plans);
__global__ void logz_tables_kernel(const Plan *plans, int nsA, int nsB, Rec *recs,
                                   unsigned rec_stride, int *K);
__global__ void tables_kernel(const Plan *plan, int ns, int R, Rec *recs, unsigned nrec, int *Kbuf);

// qbf_walk.cu
size_t walk_smem_bytes(int n, int ns, int R);
int walk_blocks_per_sm(int R, int mode, size_t smem);
cudaError_t launch_walk(int mode, int R, const Plan *plan, const Rec *recs, const WalkArgs &a,
                        int grid, cudaStream_t s);
cudaError_t copy_corrections(const int *Kbuf_dev, cudaStream_t s);

// qbf_select.cu
__global__ void reset_counters_kernel(Counters *c);
__global__ void threshold_kernel(const Plan *plan, const int *pmin, unsigned long long npref,
                                 int top_k, Counters *c);
__global__ void flag_kernel(const Plan *plan, const int *pmin, unsigned long long npref,
                            int top_k, unsigned int *flagged, Counters *c);
__global__ void rescore_kernel(const Plan *plan, const void *Q, int n, int dtype,
                               const unsigned long long *cand, const Counters *c,
                               unsigned long long cap, long long *vals);
__global__ void select_kernel(const Plan *plan, const unsigned long long *cand,
                              const long long *vals, const Counters *c, unsigned long long cap,
                              int top_k, DevResult *res);

// qbf_api.cu: report an error through qbf_last_error_string(); returns code
int record_error(int code, const char *msg);
// A named NVTX range over one library call (host side; a profiler that
// records NVTX shows each call's kernels under it, a no-op otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Host-side fault injection for the error paths: with the environment
// variable QBF_INJECT_ALLOC_FAILURE set, a scratch pool that has to grow
// reports a failed allocation instead of allocating (no GPU work involved).
inline bool inject_alloc_failure() { return std::getenv("QBF_INJECT_ALLOC_FAILURE") != nullptr; }

// qbf_api.cu: cancellation.  cancel_clear (host, before a solve enqueues or
// captures its work) clears the host flag and allocates the current device's
// flag word; cancel_word_dev is that word (nullptr if it could not be
// allocated); cancel_reset_async clears it in the solve's stream before the
// kernels; cancel_requested tells the host after the solve whether
// qbf_cancel was called meanwhile (then the call returns QBF_ECANCELED).
const volatile int *cancel_word_dev();
void cancel_clear();
cudaError_t cancel_reset_async(cudaStream_t s);
bool cancel_requested();
int cancel_all();
void release_cancel();  // frees every device's word and stream (qbf_release)

// qbf_batched.cu
// Where a batched solve copies the MIN pass's per-item minima of one instance
// (item j: prefixes 32j..32j+31, the fixed-point image's minimum over their
// states): at most max_items of them into item_min (host), their count into
// *n_items.
struct BatchItemsOut {
    int inst;
    int *item_min;
    unsigned long long max_items;
    unsigned long long *n_items;
};
int solve_batched(const void *const *Q, const int *n, const int *dtype, int count,
                  const qbf_options *opt, double *min_value, uint64_t *argmin, cudaStream_t s,
                  int *kernel_launches, qbf_batch_info *info = nullptr, int ctas_override = 0,
                  const BatchItemsOut *items_out = nullptr);
int set_tuned_batch_ns(int ns);
int tune_batched_table(int n_min, int n_max, int dtype, const char *cache_path);
int tuned_params(int n, int dtype, int *suffix_bits, int *ctas_per_sm);
int release_batched();

// qbf_logz.cu
int logz_forward(const void *Q, int n, int dtype, int batch, const double *beta, int nbeta,
                 double *logz, double *min_value, uint64_t *argmin, cudaStream_t s);
int logz_backward(const void *Q, int n, int dtype, int batch, const double *beta, int nbeta,
                  const double *upstream, double *grad, double *moment, cudaStream_t s);
int danskin(const uint64_t *argmin_host, int n, int batch, const double *upstream, double *grad,
            cudaStream_t s);
int release_logz();

// qbf_walk_f32.cu: MIN walk in packed FP32 (image bounded by 2^23, pairs of prefixes)
constexpr long long kF32Vmax = (1ll << 23) - (1ll << 12);
// qbf_walk_plain.cu: the plain Gray walk (field vector, suffix <= 20 bits) and
// the naive natural-order evaluator, on the int32 image
constexpr int kFieldMaxSuffix = 20;
cudaError_t launch_walk_field(const Plan *plan, const WalkArgs &a, int num_sms, cudaStream_t s);
cudaError_t launch_walk_naive(const Plan *plan, const WalkArgs &a, int num_sms, cudaStream_t s);

// qbf_ising.cu: Q = 4J + diag(2h - 2R - 2C) and c into a fixed device buffer
// (FP64 Q for float J, h; int32 Q for integer J, h); returns Q, its dtype, c
// and the range status on the host after synchronising s
cudaError_t ising_to_qubo(const void *J, const void *h, int n, int dtype, const void **Q,
                          int *qdtype, double *c_host, int *status_host, cudaStream_t s);

// qbf_walk_defer.cu: MIN walk with the in-block correction added after the
// minimum over eight prefixes (same image bound and geometry as the two-pipe
// walk); scratch_dev holds 130 floats.  With ftab_dev (device memory of
// walk_defer_table_floats(R, a.ns - 3) floats, when that is not 0) it runs the
// table-driven form, else the record-driven one.
cudaError_t launch_walk_defer(int R, const Plan *plan, const Rec *recs, const WalkArgs &a,
                              const int *Kbuf_dev, void *scratch_dev, int num_sms, cudaStream_t s,
                              float *ftab_dev = nullptr);
size_t walk_defer_table_floats(int R, int nsw);

// qbf_walk_mix.cu: MIN walk on both pipes (same image bound; eight prefixes per thread)
cudaError_t launch_walk_mix(int R, const Plan *plan, const Rec *recs, const WalkArgs &a,
                            const int *Kbuf_dev, unsigned long long *Kf2_dev, int num_sms,
                            cudaStream_t s);
cudaError_t launch_walk_f32(int R, const Plan *plan, const Rec *recs, const WalkArgs &a,
                            const int *Kbuf_dev, unsigned long long *Kf2_dev, int num_sms,
                            cudaStream_t s);

// qbf_tc.cu: tensor-core blocked form (tiles of 14 low bits)
constexpr int kTcTileSuffixBits = 14;
constexpr long long kTcVmax = (1ll << 22) - (1ll << 12);  // bound on sum |image| for exact FP32
cudaError_t launch_tc_min(const Plan *plan, int n, unsigned long long p_lo,
                          unsigned long long p_hi, int *pmin, Counters *ctr, int num_sms,
                          cudaStream_t s);
cudaError_t run_tc_selftest(const void *A_host, const void *B_host, float *D_host, int *err_host);

// qbf_microbench.cu
cudaError_t run_alu_microbench(int op, double *ops_per_clk_sm, double *sm_mhz, double *seconds,
                               cudaStream_t s);

}  // namespace qbf
