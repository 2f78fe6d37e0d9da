// qbf_noalloc.cu -- qbf_solve_noalloc: the same solve as qbf_solve, run on a
// fixed scratch area compiled into the library, so the call itself never asks
// the CUDA runtime for memory.
//
// Who needs this: programs that reserve the whole device up front and hand out
// memory only through their own pool, plug-ins that live inside a host
// application which owns the GPU memory budget, and latency-critical services
// that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
// cause.  Such callers provide Q and receive the result, and nothing else.
//
// The scratch is one file-scope __device__ array of QBF_NOALLOC_SCRATCH_BYTES.
// Every GPU that loads the library holds it until the process exits.  Host
// code must not pass the array's name to a kernel (on the host that name is
// only a stand-in); the first call on each device looks up the array's device
// address with cudaGetSymbolAddress while that device is current and keeps it.
// That first call should therefore happen before any stream capture begins.
//
// All calls share the one array and each call leaves its contents behind:
// every field a later step reads is rewritten or reset (the counters block is
// reset by reset_counters_kernel) before use.  Calls whose GPU work overlaps
// (different host threads on different streams, or together with qbf_solve,
// which shares the constant-bank corrections) race; calls from one thread are
// serialised, and each call waits for its stream before returning.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "qbf.h"
#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"

namespace qbf {
namespace {

constexpr int kNaMaxPrefixBits = 16;
constexpr int kNaMaxSuffixBits = 20;
constexpr unsigned long long kNaCandCap = 1ull << 16;
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[QBF_NOALLOC_SCRATCH_BYTES];

std::mutex g_na_mu;
char *g_na_base[kNaMaxDevices] = {};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NaLayout {
    size_t plan, ctr, res, kbuf, recs, pmin, flagged, cand, vals, total;
};

NaLayout na_layout(int ns, int R, unsigned long long npref)
{
    NaLayout L;
    size_t o = 0;
    L.plan = o;
    o = al256(o + sizeof(Plan));
    L.ctr = o;
    o = al256(o + sizeof(Counters));
    L.res = o;
    o = al256(o + sizeof(DevResult));
    L.kbuf = o;
    o = al256(o + sizeof(int) * kKbufInts);
    L.recs = o;
    o = al256(o + sizeof(Rec) * std::max<size_t>((size_t)1 << (ns - R), 2));
    L.pmin = o;
    o = al256(o + sizeof(int) * npref);
    L.flagged = o;
    o = al256(o + sizeof(unsigned) * npref);
    L.cand = o;
    o = al256(o + sizeof(unsigned long long) * kNaCandCap);
    L.vals = o;
    o = al256(o + sizeof(long long) * kNaCandCap);
    L.total = o;
    return L;
}

// Device address of the scratch array for the current device (looked up once).
int na_scratch(char **base)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return record_error(QBF_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kNaMaxDevices)
        return record_error(QBF_EINVAL, "qbf_solve_noalloc supports device ordinals below 64");
    if (!g_na_base[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return record_error(QBF_ECUDA, "cudaGetSymbolAddress(noalloc scratch) failed");
        g_na_base[dev] = (char *)p;
    }
    *base = g_na_base[dev];
    return QBF_OK;
}

int na_grid(int R, int mode, int n, int ns, unsigned long long nitems)
{
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int bps = walk_blocks_per_sm(R, mode, walk_smem_bytes(n, ns, R));
    const long long full = (long long)std::max(nsm, 1) * bps;
    const long long need = (long long)((nitems + (kWalkThreads / 32) - 1) / (kWalkThreads / 32));
    return (int)std::max<long long>(1, std::min(full, need));
}

int dtype_ok(int dt) { return dt == QBF_F64 || dt == QBF_F32 || dt == QBF_I32 || dt == QBF_I16; }

#define NA_CUDA(call, where)                                                                     \
    do {                                                                                         \
        cudaError_t na_e_ = (call);                                                              \
        if (na_e_ != cudaSuccess)                                                                \
            return record_error(QBF_ECUDA, where);                                               \
    } while (0)

int solve_noalloc_locked(const void *Q, int n, int dtype, const qbf_options *opt_in,
                         qbf_result *out, cudaStream_t s)
{
    if (!Q || !out)
        return record_error(QBF_EINVAL, "null pointer argument");
    if (!dtype_ok(dtype))
        return record_error(QBF_EDTYPE, "unknown dtype");
    if (n < 1 || n > QBF_NOALLOC_MAX_N)
        return record_error(QBF_EINVAL,
                            "qbf_solve_noalloc: n must be in [1, 36] (fixed scratch size)");
    qbf_options o;
    qbf_default_options(&o);
    if (opt_in)
        o = *opt_in;
    if (o.top_k == 0)
        o.top_k = 1;
    if (o.top_k < 1 || o.top_k > QBF_MAX_TOPK)
        return record_error(QBF_EINVAL, "top_k must be in [1, 64]");
    if (o.variant != QBF_VARIANT_AUTO && o.variant != QBF_VARIANT_SPLIT)
        return record_error(QBF_ENOTIMPL, "requested walk variant is not built");
    if (o.fix_bits < 0 || o.fix_bits > n - 1 || o.fix_bits > kNaMaxPrefixBits)
        return record_error(QBF_EINVAL, "qbf_solve_noalloc: fix_bits must be in [0, min(n-1, 16)]");
    if (o.fix_bits > 0 && (o.fix_value >> o.fix_bits) != 0)
        return record_error(QBF_EINVAL, "fix_value has bits above fix_bits");

    // geometry: at most 2^16 prefixes and 2^20 suffix states per thread
    const int kmin = std::max(0, n - kNaMaxSuffixBits);
    int k;
    if (o.prefix_bits >= 0) {
        k = o.prefix_bits;
        if (k < kmin || k > std::min(n - 1, kNaMaxPrefixBits))
            return record_error(QBF_EINVAL,
                                "qbf_solve_noalloc: prefix_bits must be in [max(0, n-20), min(n-1, 16)]");
    } else {
        k = (n <= 10) ? 0 : std::min(kNaMaxPrefixBits, n - 10);
        k = std::max(k, kmin);
    }
    k = std::max(k, o.fix_bits);
    if (k > kNaMaxPrefixBits || n - k > kNaMaxSuffixBits)
        return record_error(QBF_EINVAL, "qbf_solve_noalloc: problem exceeds the fixed scratch");
    const int ns = n - k;
    const int R = std::min(kRMax, ns);
    const int M = ns - R;
    const int q = std::min(M, 10);
    unsigned long long p_lo = 0, p_hi = 1ull << k;
    if (o.fix_bits > 0) {
        p_lo = o.fix_value << (k - o.fix_bits);
        p_hi = (o.fix_value + 1) << (k - o.fix_bits);
    }
    const unsigned long long npref = p_hi - p_lo;
    const NaLayout L = na_layout(ns, R, npref);
    if (L.total > (size_t)QBF_NOALLOC_SCRATCH_BYTES)
        return record_error(QBF_EINVAL, "qbf_solve_noalloc: problem exceeds the fixed scratch");

    char *base = nullptr;
    int rc = na_scratch(&base);
    if (rc)
        return rc;
    Plan *plan = (Plan *)(base + L.plan);
    Counters *ctr = (Counters *)(base + L.ctr);
    Rec *recs = (Rec *)(base + L.recs);
    int *Kbuf = (int *)(base + L.kbuf);
    int *pmin = (int *)(base + L.pmin);
    unsigned *flagged = (unsigned *)(base + L.flagged);
    unsigned long long *cand = (unsigned long long *)(base + L.cand);
    long long *vals = (long long *)(base + L.vals);
    DevResult *dres = (DevResult *)(base + L.res);

    prepare_kernel<<<1, 256, 0, s>>>(Q, n, dtype, plan, (long long)INT_MAX);
    NA_CUDA(cudaGetLastError(), "prepare_kernel launch failed");
    const unsigned nrec = 1u << M;
    tables_kernel<<<(nrec + 255) / 256, 256, 0, s>>>(plan, ns, R, recs, nrec, Kbuf);
    NA_CUDA(cudaGetLastError(), "tables_kernel launch failed");
    NA_CUDA(copy_corrections(Kbuf, s), "corrections to constant bank failed");
    reset_counters_kernel<<<1, 32, 0, s>>>(ctr);
    NA_CUDA(cudaGetLastError(), "reset_counters_kernel launch failed");

    WalkArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.ns = ns;
    a.p_lo = p_lo;
    a.p_hi = p_hi;
    a.nitems = (npref + 31) / 32;
    a.ctr = ctr;
    a.pmin = pmin;
    NA_CUDA(launch_walk(kModeMin, R, plan, recs, a, na_grid(R, kModeMin, n, ns, a.nitems), s),
            "walk (min) launch failed");
    threshold_kernel<<<1, 1024, 0, s>>>(plan, pmin, npref, o.top_k, ctr);
    NA_CUDA(cudaGetLastError(), "threshold_kernel launch failed");
    const bool is_int = (dtype == QBF_I32 || dtype == QBF_I16);
    const int fb = (int)std::min<unsigned long long>((npref + 255) / 256, 4096);
    flag_kernel<<<fb, 256, 0, s>>>(plan, pmin, npref, o.top_k, flagged, ctr);
    NA_CUDA(cudaGetLastError(), "flag_kernel launch failed");
    WalkArgs e = a;
    e.ns = ns - q;
    e.q = q;
    e.top_k = o.top_k;
    e.flagged = flagged;
    e.cand = cand;
    e.cand_cap = kNaCandCap;
    e.pmin = nullptr;
    const unsigned long long max_items = (npref << q) / 32 + 1;
    NA_CUDA(launch_walk(kModeEmit, R, plan, recs, e, na_grid(R, kModeEmit, n, e.ns, max_items), s),
            "walk (emit) launch failed");
    rescore_kernel<<<256, 256, 0, s>>>(plan, Q, n, dtype, cand, ctr, kNaCandCap, vals);
    NA_CUDA(cudaGetLastError(), "rescore_kernel launch failed");
    select_kernel<<<1, 1024, 0, s>>>(plan, cand, vals, ctr, kNaCandCap, o.top_k, dres);
    NA_CUDA(cudaGetLastError(), "select_kernel launch failed");

    DevResult R_h;
    Plan P_h;
    NA_CUDA(cudaMemcpyAsync(&R_h, dres, sizeof(DevResult), cudaMemcpyDeviceToHost, s),
            "copy result failed");
    NA_CUDA(cudaMemcpyAsync(&P_h, plan, offsetof(Plan, lin), cudaMemcpyDeviceToHost, s),
            "copy plan failed");
    NA_CUDA(cudaStreamSynchronize(s), "qbf_solve_noalloc failed on the stream");
    if (P_h.status == QBF_ENONFINITE)
        return record_error(QBF_ENONFINITE, "Q holds NaN or Inf");
    if (P_h.status == QBF_ERANGE)
        return record_error(QBF_ERANGE, "integer Q: sum |Q_ij| must stay below 2^31");
    if (P_h.status != QBF_OK)
        return record_error(P_h.status, "prepare failed");
    if (R_h.status == QBF_EOVERFLOW)
        return record_error(QBF_EOVERFLOW,
                            "qbf_solve_noalloc: more than 2^16 states inside the certification window");
    if (R_h.status != QBF_OK || R_h.count < 1)
        return record_error(QBF_ECUDA, "internal error: no candidate state selected");

    memset(out, 0, sizeof(*out));
    out->top_k = R_h.count;
    for (int i = 0; i < R_h.count; ++i) {
        out->topk_value[i] = R_h.topk_value[i];
        out->topk_index[i] = R_h.topk_index[i];
    }
    out->min_value = R_h.topk_value[0];
    out->argmin = R_h.topk_index[0];
    out->scale_bits = P_h.sigma;
    out->error_bound = is_int ? 0.0 : P_h.error_bound;
    out->n_candidates = R_h.n_candidates;
    out->prefix_bits = k;
    out->suffix_bits = ns;
    out->variant = QBF_VARIANT_SPLIT;
    out->walk_launches = 1;
    out->kernel_launches = 9;
    return QBF_OK;
}

}  // namespace
}  // namespace qbf

extern "C" int qbf_solve_noalloc(const void *Q_dev, int n, int dtype, const qbf_options *opt,
                                 qbf_result *out, void *stream)
{
    std::lock_guard<std::mutex> lk(qbf::g_na_mu);
    return qbf::solve_noalloc_locked(Q_dev, n, dtype, opt, out, (cudaStream_t)stream);
}
