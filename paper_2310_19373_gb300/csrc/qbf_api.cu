// qbf_api.cu -- host runtime of libqubobf: argument checks, planning, scratch
// pool and the launch sequence of one solve.
//
// One solve (qbf_solve) enqueues on the caller's stream:
//   prepare_kernel        A1  fixed-point image of Q, certification window
//   tables_kernel         A1  lane-invariant walk records + in-block corrections
//   corrections -> constant bank (device-to-device copy)
//   reset_counters_kernel
//   walk (MIN)            A2-A4  every prefix's minimum and the global minimum
//   threshold_kernel      A5/A7  tau = k-th smallest prefix minimum + W
//   flag_kernel           A6  prefixes that can hold a winning state
//   walk (EMIT)           A6  re-walk of those prefixes, emitting candidates
//   rescore_kernel        A6  FP64 canonical / exact int64 value per candidate
//   select_kernel         A5/A7  top-k by (value, natural index)
// then copies the small result back and waits for the stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "qbf.h"
#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"

using namespace qbf;

namespace {

thread_local std::string g_err;
std::mutex g_mu;

int set_err(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_err(cudaError_t e, const char *where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return QBF_ECUDA;
}

#define QBF_CUDA(call, where)                                                                    \
    do {                                                                                         \
        cudaError_t qbf_e_ = (call);                                                             \
        if (qbf_e_ != cudaSuccess)                                                               \
            return cuda_err(qbf_e_, where);                                                      \
    } while (0)

struct Pool {
    void *dev = nullptr;
    size_t bytes = 0;
    void *host = nullptr;  // pinned staging for the result
    size_t hbytes = 0;
};
std::vector<Pool> g_pools;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t plan, ctr, res, kbuf, recs, pmin, flagged, cand, vals, qcopy, ftab, total;
};

Layout make_layout(size_t nrec, size_t npref, size_t qbytes, bool need_cand,
                   size_t ftab_floats = 0)
{
    Layout L;
    size_t o = 0;
    L.plan = o;
    o = align256(o + sizeof(Plan));
    L.ctr = o;
    o = align256(o + sizeof(Counters));
    L.res = o;
    o = align256(o + sizeof(DevResult));
    L.kbuf = o;
    o = align256(o + sizeof(int) * kKbufInts + sizeof(unsigned long long) * 128);
    L.recs = o;
    o = align256(o + sizeof(Rec) * std::max<size_t>(nrec, 2));
    L.pmin = o;
    o = align256(o + sizeof(int) * npref);
    L.flagged = o;
    o = align256(o + sizeof(unsigned) * npref);
    L.cand = o;
    o = align256(o + (need_cand ? sizeof(unsigned long long) * kCandCap : 0));
    L.vals = o;
    o = align256(o + (need_cand ? sizeof(long long) * kCandCap : 0));
    L.qcopy = o;
    o = align256(o + qbytes);
    L.ftab = o;
    o = align256(o + sizeof(float) * ftab_floats);
    L.total = o;
    return L;
}

int pool_get(size_t bytes, size_t hbytes, Pool **out)
{
    int dev = 0;
    QBF_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if ((int)g_pools.size() <= dev)
        g_pools.resize(dev + 1);
    Pool &P = g_pools[dev];
    if (P.bytes < bytes) {
        if (inject_alloc_failure())
            return set_err(QBF_ECUDA, "cudaMalloc(scratch): failure injected by "
                                      "QBF_INJECT_ALLOC_FAILURE");
        if (P.dev) {
            QBF_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
            cudaFree(P.dev);
            P.dev = nullptr;
            P.bytes = 0;
        }
        QBF_CUDA(cudaMalloc(&P.dev, bytes), "cudaMalloc(scratch)");
        P.bytes = bytes;
    }
    if (P.hbytes < hbytes) {
        if (P.host)
            cudaFreeHost(P.host);
        P.host = nullptr;
        P.hbytes = 0;
        QBF_CUDA(cudaMallocHost(&P.host, hbytes), "cudaMallocHost");
        P.hbytes = hbytes;
    }
    *out = &P;
    return QBF_OK;
}

size_t dtype_size(int dt)
{
    switch (dt) {
    case QBF_F64: return 8;
    case QBF_F32: return 4;
    case QBF_I32: return 4;
    case QBF_I16: return 2;
    default: return 0;
    }
}

int num_sms()
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return nsm > 0 ? nsm : 1;
}

// Suffix width walked per thread when the caller leaves it to the planner:
// small n -> few long walks are not worth it, large n -> 2^24 prefixes keep the
// per-prefix set-up below 1% of the walk and give a fine-grained work queue.
// (2^14 short walks at 10 < n < 24 made an n = 20 top-8 solve slower, 144 ->
// 167 us: the top-k threshold and the flags then scan 16 times the prefixes.)
int auto_suffix_bits(int n)
{
    if (n <= 10)
        return n;
    int ns = n - 24;
    if (ns < 10)
        ns = 10;
    return ns;
}

// Suffix bits walked per lane by the table-driven deferred walk when the
// caller leaves the prefix width to the planner (the lane's three group bits
// come on top).  Measured on GB300 as the fastest MIN walk over the prefix
// widths at n = 26..40: small problems want more lanes, large ones longer
// lane walks, and from n = 36 on the lane depth of the n = 40 solve (for
// example n = 26: 0.023 against 0.039 ms with 10 bits; n = 34: 0.93 against
// 1.13 ms with 10 bits; n = 40: 16 bits, 53.0 ms, the fastest).
int defer_suffix_bits(int n)
{
    if (n <= 27)
        return 8;
    if (n == 28)
        return 9;
    if (n <= 32)
        return 11;
    if (n <= 34)
        return 12;
    if (n == 35)
        return 15;
    return 16;
}

// Prefixes per launch of a MIN walk: all of them up to 2^41 states (the n = 40
// solve is one launch), else slices of 2^41 states (multiples of 32 prefixes)
constexpr unsigned long long kLaunchStates = 1ull << 41;
unsigned long long launch_slice(unsigned long long npref, int ns)
{
    const unsigned long long per = ns >= 41 ? 1ull : kLaunchStates >> ns;
    const unsigned long long cap = std::max(32ull, per / 32 * 32);
    return npref <= cap ? npref : cap;
}

// walked blocks per thread (each 2^R states) are at most 2^kMaxBlockBits
constexpr int kMaxBlockBits = 20;

struct Geo {
    int n, k, ns, R, M, q;
    int ns_tab;  // suffix width the walk tables are built for
    unsigned long long p_lo, p_hi;
};

int plan_geometry(int n, const qbf_options &o, Geo *g)
{
    int k;
    // the automatic suffix width follows the states one call walks: with
    // fix_bits variables fixed, n - fix_bits of them vary
    const int fix = (o.fix_bits > 0 && o.fix_bits <= n - 1) ? o.fix_bits : 0;
    const int nf = n - fix;
    if (o.variant == QBF_VARIANT_TC) {
        // tiles of 14 low bits are the prefixes of the certification step
        if (n < kTcTileSuffixBits + 1 || n - kTcTileSuffixBits > 28)
            return set_err(QBF_EINVAL, "the tensor-core form needs 15 <= n <= 42");
        if (o.prefix_bits >= 0 && o.prefix_bits != n - kTcTileSuffixBits)
            return set_err(QBF_EINVAL, "the tensor-core form fixes prefix_bits = n - 14");
        k = n - kTcTileSuffixBits;
    } else if (o.variant == QBF_VARIANT_FIELD) {
        // the field vector lives in registers: at most kFieldMaxSuffix suffix bits
        if (o.prefix_bits >= 0) {
            k = o.prefix_bits;
            if (n - k < 1 || n - k > kFieldMaxSuffix || k > 28)
                return set_err(QBF_EINVAL, "the field walk needs 1 <= n - prefix_bits <= 20");
        } else {
            k = n - std::min(auto_suffix_bits(nf), kFieldMaxSuffix);
        }
    } else if (o.variant == QBF_VARIANT_SPLIT_MIX || o.variant == QBF_VARIANT_SPLIT_DEFER) {
        // a lane walks nsw bits for all eight values of the group bits nsw..nsw+2
        if (n < 4)
            return set_err(QBF_EINVAL, "the eight-prefix walks need n >= 4");
        if (o.prefix_bits >= 0) {
            k = o.prefix_bits;
            if (k > n - 4 || k > 28)
                return set_err(QBF_EINVAL, "prefix_bits must be in [0, min(n-4, 28)] for the eight-prefix walks");
        } else {
            const int want = (o.variant == QBF_VARIANT_SPLIT_DEFER) ? defer_suffix_bits(nf)
                                                                    : auto_suffix_bits(nf);
            const int nsw = std::max(1, std::min(want, nf - 3));
            k = n - nsw - 3;
        }
    } else if (o.variant == QBF_VARIANT_SPLIT_F32) {
        // a lane walks nsw bits for both values of the pair bit (variable nsw)
        if (n < 2)
            return set_err(QBF_EINVAL, "the packed FP32 walk needs n >= 2");
        if (o.prefix_bits >= 0) {
            k = o.prefix_bits;
            if (k > n - 2 || k > 28)
                return set_err(QBF_EINVAL, "prefix_bits must be in [0, min(n-2, 28)] for the packed walk");
        } else {
            const int nsw = std::max(1, std::min(auto_suffix_bits(nf), nf - 1));
            k = n - nsw - 1;
        }
    } else if (o.prefix_bits >= 0) {
        k = o.prefix_bits;
        if (k > n - 1 || k > 28)
            return set_err(QBF_EINVAL, "prefix_bits must be in [0, min(n-1, 28)]");
    } else {
        // the int32 split walk: a top-1 solve of a small problem runs fastest
        // with more, shorter lanes (whole-solve times measured on GB300: n = 16
        // 71 against 83 us, n = 22 82 against 93 us with 10 suffix bits); a
        // top-k solve keeps the wider suffix (n = 20 top-8: 101 us, against
        // 110 us with 6 bits)
        int ns = auto_suffix_bits(nf);
        if (o.top_k <= 1 && nf <= 23)
            ns = std::min(nf, std::max(6, nf - 14));
        k = n - ns;
    }
    // prefixes are numbered in 32 bits downstream (flag lists): an automatic
    // geometry keeps at most 2^28 of them, like an explicit prefix_bits
    if (o.prefix_bits < 0 && k > 28)
        k = 28;
    if (o.fix_bits < 0 || o.fix_bits > n - 1)
        return set_err(QBF_EINVAL, "fix_bits must be in [0, n-1]");
    if (o.fix_bits > 0 && (o.fix_value >> o.fix_bits) != 0)
        return set_err(QBF_EINVAL, "fix_value has bits above fix_bits");
    if (k < o.fix_bits) {
        if (o.variant == QBF_VARIANT_TC)
            return set_err(QBF_EINVAL, "fix_bits must be <= n - 14 for the tensor-core form");
        k = o.fix_bits;
    }
    g->n = n;
    g->k = k;
    g->ns = n - k;
    if (o.variant == QBF_VARIANT_SPLIT_MIX || o.variant == QBF_VARIANT_SPLIT_DEFER) {
        if (g->ns < 4)
            return set_err(QBF_EINVAL, "fix_bits must be <= n - 4 for the eight-prefix walks");
        const int nsw = g->ns - 3;
        g->R = std::min(kRMax, nsw);
        g->M = nsw - g->R;
        g->q = std::min(g->ns - g->R, 10);
        g->ns_tab = nsw;
    } else if (o.variant == QBF_VARIANT_SPLIT_F32) {
        const int nsw = g->ns - 1;
        g->R = std::min(kRMax, nsw);
        g->M = nsw - g->R;
        g->q = std::min(g->ns - g->R, 10);
        g->ns_tab = nsw;
    } else {
        g->R = std::min(kRMax, g->ns);
        g->M = g->ns - g->R;
        g->q = std::min(g->M, 10);
        g->ns_tab = g->ns;
    }
    // 2^M block records (32 B each) are built per solve and every thread walks
    // 2^(ns - k') states: bound both before anything is sized from M
    if (g->M > kMaxBlockBits)
        return set_err(QBF_EINVAL,
                       "prefix_bits too small: at most 2^20 blocks of 2^6 states per thread "
                       "(about 26 suffix bits; use more prefix bits)");
    if (o.fix_bits > 0) {
        g->p_lo = o.fix_value << (k - o.fix_bits);
        g->p_hi = (o.fix_value + 1) << (k - o.fix_bits);
    } else {
        g->p_lo = 0;
        g->p_hi = 1ull << k;
    }
    return QBF_OK;
}

int walk_grid(int R, int mode, int n, int ns, unsigned long long nitems)
{
    const size_t smem = walk_smem_bytes(n, ns, R);
    const int bps = walk_blocks_per_sm(R, mode, smem);
    const long long full = (long long)num_sms() * bps;
    const long long need = (long long)((nitems + (kWalkThreads / 32) - 1) / (kWalkThreads / 32));
    return (int)std::max<long long>(1, std::min(full, need));
}

// Enqueue prepare + tables + constant-bank copy + counter reset.
int enqueue_prepare(const void *Q, int n, int dtype, const Geo &g, char *base, const Layout &L,
                    cudaStream_t s, long long vmax = INT_MAX)
{
    Plan *plan = (Plan *)(base + L.plan);
    prepare_kernel<<<1, 256, 0, s>>>(Q, n, dtype, plan, vmax);
    QBF_CUDA(cudaGetLastError(), "prepare_kernel");
    const unsigned nrec = 1u << g.M;
    tables_kernel<<<(nrec + 255) / 256, 256, 0, s>>>(plan, g.ns_tab, g.R, (Rec *)(base + L.recs),
                                                    nrec, (int *)(base + L.kbuf));
    QBF_CUDA(cudaGetLastError(), "tables_kernel");
    QBF_CUDA(copy_corrections((const int *)(base + L.kbuf), s), "corrections to constant bank");
    reset_counters_kernel<<<1, 32, 0, s>>>((Counters *)(base + L.ctr));
    QBF_CUDA(cudaGetLastError(), "reset_counters_kernel");
    return QBF_OK;
}

int check_common(const void *Q, int n, int dtype, qbf_result *out)
{
    if (!Q || !out)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (n < 1 || n > QBF_MAX_N)
        return set_err(QBF_EINVAL, "n must be in [1, 48]");
    if (dtype_size(dtype) == 0)
        return set_err(QBF_EDTYPE, "unknown dtype");
    return QBF_OK;
}

// ---- graph replay of repeated solves ----------------------------------------

// One solve attempt is fixed by its matrix pointer, shape, options and the
// scratch pool it runs in; the kernels read Q at replay time, so new contents
// in the same buffer are solved afresh.
struct SolveKey {
    const void *Q;
    int n, dtype, top_k, variant, prefix_bits, fix_bits;
    uint64_t fix_value;
    void *dev, *host;
    size_t total;
    bool operator==(const SolveKey &o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

struct SolveGraph {
    SolveKey key;
    cudaGraphExec_t exec = nullptr;
    unsigned long long used = 0;
    bool seen = false;
};

constexpr int kSolveGraphs = 8;  // attempts remembered per device (least recently used out)

struct DevGraphs {
    cudaStream_t cap = nullptr;
    SolveGraph slot[kSolveGraphs];
    unsigned long long tick = 0;
};
std::vector<DevGraphs> g_graphs;

bool graphs_enabled()
{
    const char *e = getenv("QBF_NO_SOLVE_GRAPHS");
    return !(e && *e && *e != '0');
}

// Run one attempt: directly the first time its key is seen, captured into a
// graph and replayed from the second time on.  Called with g_mu held.
template <class F>
int run_cached(const SolveKey &key, F &&enqueue, cudaStream_t s)
{
    int dev = 0;
    QBF_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if ((int)g_graphs.size() <= dev)
        g_graphs.resize(dev + 1);
    DevGraphs &G = g_graphs[dev];
    ++G.tick;
    SolveGraph *hit = nullptr, *victim = &G.slot[0];
    for (SolveGraph &sg : G.slot) {
        if (sg.seen && sg.key == key) {
            hit = &sg;
            break;
        }
        if (!sg.seen || sg.used < victim->used)
            victim = &sg;
    }
    if (!hit) {
        if (victim->exec)
            cudaGraphExecDestroy(victim->exec);
        victim->exec = nullptr;
        victim->key = key;
        victim->seen = true;
        victim->used = G.tick;
        return enqueue(s);
    }
    hit->used = G.tick;
    if (!hit->exec) {
        if (!G.cap)
            QBF_CUDA(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t graph = nullptr;
        QBF_CUDA(cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        const int rc = enqueue(G.cap);
        const cudaError_t ce = cudaStreamEndCapture(G.cap, &graph);
        if (rc || ce != cudaSuccess) {
            if (graph)
                cudaGraphDestroy(graph);
            hit->seen = false;
            return rc ? rc : cuda_err(ce, "end capture");
        }
        const cudaError_t ie = cudaGraphInstantiate(&hit->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            hit->exec = nullptr;
            hit->seen = false;
            return cuda_err(ie, "graph instantiate");
        }
    }
    QBF_CUDA(cudaGraphLaunch(hit->exec, s), "graph launch");
    return QBF_OK;
}

void release_graphs()
{
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_graphs.size(); ++d) {
        DevGraphs &G = g_graphs[d];
        cudaSetDevice((int)d);
        for (SolveGraph &sg : G.slot) {
            if (sg.exec)
                cudaGraphExecDestroy(sg.exec);
            sg = SolveGraph();
        }
        if (G.cap)
            cudaStreamDestroy(G.cap);
        G.cap = nullptr;
    }
    cudaSetDevice(cur);
}

int solve_one(const void *Q, bool host_q, int n, int dtype, const qbf_options *opt_in,
              qbf_result *out, cudaStream_t s)
{
    const NvtxRange range("qbf_solve");
    int rc = check_common(Q, n, dtype, out);
    if (rc)
        return rc;
    qbf_options o;
    qbf_default_options(&o);
    if (opt_in)
        o = *opt_in;
    if (o.top_k == 0)
        o.top_k = 1;
    if (o.top_k < 1 || o.top_k > QBF_MAX_TOPK)
        return set_err(QBF_EINVAL, "top_k must be in [1, 64]");
    if (o.variant != QBF_VARIANT_AUTO && o.variant != QBF_VARIANT_SPLIT &&
        o.variant != QBF_VARIANT_TC && o.variant != QBF_VARIANT_SPLIT_F32 &&
        o.variant != QBF_VARIANT_SPLIT_MIX && o.variant != QBF_VARIANT_FIELD &&
        o.variant != QBF_VARIANT_NAIVE && o.variant != QBF_VARIANT_SPLIT_DEFER)
        return set_err(QBF_ENOTIMPL, "requested walk variant is not built");
    Geo g;
    if ((rc = plan_geometry(n, o, &g)))
        return rc;
    const bool tc = (o.variant == QBF_VARIANT_TC);
    const bool mix = (o.variant == QBF_VARIANT_SPLIT_MIX);
    const bool defer = (o.variant == QBF_VARIANT_SPLIT_DEFER);
    const bool field = (o.variant == QBF_VARIANT_FIELD);
    const bool naive = (o.variant == QBF_VARIANT_NAIVE);
    const bool f32 = (o.variant == QBF_VARIANT_SPLIT_F32) || mix || defer;  // same image bound

    const unsigned long long npref = g.p_hi - g.p_lo;
    const size_t qbytes = host_q ? dtype_size(dtype) * n * n : 0;
    const size_t ftab = defer ? walk_defer_table_floats(g.R, g.ns_tab) : 0;
    const Layout L = make_layout(1u << g.M, npref, qbytes, true, ftab);
    Pool *P = nullptr;
    if ((rc = pool_get(L.total, sizeof(DevResult) + sizeof(Plan) + 16, &P)))
        return rc;
    char *base = (char *)P->dev;
    const void *Qdev = host_q ? (const void *)(base + L.qcopy) : Q;
    Plan *plan = (Plan *)(base + L.plan);
    Counters *ctr = (Counters *)(base + L.ctr);
    const Rec *recs = (const Rec *)(base + L.recs);
    int *pmin = (int *)(base + L.pmin);
    unsigned *flagged = (unsigned *)(base + L.flagged);
    unsigned long long *cand = (unsigned long long *)(base + L.cand);
    long long *vals = (long long *)(base + L.vals);
    DevResult *dres = (DevResult *)(base + L.res);
    char *h = (char *)P->host;
    const bool is_int = (dtype == QBF_I32 || dtype == QBF_I16);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    const unsigned long long slice = tc ? npref : launch_slice(npref, g.ns);
    const int launches = (int)((npref + slice - 1) / slice);
    cancel_clear();
    // Every stream operation of one attempt, on stream st: replayable as a
    // graph (no host decision inside; the host reads the results afterwards)
    auto enqueue = [&](cudaStream_t s) -> int {
    QBF_CUDA(cancel_reset_async(s), "clear the cancellation word");
    if (host_q) {
        QBF_CUDA(cudaMemcpyAsync(base + L.qcopy, Q, qbytes, cudaMemcpyHostToDevice, s),
                 "copy Q to device");
    }
    int erc = enqueue_prepare(Qdev, n, dtype, g, base, L, s,
                              tc ? kTcVmax : (f32 ? kF32Vmax : (long long)INT_MAX));
    if (erc)
        return erc;

    // A2-A4: MIN walk over every prefix
    WalkArgs a_all;
    memset(&a_all, 0, sizeof(a_all));
    a_all.cancel = cancel_word_dev();
    a_all.n = n;
    a_all.ns = g.ns;
    a_all.p_lo = g.p_lo;
    a_all.p_hi = g.p_hi;
    a_all.nitems = (npref + 31) / 32;
    a_all.ctr = ctr;
    a_all.pmin = pmin;
    if (o.timing) {
        QBF_CUDA(cudaEventCreate(&ev[0]), "cudaEventCreate");
        QBF_CUDA(cudaEventCreate(&ev[1]), "cudaEventCreate");
        QBF_CUDA(cudaEventRecord(ev[0], s), "cudaEventRecord");
    }
    // Long walks run as several launches over consecutive prefix slices of at
    // most kLaunchStates states each (about 0.1 s of walking), so no single
    // kernel runs for seconds; the work counter restarts for every slice and
    // the global minimum accumulates across them.  The tensor-core form runs
    // in one launch.
    for (unsigned long long c0 = 0; c0 < npref; c0 += slice) {
        WalkArgs a = a_all;
        a.p_lo = g.p_lo + c0;
        a.p_hi = std::min(g.p_hi, a.p_lo + slice);
        a.nitems = (a.p_hi - a.p_lo + 31) / 32;
        a.pmin = pmin + c0;
        if (c0 > 0)
            QBF_CUDA(cudaMemsetAsync(&ctr->items[kModeMin], 0, sizeof(ctr->items[kModeMin]), s),
                     "restart the work counter");
        if (tc)
            QBF_CUDA(launch_tc_min(plan, n, g.p_lo, g.p_hi, pmin, ctr, num_sms(), s), "tc (min)");
        else if (field)
            QBF_CUDA(launch_walk_field(plan, a, num_sms(), s), "walk field (min)");
        else if (naive)
            QBF_CUDA(launch_walk_naive(plan, a, num_sms(), s), "naive (min)");
        else if (defer)
            QBF_CUDA(launch_walk_defer(g.R, plan, recs, a, (const int *)(base + L.kbuf),
                                       base + L.kbuf + sizeof(int) * kKbufInts, num_sms(), s,
                                       ftab ? (float *)(base + L.ftab) : nullptr),
                     "walk defer (min)");
        else if (mix)
            QBF_CUDA(launch_walk_mix(g.R, plan, recs, a, (const int *)(base + L.kbuf),
                                     (unsigned long long *)(base + L.kbuf + sizeof(int) * kKbufInts),
                                     num_sms(), s),
                     "walk mix (min)");
        else if (f32)
            QBF_CUDA(launch_walk_f32(g.R, plan, recs, a, (const int *)(base + L.kbuf),
                                     (unsigned long long *)(base + L.kbuf + sizeof(int) * kKbufInts),
                                     num_sms(), s),
                     "walk f32 (min)");
        else
            QBF_CUDA(launch_walk(kModeMin, g.R, plan, recs, a,
                                 walk_grid(g.R, kModeMin, n, g.ns, a.nitems), s),
                     "walk (min)");
    }
    if (o.timing)
        QBF_CUDA(cudaEventRecord(ev[1], s), "cudaEventRecord");

    // A5-A7: threshold, flags, re-walk of flagged prefixes, rescoring, selection
    threshold_kernel<<<1, 1024, 0, s>>>(plan, pmin, npref, o.top_k, ctr);
    QBF_CUDA(cudaGetLastError(), "threshold_kernel");
    // With exact values (W = 0: integer Q, or an all-zero float Q) and
    // top_k = 1 the kernels re-walk only the lowest flagged prefix; they read
    // W from the plan, so the host sizes the grid for the general case.
    {
        const int fb = (int)std::min<unsigned long long>((npref + 255) / 256, 4096);
        flag_kernel<<<fb, 256, 0, s>>>(plan, pmin, npref, o.top_k, flagged, ctr);
        QBF_CUDA(cudaGetLastError(), "flag_kernel");
    }
    WalkArgs e = a_all;
    e.ns = g.ns - g.q;
    e.q = g.q;
    e.top_k = o.top_k;
    e.flagged = flagged;
    e.cand = cand;
    e.cand_cap = kCandCap;
    e.pmin = nullptr;
    // the number of flagged prefixes is only known on the device: size the
    // persistent grid for the worst case, idle warps exit at once
    const unsigned long long max_items = (npref << g.q) / 32 + 1;
    QBF_CUDA(launch_walk(kModeEmit, g.R, plan, recs, e, walk_grid(g.R, kModeEmit, n, e.ns, max_items), s),
             "walk (emit)");
    rescore_kernel<<<256, 256, 0, s>>>(plan, Qdev, n, dtype, cand, ctr, kCandCap, vals);
    QBF_CUDA(cudaGetLastError(), "rescore_kernel");
    select_kernel<<<1, 1024, 0, s>>>(plan, cand, vals, ctr, kCandCap, o.top_k, dres);
    QBF_CUDA(cudaGetLastError(), "select_kernel");

    QBF_CUDA(cudaMemcpyAsync(h, dres, sizeof(DevResult), cudaMemcpyDeviceToHost, s), "copy result");
    QBF_CUDA(cudaMemcpyAsync(h + sizeof(DevResult), plan, offsetof(Plan, lin), cudaMemcpyDeviceToHost, s),
             "copy plan");
    QBF_CUDA(cudaMemcpyAsync(h + sizeof(DevResult) + sizeof(Plan), &ctr->status, sizeof(int),
                             cudaMemcpyDeviceToHost, s),
             "copy status");
    return QBF_OK;
    };
    // A repeated solve of the same device matrix with the same options replays
    // a captured graph of the attempt (one launch instead of about a dozen);
    // a first sighting runs directly, which also loads every kernel it uses
    if (!host_q && !o.timing && graphs_enabled()) {
        SolveKey key;
        memset(&key, 0, sizeof(key));
        key.Q = Q;
        key.n = n;
        key.dtype = dtype;
        key.top_k = o.top_k;
        key.variant = o.variant;
        key.prefix_bits = o.prefix_bits;
        key.fix_bits = o.fix_bits;
        key.fix_value = o.fix_value;
        key.dev = P->dev;
        key.host = P->host;
        key.total = L.total;
        if ((rc = run_cached(key, enqueue, s)))
            return rc;
    } else if ((rc = enqueue(s))) {
        return rc;
    }
    QBF_CUDA(cudaStreamSynchronize(s), "solve");
    if (cancel_requested()) {
        if (o.timing) {
            cudaEventDestroy(ev[0]);
            cudaEventDestroy(ev[1]);
        }
        return set_err(QBF_ECANCELED, "cancelled by qbf_cancel");
    }
    float walk_ms = 0.f;
    if (o.timing) {
        cudaEventElapsedTime(&walk_ms, ev[0], ev[1]);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    const DevResult *R = (const DevResult *)h;
    const Plan *PH = (const Plan *)(h + sizeof(DevResult));
    if (PH->status != QBF_OK) {
        if (PH->status == QBF_ENONFINITE)
            return set_err(QBF_ENONFINITE, "Q holds NaN or Inf");
        if (PH->status == QBF_ERANGE)
            return set_err(QBF_ERANGE,
                           tc ? "integer Q: the tensor-core form needs sum |Q_ij| < 2^22"
                              : (f32 ? "integer Q: the FP32-pipe walks need sum |Q_ij| < 2^23"
                                     : "integer Q: sum |Q_ij| must stay below 2^31"));
        return set_err(PH->status, "prepare failed");
    }
    {
        int st = 0;
        memcpy(&st, h + sizeof(DevResult) + sizeof(Plan), sizeof(int));
        if (st != QBF_OK)
            return set_err(QBF_ECUDA, "a device-side wait ran out (tensor-core pipeline)");
    }
    if (R->status == QBF_EOVERFLOW)
        return set_err(QBF_EOVERFLOW, "more than 2^22 states inside the certification window");
    if (R->status != QBF_OK || R->count < 1)
        return set_err(QBF_ECUDA, "internal error: no candidate state selected");

    memset(out, 0, sizeof(*out));
    out->top_k = R->count;
    for (int i = 0; i < R->count; ++i) {
        out->topk_value[i] = R->topk_value[i];
        out->topk_index[i] = R->topk_index[i];
    }
    out->min_value = R->topk_value[0];
    out->argmin = R->topk_index[0];
    out->scale_bits = PH->sigma;
    out->error_bound = is_int ? 0.0 : PH->error_bound;
    out->n_candidates = R->n_candidates;
    out->prefix_bits = g.k;
    out->suffix_bits = g.ns;
    out->variant = tc      ? QBF_VARIANT_TC
                   : defer ? QBF_VARIANT_SPLIT_DEFER
                   : mix   ? QBF_VARIANT_SPLIT_MIX
                   : f32   ? QBF_VARIANT_SPLIT_F32
                   : field ? QBF_VARIANT_FIELD
                   : naive ? QBF_VARIANT_NAIVE
                           : QBF_VARIANT_SPLIT;
    out->walk_launches = launches;
    // prepare, tables, reset, walk(min), threshold, flag, walk(emit), rescore, select
    // (+ the correction-pair conversion of the packed walk)
    // the FP32-pipe walks convert the correction pairs (or build the suffix
    // table) before every MIN launch
    out->kernel_launches = (f32 ? 10 : 9) + (launches - 1) * (f32 ? 2 : 1);
    out->walk_seconds = walk_ms * 1e-3;
    return QBF_OK;
}

// QBF_VARIANT_AUTO with n >= kAutoMixMinN takes the deferred-correction walk
// (the fastest form on this part).  Its image is bounded by 2^23 instead of 2^31:
// integer Q with a larger sum |Q_ij| is rejected by prepare (QBF_ERANGE)
// before any walk work, and for float Q the certification window is 2^8
// times wider, so if it flags more candidates than the candidate buffer holds
// (QBF_EOVERFLOW) the solve is repeated on the int32 walk.
constexpr int kAutoMixMinN = 24;

int solve_locked(const void *Q, bool host_q, int n, int dtype, const qbf_options *opt_in,
                 qbf_result *out, cudaStream_t s)
{
    qbf_options o;
    qbf_default_options(&o);
    if (opt_in)
        o = *opt_in;
    if (o.variant == QBF_VARIANT_AUTO && n >= kAutoMixMinN && o.prefix_bits <= n - 4 &&
        o.fix_bits <= n - 4) {
        qbf_options om = o;
        om.variant = QBF_VARIANT_SPLIT_DEFER;
        const int rc = solve_one(Q, host_q, n, dtype, &om, out, s);
        if (rc != QBF_EOVERFLOW && rc != QBF_ERANGE)
            return rc;
    }
    return solve_one(Q, host_q, n, dtype, &o, out, s);
}

// ---- chunked enumeration: host-side bookkeeping ---------------------------

uint64_t fnv1a(const unsigned char *p, size_t len)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < len; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

int q_fingerprint(const void *Q_dev, int n, int dtype, cudaStream_t s, uint64_t *h)
{
    const size_t bytes = dtype_size(dtype) * (size_t)n * n;
    std::vector<unsigned char> buf(bytes);
    QBF_CUDA(cudaMemcpyAsync(buf.data(), Q_dev, bytes, cudaMemcpyDeviceToHost, s), "copy Q");
    QBF_CUDA(cudaStreamSynchronize(s), "fingerprint Q");
    *h = fnv1a(buf.data(), bytes) ^ ((uint64_t)n << 56) ^ ((uint64_t)dtype << 48);
    return QBF_OK;
}

// merge two ascending (value, index) lists into `val`/`idx`, keeping `cap`
int merge_lists(const double *va, const uint64_t *ia, int na, const double *vb,
                const uint64_t *ib, int nb, int cap, double *val, uint64_t *idx)
{
    double tv[2 * QBF_MAX_TOPK];
    uint64_t ti[2 * QBF_MAX_TOPK];
    int a = 0, b = 0, c = 0;
    while (c < cap && (a < na || b < nb)) {
        const bool take_a =
            b >= nb || (a < na && (va[a] < vb[b] || (va[a] == vb[b] && ia[a] < ib[b])));
        if (take_a) {
            tv[c] = va[a];
            ti[c++] = ia[a++];
        } else {
            tv[c] = vb[b];
            ti[c++] = ib[b++];
        }
    }
    for (int i = 0; i < c; ++i) {
        val[i] = tv[i];
        idx[i] = ti[i];
    }
    return c;
}

uint64_t all_shards(int nshards)
{
    return nshards >= 64 ? ~0ull : ((1ull << nshards) - 1);
}

}  // namespace

namespace qbf {
// Lets other translation units of the library report errors through
// qbf_last_error_string().
int record_error(int code, const char *msg) { return set_err(code, msg); }

namespace {
// Cancellation: a host flag (set by qbf_cancel, read by the host after a
// solve) and, per device, a flag word in device memory that the kernels read.
// qbf_cancel writes the device words with the copy engine on a stream of its
// own, so the write lands while a solve's kernels run; a solve clears its
// device word in its own stream before its kernels.
std::mutex g_cancel_mu;
int g_cancel_host = 0;
struct CancelDev {
    int *flag = nullptr;
    cudaStream_t stream = nullptr;
};
std::vector<CancelDev> g_cancel_dev;  // by device
const int g_one = 1;
}  // namespace

const volatile int *cancel_word_dev()
{
    std::lock_guard<std::mutex> lk(g_cancel_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= (int)g_cancel_dev.size()) {
        cudaGetLastError();
        return nullptr;
    }
    return g_cancel_dev[dev].flag;  // allocated by cancel_clear, outside any capture
}

void cancel_clear()
{
    std::lock_guard<std::mutex> lk(g_cancel_mu);
    __atomic_store_n(&g_cancel_host, 0, __ATOMIC_SEQ_CST);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if ((int)g_cancel_dev.size() <= dev)
        g_cancel_dev.resize(dev + 1);
    CancelDev &C = g_cancel_dev[dev];
    if (C.flag)
        return;
    int *f = nullptr;
    cudaStream_t cs = nullptr;
    if (cudaMalloc(&f, sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemset(f, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (f)
            cudaFree(f);
        if (cs)
            cudaStreamDestroy(cs);
        return;  // no cancellation on this device; the solves still run
    }
    C.flag = f;
    C.stream = cs;
}

cudaError_t cancel_reset_async(cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    int *f = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_cancel_mu);
        if (dev < (int)g_cancel_dev.size())
            f = g_cancel_dev[dev].flag;
    }
    return f ? cudaMemsetAsync(f, 0, sizeof(int), s) : cudaSuccess;
}

bool cancel_requested()
{
    return __atomic_load_n(&g_cancel_host, __ATOMIC_SEQ_CST) != 0;
}

void release_cancel()
{
    std::lock_guard<std::mutex> lk(g_cancel_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_cancel_dev.size(); ++d) {
        CancelDev &C = g_cancel_dev[d];
        if (!C.flag && !C.stream)
            continue;
        cudaSetDevice((int)d);
        if (C.stream) {
            cudaStreamSynchronize(C.stream);
            cudaStreamDestroy(C.stream);
        }
        if (C.flag)
            cudaFree(C.flag);
        C = CancelDev();
    }
    cudaSetDevice(cur);
    cudaGetLastError();
}

int cancel_all()
{
    std::lock_guard<std::mutex> lk(g_cancel_mu);
    __atomic_store_n(&g_cancel_host, 1, __ATOMIC_SEQ_CST);
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_cancel_dev.size(); ++d) {
        CancelDev &C = g_cancel_dev[d];
        if (!C.flag)
            continue;
        cudaSetDevice((int)d);
        cudaMemcpyAsync(C.flag, &g_one, sizeof(int), cudaMemcpyHostToDevice, C.stream);
        cudaStreamSynchronize(C.stream);
    }
    cudaSetDevice(cur);
    cudaGetLastError();  // a failed write only delays the stop to the call's end
    return QBF_OK;
}
}  // namespace qbf

extern "C" {

void qbf_default_options(qbf_options *opt)
{
    if (!opt)
        return;
    memset(opt, 0, sizeof(*opt));
    opt->top_k = 1;
    opt->variant = QBF_VARIANT_AUTO;
    opt->prefix_bits = -1;
}

int qbf_solve(const void *Q_dev, int n, int dtype, const qbf_options *opt, qbf_result *out,
              void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return solve_locked(Q_dev, false, n, dtype, opt, out, (cudaStream_t)stream);
}

int qbf_solve_host(const void *Q_host, int n, int dtype, const qbf_options *opt,
                   qbf_result *out, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return solve_locked(Q_host, true, n, dtype, opt, out, (cudaStream_t)stream);
}

int qbf_solve_ising(const void *J_dev, const void *h_dev, int n, int dtype,
                    const qbf_options *opt, qbf_result *out, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (!J_dev || !h_dev || !out)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (n < 1 || n > QBF_MAX_N)
        return set_err(QBF_EINVAL, "n must be in [1, 48]");
    if (dtype_size(dtype) == 0)
        return set_err(QBF_EDTYPE, "unknown dtype");
    const void *Q = nullptr;
    int qdtype = 0, st = QBF_OK;
    double c = 0.0;
    QBF_CUDA(ising_to_qubo(J_dev, h_dev, n, dtype, &Q, &qdtype, &c, &st, s), "ising to qubo");
    if (st != QBF_OK)
        return set_err(QBF_ERANGE, "integer J, h: an entry of 4J + diag(2h - 2R - 2C) leaves int32");
    const int rc = solve_locked(Q, false, n, qdtype, opt, out, s);
    if (rc)
        return rc;
    out->min_value += c;
    for (int i = 0; i < out->top_k; ++i)
        out->topk_value[i] += c;
    return QBF_OK;
}

int qubo_bf_solve(const void *Q_host, int n, int dtype, double *min_value, uint64_t *argmin,
                  int top_k, double *topk_value, uint64_t *topk_index, int *count)
{
    if (!Q_host || !min_value || !argmin)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (top_k < 0 || top_k > QBF_MAX_TOPK)
        return set_err(QBF_EINVAL, "top_k must be in [0, 64]");
    if (top_k > 0 && (!topk_value || !topk_index))
        return set_err(QBF_EINVAL, "null top-k output");
    qbf_options o;
    qbf_default_options(&o);
    o.top_k = top_k > 0 ? top_k : 1;
    qbf_result r;
    int rc;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        rc = solve_locked(Q_host, true, n, dtype, &o, &r, (cudaStream_t)0);
    }
    if (rc)
        return rc;
    *min_value = r.min_value;
    *argmin = r.argmin;
    for (int i = 0; i < top_k && i < r.top_k; ++i) {
        topk_value[i] = r.topk_value[i];
        topk_index[i] = r.topk_index[i];
    }
    if (count)
        *count = top_k > 0 ? std::min(top_k, r.top_k) : 0;
    return QBF_OK;
}

int qbf_chunked_init(qbf_checkpoint *ck, const void *Q_dev, int n, int dtype, int top_k,
                     int chunk_bits, int shard, int nshards, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!ck || !Q_dev)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (n < 2 || n > QBF_MAX_N)
        return set_err(QBF_EINVAL, "n must be in [2, 48]");
    if (dtype_size(dtype) == 0)
        return set_err(QBF_EDTYPE, "unknown dtype");
    if (top_k < 1 || top_k > QBF_MAX_TOPK)
        return set_err(QBF_EINVAL, "top_k must be in [1, 64]");
    if (chunk_bits < 1 || chunk_bits > std::min(n - 1, 24))
        return set_err(QBF_EINVAL, "chunk_bits must be in [1, min(n-1, 24)]");
    if (nshards < 1 || nshards > 64 || shard < 0 || shard >= nshards)
        return set_err(QBF_EINVAL, "need 0 <= shard < nshards <= 64");
    memset(ck, 0, sizeof(*ck));
    ck->version = QBF_CKPT_VERSION;
    ck->n = n;
    ck->dtype = dtype;
    ck->top_k = top_k;
    ck->chunk_bits = chunk_bits;
    ck->shard = shard;
    ck->nshards = nshards;
    if ((uint64_t)shard >= (1ull << chunk_bits))
        ck->done_mask = 1ull << shard;  // no chunk falls to this shard
    return q_fingerprint(Q_dev, n, dtype, (cudaStream_t)stream, &ck->q_hash);
}

int qbf_chunked_step(qbf_checkpoint *ck, const void *Q_dev, const qbf_options *opt,
                     uint64_t max_chunks, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (!ck || !Q_dev)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (ck->version != QBF_CKPT_VERSION || ck->nshards < 1 || ck->nshards > 64)
        return set_err(QBF_EINVAL, "not a checkpoint of this library version");
    uint64_t h = 0;
    int rc = q_fingerprint(Q_dev, ck->n, ck->dtype, s, &h);
    if (rc)
        return rc;
    if (h != ck->q_hash)
        return set_err(QBF_EINVAL, "the checkpoint belongs to another Q");
    const uint64_t nchunks = 1ull << ck->chunk_bits;
    qbf_options o;
    qbf_default_options(&o);
    if (opt)
        o = *opt;
    o.top_k = ck->top_k;
    o.fix_bits = ck->chunk_bits;
    for (uint64_t done = 0; done < max_chunks; ++done) {
        const uint64_t chunk = (uint64_t)ck->shard + ck->next * (uint64_t)ck->nshards;
        if (chunk >= nchunks) {
            ck->done_mask |= 1ull << ck->shard;
            break;
        }
        o.fix_value = chunk;
        qbf_result r;
        if ((rc = solve_locked(Q_dev, false, ck->n, ck->dtype, &o, &r, s)))
            return rc;
        ck->count = merge_lists(ck->best_value, ck->best_index, ck->count, r.topk_value,
                                r.topk_index, r.top_k, ck->top_k, ck->best_value, ck->best_index);
        ck->error_bound = std::max(ck->error_bound, r.error_bound);
        ck->n_candidates += r.n_candidates;
        ck->chunks_done += 1;
        ck->next += 1;
        if ((uint64_t)ck->shard + ck->next * (uint64_t)ck->nshards >= nchunks)
            ck->done_mask |= 1ull << ck->shard;
    }
    return QBF_OK;
}

int qbf_chunked_merge(qbf_checkpoint *into, const qbf_checkpoint *other)
{
    if (!into || !other)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (into->version != QBF_CKPT_VERSION || other->version != QBF_CKPT_VERSION)
        return set_err(QBF_EINVAL, "not a checkpoint of this library version");
    if (into->n != other->n || into->dtype != other->dtype || into->top_k != other->top_k ||
        into->chunk_bits != other->chunk_bits || into->nshards != other->nshards ||
        into->q_hash != other->q_hash)
        return set_err(QBF_EINVAL, "checkpoints of different problems or splits");
    if (!into->done_mask || !other->done_mask)
        return set_err(QBF_EINVAL, "only finished shards merge");
    if (into->done_mask & other->done_mask)
        return set_err(QBF_EINVAL, "the checkpoints share a shard");
    into->count = merge_lists(into->best_value, into->best_index, into->count, other->best_value,
                              other->best_index, other->count, into->top_k, into->best_value,
                              into->best_index);
    into->chunks_done += other->chunks_done;
    into->n_candidates += other->n_candidates;
    into->error_bound = std::max(into->error_bound, other->error_bound);
    into->done_mask |= other->done_mask;
    return QBF_OK;
}

int qbf_chunked_result(const qbf_checkpoint *ck, qbf_result *out)
{
    if (!ck || !out)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (ck->version != QBF_CKPT_VERSION || ck->nshards < 1 || ck->nshards > 64)
        return set_err(QBF_EINVAL, "not a checkpoint of this library version");
    if (ck->done_mask != all_shards(ck->nshards) || ck->chunks_done != (1ull << ck->chunk_bits) ||
        ck->count < 1)
        return set_err(QBF_EINVAL, "chunks are still missing");
    memset(out, 0, sizeof(*out));
    out->top_k = ck->count;
    for (int i = 0; i < ck->count; ++i) {
        out->topk_value[i] = ck->best_value[i];
        out->topk_index[i] = ck->best_index[i];
    }
    out->min_value = ck->best_value[0];
    out->argmin = ck->best_index[0];
    out->error_bound = ck->error_bound;
    out->n_candidates = ck->n_candidates;
    return QBF_OK;
}

int qbf_walk_trace(const void *Q_dev, int n, int dtype, int prefix_bits, uint64_t *idx_dev,
                   int64_t *val_dev, int *sigma_out, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (!Q_dev || !idx_dev || !val_dev || !sigma_out)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (n < 1 || n > 24)
        return set_err(QBF_EINVAL, "trace needs 1 <= n <= 24");
    if (dtype_size(dtype) == 0)
        return set_err(QBF_EDTYPE, "unknown dtype");
    qbf_options o;
    qbf_default_options(&o);
    o.prefix_bits = prefix_bits;
    Geo g;
    int rc = plan_geometry(n, o, &g);
    if (rc)
        return rc;
    const unsigned long long npref = g.p_hi - g.p_lo;
    const Layout L = make_layout(1u << g.M, npref, 0, false);
    Pool *P = nullptr;
    if ((rc = pool_get(L.total, sizeof(DevResult) + sizeof(Plan), &P)))
        return rc;
    char *base = (char *)P->dev;
    if ((rc = enqueue_prepare(Q_dev, n, dtype, g, base, L, s)))
        return rc;
    WalkArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.ns = g.ns;
    a.p_lo = g.p_lo;
    a.p_hi = g.p_hi;
    a.nitems = (npref + 31) / 32;
    a.ctr = (Counters *)(base + L.ctr);
    a.trace_idx = (unsigned long long *)idx_dev;
    a.trace_val = (long long *)val_dev;
    const Plan *plan = (const Plan *)(base + L.plan);
    QBF_CUDA(launch_walk(kModeTrace, g.R, plan, (const Rec *)(base + L.recs), a,
                         walk_grid(g.R, kModeTrace, n, g.ns, a.nitems), s),
             "walk (trace)");
    char *h = (char *)P->host;
    QBF_CUDA(cudaMemcpyAsync(h, plan, offsetof(Plan, lin), cudaMemcpyDeviceToHost, s), "copy plan");
    QBF_CUDA(cudaStreamSynchronize(s), "trace");
    const Plan *PH = (const Plan *)h;
    if (PH->status != QBF_OK)
        return set_err(PH->status, "prepare failed");
    *sigma_out = PH->sigma;
    return QBF_OK;
}

static int prefix_minima_impl(const void *Q_dev, int n, int dtype, int prefix_bits, int variant,
                              int fix_bits, uint64_t fix_value, int32_t *pmin_dev, int *sigma_out,
                              void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (!Q_dev || !pmin_dev || !sigma_out)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (n < 1 || n > QBF_MAX_N)
        return set_err(QBF_EINVAL, "n must be in [1, 48]");
    if (dtype_size(dtype) == 0)
        return set_err(QBF_EDTYPE, "unknown dtype");
    if (prefix_bits < 0)
        return set_err(QBF_EINVAL, "prefix_bits must be given");
    if (variant != QBF_VARIANT_AUTO && variant != QBF_VARIANT_SPLIT && variant != QBF_VARIANT_TC &&
        variant != QBF_VARIANT_SPLIT_F32 && variant != QBF_VARIANT_SPLIT_MIX &&
        variant != QBF_VARIANT_FIELD && variant != QBF_VARIANT_NAIVE &&
        variant != QBF_VARIANT_SPLIT_DEFER)
        return set_err(QBF_ENOTIMPL, "requested walk variant is not built");
    if (fix_bits < 0 || fix_bits > prefix_bits)
        return set_err(QBF_EINVAL, "fix_bits must be in [0, prefix_bits]");
    if (fix_bits < 64 && (fix_value >> fix_bits) != 0)
        return set_err(QBF_EINVAL, "fix_value has bits above fix_bits");
    qbf_options o;
    qbf_default_options(&o);
    o.prefix_bits = prefix_bits;
    o.variant = variant;
    o.fix_bits = fix_bits;
    o.fix_value = fix_value;
    const bool tc = (variant == QBF_VARIANT_TC);
    const bool mix = (variant == QBF_VARIANT_SPLIT_MIX);
    const bool defer = (variant == QBF_VARIANT_SPLIT_DEFER);
    const bool field = (variant == QBF_VARIANT_FIELD);
    const bool naive = (variant == QBF_VARIANT_NAIVE);
    const bool f32 = (variant == QBF_VARIANT_SPLIT_F32) || mix || defer;  // same image bound
    Geo g;
    int rc = plan_geometry(n, o, &g);
    if (rc)
        return rc;
    const size_t ftab = defer ? walk_defer_table_floats(g.R, g.ns_tab) : 0;
    const Layout L = make_layout(1u << g.M, 0, 0, false, ftab);
    Pool *P = nullptr;
    if ((rc = pool_get(L.total, sizeof(DevResult) + sizeof(Plan), &P)))
        return rc;
    char *base = (char *)P->dev;
    if ((rc = enqueue_prepare(Q_dev, n, dtype, g, base, L, s,
                              tc ? kTcVmax : (f32 ? kF32Vmax : (long long)INT_MAX))))
        return rc;
    WalkArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.ns = g.ns;
    a.p_lo = g.p_lo;
    a.p_hi = g.p_hi;
    a.nitems = (g.p_hi - g.p_lo + 31) / 32;
    a.ctr = (Counters *)(base + L.ctr);
    a.pmin = pmin_dev;
    const Plan *plan = (const Plan *)(base + L.plan);
    if (tc)
        QBF_CUDA(launch_tc_min(plan, n, g.p_lo, g.p_hi, pmin_dev, a.ctr, num_sms(), s), "tc (min)");
    else if (field)
        QBF_CUDA(launch_walk_field(plan, a, num_sms(), s), "walk field (min)");
    else if (naive)
        QBF_CUDA(launch_walk_naive(plan, a, num_sms(), s), "naive (min)");
    else if (defer)
        QBF_CUDA(launch_walk_defer(g.R, plan, (const Rec *)(base + L.recs), a,
                                   (const int *)(base + L.kbuf),
                                   base + L.kbuf + sizeof(int) * kKbufInts, num_sms(), s,
                                   ftab ? (float *)(base + L.ftab) : nullptr),
                 "walk defer (min)");
    else if (mix)
        QBF_CUDA(launch_walk_mix(g.R, plan, (const Rec *)(base + L.recs), a,
                                 (const int *)(base + L.kbuf),
                                 (unsigned long long *)(base + L.kbuf + sizeof(int) * kKbufInts),
                                 num_sms(), s),
                 "walk mix (min)");
    else if (f32)
        QBF_CUDA(launch_walk_f32(g.R, plan, (const Rec *)(base + L.recs), a,
                                 (const int *)(base + L.kbuf),
                                 (unsigned long long *)(base + L.kbuf + sizeof(int) * kKbufInts),
                                 num_sms(), s),
                 "walk f32 (min)");
    else
        QBF_CUDA(launch_walk(kModeMin, g.R, plan, (const Rec *)(base + L.recs), a,
                             walk_grid(g.R, kModeMin, n, g.ns, a.nitems), s),
                 "walk (min)");
    char *h = (char *)P->host;
    QBF_CUDA(cudaMemcpyAsync(h, plan, offsetof(Plan, lin), cudaMemcpyDeviceToHost, s), "copy plan");
    QBF_CUDA(cudaStreamSynchronize(s), "prefix minima");
    const Plan *PH = (const Plan *)h;
    if (PH->status != QBF_OK)
        return set_err(PH->status, "prepare failed");
    *sigma_out = PH->sigma;
    return QBF_OK;
}

int qbf_prefix_minima(const void *Q_dev, int n, int dtype, int prefix_bits, int variant,
                      int32_t *pmin_dev, int *sigma_out, void *stream)
{
    return prefix_minima_impl(Q_dev, n, dtype, prefix_bits, variant, 0, 0, pmin_dev, sigma_out,
                              stream);
}

int qbf_prefix_minima_fixed(const void *Q_dev, int n, int dtype, int prefix_bits, int variant,
                            int fix_bits, uint64_t fix_value, int32_t *pmin_dev, int *sigma_out,
                            void *stream)
{
    return prefix_minima_impl(Q_dev, n, dtype, prefix_bits, variant, fix_bits, fix_value,
                              pmin_dev, sigma_out, stream);
}

int qbf_tc_selftest(const uint16_t *A_host, const uint16_t *B_host, float *D_host)
{
    if (!A_host || !B_host || !D_host)
        return set_err(QBF_EINVAL, "null pointer argument");
    std::lock_guard<std::mutex> lk(g_mu);
    int err = 0;
    cudaError_t e = run_tc_selftest(A_host, B_host, D_host, &err);
    if (e != cudaSuccess)
        return cuda_err(e, "tensor-core self-test");
    if (err)
        return set_err(QBF_ECUDA, "tensor-core self-test: the MMA completion wait ran out");
    return QBF_OK;
}

int qbf_alu_microbench(int op, double *ops_per_clk_sm, double *sm_mhz, double *seconds,
                       void *stream)
{
    if (!ops_per_clk_sm || !sm_mhz || !seconds)
        return set_err(QBF_EINVAL, "null pointer argument");
    if (op < 0 || op > 14)
        return set_err(QBF_EINVAL, "op must be in [0, 14]");
    std::lock_guard<std::mutex> lk(g_mu);
    cudaError_t e = run_alu_microbench(op, ops_per_clk_sm, sm_mhz, seconds, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_err(e, "alu microbench");
    return QBF_OK;
}

int qbf_solve_batched(const void *const *Q_dev, const int *n, const int *dtype, int count,
                      const qbf_options *opt, double *min_value, uint64_t *argmin, void *stream)
{
    return solve_batched(Q_dev, n, dtype, count, opt, min_value, argmin, (cudaStream_t)stream,
                         nullptr);
}

int qbf_solve_batched_info(const void *const *Q_dev, const int *n, const int *dtype, int count,
                           const qbf_options *opt, double *min_value, uint64_t *argmin,
                           qbf_batch_info *info, void *stream)
{
    return solve_batched(Q_dev, n, dtype, count, opt, min_value, argmin, (cudaStream_t)stream,
                         nullptr, info, 0);
}

int qbf_solve_batched_item_minima(const void *const *Q_dev, const int *n, const int *dtype,
                                  int count, const qbf_options *opt, int inst, int32_t *item_min,
                                  uint64_t max_items, uint64_t *n_items, qbf_batch_info *info,
                                  void *stream)
{
    if (!n_items)
        return set_err(QBF_EINVAL, "n_items must not be null");
    if (count < 1 || count > QBF_BATCH_MAX_COUNT)
        return set_err(QBF_EINVAL, "count must be in [1, 65536]");
    std::vector<double> vmin(count);
    std::vector<uint64_t> am(count);
    unsigned long long ni = 0;
    const BatchItemsOut out{inst, item_min, (unsigned long long)max_items, &ni};
    const int rc = solve_batched(Q_dev, n, dtype, count, opt, vmin.data(), am.data(),
                                 (cudaStream_t)stream, nullptr, info, 0, &out);
    *n_items = ni;
    return rc;
}

int qbf_tune(int n_min, int n_max, int dtype, const char *cache_path)
{
    return tune_batched_table(n_min, n_max, dtype, cache_path);
}

int qbf_tuned_params(int n, int dtype, int *suffix_bits, int *ctas_per_sm)
{
    return tuned_params(n, dtype, suffix_bits, ctas_per_sm);
}

int qbf_tune_batched(const void *const *Q_dev, const int *n, const int *dtype, int count,
                     int lo_bits, int hi_bits, int *best_bits, double *best_seconds, void *stream)
{
    if (!best_bits || !best_seconds)
        return set_err(QBF_EINVAL, "null pointer argument");
    lo_bits = std::max(lo_bits, kRMax);
    hi_bits = std::min(hi_bits, 18);
    if (lo_bits > hi_bits)
        return set_err(QBF_EINVAL, "empty suffix-width range (valid: 6..18)");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> vmin(count);
    std::vector<uint64_t> am(count);
    int best = -1;
    double best_t = 1e300;
    for (int b = lo_bits; b <= hi_bits; ++b) {
        qbf_options o;
        qbf_default_options(&o);
        o.batch_suffix_bits = b;
        int rc = solve_batched(Q_dev, n, dtype, count, &o, vmin.data(), am.data(), s, nullptr);
        if (rc)
            return rc;
        cudaEvent_t e0, e1;
        QBF_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
        QBF_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
        QBF_CUDA(cudaEventRecord(e0, s), "cudaEventRecord");
        rc = solve_batched(Q_dev, n, dtype, count, &o, vmin.data(), am.data(), s, nullptr);
        QBF_CUDA(cudaEventRecord(e1, s), "cudaEventRecord");
        QBF_CUDA(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc)
            return rc;
        if (ms * 1e-3 < best_t) {
            best_t = ms * 1e-3;
            best = b;
        }
    }
    *best_bits = best;
    *best_seconds = best_t;
    int rc = set_tuned_batch_ns(best);
    if (rc)
        return rc;
    if (const char *path = getenv("QBF_TUNE_CACHE")) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceProp prop;
        memset(&prop, 0, sizeof(prop));
        cudaGetDeviceProperties(&prop, dev);
        if (FILE *f = fopen(path, "a")) {
            for (char *c = prop.name; *c; ++c)
                if (*c == ' ')
                    *c = '_';
            fprintf(f, "%s %d %d %.6f\n", prop.name, nsm, best, best_t);
            fclose(f);
        }
    }
    return QBF_OK;
}

int qbf_logz(const void *Q_dev, int n, int dtype, int batch, const double *beta, int nbeta,
             double *logz, double *min_value, uint64_t *argmin, void *stream)
{
    return logz_forward(Q_dev, n, dtype, batch, beta, nbeta, logz, min_value, argmin,
                        (cudaStream_t)stream);
}

int qbf_logz_backward(const void *Q_dev, int n, int dtype, int batch, const double *beta,
                      int nbeta, const double *upstream_dev, double *grad_dev, double *moment_dev,
                      void *stream)
{
    return logz_backward(Q_dev, n, dtype, batch, beta, nbeta, upstream_dev, grad_dev, moment_dev,
                         (cudaStream_t)stream);
}

int qbf_danskin(const uint64_t *argmin_host, int n, int batch, const double *upstream_dev,
                double *grad_dev, void *stream)
{
    return danskin(argmin_host, n, batch, upstream_dev, grad_dev, (cudaStream_t)stream);
}

const char *qbf_last_error_string(void) { return g_err.c_str(); }

int qbf_cancel(void) { return cancel_all(); }

int qbf_release(void)
{
    release_batched();
    release_logz();
    std::lock_guard<std::mutex> lk(g_mu);
    release_graphs();
    release_cancel();
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_pools.size(); ++d) {
        Pool &P = g_pools[d];
        if (!P.dev && !P.host)
            continue;
        cudaSetDevice((int)d);
        cudaDeviceSynchronize();
        if (P.dev)
            cudaFree(P.dev);
        if (P.host)
            cudaFreeHost(P.host);
        P = Pool();
    }
    cudaSetDevice(cur);
    return QBF_OK;
}

int qbf_version(void) { return 100; }

}  // extern "C"
