// qbf_microbench.cu -- ALU throughput of the instruction classes the walk uses.
//
// The walk is bound by integer/float ALU issue, not by HBM, so its roofline
// denominator is the number of lane operations an SM retires per clock.
// Each kernel below runs 8 independent dependency chains per thread of one
// instruction class, fills every SM with one wave of resident blocks, and is
// timed with CUDA events and with the blocks' SM cycle counters (read after a
// barrier: warps of one block finish far apart, the first ones early, so a
// single warp's count understates the block's time).  The result is lane
// operations per SM clock per SM
// (a packed f32x2 add counts as two; each instruction of a pair counts one).
// The figures count the operations written in PTX: the assembler may merge two
// consecutive dependent mins of a chain into one three-input min, so the
// two-input min classes can read up to twice the instruction rate (in the
// walk kernels every ALU instruction, two- or three-input, holds the pipe two
// cycles, per ncu).  Ops 10-13 (the exponential unit, FP64 add, integer
// multiply-add, int/float conversions) serve the log Z and rescoring rooflines.
#include <cstdint>
#include <cstring>
#include <vector>

#include "qbf_kernels.cuh"

namespace qbf {

namespace {

constexpr int kMbThreads = 512;
constexpr int kRounds = 16;  // unrolled rounds per iteration, 8 chains each

template <int OP>
__global__ void __launch_bounds__(kMbThreads) alu_kernel(int iters, unsigned seed, unsigned *sink,
                                                         long long *cycles)
{
    int x[8], y[8];
    float f[8], g[8];
    unsigned long long p[8];
    double dd[8];
    const int ia = (int)(seed ^ threadIdx.x), ib = (int)(seed >> 3);
    const float fa = 1.0f + (float)(threadIdx.x & 7) * 1e-7f, fb = 0.999f;
    const unsigned long long pc = ((unsigned long long)__float_as_uint(fa) << 32) | __float_as_uint(fb);
    for (int j = 0; j < 8; ++j) {
        x[j] = (int)(seed * (threadIdx.x + 1)) + j * 7919;
        y[j] = x[j] ^ 0x5bd1e995;
        f[j] = (float)(x[j] & 0xffff) * 1e-3f;
        g[j] = f[j] + 1.0f;
        p[j] = ((unsigned long long)__float_as_uint(f[j]) << 32) | __float_as_uint(g[j]);
        dd[j] = (double)f[j];
    }
    const double da = 1.0000001;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if constexpr (OP == 0 || OP == 8)
                    asm volatile("{.reg .s32 t; add.s32 t, %0, %1; add.s32 %0, t, %2;}"
                                 : "+r"(x[j]) : "r"(ia), "r"(ib));
                if constexpr (OP == 1 || OP == 8)
                    asm volatile("min.s32 %0, %0, %1;" : "+r"(y[j]) : "r"(ia));
                if constexpr (OP == 2)
                    x[j] = __vimin3_s32(x[j], ia, ib + j);
                if constexpr (OP == 3 || OP == 9)
                    asm volatile("add.rn.f32 %0, %0, %1;" : "+f"(f[j]) : "f"(fa));
                if constexpr (OP == 4)
                    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[j]) : "f"(fa), "f"(fb));
                if constexpr (OP == 5 || OP == 9)
                    asm volatile("min.f32 %0, %0, %1;" : "+f"(g[j]) : "f"(fa));
                if constexpr (OP == 6)
                    asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(g[j]) : "f"(fa), "f"(fb));
                if constexpr (OP == 7)
                    asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(p[j]) : "l"(pc));
                if constexpr (OP == 10)  // f <- 2^(-f): stays near 0.64, never folds
                    asm volatile("{.reg .f32 t; neg.f32 t, %0; ex2.approx.ftz.f32 %0, t;}"
                                 : "+f"(f[j]));
                if constexpr (OP == 11)
                    asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(dd[j]) : "d"(da));
                if constexpr (OP == 12)
                    asm volatile("mad.lo.s32 %0, %0, %1, %2;" : "+r"(x[j]) : "r"(ia), "r"(ib));
                if constexpr (OP == 13)  // int -> float -> int chain: one I2F and one F2I
                    asm volatile("{.reg .f32 t; cvt.rn.f32.s32 t, %0; cvt.rzi.s32.f32 %0, t;}"
                                 : "+r"(x[j]));
            }
        }
    }
    __syncthreads();  // the block's time, not its first warp's
    const long long t1 = clock64();
    unsigned acc = 0;
    for (int j = 0; j < 8; ++j)
        acc ^= (unsigned)x[j] ^ (unsigned)y[j] ^ __float_as_uint(f[j]) ^ __float_as_uint(g[j]) ^
               (unsigned)p[j] ^ (unsigned)(p[j] >> 32) ^ (unsigned)__double2loint(dd[j]);
    if (acc == 0x12345678u)
        sink[0] = acc;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = t1 - t0;
}

// Op 14: the step of the table-driven deferred walk with no global memory
// traffic -- per step and thread 4 packed adds of field pairs, the eight-value
// min tree, and per two steps one packed add of an F pair read from shared
// memory and a three-input min into a running minimum -- at the walk's launch
// shape (256 threads, three CTAs per SM).  Its rate is the ceiling of that
// instruction mix on this part, against which the walk's own rate (with its
// block transitions, table staging and per-prefix set-up) is compared.
constexpr int kMixThreads = 256;
__device__ __forceinline__ unsigned long long mx_add(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long mx_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long mx_pack(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void mx_unpack(unsigned long long v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ float mx_min3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ unsigned long long mx_lds(const unsigned long long *p)
{
    unsigned long long r;  // volatile: one load per use, as in the walk
    asm volatile("ld.shared.u64 %0, [%1];" : "=l"(r) : "r"((unsigned)__cvta_generic_to_shared(p)));
    return r;
}
__host__ __device__ constexpr int mx_ctz(int u)
{
    int l = 0;
    while (!((u >> l) & 1))
        ++l;
    return l;
}

__global__ void __launch_bounds__(kMixThreads, 3)
    step_mix_kernel(int blocks, const unsigned long long *init, unsigned *sink, long long *cycles)
{
    __shared__ __align__(16) unsigned long long sF[kMixThreads / 32][32];
    unsigned long long w[4], GF[4][6];
    float m0 = 3e38f, m1 = 3e38f;
    const int b = (threadIdx.x & 63) * 32;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        w[s] = init[b + s];
#pragma unroll
        for (int l = 0; l < 6; ++l)
            GF[s][l] = init[b + 4 + s * 6 + l];
    }
    sF[threadIdx.x >> 5][threadIdx.x & 31] = init[b + (threadIdx.x & 31)];
    __syncwarp();
    const unsigned long long *Fs = sF[threadIdx.x >> 5];
    const long long t0 = clock64();
    for (int B = 0; B < blocks; ++B) {
        float tp = 0.f;
#pragma unroll
        for (int u = 0; u < 64; ++u) {
            if (u > 0) {
                const int l = mx_ctz(u);
                const int nb = ((u ^ (u >> 1)) >> l) & 1;
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    w[s] = (nb ^ (l == 5 ? (B & 1) : 0)) ? mx_add(w[s], GF[s][l])
                                                         : mx_sub(w[s], GF[s][l]);
            }
            float x[8];
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mx_unpack(w[s], x[2 * s], x[2 * s + 1]);
            const float a = mx_min3(x[0], x[1], x[2]), c3 = mx_min3(x[3], x[4], x[5]);
            const float t = fminf(c3, mx_min3(x[6], x[7], a));
            if (u & 1) {
                const unsigned long long y = mx_add(mx_pack(tp, t), mx_lds(Fs + ((u >> 1) & 31)));
                float lo, hi;
                mx_unpack(y, lo, hi);
                if ((u >> 1) & 1)
                    m1 = mx_min3(m1, lo, hi);
                else
                    m0 = mx_min3(m0, lo, hi);
            } else {
                tp = t;
            }
        }
    }
    __syncthreads();  // the block's time, not its first warp's
    const long long t1 = clock64();
    if (__float_as_uint(fminf(m0, m1)) == 0x12345678u)
        sink[0] = 1;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = t1 - t0;
}

cudaError_t run_step_mix(double *value_ops_per_clk_sm, double *sm_mhz, double *seconds,
                         cudaStream_t s)
{
    int dev = 0, nsm = 0, bps = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, step_mix_kernel, kMixThreads,
                                                           0)) != cudaSuccess)
        return e;
    if (bps < 1)
        bps = 1;
    const int grid = nsm * bps, blocks = 2048;
    unsigned *sink = nullptr;
    long long *cyc = nullptr;
    unsigned long long *init = nullptr;
    std::vector<unsigned long long> h_init(64 * 32);
    for (size_t i = 0; i < h_init.size(); ++i) {
        const float a = (float)(i % 97), c = (float)(i % 89);
        unsigned ua, uc;
        memcpy(&ua, &a, 4);
        memcpy(&uc, &c, 4);
        h_init[i] = ((unsigned long long)uc << 32) | ua;
    }
    if ((e = cudaMalloc(&sink, sizeof(unsigned))) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&cyc, sizeof(long long) * grid)) == cudaSuccess &&
        (e = cudaMalloc(&init, sizeof(unsigned long long) * h_init.size())) == cudaSuccess)
        e = cudaMemcpy(init, h_init.data(), sizeof(unsigned long long) * h_init.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(sink);
        cudaFree(cyc);
        cudaFree(init);
        return e;
    }
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    step_mix_kernel<<<grid, kMixThreads, 0, s>>>(4, init, sink, cyc);  // warm-up
    cudaEventRecord(ev0, s);
    step_mix_kernel<<<grid, kMixThreads, 0, s>>>(blocks, init, sink, cyc);
    cudaEventRecord(ev1, s);
    e = cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    std::vector<long long> h(grid);
    if (e == cudaSuccess)
        e = cudaMemcpy(h.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaFree(sink);
    cudaFree(cyc);
    cudaFree(init);
    if (e != cudaSuccess)
        return e;
    double mean_cyc = 0;
    for (long long c : h)
        mean_cyc += (double)c;
    mean_cyc /= grid;
    // 8 states per thread and step, 2 value-ops per state
    const double ops_per_sm = (double)blocks * 64 * 8 * 2 * kMixThreads * bps;
    *value_ops_per_clk_sm = ops_per_sm / mean_cyc;
    *seconds = ms * 1e-3;
    *sm_mhz = mean_cyc / (ms * 1e-3) * 1e-6;
    return cudaSuccess;
}

template <int OP>
cudaError_t run_op(int iters, double *ops_per_clk_sm, double *sm_mhz, double *seconds,
                   cudaStream_t s)
{
    int dev = 0, nsm = 0, bps = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, alu_kernel<OP>, kMbThreads, 0)) !=
        cudaSuccess)
        return e;
    if (bps < 1)
        bps = 1;
    const int grid = nsm * bps;
    unsigned *sink = nullptr;
    long long *cyc = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(unsigned))) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&cyc, sizeof(long long) * grid)) != cudaSuccess) {
        cudaFree(sink);
        return e;
    }
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    alu_kernel<OP><<<grid, kMbThreads, 0, s>>>(8, 12345u, sink, cyc);  // warm-up
    cudaEventRecord(ev0, s);
    alu_kernel<OP><<<grid, kMbThreads, 0, s>>>(iters, 12345u, sink, cyc);
    cudaEventRecord(ev1, s);
    e = cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    std::vector<long long> h(grid);
    if (e == cudaSuccess)
        e = cudaMemcpy(h.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaFree(sink);
    cudaFree(cyc);
    if (e != cudaSuccess)
        return e;
    double mean_cyc = 0;
    for (long long c : h)
        mean_cyc += (double)c;
    mean_cyc /= grid;
    const double ops_per_thread =
        (double)iters * kRounds * 8 * ((OP == 7 || OP == 8 || OP == 9 || OP == 13) ? 2 : 1);
    const double ops_per_sm = ops_per_thread * kMbThreads * bps;
    *ops_per_clk_sm = ops_per_sm / mean_cyc;
    *seconds = ms * 1e-3;
    *sm_mhz = mean_cyc / (ms * 1e-3) * 1e-6;
    return cudaSuccess;
}

}  // namespace

cudaError_t run_alu_microbench(int op, double *ops_per_clk_sm, double *sm_mhz, double *seconds,
                               cudaStream_t s)
{
    const int iters = 20000;
    switch (op) {
    case 0: return run_op<0>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 1: return run_op<1>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 2: return run_op<2>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 3: return run_op<3>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 4: return run_op<4>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 5: return run_op<5>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 6: return run_op<6>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 7: return run_op<7>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 8: return run_op<8>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 9: return run_op<9>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 10: return run_op<10>(iters / 4, ops_per_clk_sm, sm_mhz, seconds, s);
    case 11: return run_op<11>(iters / 16, ops_per_clk_sm, sm_mhz, seconds, s);
    case 12: return run_op<12>(iters, ops_per_clk_sm, sm_mhz, seconds, s);
    case 13: return run_op<13>(iters / 4, ops_per_clk_sm, sm_mhz, seconds, s);
    case 14: return run_step_mix(ops_per_clk_sm, sm_mhz, seconds, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qbf
