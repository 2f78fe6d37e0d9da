// qbf_microbench.cu -- ALU throughput of the instruction classes the walk uses.
//
// The walk is bound by integer/float ALU issue, not by HBM, so its roofline
// denominator is the number of lane operations an SM retires per clock.
// Each kernel below runs 8 independent dependency chains per thread of one
// instruction class, fills every SM with one wave of resident blocks, and is
// timed with CUDA events.  The result is lane operations per SM clock per SM
// (a packed f32x2 add counts as two; each instruction of a pair counts one).
// The figures count the operations written in PTX: the assembler may merge two
// consecutive dependent mins of a chain into one three-input min, so the
// two-input min classes can read up to twice the instruction rate (in the
// walk kernels every ALU instruction, two- or three-input, holds the pipe two
// cycles, per ncu).  Ops 10-13 (the exponential unit, FP64 add, integer
// multiply-add, int/float conversions) serve the log Z and rescoring rooflines.
#include <cstdint>
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
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qbf
