// qbf_ising.cu -- Ising-spin input for the solver.
//
// The paper motivates QUBO through its equivalence with the Ising model
// (introduction): with spins s_i = 2 x_i - 1 in {-1, +1},
//     E(s) = s^T J s + h^T s
//          = 4 x^T J x - 2 sum_i x_i (R_i + C_i) + 2 h^T x + sum_ij J_ij - sum_i h_i
// (R_i, C_i: row and column sums of J; x_i^2 = x_i puts the linear terms on
// the diagonal), so E(s) = x^T Q x + c with
//     Q = 4 J + diag(2 h - 2 R - 2 C),   c = sum_ij J_ij - sum_i h_i.
// ising_to_qubo_kernel builds Q and c in a fixed device buffer; the solve then
// runs on Q unchanged, and the caller adds c.  Float J, h give an FP64 Q (the
// off-diagonal entries exactly, the diagonal with one rounding per term);
// integer J, h give an int32 Q computed in int64 and range-checked.
#include <climits>
#include <cstdint>

#include "qbf_internal.cuh"
#include "qbf_kernels.cuh"

namespace qbf {

namespace {

struct IsingScratch {
    double qf[kMaxN * kMaxN];
    int qi[kMaxN * kMaxN];
    double c;
    long long ci;
    int status;
};

__device__ IsingScratch g_ising;

__device__ __forceinline__ double load_f(const void *p, int dtype, int e)
{
    switch (dtype) {
    case QBF_F64: return static_cast<const double *>(p)[e];
    case QBF_F32: return (double) static_cast<const float *>(p)[e];
    case QBF_I32: return (double) static_cast<const int32_t *>(p)[e];
    default: return (double) static_cast<const int16_t *>(p)[e];
    }
}

__device__ __forceinline__ long long load_i(const void *p, int dtype, int e)
{
    return dtype == QBF_I32 ? (long long) static_cast<const int32_t *>(p)[e]
                            : (long long) static_cast<const int16_t *>(p)[e];
}

// One block; thread i < n owns row/column i.  Sums run in a fixed order, so
// the result does not depend on the launch.
__global__ void ising_to_qubo_kernel(const void *J, const void *h, int n, int dtype)
{
    const int i = threadIdx.x;
    const bool is_int = (dtype == QBF_I32 || dtype == QBF_I16);
    __shared__ int bad;
    if (i == 0)
        bad = 0;
    __syncthreads();
    if (i < n) {
        if (is_int) {
            long long rc = 0;
            for (int j = 0; j < n; ++j)
                rc += load_i(J, dtype, i * n + j) + load_i(J, dtype, j * n + i);
            for (int j = 0; j < n; ++j) {
                long long q = 4 * load_i(J, dtype, i * n + j);
                if (j == i)
                    q += 2 * load_i(h, dtype, i) - 2 * rc;
                if (q > INT_MAX || q < -(long long)INT_MAX)
                    atomicExch(&bad, 1);
                g_ising.qi[i * n + j] = (int)q;
            }
        } else {
            double r = 0.0, c = 0.0;
            for (int j = 0; j < n; ++j) {
                r += load_f(J, dtype, i * n + j);
                c += load_f(J, dtype, j * n + i);
            }
            for (int j = 0; j < n; ++j) {
                double q = 4.0 * load_f(J, dtype, i * n + j);
                if (j == i)
                    q = (q + 2.0 * load_f(h, dtype, i)) - (2.0 * r + 2.0 * c);
                g_ising.qf[i * n + j] = q;
            }
        }
    }
    __syncthreads();
    if (i == 0) {
        // c = sum_ij J_ij - sum_i h_i, row by row in natural order
        if (is_int) {
            long long c = 0;
            for (int e = 0; e < n * n; ++e)
                c += load_i(J, dtype, e);
            for (int k = 0; k < n; ++k)
                c -= load_i(h, dtype, k);
            g_ising.ci = c;
            g_ising.c = (double)c;
        } else {
            double c = 0.0;
            for (int e = 0; e < n * n; ++e)
                c += load_f(J, dtype, e);
            for (int k = 0; k < n; ++k)
                c -= load_f(h, dtype, k);
            g_ising.c = c;
        }
        g_ising.status = bad ? QBF_ERANGE : QBF_OK;
    }
}

}  // namespace

cudaError_t ising_to_qubo(const void *J, const void *h, int n, int dtype, const void **Q,
                          int *qdtype, double *c_host, int *status_host, cudaStream_t s)
{
    ising_to_qubo_kernel<<<1, 64, 0, s>>>(J, h, n, dtype);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    IsingScratch *dev = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&dev, g_ising)) != cudaSuccess)
        return e;
    const bool is_int = (dtype == QBF_I32 || dtype == QBF_I16);
    *Q = is_int ? (const void *)dev->qi : (const void *)dev->qf;
    *qdtype = is_int ? QBF_I32 : QBF_F64;
    if ((e = cudaMemcpyAsync(c_host, &dev->c, sizeof(double), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(status_host, &dev->status, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);
}

}  // namespace qbf
