// Standalone dense LDL^T factor and solve of a symmetric n x n block (FP64),
// the factorization used for the first-stage (border) Schur complement of
// eq. (newtonsystem).  Exposed on its own so that callers and tests can use
// the coupling factor without a model handle.
#include <cuda_runtime.h>

#include "../../include/scopf.h"
#include "dense_ldlt.cuh"
#include "kernels.h"

namespace scopf {

namespace {

constexpr int kDT = 1024;

__global__ void __launch_bounds__(kDT) k_dense_rhs_solve(const double *__restrict__ F, int n,
                                                         const double *__restrict__ b,
                                                         double *__restrict__ x,
                                                         double *__restrict__ y) {
    for (int i = threadIdx.x; i < n; i += kDT) y[i] = b[i];
    __syncthreads();
    block_ldlt_solve<kDT>(F, n, y);
    for (int i = threadIdx.x; i < n; i += kDT) x[i] = y[i];
}

}  // namespace

// F (n x n, column-major, overwritten by L and D), y (n) scratch, st counters
int dense_factor_solve(double *F, int n, const double *b, double *x, double *y, FactorStatus *st,
                       int32_t inertia[3], cudaStream_t s) {
    cudaMemsetAsync(st, 0, sizeof(FactorStatus), s);
    if (launch_dense_ldlt(F, n, st, 0.0, s) != cudaSuccess) return SCOPF_ERR_CUDA;
    note_launch(), k_dense_rhs_solve<<<1, kDT, 0, s>>>(F, n, b, x, y);
    FactorStatus fs;
    cudaMemcpyAsync(&fs, st, sizeof(fs), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return SCOPF_ERR_CUDA;
    if (fs.error) return SCOPF_ERR_TIMEOUT;
    if (inertia) {
        inertia[0] = fs.n_pos;
        inertia[1] = fs.n_neg;
        inertia[2] = fs.n_zero;
    }
    return SCOPF_OK;
}

}  // namespace scopf

extern "C" int scopf_dense_ldlt_solve(const double *S, int32_t n, const double *b, double *x,
                                      int32_t inertia[3], void *stream) {
    using namespace scopf;
    if (n <= 0 || !S || !b || !x) return SCOPF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double *F = nullptr, *y = nullptr;
    FactorStatus *st = nullptr;
    if (cudaMalloc(&F, sizeof(double) * (size_t)n * n) != cudaSuccess) return SCOPF_ERR_OOM;
    if (cudaMalloc(&y, sizeof(double) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&st, sizeof(FactorStatus)) != cudaSuccess) {
        cudaFree(F);
        cudaFree(y);
        return SCOPF_ERR_OOM;
    }
    cudaMemcpyAsync(F, S, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice, s);
    const int r = dense_factor_solve(F, n, b, x, y, st, inertia, s);
    cudaFree(F);
    cudaFree(y);
    cudaFree(st);
    return r;
}
