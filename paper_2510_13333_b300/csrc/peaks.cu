// Arithmetic-throughput probes for the roofline denominators of the block
// factorization and the dense border factor: FP32 FFMA and FP64 DFMA
// (independent dependent-FMA chains per thread, enough of them to cover the
// pipelines' latency) and FP64 tensor MMA (mma.sync m8n8k4, several
// independent accumulators per warp).  The caller times one launch with CUDA
// events on the stream it passes; the entry point returns the launch's flop
// count.  Not part of the paper's method: measurement support only.
#include <cuda_runtime.h>

#include "../../include/scopf.h"
#include "kernels.h"

namespace {

constexpr int kPT = 256;     // threads per CTA
constexpr int kChains = 8;   // independent FMA chains per thread
constexpr int kAcc = 4;      // independent MMA accumulators per warp

template <typename T>
__global__ void __launch_bounds__(kPT) k_fma_chains(int64_t iters, T *__restrict__ out) {
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
    const T b = (T)0.999999, c = (T)1e-6;
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < kChains; j++) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) s += a[j];
    if (s == (T)-1.2345) out[0] = s;   // never true: keeps the chains live
}

// FP64 FMA chains on lane 0 of every warp only (the other lanes idle): how
// the FP64 pipe charges a warp instruction with one active lane
__global__ void __launch_bounds__(kPT) k_fma_chains_one_lane(int64_t iters, double *__restrict__ out) {
    if ((threadIdx.x & 31) != 0) return;
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = (double)(threadIdx.x + j) * 1e-3;
    const double b = 0.999999, c = 1e-6;
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < kChains; j++) a[j] = fma(a[j], b, c);
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) s += a[j];
    if (s == -1.2345) out[0] = s;
}

__global__ void __launch_bounds__(kPT) k_dmma_chains(int64_t iters, double *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const double a = 1e-3 * (lane + 1), b = 1e-3 * (32 - lane);
    double d[kAcc][2];
#pragma unroll
    for (int j = 0; j < kAcc; j++) d[j][0] = d[j][1] = 0.0;
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < kAcc; j++)
            asm volatile(
                "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                : "+d"(d[j][0]), "+d"(d[j][1])
                : "d"(a), "d"(b));
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < kAcc; j++) s += d[j][0] + d[j][1];
    if (s == -1.2345) out[0] = s;
}

// Even warps run FP64 FMA chains (4 x iters steps), odd warps FP64 MMA
// chains (iters steps): equal flops per warp pair, so the launch takes the
// time of the slower half.  Whether the two FP64 paths share one pipe.
__global__ void __launch_bounds__(kPT) k_fma_and_dmma(int64_t iters, double *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    double s = 0;
    if ((threadIdx.x >> 5) & 1) {
        const double a = 1e-3 * (lane + 1), b = 1e-3 * (32 - lane);
        double d[kAcc][2];
#pragma unroll
        for (int j = 0; j < kAcc; j++) d[j][0] = d[j][1] = 0.0;
        for (int64_t i = 0; i < iters; i++) {
#pragma unroll
            for (int j = 0; j < kAcc; j++)
                asm volatile(
                    "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                    : "+d"(d[j][0]), "+d"(d[j][1])
                    : "d"(a), "d"(b));
        }
#pragma unroll
        for (int j = 0; j < kAcc; j++) s += d[j][0] + d[j][1];
    } else {
        double a[kChains];
#pragma unroll
        for (int j = 0; j < kChains; j++) a[j] = (double)(threadIdx.x + j) * 1e-3;
        const double b = 0.999999, c = 1e-6;
        for (int64_t i = 0; i < 4 * iters; i++) {
#pragma unroll
            for (int j = 0; j < kChains; j++) a[j] = fma(a[j], b, c);
        }
#pragma unroll
        for (int j = 0; j < kChains; j++) s += a[j];
    }
    if (s == -1.2345) out[0] = s;
}

}  // namespace

extern "C" int scopf_peak_probe(int32_t kind, int64_t iters, double *out, void *stream,
                                double *flops) {
    using namespace scopf;
    if (!out || iters <= 0 || kind < 0 || kind > 4) return SCOPF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = sm_count() * (2048 / kPT);
    const double threads = (double)grid * kPT;
    double f = 0;
    if (kind == 0) {
        note_launch(), k_fma_chains<float><<<grid, kPT, 0, s>>>(iters, reinterpret_cast<float *>(out));
        f = threads * kChains * 2.0 * (double)iters;
    } else if (kind == 1) {
        note_launch(), k_fma_chains<double><<<grid, kPT, 0, s>>>(iters, out);
        f = threads * kChains * 2.0 * (double)iters;
    } else if (kind == 2) {
        note_launch(), k_dmma_chains<<<grid, kPT, 0, s>>>(iters, out);
        f = threads / 32.0 * kAcc * (8.0 * 8.0 * 4.0 * 2.0) * (double)iters;
    } else if (kind == 3) {
        note_launch(), k_fma_chains_one_lane<<<grid, kPT, 0, s>>>(iters, out);
        f = threads / 32.0 * kChains * 2.0 * (double)iters;   // active lanes only
    } else {
        note_launch(), k_fma_and_dmma<<<grid, kPT, 0, s>>>(iters, out);
        f = threads / 2.0 * kChains * 2.0 * 4.0 * (double)iters +
            threads / 64.0 * kAcc * (8.0 * 8.0 * 4.0 * 2.0) * (double)iters;
    }
    if (cudaGetLastError() != cudaSuccess) return SCOPF_ERR_CUDA;
    if (flops) *flops = f;
    return SCOPF_OK;
}

extern "C" int scopf_pivot_reciprocal(const double *d, double *out, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!d || !out))) return SCOPF_ERR_INVALID_ARG;
    return scopf::launch_reciprocal(n, d, out, (cudaStream_t)stream) == 0 ? SCOPF_OK
                                                                          : SCOPF_ERR_CUDA;
}
