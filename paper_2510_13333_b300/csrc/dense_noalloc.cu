// Dense LDL^T factor + solve of the border (Schur complement) block without
// any device allocation.
//
// Who needs it: callers that must not allocate device memory during the
// call -- for example an application whose device memory is entirely
// reserved by its own pool allocator (so cudaMalloc would fail or fragment
// that pool), or a latency-critical loop that cannot afford the implicit
// device-wide synchronisation of cudaMalloc / cudaFree.  The regular
// scopf_dense_ldlt_solve allocates its scratch on every call; this variant
// uses one statically sized scratch array per device instead.
//
// The scratch is a file-scope __device__ array of
// SCOPF_NOALLOC_MAX_N^2 + SCOPF_NOALLOC_MAX_N doubles plus a status word
// (about 4.7 MB for the maximum order 768).  Every GPU that loads this
// library holds it until the process exits.  Its device address is looked
// up once per device (cudaGetSymbolAddress, with that device current) by the
// first call made on that device.  The address is cached per device ordinal
// for the life of the process, so it goes stale if the caller resets the
// device (cudaDeviceReset) and keeps using the library.  All calls on a device
// share the array and it keeps the last call's contents; each call
// synchronises its stream before returning, so calls can only overlap on the
// GPU when several host threads call at once (on different streams) --
// those race and must be ordered by the caller.
#include <cuda_runtime.h>

#include <atomic>

#include "../../include/scopf.h"
#include "kernels.h"

#define SCOPF_NOALLOC_MAX_N 768

namespace scopf {
int dense_factor_solve(double *F, int n, const double *b, double *x, double *y, FactorStatus *st,
                       int32_t inertia[3], cudaStream_t s);
}

namespace {

constexpr size_t kScratchDoubles =
    (size_t)SCOPF_NOALLOC_MAX_N * SCOPF_NOALLOC_MAX_N + SCOPF_NOALLOC_MAX_N +
    (sizeof(scopf::FactorStatus) + sizeof(double) - 1) / sizeof(double);

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
// Per device ordinal, the array's device address once looked up.  Atomic
// because concurrent first calls from several host threads may all look it
// up; each stores the same value.  The cached address belongs to the CUDA
// context it was taken in: after cudaDeviceReset the next context may place
// the array elsewhere, and the stale entry would be used.
std::atomic<double *> g_scratch_ptr[kMaxDevices];

// device address of the scratch array on the current device (set up once)
int scratch_on_current_device(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SCOPF_ERR_CUDA;
    double *ptr = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!ptr) {
        if (cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
            return SCOPF_ERR_CUDA;
        g_scratch_ptr[dev].store(ptr, std::memory_order_release);
    }
    *out = ptr;
    return SCOPF_OK;
}

}  // namespace

extern "C" int scopf_dense_ldlt_solve_noalloc(const double *S, int32_t n, const double *b,
                                              double *x, int32_t inertia[3], void *stream) {
    using namespace scopf;
    if (!S || !b || !x || n <= 0) return SCOPF_ERR_INVALID_ARG;
    if (n > SCOPF_NOALLOC_MAX_N) return SCOPF_ERR_INVALID_ARG;  // beyond the static scratch
    double *base = nullptr;
    const int r = scratch_on_current_device(&base);
    if (r != SCOPF_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    double *F = base;                                   // n x n factor (copy of S)
    double *y = base + (size_t)SCOPF_NOALLOC_MAX_N * SCOPF_NOALLOC_MAX_N;
    FactorStatus *st = reinterpret_cast<FactorStatus *>(y + SCOPF_NOALLOC_MAX_N);
    if (cudaMemcpyAsync(F, S, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return SCOPF_ERR_CUDA;
    // the status counters are cleared by dense_factor_solve before use
    return dense_factor_solve(F, n, b, x, y, st, inertia, s);
}
