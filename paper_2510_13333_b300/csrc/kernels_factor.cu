// Pivot-free multifrontal LDL^T of every contingency block, Schur complement
// onto the first-stage border, dense LDL^T of the border block, and the
// triangular solves (Section IV-B: the NCL term makes eq. (newtonsystem)
// factorizable without numerical pivoting).
//
// Work decomposition.  Every supernode of every block is one task; tasks are
// stored sorted by (tree level, block, supernode) and a persistent grid of
// CTAs pulls them from a global counter.  A task waits (bounded poll) until
// its children have published their update blocks, extend-adds them into its
// own dense front, eliminates its pivot columns and publishes.  Because tasks
// are handed out in level order, every awaited child has already been taken
// by a running CTA, so the waits always end; a poll limit still turns a
// broken dependency into an error status instead of a hang.
//
// Fronts are dense, column-major, lower triangle used, one slot per
// supernode (HBM is large enough to keep every front resident, so no stack
// management is needed).  The last "supernode" of each block is its border
// front: it receives the trailing updates of the block's roots, i.e. the
// block's contribution -K_ck K_kk^-1 K_kc to the Schur complement.
#include <cmath>

#include "kernels.h"

namespace scopf {

namespace {

constexpr int kFT = 128;  // threads per task CTA

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until done[dep] == epoch for the given dependencies (thread-parallel).
__device__ bool wait_deps(const int *deps, int ndeps, const int *done, int epoch, int spin_limit) {
    __shared__ int s_fail;
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < ndeps; i += blockDim.x) {
        const int d = deps[i];
        int spins = 0;
        while (ld_acquire(&done[d]) != epoch) {
            if (++spins > spin_limit) {
                atomicExch(&s_fail, 1);
                break;
            }
            __nanosleep(64);
        }
    }
    __syncthreads();
    return s_fail == 0;
}

template <typename T>
__global__ void k_front_scatter(int64_t nnz, const int64_t *__restrict__ map,
                                const double *__restrict__ kval, T *__restrict__ fronts) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nnz) return;
    const int64_t off = map[j];
    if (off >= 0) fronts[off] = (T)kval[j];
}

template <typename T>
__global__ void __launch_bounds__(kFT) k_factor(DevFront F, T *__restrict__ fronts, FactorStatus *st,
                                                int *queue, int *done, int epoch, double pivot_tol,
                                                int spin_limit) {
    __shared__ int s_task;
    __shared__ int s_pos, s_neg, s_zero;
    while (true) {
        if (threadIdx.x == 0) {
            s_task = atomicAdd(queue, 1);
            s_pos = s_neg = s_zero = 0;
        }
        __syncthreads();
        const int task = s_task;
        if (task >= F.n_tasks) break;
        const int c0 = F.child_ptr[task], c1 = F.child_ptr[task + 1];
        if (!wait_deps(F.child + c0, c1 - c0, done, epoch, spin_limit)) {
            if (threadIdx.x == 0) {
                atomicExch(&st->error, 1);
                atomicExch(&st->timeout_task, task);
            }
        }
        T *Fr = fronts + F.front_off[task];
        const int f = F.f[task];
        const int np = F.npiv[task];
        // extend-add the children's update blocks (fixed child order)
        for (int ci = c0; ci < c1; ci++) {
            const int ch = F.child[ci];
            const T *Fc = fronts + F.front_off[ch];
            const int fc = F.f[ch], npc = F.npiv[ch], nu = fc - npc;
            const int32_t *rel = F.rel + F.rel_off[ch];
            const int tot = nu * nu;
            for (int t = threadIdx.x; t < tot; t += blockDim.x) {
                const int jj = t / nu, ii = t - jj * nu;
                if (ii < jj) continue;
                Fr[(int64_t)rel[jj] * f + rel[ii]] += Fc[(int64_t)(npc + jj) * fc + npc + ii];
            }
            __syncthreads();
        }
        // eliminate the pivot columns: rank-1 updates, D diagonal, no pivoting
        for (int c = 0; c < np; c++) {
            const T d = Fr[(int64_t)c * f + c];
            if (threadIdx.x == 0) {
                const double dd = (double)d;
                if (dd > pivot_tol)
                    s_pos++;
                else if (dd < -pivot_tol)
                    s_neg++;
                else
                    s_zero++;
            }
            const T dsafe = (d == (T)0) ? (sizeof(T) == 4 ? (T)1e-30 : (T)1e-300) : d;
            T *colc = Fr + (int64_t)c * f;
            for (int i = c + 1 + threadIdx.x; i < f; i += blockDim.x) colc[i] = colc[i] / dsafe;
            __syncthreads();
            const int mrem = f - c - 1;
            const int tot = mrem * mrem;
            for (int t = threadIdx.x; t < tot; t += blockDim.x) {
                const int jj = t / mrem, ii = t - jj * mrem;
                if (ii < jj) continue;
                const int j = c + 1 + jj, i = c + 1 + ii;
                Fr[(int64_t)j * f + i] -= colc[i] * colc[j] * d;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (s_pos) atomicAdd(&st->n_pos, s_pos);
            if (s_neg) atomicAdd(&st->n_neg, s_neg);
            if (s_zero) atomicAdd(&st->n_zero, s_zero);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release(&done[task], epoch);
    }
}

// S = sum over blocks of the border fronts (lower triangle, fixed block order)
template <typename T>
__global__ void k_schur_sum(int n_blocks, int nb, const int64_t *__restrict__ boff,
                            const T *__restrict__ fronts, double *__restrict__ S) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nb * nb) return;
    const int j = idx / nb, i = idx - j * nb;
    if (i < j) return;
    double acc = 0.0;
    for (int k = 0; k < n_blocks; k++) acc += (double)fronts[boff[k] + (int64_t)j * nb + i];
    S[(int64_t)j * nb + i] = acc;
    S[(int64_t)i * nb + j] = acc;
}

// Dense pivot-free LDL^T of the n x n border block (FP64, one CTA, in place,
// lower triangle: L below the diagonal, D on it).
__global__ void k_dense_ldlt(double *S, int n, FactorStatus *st, double pivot_tol) {
    __shared__ int s_pos, s_neg, s_zero;
    if (threadIdx.x == 0) s_pos = s_neg = s_zero = 0;
    __syncthreads();
    for (int c = 0; c < n; c++) {
        const double d = S[(int64_t)c * n + c];
        if (threadIdx.x == 0) {
            if (d > pivot_tol)
                s_pos++;
            else if (d < -pivot_tol)
                s_neg++;
            else
                s_zero++;
        }
        const double dsafe = d == 0.0 ? 1e-300 : d;
        double *colc = S + (int64_t)c * n;
        for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) colc[i] /= dsafe;
        __syncthreads();
        const int mrem = n - c - 1;
        for (int t = threadIdx.x; t < mrem * mrem; t += blockDim.x) {
            const int jj = t / mrem, ii = t - jj * mrem;
            if (ii < jj) continue;
            const int j = c + 1 + jj, i = c + 1 + ii;
            S[(int64_t)j * n + i] -= colc[i] * colc[j] * d;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&st->n_pos, s_pos);
        atomicAdd(&st->n_neg, s_neg);
        atomicAdd(&st->n_zero, s_zero);
    }
}

// ---------------------------------------------------------------- solves
template <typename T>
__global__ void __launch_bounds__(kFT) k_solve_fwd(DevFront F, const T *__restrict__ fronts,
                                                   T *__restrict__ vec, const double *__restrict__ b,
                                                   int *queue, int *done, int epoch,
                                                   FactorStatus *st, int spin_limit) {
    __shared__ int s_task;
    while (true) {
        if (threadIdx.x == 0) s_task = atomicAdd(queue, 1);
        __syncthreads();
        const int task = s_task;
        if (task >= F.n_tasks) break;
        const int c0 = F.child_ptr[task], c1 = F.child_ptr[task + 1];
        if (!wait_deps(F.child + c0, c1 - c0, done, epoch, spin_limit) && threadIdx.x == 0)
            atomicExch(&st->error, 2);
        const int f = F.f[task], np = F.npiv[task];
        const T *L = fronts + F.front_off[task];
        T *v = vec + F.vec_off[task];
        const int64_t *rows = F.rows + F.rows_off[task];
        for (int i = threadIdx.x; i < f; i += blockDim.x) v[i] = i < np ? (T)b[rows[i]] : (T)0;
        __syncthreads();
        for (int ci = c0; ci < c1; ci++) {
            const int ch = F.child[ci];
            const int fc = F.f[ch], npc = F.npiv[ch], nu = fc - npc;
            const T *vc = vec + F.vec_off[ch];
            const int32_t *rel = F.rel + F.rel_off[ch];
            for (int i = threadIdx.x; i < nu; i += blockDim.x) v[rel[i]] += vc[npc + i];
            __syncthreads();
        }
        for (int c = 0; c < np; c++) {
            const T xc = v[c];
            const T *col = L + (int64_t)c * f;
            for (int i = c + 1 + threadIdx.x; i < f; i += blockDim.x) v[i] -= col[i] * xc;
            __syncthreads();
        }
        // diagonal: y = D^-1 (L^-1 b) on the pivot rows
        for (int c = threadIdx.x; c < np; c += blockDim.x) v[c] = v[c] / L[(int64_t)c * f + c];
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release(&done[task], epoch);
    }
}

// Border right-hand side, then the dense border solve with S = L_S D_S L_S'.
template <typename T>
__global__ void k_border_solve(DevFront F, const T *__restrict__ vec, const double *__restrict__ S,
                               int n, const double *__restrict__ b, double *__restrict__ x,
                               double *__restrict__ y) {
    // y = b_border + sum_k (update vector of block k's border front), fixed order
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double acc = b[F.border_rows[j]];
        for (int t = 0; t < F.n_tasks; t++)
            if (F.is_border[t]) acc += (double)vec[F.vec_off[t] + j];
        y[j] = acc;
    }
    __syncthreads();
    for (int c = 0; c < n; c++) {
        const double yc = y[c];
        for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) y[i] -= S[(int64_t)c * n + i] * yc;
        __syncthreads();
    }
    for (int c = threadIdx.x; c < n; c += blockDim.x) y[c] /= S[(int64_t)c * n + c];
    __syncthreads();
    __shared__ double red[kFT];
    for (int c = n - 1; c >= 0; c--) {
        double acc = 0.0;
        for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) acc += S[(int64_t)c * n + i] * y[i];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) y[c] -= red[0];
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) x[F.border_rows[j]] = y[j];
}

template <typename T>
__global__ void __launch_bounds__(kFT) k_solve_bwd(DevFront F, const T *__restrict__ fronts,
                                                   T *__restrict__ vec, double *__restrict__ x,
                                                   int *queue, int *done, int epoch,
                                                   FactorStatus *st, int spin_limit) {
    __shared__ int s_task;
    __shared__ T red[kFT];
    while (true) {
        if (threadIdx.x == 0) s_task = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_task;
        if (q >= F.n_tasks) break;
        const int task = F.n_tasks - 1 - q;
        if (F.is_border[task]) {
            __syncthreads();
            if (threadIdx.x == 0) st_release(&done[task], epoch);
            continue;
        }
        const int par = F.parent[task];
        if (par >= 0 && !wait_deps(&par, 1, done, epoch, spin_limit) && threadIdx.x == 0)
            atomicExch(&st->error, 3);
        const int f = F.f[task], np = F.npiv[task];
        const T *L = fronts + F.front_off[task];
        T *v = vec + F.vec_off[task];
        const int64_t *rows = F.rows + F.rows_off[task];
        for (int i = np + threadIdx.x; i < f; i += blockDim.x) v[i] = (T)x[rows[i]];
        __syncthreads();
        for (int c = np - 1; c >= 0; c--) {
            const T *col = L + (int64_t)c * f;
            T acc = 0;
            for (int i = c + 1 + threadIdx.x; i < f; i += blockDim.x) acc += col[i] * v[i];
            red[threadIdx.x] = acc;
            __syncthreads();
            for (int s = blockDim.x / 2; s > 0; s >>= 1) {
                if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
                __syncthreads();
            }
            if (threadIdx.x == 0) v[c] -= red[0];
            __syncthreads();
        }
        for (int c = threadIdx.x; c < np; c += blockDim.x) x[rows[c]] = (double)v[c];
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release(&done[task], epoch);
    }
}

int persistent_grid(int threads) {
    static int grid = 0;
    if (!grid) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        per = 2048 / threads;
        if (per > 16) per = 16;
        grid = sms * per;
        if (grid <= 0) grid = 148;
    }
    return grid;
}

}  // namespace

template <typename T>
void launch_front_init(const DevFront &F, const double *kval, T *fronts, cudaStream_t s) {
    cudaMemsetAsync(fronts, 0, sizeof(T) * F.front_elems, s);
    const int t = 256;
    k_front_scatter<T><<<(int)((F.nnz + t - 1) / t), t, 0, s>>>(F.nnz, F.scatter, kval, fronts);
}

template <typename T>
void launch_factor(const DevFront &F, T *fronts, FactorStatus *st, int *queue, int *done, int epoch,
                   double pivot_tol, int spin_limit, cudaStream_t s) {
    cudaMemsetAsync(queue, 0, sizeof(int), s);
    int grid = persistent_grid(kFT);
    if (grid > F.n_tasks) grid = F.n_tasks;
    k_factor<T><<<grid, kFT, 0, s>>>(F, fronts, st, queue, done, epoch, pivot_tol, spin_limit);
}

template <typename T>
void launch_schur_sum(const DevFront &F, const T *fronts, double *S, cudaStream_t s) {
    const int nb = F.n_border;
    if (nb == 0) return;
    k_schur_sum<T><<<(nb * nb + 255) / 256, 256, 0, s>>>(F.n_blocks, nb, F.border_off, fronts, S);
}

void launch_dense_ldlt(double *S, int n, FactorStatus *st, double pivot_tol, cudaStream_t s) {
    if (n == 0) return;
    k_dense_ldlt<<<1, 1024, 0, s>>>(S, n, st, pivot_tol);
}

template <typename T>
void launch_solve(const DevFront &F, const T *fronts, T *vec, const double *S, int nS,
                  const double *b, double *x, double *border_work, int *queue, int *done,
                  int epoch, FactorStatus *st, int spin_limit, cudaStream_t s) {
    int grid = persistent_grid(kFT);
    if (grid > F.n_tasks) grid = F.n_tasks;
    cudaMemsetAsync(queue, 0, sizeof(int), s);
    k_solve_fwd<T><<<grid, kFT, 0, s>>>(F, fronts, vec, b, queue, done, epoch, st, spin_limit);
    k_border_solve<T><<<1, kFT, 0, s>>>(F, vec, S, nS, b, x, border_work);
    cudaMemsetAsync(queue, 0, sizeof(int), s);
    k_solve_bwd<T><<<grid, kFT, 0, s>>>(F, fronts, vec, x, queue, done, epoch + 1, st,
                                        spin_limit);
}

#define INST(T)                                                                                    \
    template void launch_front_init<T>(const DevFront &, const double *, T *, cudaStream_t);      \
    template void launch_factor<T>(const DevFront &, T *, FactorStatus *, int *, int *, int,     \
                                   double, int, cudaStream_t);                                   \
    template void launch_schur_sum<T>(const DevFront &, const T *, double *, cudaStream_t);      \
    template void launch_solve<T>(const DevFront &, const T *, T *, const double *, int,          \
                                  const double *, double *, double *, int *, int *, int,         \
                                  FactorStatus *, int, cudaStream_t);
INST(float)
INST(double)

}  // namespace scopf
