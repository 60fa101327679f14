// Pivot-free multifrontal LDL^T of every contingency block, Schur complement
// onto the first-stage border, dense LDL^T of the border block, and the
// triangular solves (Section IV-B: the NCL term makes eq. (newtonsystem)
// factorizable without numerical pivoting).
//
// Work decomposition.  Every supernode of every block is one task; tasks are
// stored sorted by (tree level, block, supernode) and a persistent grid of
// warps pulls them from a global counter.  Fronts of these power-grid KKT
// blocks are small (about 14 rows on average, at most the 180-row border plus
// a few pivots), so one warp owns one front: no block-wide barriers, only
// warp shuffles and __syncwarp.  A task waits (bounded poll) until its
// children have published their update blocks, extend-adds them into its
// own dense front, eliminates its pivot columns and publishes.  Because tasks
// are handed out in level order, every awaited child has already been taken
// by a running warp, so the waits always end; a poll limit still turns a
// broken dependency into an error status instead of a hang.
//
// Fronts are dense, column-major, lower triangle used, one slot per
// supernode (HBM is large enough to keep every front resident, so no stack
// management is needed).  The last "supernode" of each block is its border
// front: it receives the trailing updates of the block's roots, i.e. the
// block's contribution -K_ck K_kk^-1 K_kc to the Schur complement.
//
// The matrix handed to the factorization is the symmetric equilibration
// D K D (Ruiz scaling, D > 0 diagonal): the inertia is unchanged (Sylvester)
// and FP32 fronts keep far more accuracy than on the raw barrier-scaled KKT.
#include <cmath>

#include "dense_ldlt.cuh"
#include "kernels.h"

namespace scopf {

namespace {

constexpr int kWT = 128;  // threads per CTA of the warp-task kernels

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- ready queue ----------------------------------------------------------
// Tasks become ready when their dependencies complete (bottom-up: the last
// child pushes its parent; top-down: a parent pushes its children) and are
// appended to a slot array; workers claim slots in order and wait (bounded)
// for a claimed slot to be filled.  Every task is pushed exactly once, so
// slot s is filled by the s-th push.  If every worker waits, all filled
// slots have been claimed and finished, and in a tree that means every task
// is done (an unfinished task has an unfinished descendant, down to a seeded
// leaf); so a wait always ends while the run has work, and workers that have
// not started hold no slot.
struct QueueView {
    int *slots;     // -1 = not yet filled
    int *ctr;       // [0] next slot to claim, [1] next slot to fill
    int *pending;   // outstanding dependencies per task
    int n_items;    // tasks pushed in this run
};

// lane 0 claims a slot and waits for it; returns the task, -1 when the run
// is finished, -2 when the wait ran out (error)
__device__ __forceinline__ int claim_slot(const QueueView &Q, int spin_limit) {
    const int s = atomicAdd(&Q.ctr[0], 1);
    if (s >= Q.n_items) return -1;
    int t, spins = 0;
    while ((t = ld_acquire(&Q.slots[s])) < 0) {
        if (++spins > spin_limit) return -2;
        __nanosleep(32);
    }
    return t;
}

// warp-wide claim: the task id in every lane; the warp barrier orders lane
// 0's acquire before the other lanes' reads of the task's inputs
__device__ __forceinline__ int warp_claim(const QueueView &Q, int spin_limit, FactorStatus *st,
                                          int err) {
    int task = 0;
    if ((threadIdx.x & 31) == 0) {
        task = claim_slot(Q, spin_limit);
        if (task == -2) atomicExch(&st->error, err);
    }
    task = __shfl_sync(0xffffffffu, task, 0);
    __syncwarp();
    return task;
}

__device__ __forceinline__ void push_task(const QueueView &Q, int task) {
    const int s = atomicAdd(&Q.ctr[1], 1);
    st_release(&Q.slots[s], task);
}

// one thread, after a barrier that ordered its group's writes: count the task
// off at its parent; the last child pushes the parent
__device__ __forceinline__ void complete_child(const QueueView &Q, int parent) {
    __threadfence();
    if (atomicSub(&Q.pending[parent], 1) == 1) {
        __threadfence();
        push_task(Q, parent);
    }
}

// whole warp, after __syncwarp: push every child of `task`
__device__ __forceinline__ void push_children(const QueueView &Q, const DevFront &F, int task) {
    const int lane = threadIdx.x & 31;
    const int c0 = F.child_ptr[task], nc = F.child_ptr[task + 1] - c0;
    if (nc == 0) return;
    __threadfence();
    int base = 0;
    if (lane == 0) base = atomicAdd(&Q.ctr[1], nc);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < nc; i += 32) st_release(&Q.slots[base + i], F.child[c0 + i]);
}

// both queues of a run: slots from their seed lists, counters, pending
__global__ void k_queue_reset(int n, int *slots_a, const int32_t *init_a, int n_a, int *slots_b,
                              const int32_t *init_b, int n_b, int *pending,
                              const int32_t *pend, int *ctr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        slots_a[i] = i < n_a ? init_a[i] : -1;
        slots_b[i] = i < n_b ? init_b[i] : -1;
        pending[i] = pend ? pend[i] : 0;
    }
    if (i == 0) {
        ctr[0] = 0;
        ctr[1] = n_a;
        ctr[2] = 0;
        ctr[3] = n_b;
    }
}

QueueView queue_a(const DevFront &F, int n_items) {
    return QueueView{F.q_slots_a, F.q_ctr, F.q_pending, n_items};
}
QueueView queue_b(const DevFront &F, int n_items) {
    return QueueView{F.q_slots_b, F.q_ctr + 2, F.q_pending, n_items};
}

// (column j, row i) of element e of the column-major lower triangle of an
// m x m matrix (diagonal included)
__device__ __forceinline__ void tri_index(int e, int m, int &j, int &i) {
    const float b = 2.0f * m + 1.0f;
    int jj = (int)((b - sqrtf(fmaxf(b * b - 8.0f * (float)e, 0.0f))) * 0.5f);
    if (jj < 0) jj = 0;
    if (jj > m - 1) jj = m - 1;
    int st = jj * m - (jj * (jj - 1)) / 2;
    while (st > e) {
        jj--;
        st = jj * m - (jj * (jj - 1)) / 2;
    }
    while (st + (m - jj) <= e) {
        st += m - jj;
        jj++;
    }
    j = jj;
    i = jj + (e - st);
}

template <int GS>
__device__ __forceinline__ void gsync() {
    if (GS == 32)
        __syncwarp();
    else
        __syncthreads();
}

// Extend-add the children's update blocks into the front, then eliminate
// its np pivot columns without pivoting: panel factorization (rank-1 updates
// restricted to the np panel columns) followed by one pass of the trailing
// update U -= L21 D L21' over the (f - np)^2 lower triangle.  GS threads
// (one warp or one CTA) cooperate; tid in [0, GS).
template <typename T, int GS>
__device__ void eliminate_front(const DevFront &F, T *__restrict__ fronts, int task, int tid,
                                double pivot_tol, int &n_pos, int &n_neg, int &n_zero) {
    T *Fr = fronts + F.front_off[task];
    const int f = F.f[task];
    const int np = F.npiv[task];
    const int c0 = F.child_ptr[task], c1 = F.child_ptr[task + 1];
    // the front's own original entries (scaled), zeros elsewhere
    for (int e = tid; e < f * f; e += GS) Fr[e] = (T)0;
    gsync<GS>();
    for (int64_t q = F.orig_ptr[task] + tid; q < F.orig_ptr[task + 1]; q += GS)
        Fr[F.orig_off[q]] = (T)F.ovals[q];
    gsync<GS>();
    for (int ci = c0; ci < c1; ci++) {
        const int ch = F.child[ci];
        const T *Fc = fronts + F.front_off[ch];
        const int fc = F.f[ch], npc = F.npiv[ch], nu = fc - npc;
        const int32_t *rel = F.rel + F.rel_off[ch];
        const int tot = nu * nu;
        for (int e = tid; e < tot; e += GS) {
            const int jj = e / nu, ii = e - jj * nu;
            if (ii >= jj)
                Fr[(int64_t)rel[jj] * f + rel[ii]] += Fc[(int64_t)(npc + jj) * fc + npc + ii];
        }
        gsync<GS>();
    }
    for (int c = 0; c < np; c++) {
        T *colc = Fr + (int64_t)c * f;
        const T d = colc[c];
        if (tid == 0) {
            const double dd = (double)d;
            if (dd > pivot_tol) n_pos++;
            else if (dd < -pivot_tol) n_neg++;
            else n_zero++;
        }
        const T dinv = (T)1 / (d == (T)0 ? (sizeof(T) == 4 ? (T)1e-30 : (T)1e-300) : d);
        for (int i = c + 1 + tid; i < f; i += GS) colc[i] *= dinv;
        gsync<GS>();
        for (int j = c + 1; j < np; j++) {
            const T lj = colc[j] * d;
            T *colj = Fr + (int64_t)j * f;
            for (int i = j + tid; i < f; i += GS) colj[i] -= colc[i] * lj;
        }
        gsync<GS>();
    }
    const int m = f - np;
    if (np > 0 && m > 0) {
        const int tot = m * m;
        for (int e = tid; e < tot; e += GS) {
            const int jj = e / m, ii = e - jj * m;
            if (ii < jj) continue;
            const int i = np + ii, j = np + jj;
            T acc = 0;
            for (int c = 0; c < np; c++) {
                const T *col = Fr + (int64_t)c * f;
                acc += col[i] * (col[j] * col[c]);
            }
            Fr[(int64_t)j * f + i] -= acc;
        }
        gsync<GS>();
    }
}

// A front with f <= 32 rows held in one warp's shared-memory tile (lane i
// owns row i): originals, extend-add, unblocked right-looking elimination,
// then one coalesced write of the whole front (L panel, D, update block).
template <typename T>
__device__ void eliminate_front_tile(const DevFront &F, T *__restrict__ fronts, int task,
                                     int lane, T (*tile)[33], double pivot_tol, int &n_pos,
                                     int &n_neg, int &n_zero) {
    T *Fr = fronts + F.front_off[task];
    const int f = F.f[task];
    const int np = F.npiv[task];
    const int c0 = F.child_ptr[task], c1 = F.child_ptr[task + 1];
    for (int j = 0; j < 32; j++) tile[lane][j] = (T)0;
    __syncwarp();
    const int64_t o0 = F.orig_ptr[task], o1 = F.orig_ptr[task + 1];
    for (int64_t q = o0 + lane; q < o1; q += 32) {
        const int off = F.orig_off[q];
        const int col = off / f, row = off - col * f;
        tile[row][col] = (T)F.ovals[q];
    }
    __syncwarp();
    for (int ci = c0; ci < c1; ci++) {
        const int ch = F.child[ci];
        const T *Fc = fronts + F.front_off[ch];
        const int fc = F.f[ch], npc = F.npiv[ch], nu = fc - npc;
        const int32_t *rel = F.rel + F.rel_off[ch];
        const int myrel = lane < nu ? rel[lane] : 0;
        // eight independent column loads in flight per step
        for (int j0 = 0; j0 < nu; j0 += 8) {
            T v[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int jj = j0 + k;
                v[k] = (jj < nu && lane >= jj && lane < nu)
                           ? Fc[(int64_t)(npc + jj) * fc + npc + lane] : (T)0;
            }
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int jj = j0 + k;
                const int rj = __shfl_sync(0xffffffffu, myrel, jj & 31);
                if (jj < nu && lane >= jj && lane < nu) tile[myrel][rj] += v[k];
            }
        }
        __syncwarp();
    }
    for (int c = 0; c < np; c++) {
        const T d = tile[c][c];
        if (lane == 0) {
            const double dd = (double)d;
            if (dd > pivot_tol) n_pos++;
            else if (dd < -pivot_tol) n_neg++;
            else n_zero++;
        }
        const T dinv = (T)1 / (d == (T)0 ? (sizeof(T) == 4 ? (T)1e-30 : (T)1e-300) : d);
        T l = (T)0;
        if (lane > c && lane < f) {
            l = tile[lane][c] * dinv;
            tile[lane][c] = l;
        }
        __syncwarp();
        for (int j = c + 1; j < f; j++) {
            const T lj = __shfl_sync(0xffffffffu, l, j) * d;
            if (lane >= j && lane < f) tile[lane][j] -= l * lj;
        }
        __syncwarp();
    }
    for (int j = 0; j < f; j++)
        if (lane < f) Fr[(int64_t)j * f + lane] = tile[lane][j];
}

// Phase 1: small fronts, one warp per front.
template <typename T>
__global__ void __launch_bounds__(kWT) k_factor(DevFront F, T *__restrict__ fronts,
                                                FactorStatus *st, QueueView Q, double pivot_tol,
                                                int spin_limit) {
    __shared__ T tiles[kWT / 32][32][33];
    const int lane = threadIdx.x & 31;
    T (*tile)[33] = tiles[threadIdx.x >> 5];
    int n_pos = 0, n_neg = 0, n_zero = 0;
    while (true) {
        const int task = warp_claim(Q, spin_limit, st, 1);
        if (task < 0) break;
        if (F.f[task] <= 32)
            eliminate_front_tile<T>(F, fronts, task, lane, tile, pivot_tol, n_pos, n_neg, n_zero);
        else
            eliminate_front<T, 32>(F, fronts, task, lane, pivot_tol, n_pos, n_neg, n_zero);
        __syncwarp();
        const int par = F.parent[task];
        if (lane == 0 && par >= 0 && par < F.n_small) complete_child(Q, par);
    }
    if (lane == 0) {
        if (n_pos) atomicAdd(&st->n_pos, n_pos);
        if (n_neg) atomicAdd(&st->n_neg, n_neg);
        if (n_zero) atomicAdd(&st->n_zero, n_zero);
    }
}

// Phase 2: large fronts near the tree tops (they carry the border rows), one
// CTA per front.  Launched after phase 1, so small children are complete.
constexpr int kBT = 256;
constexpr int kBigPanelBytes = 96 * 1024;
constexpr int kBigPanel = kBigPanelBytes / 8;   // panel elements that fit (FP64 bound)

// Large front: zero + originals and extend-add in global memory, then the
// np x f panel is copied to shared memory and eliminated there (rank-1
// updates restricted to the panel columns, columns spread over warps), and
// the trailing update U -= L21 D L21' makes one pass over the update block
// with L read from shared memory.
template <typename T>
__device__ void eliminate_front_big(const DevFront &F, T *__restrict__ fronts, int task,
                                    double pivot_tol, int &n_pos, int &n_neg, int &n_zero) {
    extern __shared__ unsigned char big_smem[];
    T *P = reinterpret_cast<T *>(big_smem);   // P[c * f + i]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kBT >> 5;
    T *Fr = fronts + F.front_off[task];
    const int f = F.f[task];
    const int np = F.npiv[task];
    const int c0 = F.child_ptr[task], c1 = F.child_ptr[task + 1];
    for (int e = tid; e < f * f; e += kBT) Fr[e] = (T)0;
    __syncthreads();
    for (int64_t q = F.orig_ptr[task] + tid; q < F.orig_ptr[task + 1]; q += kBT)
        Fr[F.orig_off[q]] = (T)F.ovals[q];
    __syncthreads();
    for (int ci = c0; ci < c1; ci++) {
        const int ch = F.child[ci];
        const T *Fc = fronts + F.front_off[ch];
        const int fc = F.f[ch], npc = F.npiv[ch], nu = fc - npc;
        const int32_t *rel = F.rel + F.rel_off[ch];
        for (int jj = warp; jj < nu; jj += nw) {
            const int64_t dst = (int64_t)rel[jj] * f;
            const T *src = Fc + (int64_t)(npc + jj) * fc + npc;
            for (int ii = jj + lane; ii < nu; ii += 32) Fr[dst + rel[ii]] += src[ii];
        }
        __syncthreads();
    }
    if (np == 0) return;
    for (int e = tid; e < np * f; e += kBT) P[e] = Fr[e];
    __syncthreads();
    for (int c = 0; c < np; c++) {
        T *colc = P + c * f;
        const T d = colc[c];
        if (tid == 0) {
            const double dd = (double)d;
            if (dd > pivot_tol) n_pos++;
            else if (dd < -pivot_tol) n_neg++;
            else n_zero++;
        }
        const T dinv = (T)1 / (d == (T)0 ? (sizeof(T) == 4 ? (T)1e-30 : (T)1e-300) : d);
        for (int i = c + 1 + tid; i < f; i += kBT) colc[i] *= dinv;
        __syncthreads();
        for (int j = c + 1 + warp; j < np; j += nw) {
            const T lj = colc[j] * d;
            T *colj = P + j * f;
            for (int i = j + lane; i < f; i += 32) colj[i] -= colc[i] * lj;
        }
        __syncthreads();
    }
    for (int e = tid; e < np * f; e += kBT) Fr[e] = P[e];
    const int m = f - np;
    for (int jj = warp; jj < m; jj += nw) {
        const int j = np + jj;
        T *colj = Fr + (int64_t)j * f;
        for (int i = j + lane; i < f; i += 32) {
            T acc = 0;
            for (int c = 0; c < np; c++) acc += P[c * f + i] * (P[c * f + j] * P[c * f + c]);
            colj[i] -= acc;
        }
    }
    __syncthreads();
}
template <typename T>
__global__ void __launch_bounds__(kBT) k_factor_big(DevFront F, T *__restrict__ fronts,
                                                    FactorStatus *st, QueueView Q,
                                                    double pivot_tol, int spin_limit) {
    __shared__ int s_task;
    int n_pos = 0, n_neg = 0, n_zero = 0;
    while (true) {
        if (threadIdx.x == 0) {
            s_task = claim_slot(Q, spin_limit);
            if (s_task == -2) atomicExch(&st->error, 1);
        }
        __syncthreads();
        const int task = s_task;
        __syncthreads();
        if (task < 0) break;
        if ((int64_t)F.f[task] * F.npiv[task] <= kBigPanel)
            eliminate_front_big<T>(F, fronts, task, pivot_tol, n_pos, n_neg, n_zero);
        else
            eliminate_front<T, kBT>(F, fronts, task, threadIdx.x, pivot_tol, n_pos, n_neg, n_zero);
        __syncthreads();   // orders every thread's writes before the release below
        const int par = F.parent[task];
        if (threadIdx.x == 0 && par >= 0) complete_child(Q, par);
    }
    if (threadIdx.x == 0) {
        if (n_pos) atomicAdd(&st->n_pos, n_pos);
        if (n_neg) atomicAdd(&st->n_neg, n_neg);
        if (n_zero) atomicAdd(&st->n_zero, n_zero);
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
    // eight independent partial sums (fixed assignment k mod 8), combined in order
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t off = (int64_t)j * nb + i;
    int k = 0;
    for (; k + 8 <= n_blocks; k += 8) {
#pragma unroll
        for (int u = 0; u < 8; u++) a[u] += (double)fronts[boff[k + u] + off];
    }
    for (int u = 0; k < n_blocks; k++, u++) a[u] += (double)fronts[boff[k] + off];
    const double acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    S[(int64_t)j * nb + i] = acc;
    S[(int64_t)i * nb + j] = acc;
}

// ---- dense LDL^T of the border block (FP64, blocked right-looking) -------
constexpr int kPanel = 32;

// Factor columns [k0, k1) of S in place (rows >= k0), counting inertia.  The
// panel (n - k0 rows x pw columns) is staged in shared memory; panel columns
// are updated by different warps in parallel.
__global__ void k_dense_panel(double *S, int n, int k0, int k1, FactorStatus *st,
                              double pivot_tol) {
    extern __shared__ double P[];   // P[cl * R + il], R = n - k0
    __shared__ int s_pos, s_neg, s_zero;
    const int R = n - k0, pw = k1 - k0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_pos = s_neg = s_zero = 0;
    for (int t = threadIdx.x; t < pw * R; t += blockDim.x) {
        const int cl = t / R, il = t - cl * R;
        P[t] = S[(int64_t)(k0 + cl) * n + k0 + il];
    }
    __syncthreads();
    for (int c = 0; c < pw; c++) {
        double *colc = P + c * R;
        const double d = colc[c];
        if (threadIdx.x == 0) {
            if (d > pivot_tol) s_pos++;
            else if (d < -pivot_tol) s_neg++;
            else s_zero++;
        }
        const double dinv = 1.0 / (d == 0.0 ? 1e-300 : d);
        for (int i = c + 1 + threadIdx.x; i < R; i += blockDim.x) colc[i] *= dinv;
        __syncthreads();
        for (int j = c + 1 + warp; j < pw; j += nw) {
            const double lj = colc[j] * d;
            double *colj = P + j * R;
            for (int i = j + lane; i < R; i += 32) colj[i] -= colc[i] * lj;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < pw * R; t += blockDim.x) {
        const int cl = t / R, il = t - cl * R;
        if (il >= cl) S[(int64_t)(k0 + cl) * n + k0 + il] = P[t];
    }
    if (threadIdx.x == 0) {
        atomicAdd(&st->n_pos, s_pos);
        atomicAdd(&st->n_neg, s_neg);
        atomicAdd(&st->n_zero, s_zero);
    }
}

// Trailing update S[i,j] -= sum_{c in [k0,k1)} L[i,c] d_c L[j,c], i >= j >= k1
// (one 32x32 tile per CTA of the lower triangle)
__global__ void k_dense_trailing(double *S, int n, int k0, int k1) {
    const int tj = blockIdx.x, ti = blockIdx.y;
    if (ti < tj) return;
    __shared__ double Li[kPanel][33], Lj[kPanel][33], dd[kPanel];
    const int pw = k1 - k0;
    const int i0 = k1 + ti * 32, j0 = k1 + tj * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int c = ty; c < pw; c += 8) {
        const double *col = S + (int64_t)(k0 + c) * n;
        Li[c][tx] = (i0 + tx < n) ? col[i0 + tx] : 0.0;
        Lj[c][tx] = (j0 + tx < n) ? col[j0 + tx] : 0.0;
        if (tx == 0) dd[c] = col[k0 + c];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + tx, j = j0 + r;
        if (i >= n || j >= n || i < j) continue;
        double acc = 0.0;
        for (int c = 0; c < pw; c++) acc += Li[c][tx] * dd[c] * Lj[c][r];
        S[(int64_t)j * n + i] -= acc;
    }
}

// ---------------------------------------------------------------- solves
// Forward sweep of one front: gather D b on its pivot rows plus the
// children's update vectors, then y = D^-1 L^-1 (.) on the pivot rows and
// the update vector -L21 y for the parent on the others.
template <typename T>
__device__ __forceinline__ void fwd_front(const DevFront &F, const T *__restrict__ fronts,
                                          T *__restrict__ vec, const double *__restrict__ b,
                                          const double *__restrict__ scale, int task, int lane,
                                          T *sv) {
    const int c0 = F.child_ptr[task], c1 = F.child_ptr[task + 1];
    const int f = F.f[task], np = F.npiv[task];
    const T *L = fronts + F.front_off[task];
    T *v = vec + F.vec_off[task];
    const int64_t *rows = F.rows + F.rows_off[task];
    if (f <= 32) {
        // lane i owns row i; its row of the L panel is prefetched into registers
        T Lr[32];
#pragma unroll
        for (int c = 0; c < 32; c++) Lr[c] = (c < np && lane < f) ? L[(int64_t)c * f + lane] : (T)0;
        const T dl = lane < np ? L[(int64_t)lane * f + lane] : (T)1;
        T vi = (T)0;
        if (lane < np) {
            const int64_t r = rows[lane];
            vi = (T)(scale[r] * b[r]);
        }
        sv[lane] = vi;
        __syncwarp();
        for (int ci = c0; ci < c1; ci++) {
            const int ch = F.child[ci];
            const int nu = F.f[ch] - F.npiv[ch];
            if (lane < nu) sv[F.rel[F.rel_off[ch] + lane]] += vec[F.vec_off[ch] + F.npiv[ch] + lane];
            __syncwarp();
        }
        vi = sv[lane];
#pragma unroll
        for (int c = 0; c < 32; c++) {
            if (c < np) {
                const T xc = __shfl_sync(0xffffffffu, vi, c);
                if (lane > c) vi -= Lr[c] * xc;
            }
        }
        if (lane < np) vi /= dl;
        if (lane < f) v[lane] = vi;
        return;
    }
    for (int i = lane; i < f; i += 32) {
        T x = (T)0;
        if (i < np) {
            const int64_t r = rows[i];
            x = (T)(scale[r] * b[r]);
        }
        v[i] = x;
    }
    __syncwarp();
    for (int ci = c0; ci < c1; ci++) {
        const int ch = F.child[ci];
        const int fc = F.f[ch], npc = F.npiv[ch], nu = fc - npc;
        const T *vc = vec + F.vec_off[ch] + npc;
        const int32_t *rel = F.rel + F.rel_off[ch];
        for (int i = lane; i < nu; i += 32) v[rel[i]] += vc[i];
        __syncwarp();
    }
    for (int c = 0; c < np; c++) {
        const T xc = v[c];
        const T *col = L + (int64_t)c * f;
        for (int i = c + 1 + lane; i < f; i += 32) v[i] -= col[i] * xc;
        __syncwarp();
    }
    // diagonal: y = D^-1 (L^-1 b) on the pivot rows
    for (int c = lane; c < np; c += 32) v[c] = v[c] / L[(int64_t)c * f + c];
}

// bottom-up over every task (border fronts included: they collect the
// block's contribution to the border right-hand side)
template <typename T>
__global__ void __launch_bounds__(kWT) k_solve_fwd(DevFront F, const T *__restrict__ fronts,
                                                   T *__restrict__ vec, const double *__restrict__ b,
                                                   const double *__restrict__ scale, QueueView Q,
                                                   FactorStatus *st, int spin_limit) {
    __shared__ T sv_all[kWT / 32][32];
    const int lane = threadIdx.x & 31;
    T *sv = sv_all[threadIdx.x >> 5];
    while (true) {
        const int task = warp_claim(Q, spin_limit, st, 2);
        if (task < 0) break;
        fwd_front<T>(F, fronts, vec, b, scale, task, lane, sv);
        __syncwarp();
        const int par = F.parent[task];
        if (lane == 0 && par >= 0) complete_child(Q, par);
    }
}

// Border right-hand side y = D b_border + sum_k (update vector of block k's
// border front), then the dense border solve with S = L_S D_S L_S' by one
// warp (column sweeps, warp-shuffle dot products).
constexpr int kBS = 1024;   // threads of the border solve
template <typename T>
__global__ void __launch_bounds__(kBS) k_border_solve(DevFront F, const T *__restrict__ vec,
                                                      const double *__restrict__ S, int n,
                                                      const double *__restrict__ b,
                                                      const double *__restrict__ scale,
                                                      double *__restrict__ x,
                                                      double *__restrict__ y) {
    extern __shared__ double sm[];          // partial sums, then the 32x32 diagonal blocks
    const int tid = threadIdx.x;
    // y = D b_border + sum over blocks of the border update vectors:
    // G groups of threads split the blocks, fixed combination order
    const int G = kBS / n > 0 ? kBS / n : 1;
    for (int t = tid; t < G * n; t += kBS) {
        const int g = t / n, j = t - g * n;
        double a0 = 0, a1 = 0;
        int k = g;
        for (; k + G < F.n_blocks; k += 2 * G) {
            a0 += (double)vec[F.border_vec_off[k] + j];
            a1 += (double)vec[F.border_vec_off[k + G] + j];
        }
        if (k < F.n_blocks) a0 += (double)vec[F.border_vec_off[k] + j];
        sm[t] = a0 + a1;
    }
    __syncthreads();
    for (int j = tid; j < n; j += kBS) {
        const int64_t r = F.border_rows[j];
        double acc = scale[r] * b[r];
        for (int g = 0; g < G; g++) acc += sm[g * n + j];
        y[j] = acc;
    }
    __syncthreads();
    block_ldlt_solve<kBS>(S, n, y);
    for (int j = tid; j < n; j += kBS) {
        const int64_t r = F.border_rows[j];
        x[r] = scale[r] * y[j];
    }
}

// Backward sweep of one (non-border) front: its update rows hold the final
// solution of ancestors and border, the pivot rows solve L11' x = y - L21' x2.
template <typename T>
__device__ __forceinline__ void bwd_front(const DevFront &F, const T *__restrict__ fronts,
                                          T *__restrict__ vec, const double *__restrict__ scale,
                                          double *__restrict__ x, int task, int lane) {
    const int f = F.f[task], np = F.npiv[task];
    const T *L = fronts + F.front_off[task];
    T *v = vec + F.vec_off[task];
    const int64_t *rows = F.rows + F.rows_off[task];
    if (f <= 32) {
        T Lr[32];
#pragma unroll
        for (int c = 0; c < 32; c++) Lr[c] = (c < np && lane < f) ? L[(int64_t)c * f + lane] : (T)0;
        T vi = (T)0;
        int64_t r = 0;
        if (lane < f) r = rows[lane];
        if (lane < np)
            vi = v[lane];
        else if (lane < f)
            vi = (T)(x[r] / scale[r]);
#pragma unroll
        for (int c = 31; c >= 0; c--) {
            if (c < np) {
                T p = (lane > c && lane < f) ? Lr[c] * vi : (T)0;
                for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
                if (lane == c) vi -= p;
            }
        }
        if (lane < np) x[r] = scale[r] * (double)vi;
        return;
    }
    for (int i = np + lane; i < f; i += 32) {
        const int64_t r = rows[i];
        v[i] = (T)(x[r] / scale[r]);
    }
    __syncwarp();
    for (int c = np - 1; c >= 0; c--) {
        const T *col = L + (int64_t)c * f;
        T acc = 0;
        for (int i = c + 1 + lane; i < f; i += 32) acc += col[i] * v[i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) v[c] -= acc;
        __syncwarp();
    }
    for (int c = lane; c < np; c += 32) {
        const int64_t r = rows[c];
        x[r] = scale[r] * (double)v[c];
    }
}

// top-down from the block roots (the border solution is already in x); a
// finished front pushes its children
template <typename T>
__global__ void __launch_bounds__(kWT) k_solve_bwd(DevFront F, const T *__restrict__ fronts,
                                                   T *__restrict__ vec, const double *__restrict__ scale,
                                                   double *__restrict__ x, QueueView Q,
                                                   FactorStatus *st, int spin_limit) {
    const int lane = threadIdx.x & 31;
    while (true) {
        const int task = warp_claim(Q, spin_limit, st, 3);
        if (task < 0) break;
        bwd_front<T>(F, fronts, vec, scale, x, task, lane);
        __syncwarp();
        push_children(Q, F, task);
    }
}

// ---- Ruiz equilibration: s_i <- s_i / sqrt(max_j |s_i K_ij s_j|) ---------
__global__ void k_ruiz(int64_t n, const int64_t *__restrict__ ptr, const int64_t *__restrict__ col,
                       const double *__restrict__ kval, const double *__restrict__ s_in,
                       double *__restrict__ s_out, const int8_t *__restrict__ is_long) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || is_long[i]) return;
    double mx = 0.0;
    const double si = s_in[i];
    for (int64_t q = ptr[i]; q < ptr[i + 1]; q++) mx = fmax(mx, fabs(si * kval[q] * s_in[col[q]]));
    s_out[i] = mx > 0.0 ? si / sqrt(mx) : si;
}

__global__ void k_ruiz_long(int64_t n_long, const int64_t *__restrict__ rows,
                            const int64_t *__restrict__ ptr, const int64_t *__restrict__ col,
                            const double *__restrict__ kval, const double *__restrict__ s_in,
                            double *__restrict__ s_out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_long) return;
    const int64_t i = rows[w];
    const double si = s_in[i];
    double mx = 0.0;
    for (int64_t q = ptr[i] + lane; q < ptr[i + 1]; q += 32)
        mx = fmax(mx, fabs(si * kval[q] * s_in[col[q]]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_out[i] = mx > 0.0 ? si / sqrt(mx) : si;
}

// scaled original entries of every front, in task order
__global__ void k_orig_vals(int64_t n_orig, const int64_t *__restrict__ nz,
                            const int32_t *__restrict__ row, const int64_t *__restrict__ col,
                            const double *__restrict__ scale, const double *__restrict__ kval,
                            double *__restrict__ ovals) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_orig) return;
    const int64_t q = nz[p];
    ovals[p] = scale[row[q]] * kval[q] * scale[col[q]];
}

__global__ void k_fill(int64_t n, double v, double *x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

int warp_grid() {
    static int grid = 0;
    if (!grid) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = sms * (2048 / kWT);
        if (grid <= 0) grid = 148 * 16;
    }
    return grid;
}

}  // namespace

void launch_equilibrate(const DevModel &M, const double *kval, double *scale, double *tmp,
                        int iters, cudaStream_t s) {
    const int t = 256;
    const int64_t n = M.n_kkt;
    const int g = (int)((n + t - 1) / t);
    const int gl = (int)((32 * M.n_long + t - 1) / t);
    k_fill<<<g, t, 0, s>>>(n, 1.0, scale);
    double *a = scale, *b = tmp;
    for (int it = 0; it < iters; it++) {
        k_ruiz<<<g, t, 0, s>>>(n, M.kkt_ptr, M.kkt_col, kval, a, b, M.is_long);
        if (M.n_long)
            k_ruiz_long<<<gl, t, 0, s>>>(M.n_long, M.long_rows, M.kkt_ptr, M.kkt_col, kval, a, b);
        double *c = a;
        a = b;
        b = c;
    }
    if (a != scale) cudaMemcpyAsync(scale, a, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
}

void launch_orig_vals(const DevFront &F, double *ovals, cudaStream_t s) {
    const int t = 256;
    if (F.n_orig > 0)
        k_orig_vals<<<(int)((F.n_orig + t - 1) / t), t, 0, s>>>(F.n_orig, F.orig_nz, F.kkt_row,
                                                               F.kkt_col, F.scale, F.kval, ovals);
}

void launch_queue_reset(const DevFront &F, const int32_t *init_a, int n_a, const int32_t *init_b,
                        int n_b, const int32_t *pend, cudaStream_t s) {
    const int t = 256;
    const int n = F.n_tasks > 0 ? F.n_tasks : 1;
    k_queue_reset<<<(n + t - 1) / t, t, 0, s>>>(F.n_tasks, F.q_slots_a, init_a, n_a, F.q_slots_b,
                                                init_b, n_b, F.q_pending, pend, F.q_ctr);
}

template <typename T>
void launch_factor(const DevFront &F, T *fronts, FactorStatus *st, double pivot_tol,
                   int spin_limit, cudaStream_t s) {
    // queue a: phase 1 (small fronts), queue b: phase 2 (large fronts)
    launch_queue_reset(F, F.init_small, F.n_init_small, F.init_big, F.n_init_big, F.pend_factor, s);
    int grid = warp_grid();
    const int need = (F.n_small + kWT / 32 - 1) / (kWT / 32);
    if (grid > need) grid = need;
    if (F.n_small > 0)
        k_factor<T><<<grid, kWT, 0, s>>>(F, fronts, st, queue_a(F, F.n_small), pivot_tol,
                                         spin_limit);
    const int nbig = F.n_tasks - F.n_small;
    if (nbig > 0) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_factor_big<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kBigPanelBytes);
            cudaFuncSetAttribute(k_factor_big<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kBigPanelBytes);
            attr = true;
        }
        int g2 = sms * 2;
        if (g2 > nbig) g2 = nbig;
        k_factor_big<T><<<g2, kBT, kBigPanelBytes, s>>>(F, fronts, st, queue_b(F, nbig), pivot_tol,
                                                        spin_limit);
    }
}

template <typename T>
void launch_schur_sum(const DevFront &F, const T *fronts, double *S, cudaStream_t s) {
    const int nb = F.n_border;
    if (nb == 0) return;
    k_schur_sum<T><<<(nb * nb + 255) / 256, 256, 0, s>>>(F.n_blocks, nb, F.border_off, fronts, S);
}

void launch_dense_ldlt(double *S, int n, FactorStatus *st, double pivot_tol, cudaStream_t s) {
    for (int k0 = 0; k0 < n; k0 += kPanel) {
        const int k1 = k0 + kPanel < n ? k0 + kPanel : n;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_dense_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr = true;
        }
        k_dense_panel<<<1, 256, sizeof(double) * (size_t)(n - k0) * (k1 - k0), s>>>(S, n, k0, k1, st, pivot_tol);
        const int rem = n - k1;
        if (rem > 0) {
            const int tiles = (rem + 31) / 32;
            k_dense_trailing<<<dim3(tiles, tiles), 256, 0, s>>>(S, n, k0, k1);
        }
    }
}

template <typename T>
void launch_solve(const DevFront &F, const T *fronts, T *vec, const double *S, int nS,
                  const double *scale, const double *b, double *x, double *border_work,
                  FactorStatus *st, int spin_limit, cudaStream_t s) {
    // queue a: forward sweep (all tasks), queue b: backward sweep (non-border)
    launch_queue_reset(F, F.init_fwd, F.n_init_fwd, F.init_bwd, F.n_init_bwd, F.nchild, s);
    int grid = warp_grid();
    const int need = (F.n_tasks + kWT / 32 - 1) / (kWT / 32);
    if (grid > need) grid = need;
    k_solve_fwd<T><<<grid, kWT, 0, s>>>(F, fronts, vec, b, scale, queue_a(F, F.n_tasks), st,
                                        spin_limit);
    {
        const int G = nS > 0 && kBS / nS > 0 ? kBS / nS : 1;
        k_border_solve<T><<<1, kBS, sizeof(double) * (size_t)G * (nS > 0 ? nS : 1), s>>>(
            F, vec, S, nS, b, scale, x, border_work);
    }
    const int nb = F.n_tasks - F.n_blocks;
    if (nb > 0)
        k_solve_bwd<T><<<grid, kWT, 0, s>>>(F, fronts, vec, scale, x, queue_b(F, nb), st,
                                            spin_limit);
}

#define INST(T)                                                                                    \
    template void launch_factor<T>(const DevFront &, T *, FactorStatus *, double, int,           \
                                   cudaStream_t);                                                \
    template void launch_schur_sum<T>(const DevFront &, const T *, double *, cudaStream_t);      \
    template void launch_solve<T>(const DevFront &, const T *, T *, const double *, int,          \
                                  const double *, const double *, double *, double *,             \
                                  FactorStatus *, int, cudaStream_t);
INST(float)
INST(double)

}  // namespace scopf
