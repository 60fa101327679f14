// Pivot-free multifrontal LDL^T of every contingency block, Schur complement
// onto the first-stage border, dense LDL^T of the border block, and the
// triangular solves (Section IV-B: the NCL term makes eq. (newtonsystem)
// factorizable without numerical pivoting).
//
// Work decomposition.  Every supernode of every block is one task (one dense
// front).  Fronts of these power-grid KKT blocks are small (about 14 rows on
// average, at most the 180-row border plus a few pivots), so one warp owns one
// front: no block-wide barriers, only warp shuffles and __syncwarp.  Tasks are
// grouped into work items -- a subtree of up to a few dozen small fronts,
// which one warp runs in postorder with nothing but __syncwarp in between, or
// a single front near the tree tops -- and items are scheduled by ready
// queues: the last child item to finish pushes its parent (factorization,
// forward sweep), a finished item pushes its children (backward sweep).  A
// persistent grid of warps claims items in the order they became ready, so
// no warp ever waits on a dependency; waits on a claimed, not yet filled
// slot are bounded and turn into an error status instead of a hang.
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
#include <algorithm>
#include <climits>
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
// Items become ready when their dependencies complete (bottom-up: the last
// child's worker; top-down: the parent's worker) and are appended to a slot
// array; workers claim slots in order and wait (bounded) for a claimed slot
// to be filled.  The worker that makes an item ready usually runs it itself
// next (the parent after its last child; one child after its parent), so
// dependency chains skip the queue; it then pushes a skip marker in the
// item's place, so every run still fills exactly n_items slots and slot s
// is filled by the s-th push.  If every worker waits, all filled slots have
// been claimed and finished, and in a tree that means every item is done
// (an unfinished item has an unfinished descendant, down to a seeded leaf);
// so a wait always ends while the run has work, and workers that have not
// started hold no slot.
constexpr int kSkip = 0x7fffffff;   // slot value of an item run by continuation
struct QueueView {
    int *slots;     // -1 = not yet filled
    int *ctr;       // [0] next slot to claim, [1] next slot to fill
    int *pending;   // outstanding dependencies per item
    int n_items;    // slots filled in this run
};

// lane 0 claims a slot and waits for it; returns the item, kSkip, -1 when
// the run is finished, -2 when the wait ran out (error)
__device__ __forceinline__ int claim_slot(const QueueView &Q, int spin_limit) {
    const int s = atomicAdd(&Q.ctr[0], 1);
    if (s >= Q.n_items) return -1;
    // exponential backoff (32 ns .. 1 us): idle workers leave the issue
    // slots to the ones that have work
    int t, spins = 0;
    unsigned ns = 32;
    while ((t = ld_acquire(&Q.slots[s])) < 0) {
        if (++spins > spin_limit) return -2;
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
    return t;
}

// warp-wide claim of the next item to run (skip markers are passed over):
// the item in every lane, -1 when the run is finished; the warp barrier
// orders lane 0's acquire before the other lanes' reads of the item's inputs
__device__ __forceinline__ int warp_claim(const QueueView &Q, int spin_limit, FactorStatus *st,
                                          int err) {
    int item = 0;
    if ((threadIdx.x & 31) == 0) {
        do {
            item = claim_slot(Q, spin_limit);
        } while (item == kSkip);
        if (item == -2) {
            atomicExch(&st->error, err);
            item = -1;
        }
    }
    item = __shfl_sync(0xffffffffu, item, 0);
    __syncwarp();
    return item;
}

__device__ __forceinline__ void push_task(const QueueView &Q, int item) {
    const int s = atomicAdd(&Q.ctr[1], 1);
    st_release(&Q.slots[s], item);
}

// one thread, after a barrier that ordered its group's writes: count the
// item off at its parent.  Returns true if it was the last child: the
// caller then runs the parent itself (a skip marker takes its slot; the
// fence after the count orders the other children's writes before the
// caller's reads).
__device__ __forceinline__ bool complete_child(const QueueView &Q, int parent) {
    __threadfence();
    if (atomicSub(&Q.pending[parent], 1) == 1) {
        __threadfence();
        push_task(Q, kSkip);
        return true;
    }
    return false;
}

// warp-wide version: lane 0 counts, every lane learns the outcome
__device__ __forceinline__ bool warp_complete_child(const QueueView &Q, int parent) {
    int last = 0;
    if ((threadIdx.x & 31) == 0) last = complete_child(Q, parent) ? 1 : 0;
    last = __shfl_sync(0xffffffffu, last, 0);
    __syncwarp();
    return last != 0;
}

// whole warp, after __syncwarp: push every child item of `item` except
// `keep` (run next by this warp; a skip marker takes its slot)
__device__ __forceinline__ void push_children(const QueueView &Q, const DevFront &F, int item,
                                              int keep) {
    const int lane = threadIdx.x & 31;
    const int c0 = F.item_child_ptr[item], nc = F.item_child_ptr[item + 1] - c0;
    if (nc == 0) return;
    __threadfence();
    int base = 0;
    if (lane == 0) base = atomicAdd(&Q.ctr[1], nc);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < nc; i += 32) {
        const int c = F.item_child[c0 + i];
        st_release(&Q.slots[base + i], c == keep ? kSkip : c);
    }
}

// the queues of a run: slots from their seed lists, counters, pending
struct QueueSeeds {
    const int32_t *init[3];
    int n[3];
};
__global__ void k_queue_reset(int n, int *slots_a, int *slots_b, int *slots_c, QueueSeeds seeds,
                              int *pending, const int32_t *pend, int *ctr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        slots_a[i] = i < seeds.n[0] ? seeds.init[0][i] : -1;
        slots_b[i] = i < seeds.n[1] ? seeds.init[1][i] : -1;
        slots_c[i] = i < seeds.n[2] ? seeds.init[2][i] : -1;
        pending[i] = pend ? pend[i] : 0;
    }
    if (i < 3) {
        ctr[2 * i] = 0;
        ctr[2 * i + 1] = seeds.n[i];
    }
}

// ---- scheduler trace (see scopf_trace): per item, claim start, claim end,
// finish (device clock, ns) and SM
__device__ __forceinline__ unsigned long long dev_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void trace_item(const DevFront &F, int kind, int item,
                                           unsigned long long tc, unsigned long long ts) {
    unsigned sm;
    asm("mov.u32 %0, %%smid;" : "=r"(sm));
    unsigned long long *r = F.trace + ((size_t)kind * F.n_items + item) * 4;
    r[0] = tc;
    r[1] = ts;
    r[2] = dev_clock_ns();
    r[3] = sm;
}

QueueView queue_a(const DevFront &F, int n_items) {
    return QueueView{F.q_slots_a, F.q_ctr, F.q_pending, n_items};
}
QueueView queue_b(const DevFront &F, int n_items) {
    return QueueView{F.q_slots_b, F.q_ctr + 2, F.q_pending, n_items};
}
QueueView queue_c(const DevFront &F, int n_items) {
    return QueueView{F.q_slots_c, F.q_ctr + 4, F.q_pending, n_items};
}

template <int GS>
__device__ __forceinline__ void gsync() {
    if (GS == 32)
        __syncwarp();
    else
        __syncthreads();
}

// ---- packed records: every thread loads the same words (broadcast loads),
// so a front's whole description arrives in one round trip
struct TaskInfo {
    int64_t front_off, vo;   // vo: offset of the front's rows and vector
    int f, np, c0, c1;       // rows, pivots, child slots [c0, c1)
    int o0, o1, parent;      // original entries [o0, o1)
};
__device__ __forceinline__ int64_t join64(int lo, int hi) {
    return (int64_t)(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo);
}
// an item record of DevFront::item_fwd / item_bwd: the task record, and in
// (e0, e1, e2) words 7, 8, 9
__device__ __forceinline__ TaskInfo item_task(const int4 *rec, int item, int &e0, int &e1,
                                              int &e2) {
    const int4 a = rec[3 * item], b = rec[3 * item + 1], c = rec[3 * item + 2];
    TaskInfo ti;
    ti.front_off = join64(a.x, a.y);
    ti.vo = join64(a.z, a.w);
    ti.f = b.x & 0xffff;
    ti.np = b.x >> 16;
    ti.c0 = b.y;
    ti.c1 = b.z;
    ti.o0 = c.z;
    ti.o1 = c.w;
    ti.parent = -1;
    e0 = b.w;
    e1 = c.x;
    e2 = c.y;
    return ti;
}
__device__ __forceinline__ TaskInfo task_info(const DevFront &F, int t) {
    const int4 a = F.task_rec[2 * t], b = F.task_rec[2 * t + 1], n = F.task_rec[2 * t + 3];
    TaskInfo ti;
    ti.front_off = join64(a.x, a.y);
    ti.vo = join64(a.z, a.w);
    ti.f = b.x & 0xffff;
    ti.np = b.x >> 16;
    ti.c0 = b.y;
    ti.o0 = b.z;
    ti.parent = b.w;
    ti.c1 = n.y;
    ti.o1 = n.z;
    return ti;
}
struct ChildInfo {
    int64_t front_off, vo;
    int rel_off, fc, npc, task;
};
__device__ __forceinline__ ChildInfo child_info(const DevFront &F, int q) {
    const int4 a = F.child_rec[2 * q], b = F.child_rec[2 * q + 1];
    ChildInfo c;
    c.front_off = join64(a.x, a.y);
    c.vo = join64(a.z, a.w);
    c.rel_off = b.x;
    c.fc = b.y & 0xffff;
    c.npc = b.y >> 16;
    c.task = b.z;
    return c;
}

// 1 / d in FP64 by Newton's method for the reciprocal, x <- x (2 - d x) in FMA
// form, two steps from a single-precision seed: the hardware reciprocal of
// d's leading 24 mantissa bits, with d's exponent handled in integer
// arithmetic.  A 2^-23 seed becomes 2^-46 and then exact to rounding: the
// result is within one unit in the last place of the quotient (tested against
// 1.0 / d).  It costs four FP64 instructions, fewer than a full-precision
// division; B300's FP64 pipe charges every warp instruction in full, and the
// pivots' divisions were a large share of the FP64 factorization's
// instructions.  Exponents outside single range (zero, subnormal, huge or
// non-finite d) take the plain division.
__device__ __forceinline__ double rcp_newton(double d) {
    const int hi = __double2hiint(d), lo = __double2loint(d);
    const int e = ((hi >> 20) & 0x7ff) - 1023;
    if (e < -126 || e > 126) return 1.0 / d;
    const unsigned m23 = ((unsigned)(hi & 0xfffff) << 3) | ((unsigned)lo >> 29);
    const float y = __frcp_rn(__uint_as_float(0x3f800000u | m23));   // in (0.5, 1]
    const unsigned fy = __float_as_uint(y);
    const int ey = (int)((fy >> 23) & 0xff) - 127;
    const unsigned my = fy & 0x7fffffu;
    const int rhi = (int)((unsigned)hi & 0x80000000u) | ((ey - e + 1023) << 20) | (int)(my >> 3);
    double r = __hiloint2double(rhi, (int)((my & 7u) << 29));
    double t = fma(-d, r, 1.0);
    r = fma(r, t, r);
    t = fma(-d, r, 1.0);
    return fma(r, t, r);
}

// Inertia count of one pivot.  With a zero tolerance an FP64 pivot is
// classified from its bit pattern (integer instructions: the FP64 pipe is the
// scarce one); zero and NaN count as zero pivots.
template <typename T>
__device__ __forceinline__ void count_pivot(T d, T ptol, bool ptol_zero, int &n_pos, int &n_neg,
                                            int &n_zero) {
    if constexpr (sizeof(T) == 8) {
        if (ptol_zero) {
            const long long b = __double_as_longlong(d);
            const long long a = b & 0x7fffffffffffffffLL;
            if (a == 0 || a > 0x7ff0000000000000LL) n_zero++;
            else if (b > 0) n_pos++;
            else n_neg++;
            return;
        }
    }
    if (d > ptol) n_pos++;
    else if (d < -ptol) n_neg++;
    else n_zero++;
}

// the reciprocal of a pivot (a zero pivot is replaced by a tiny one; it is
// counted as zero by the caller)
template <typename T>
__device__ __forceinline__ T pivot_reciprocal(T d) {
    if constexpr (sizeof(T) == 4) {
        return 1.0f / (d == 0.0f ? 1e-30f : d);
    } else {
        // zero test on the bit pattern (an integer instruction)
        const bool z = (__double_as_longlong(d) << 1) == 0;
        return rcp_newton(z ? 1e-300 : d);
    }
}

__global__ void k_reciprocal(int64_t n, const double *__restrict__ d, double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = rcp_newton(d[i]);
}

// Extend-add the children's update blocks into the front, then eliminate
// its np pivot columns without pivoting: panel factorization (rank-1 updates
// restricted to the np panel columns) followed by one pass of the trailing
// update U -= L21 D L21' over the (f - np)^2 lower triangle.  GS threads
// (one warp or one CTA) cooperate; tid in [0, GS).
template <typename T, int GS>
__device__ void eliminate_front(const DevFront &F, T *__restrict__ fronts, const TaskInfo &ti,
                                int tid, double pivot_tol, int &n_pos, int &n_neg, int &n_zero) {
    const T ptol = (T)pivot_tol;
    const bool ptol_zero = pivot_tol == 0.0;
    T *Fr = fronts + ti.front_off;
    const int f = ti.f;
    const int np = ti.np;
    // the front's own original entries (scaled), zeros elsewhere
    for (int e = tid; e < f * f; e += GS) Fr[e] = (T)0;
    gsync<GS>();
    for (int q = ti.o0 + tid; q < ti.o1; q += GS) Fr[F.orig_off[q]] = static_cast<const T *>(F.ovals)[q];
    gsync<GS>();
    for (int ci = ti.c0; ci < ti.c1; ci++) {
        const ChildInfo c = child_info(F, ci);
        const T *Fc = fronts + c.front_off;
        const int fc = c.fc, npc = c.npc, nu = fc - npc;
        const int32_t *rel = F.rel + c.rel_off;
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
            // counted in the factor precision (no FP64 instructions in FP32 fronts)
            count_pivot<T>(d, ptol, ptol_zero, n_pos, n_neg, n_zero);
        }
        const T dinv = pivot_reciprocal<T>(d);
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

// Rank-1 update of pivot step c restricted to the panel columns, packed for
// FP64: the entries (i, j) with c < j < np, j <= i < f are numbered column
// by column (column u = j - c - 1 holds rows j..f-1 and starts at entry
// u L0 - u (u - 1) / 2, L0 = f - c - 1) and dealt to the lanes 32 at a time,
// so every issued FP64 multiply-add updates an entry (the row-per-lane form
// idles the lanes above each column's diagonal).  Column c holds l = L[., c]
// (already divided by d) and row c of the unused upper triangle holds
// l_j d for the panel columns (column c before it was scaled); the update is
// M[i][j] -= l_i (l_j d).
template <typename T, int S>
__device__ __forceinline__ void panel_update_packed(T (*M)[S], int f, int np, int c, int lane) {
    const int j0 = c + 1, ncol = np - j0, L0 = f - j0;
    if (ncol <= 0) return;
    const int total = ncol * L0 - ncol * (ncol - 1) / 2;
    const float b = 2.0f * (float)L0 + 1.0f;
    for (int e = lane; e < total; e += 32) {
        // column from the quadratic u L0 - u (u - 1) / 2 <= e, then corrected
        int u = (int)(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)e, 0.0f))));
        u = min(max(u, 0), ncol - 1);
        while (u > 0 && u * L0 - u * (u - 1) / 2 > e) u--;
        while (u + 1 < ncol && (u + 1) * L0 - (u + 1) * u / 2 <= e) u++;
        const int j = j0 + u;
        const int i = j + (e - (u * L0 - u * (u - 1) / 2));
        M[i][j] -= M[i][c] * M[c][j];
    }
}

// Column index u of entry e when the lower triangle of an m-column block is
// numbered column by column (column u holds m - u entries and starts at
// u m - u (u - 1) / 2): the root of the quadratic, then corrected in integer
// arithmetic.  e < m (m + 1) / 2.
__device__ __forceinline__ int packed_column(int e, int m) {
    const float b = 2.0f * (float)m + 1.0f;
    int u = (int)(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)e, 0.0f))));
    u = min(max(u, 0), m - 1);
    while (u > 0 && u * m - u * (u - 1) / 2 > e) u--;
    while (u + 1 < m && (u + 1) * m - (u + 1) * u / 2 <= e) u++;
    return u;
}

// Trailing update U -= L21 D L21' of a front held in a shared tile with
// row stride S (lower triangle; columns < np hold L, the diagonal D), for all
// entries np <= j <= i < f.  W = L D is first written to the unused upper
// triangle (W[c][j] at tile[c][j], c < np <= j); then the m (m + 1) / 2
// entries (m = f - np) are numbered column by column and dealt to the lanes
// 32 at a time, one entry per lane: np multiply-adds per entry and no idle
// lanes but in the last round (B300's FP64 pipe charges every warp
// instruction in full, whatever its active lanes).
template <typename T, int S>
__device__ __forceinline__ void trailing_update(T (*tile)[S], int f, int np, int lane) {
    const int m = f - np;
    if (np == 0 || m <= 0) return;
    // W = L D in the upper triangle: FP64 panels stored it at each pivot (the
    // column before scaling), FP32 ones form it here
    if (sizeof(T) == 4)
        for (int c = 0; c < np; c++) {
            const T d = tile[c][c];
            for (int j = np + lane; j < f; j += 32) tile[c][j] = tile[j][c] * d;
        }
    __syncwarp();
    const int total = m * (m + 1) / 2;
    for (int e = lane; e < total; e += 32) {
        const int u = packed_column(e, m);
        const int j = np + u;
        const int i = j + (e - (u * m - u * (u - 1) / 2));
        T acc = (T)0;
#pragma unroll 4
        for (int c = 0; c < np; c++) acc += tile[i][c] * tile[c][j];
        tile[i][j] -= acc;
    }
    __syncwarp();
}

// FP64 extend-add of one child's update block (nu <= 32 rows, lower
// triangle, column stride fc) into a warp's 32-row shared tile.  The entries
// are numbered column by column and dealt to the lanes 32 at a time, so
// every issued FP64 add updates an entry; four rounds' loads are in flight
// together.  rel[i] of the child's update row i is held by lane i.  A
// child's destinations are distinct, and the children are added one after
// another, so every entry's sum keeps the child order.  (The 64-row fronts
// keep the column-by-column extend-add and panel update: with one warp per
// CTA and few CTAs per SM they are latency-bound, and this index arithmetic
// lengthens each round; measured, their FP64 kernel took 16% longer with it.)
__device__ __forceinline__ void extend_add_packed(double (*M)[33], const double *__restrict__ Fc,
                                                  int fc, int nu, int rel, int lane) {
    const int total = nu * (nu + 1) / 2;
    for (int e0 = 0; e0 < total; e0 += 128) {
        int di[4], dj[4];
        double v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int e = e0 + 32 * k + lane;
            int i = 0, j = 0;
            if (e < total) {
                j = packed_column(e, nu);
                i = j + (e - (j * nu - j * (j - 1) / 2));
            }
            di[k] = i;
            dj[k] = j;
            v[k] = e < total ? Fc[(int64_t)j * fc + i] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int ri = __shfl_sync(0xffffffffu, rel, di[k]);
            const int rj = __shfl_sync(0xffffffffu, rel, dj[k]);
            if (e0 + 32 * k + lane < total) M[ri][rj] += v[k];
        }
    }
}

// A front with f <= 32 rows held in one warp's shared-memory tile (lane i
// owns row i): originals, extend-add, unblocked right-looking elimination,
// then one coalesced write of the whole front (L panel, D, update block).
template <typename T>
__device__ void eliminate_front_tile(const DevFront &F, T *__restrict__ fronts, const TaskInfo &ti,
                                     int lane, T (*tile)[33], double pivot_tol, int &n_pos,
                                     int &n_neg, int &n_zero) {
    const T ptol = (T)pivot_tol;
    const bool ptol_zero = pivot_tol == 0.0;
    T *Fr = fronts + ti.front_off;
    const int f = ti.f;
    const int np = ti.np;
    for (int j = 0; j < 32; j++) tile[lane][j] = (T)0;
    __syncwarp();
    for (int q = ti.o0 + lane; q < ti.o1; q += 32) {
        const int off = F.orig_off[q];
        const int col = off / f, row = off - col * f;
        tile[row][col] = static_cast<const T *>(F.ovals)[q];
    }
    __syncwarp();
    for (int ci = ti.c0; ci < ti.c1; ci++) {
        const ChildInfo c = child_info(F, ci);
        const T *Fc = fronts + c.front_off + (int64_t)c.npc * c.fc + c.npc;
        const int fc = c.fc, nu = fc - c.npc;
        const int myrel = lane < nu ? F.rel[c.rel_off + lane] : 0;
        if constexpr (sizeof(T) == 8) {
            // FP64: the update block's entries dealt to the lanes (the pipe
            // charges the whole warp per instruction)
            extend_add_packed(tile, Fc, fc, nu, myrel, lane);
            __syncwarp();
            continue;
        }
        // sixteen independent column loads in flight per step (lane = row)
        for (int j0 = 0; j0 < nu; j0 += 16) {
            T v[16];
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const int jj = j0 + k;
                v[k] = (jj < nu && lane >= jj && lane < nu) ? Fc[(int64_t)jj * fc + lane] : (T)0;
            }
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const int jj = j0 + k;
                const int rj = __shfl_sync(0xffffffffu, myrel, jj & 31);
                if (jj < nu && lane >= jj && lane < nu) tile[myrel][rj] += v[k];
            }
        }
        __syncwarp();
    }
    // panel: the np pivot columns, rank-1 updates restricted to the panel
    for (int c = 0; c < np; c++) {
        const T d = tile[c][c];
        if (lane == 0) {
            // counted in the factor precision (no FP64 instructions in FP32 fronts)
            count_pivot<T>(d, ptol, ptol_zero, n_pos, n_neg, n_zero);
        }
        const T dinv = pivot_reciprocal<T>(d);
        if (sizeof(T) == 8) {
            // column c before scaling is l d: kept in the unused upper
            // triangle for the panel update and as W = L D for the trailing
            // update (no multiply), then scaled to l
            if (lane > c && lane < f) {
                const T a = tile[lane][c];
                tile[c][lane] = a;
                tile[lane][c] = a * dinv;
            }
            __syncwarp();
            panel_update_packed<T, 33>(tile, f, np, c, lane);
            __syncwarp();
            continue;
        }
        T l = (T)0;
        if (lane > c && lane < f) {
            l = tile[lane][c] * dinv;
            tile[lane][c] = l;
        }
        const T ld = l * d;
        __syncwarp();
        for (int j = c + 1; j < np; j++) {
            const T lj = __shfl_sync(0xffffffffu, ld, j);
            if (lane >= j && lane < f) tile[lane][j] -= l * lj;
        }
        __syncwarp();
    }
    trailing_update<T, 33>(tile, f, np, lane);
    for (int j = 0; j < f; j++)
        if (lane < f) Fr[(int64_t)j * f + lane] = tile[lane][j];
}

// A front with 32 < f <= 64 rows: the whole front in a 64 x 65 shared
// buffer (lane owns rows lane and lane + 32), otherwise the same steps as
// the 32-row tile: originals, extend-add, right-looking elimination of the
// np pivots, one coalesced write of the front.
constexpr int kMedF = 64;
template <typename T>
__device__ void eliminate_front_medium(const DevFront &F, T *__restrict__ fronts,
                                       const TaskInfo &ti, int lane, T (*M)[kMedF + 1],
                                       double pivot_tol, int &n_pos, int &n_neg, int &n_zero) {
    const T ptol = (T)pivot_tol;
    const bool ptol_zero = pivot_tol == 0.0;
    T *Fr = fronts + ti.front_off;
    const int f = ti.f, np = ti.np;
    const int i0 = lane, i1 = lane + 32;
    for (int c = 0; c < kMedF; c++) {
        M[i0][c] = (T)0;
        M[i1][c] = (T)0;
    }
    __syncwarp();
    for (int q = ti.o0 + lane; q < ti.o1; q += 32) {
        const int off = F.orig_off[q];
        const int col = off / f, row = off - col * f;
        M[row][col] = static_cast<const T *>(F.ovals)[q];
    }
    __syncwarp();
    for (int ci = ti.c0; ci < ti.c1; ci++) {
        const ChildInfo c = child_info(F, ci);
        const int fc = c.fc, nu = fc - c.npc;
        const T *Fc = fronts + c.front_off + (int64_t)c.npc * fc + c.npc;
        const int32_t *rel = F.rel + c.rel_off;
        const int r0 = lane < nu ? rel[lane] : 0, r1 = lane + 32 < nu ? rel[lane + 32] : 0;
        // kMB columns' loads in flight per step; column jj's map entry comes
        // from the lane holding it (a shuffle)
        constexpr int kMB = sizeof(T) == 4 ? 16 : 8;
        for (int j0 = 0; j0 < nu; j0 += kMB) {
            T v0[kMB], v1[kMB];
#pragma unroll
            for (int k = 0; k < kMB; k++) {
                const int jj = j0 + k;
                v0[k] = (jj < nu && lane < nu && lane >= jj) ? Fc[(int64_t)jj * fc + lane] : (T)0;
                v1[k] = (jj < nu && lane + 32 < nu) ? Fc[(int64_t)jj * fc + lane + 32] : (T)0;
            }
#pragma unroll
            for (int k = 0; k < kMB; k++) {
                const int jj = j0 + k;
                const int rj = __shfl_sync(0xffffffffu, jj < 32 ? r0 : r1, jj & 31);
                if (jj < nu) {
                    if (lane < nu && lane >= jj) M[r0][rj] += v0[k];
                    if (lane + 32 < nu) M[r1][rj] += v1[k];
                }
            }
        }
        __syncwarp();
    }
    for (int c = 0; c < np; c++) {
        const T d = M[c][c];
        if (lane == 0) {
            // counted in the factor precision (no FP64 instructions in FP32 fronts)
            count_pivot<T>(d, ptol, ptol_zero, n_pos, n_neg, n_zero);
        }
        const T dinv = pivot_reciprocal<T>(d);
        if (sizeof(T) == 8) {
            // FP64 runs at a fraction of the FP32 rate: lanes take rows j, j+1, ...
            // of each updated column, so no instruction carries the idle rows
            // above the diagonal (one or two chunks of 32 per column)
            // column c before scaling (l d) into the unused upper triangle:
            // the panel update's l_j d and the trailing update's W = L D
            for (int i = c + 1 + lane; i < f; i += 32) {
                const T a = M[i][c];
                M[c][i] = a;
                M[i][c] = a * dinv;
            }
            __syncwarp();
            for (int j = c + 1; j < np; j++) {   // panel columns only
                const T lj = M[c][j];
                for (int i = j + lane; i < f; i += 32) M[i][j] -= M[i][c] * lj;
            }
            __syncwarp();
            continue;
        }
        T l0 = (T)0, l1 = (T)0;
        if (i0 > c && i0 < f) {
            l0 = M[i0][c] * dinv;
            M[i0][c] = l0;
        }
        if (i1 > c && i1 < f) {
            l1 = M[i1][c] * dinv;
            M[i1][c] = l1;
        }
        __syncwarp();
        for (int j = c + 1; j < np; j++) {   // panel columns only
            const T lj = M[j][c] * d;
            if (i0 >= j && i0 < f) M[i0][j] -= l0 * lj;
            if (i1 >= j && i1 < f) M[i1][j] -= l1 * lj;
        }
        __syncwarp();
    }
    trailing_update<T, kMedF + 1>(M, f, np, lane);
    for (int j = 0; j < f; j++) {
        T *colj = Fr + (int64_t)j * f;
        if (i0 < f) colj[i0] = M[i0][j];
        if (i1 < f) colj[i1] = M[i1][j];
    }
}

// Phase 1: tile-sized fronts, one warp per front (32 x 33 shared tile each).
constexpr int kFT = 256;   // threads per CTA of the warp-per-front phases
template <typename T>
__global__ void __launch_bounds__(kFT, sizeof(T) == 4 ? 4 : 3)
    k_factor(DevFront F, T *__restrict__ fronts, FactorStatus *st, QueueView Q, double pivot_tol,
             int spin_limit) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    const int lane = threadIdx.x & 31;
    T (*tile)[33] = reinterpret_cast<T (*)[33]>(tile_smem) + 32 * (threadIdx.x >> 5);
    int n_pos = 0, n_neg = 0, n_zero = 0;
    int item = -1;
    while (true) {
        const unsigned long long tc = F.trace ? dev_clock_ns() : 0;
        if (item < 0) item = warp_claim(Q, spin_limit, st, 1);
        if (item < 0) break;
        const unsigned long long ts = F.trace ? dev_clock_ns() : 0;
        int t0, t1, par;   // one record load starts the item
        TaskInfo ti = item_task(F.item_fwd, item, t1, t0, par);
        for (int task = t0; task < t1; task++) {
            const TaskInfo nx = task_info(F, task + 1 < t1 ? task + 1 : task);   // prefetch
            if (ti.f <= 32)
                eliminate_front_tile<T>(F, fronts, ti, lane, tile, pivot_tol, n_pos, n_neg,
                                        n_zero);
            else   // not produced by the phase split; kept as a safe fallback
                eliminate_front<T, 32>(F, fronts, ti, lane, pivot_tol, n_pos, n_neg, n_zero);
            __syncwarp();   // the next front of the item reads this one
            ti = nx;
        }
        if (F.trace && lane == 0) trace_item(F, 2, item, tc, ts);
        item = (par >= 0 && par < F.n_items_small && warp_complete_child(Q, par)) ? par : -1;
    }
    if (lane == 0) {
        if (n_pos) atomicAdd(&st->n_pos, n_pos);
        if (n_neg) atomicAdd(&st->n_neg, n_neg);
        if (n_zero) atomicAdd(&st->n_zero, n_zero);
    }
}

// Phase 2: medium fronts and their ancestors (all f <= 64), one warp per
// front with its own 64 x 65 shared front.  FP64 fronts take 33 KB: one
// warp per CTA lets six of them share an SM (four-warp CTAs fit only one).
template <typename T>
constexpr int med_threads() { return sizeof(T) == 4 ? kWT : 32; }
template <typename T>
__global__ void __launch_bounds__(med_threads<T>())
    k_factor_med(DevFront F, T *__restrict__ fronts, FactorStatus *st, QueueView Q,
                 double pivot_tol, int spin_limit) {
    extern __shared__ __align__(16) unsigned char med_smem[];
    const int lane = threadIdx.x & 31;
    T (*M)[kMedF + 1] = reinterpret_cast<T (*)[kMedF + 1]>(med_smem) + kMedF * (threadIdx.x >> 5);
    int n_pos = 0, n_neg = 0, n_zero = 0;
    int item = -1;
    while (true) {
        const unsigned long long tc = F.trace ? dev_clock_ns() : 0;
        if (item < 0) item = warp_claim(Q, spin_limit, st, 1);
        if (item < 0) break;
        const unsigned long long ts = F.trace ? dev_clock_ns() : 0;
        int t0, t1, par;   // one front per item
        const TaskInfo ti = item_task(F.item_fwd, item, t1, t0, par);
        if (ti.f <= kMedF)
            eliminate_front_medium<T>(F, fronts, ti, lane, M, pivot_tol, n_pos, n_neg, n_zero);
        else   // not produced by the phase split; kept as a safe fallback
            eliminate_front<T, 32>(F, fronts, ti, lane, pivot_tol, n_pos, n_neg, n_zero);
        __syncwarp();
        if (F.trace && lane == 0) trace_item(F, 3, item, tc, ts);
        item = (par >= F.n_items_small && par < F.n_items_med && warp_complete_child(Q, par))
                   ? par : -1;
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
// row chunks of 32 per column in one extend-add / trailing-update pass
template <typename T>
__host__ __device__ constexpr int big_chunks() { return sizeof(T) == 4 ? 4 : 2; }
// Shared memory of the large-front kernel: the np x f panel, then per warp
// the products l_j d of its current pair of update columns (2 x big_np), then
// the staged child->parent map of one child.
template <typename T>
__host__ __device__ constexpr size_t big_w_offset(int big_panel) {
    return (sizeof(T) * (size_t)(big_panel > 1 ? big_panel : 1) + 15) & ~(size_t)15;
}
template <typename T>
__host__ __device__ constexpr size_t big_rel_offset(int big_panel, int big_np) {
    return big_w_offset<T>(big_panel) +
           ((sizeof(T) * (size_t)(kBT / 32) * 2 * (size_t)(big_np > 1 ? big_np : 1) + 15) &
            ~(size_t)15);
}

// Large front: zero + originals and extend-add in global memory, then the
// np x f panel is copied to shared memory and eliminated there (rank-1
// updates restricted to the panel columns, columns spread over warps), and
// the trailing update U -= L21 D L21' makes one pass over the update block
// with L read from shared memory.
template <typename T>
__device__ void eliminate_front_big(const DevFront &F, T *__restrict__ fronts, const TaskInfo &ti,
                                    double pivot_tol, int &n_pos, int &n_neg, int &n_zero) {
    const T ptol = (T)pivot_tol;
    const bool ptol_zero = pivot_tol == 0.0;
    extern __shared__ unsigned char big_smem[];
    T *P = reinterpret_cast<T *>(big_smem);   // P[c * f + i]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kBT >> 5;
    constexpr int kEA = big_chunks<T>();
    T *Fr = fronts + ti.front_off;
    const int f = ti.f;
    const int np = ti.np;
    for (int e = tid; e < f * f; e += kBT) Fr[e] = (T)0;
    __syncthreads();
    for (int q = ti.o0 + tid; q < ti.o1; q += kBT) Fr[F.orig_off[q]] = static_cast<const T *>(F.ovals)[q];
    __syncthreads();
    // children's update blocks: the child->parent map is staged in shared
    // memory, and each warp pass takes two columns with up to kEA row chunks
    // of 32 each, all their loads in flight before the adds (a child's
    // destinations are distinct; children are added one after another)
    int *srel = reinterpret_cast<int *>(big_smem + big_rel_offset<T>(F.big_panel, F.big_np));
    for (int ci = ti.c0; ci < ti.c1; ci++) {
        const ChildInfo c = child_info(F, ci);
        const T *Fc = fronts + c.front_off;
        const int fc = c.fc, npc = c.npc, nu = fc - npc;
        const int32_t *rel = F.rel + c.rel_off;
        for (int i = tid; i < nu; i += kBT) srel[i] = rel[i];
        __syncthreads();
        for (int j0 = 2 * warp; j0 < nu; j0 += 2 * nw) {
            const int j1 = j0 + 1;
            const int d0 = srel[j0] * f;
            const int d1 = j1 < nu ? srel[j1] * f : 0;
            const T *s0 = Fc + (int64_t)(npc + j0) * fc + npc;
            const T *s1 = s0 + fc;
            for (int r0 = 0; j0 + r0 < nu; r0 += 32 * kEA) {
                T a[2][kEA], b[2][kEA];
                int q[2][kEA];
#pragma unroll
                for (int k = 0; k < kEA; k++) {
                    const int i0 = j0 + r0 + 32 * k + lane, i1 = i0 + 1;
                    q[0][k] = i0 < nu ? d0 + srel[i0] : -1;
                    q[1][k] = (j1 < nu && i1 < nu) ? d1 + srel[i1] : -1;
                }
#pragma unroll
                for (int k = 0; k < kEA; k++) {
                    const int i0 = j0 + r0 + 32 * k + lane, i1 = i0 + 1;
                    a[0][k] = q[0][k] >= 0 ? s0[i0] : (T)0;
                    a[1][k] = q[1][k] >= 0 ? s1[i1] : (T)0;
                    b[0][k] = q[0][k] >= 0 ? Fr[q[0][k]] : (T)0;
                    b[1][k] = q[1][k] >= 0 ? Fr[q[1][k]] : (T)0;
                }
#pragma unroll
                for (int k = 0; k < kEA; k++) {
                    if (q[0][k] >= 0) Fr[q[0][k]] = b[0][k] + a[0][k];
                    if (q[1][k] >= 0) Fr[q[1][k]] = b[1][k] + a[1][k];
                }
            }
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
            // counted in the factor precision (no FP64 instructions in FP32 fronts)
            count_pivot<T>(d, ptol, ptol_zero, n_pos, n_neg, n_zero);
        }
        const T dinv = pivot_reciprocal<T>(d);
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
    // trailing update: two columns per warp pass, the pass's destination
    // values loaded before the dot products (from the shared panel) run; the
    // column factors l_j d_c are formed once per pass (not once per row)
    T *wb = reinterpret_cast<T *>(big_smem + big_w_offset<T>(F.big_panel)) + warp * 2 * F.big_np;
    for (int j0 = np + 2 * warp; j0 < f; j0 += 2 * nw) {
        const int j1 = j0 + 1;
        T *col0 = Fr + (int64_t)j0 * f;
        T *col1 = col0 + f;
        __syncwarp();
        for (int c = lane; c < np; c += 32) {
            const T dc = P[c * f + c];
            wb[c] = P[c * f + j0] * dc;
            wb[F.big_np + c] = j1 < f ? P[c * f + j1] * dc : (T)0;
        }
        __syncwarp();
        for (int r0 = 0; j0 + r0 < f; r0 += 32 * kEA) {
            T u[2][kEA];
#pragma unroll
            for (int k = 0; k < kEA; k++) {
                const int i0 = j0 + r0 + 32 * k + lane, i1 = i0 + 1;
                u[0][k] = i0 < f ? col0[i0] : (T)0;
                u[1][k] = (j1 < f && i1 < f) ? col1[i1] : (T)0;
            }
#pragma unroll
            for (int k = 0; k < kEA; k++) {
                const int i0 = j0 + r0 + 32 * k + lane, i1 = i0 + 1;
                if (i0 < f) {
                    T a0 = 0, a1 = 0;
                    for (int c = 0; c < np; c++) {
                        const T *pc = P + c * f;
                        a0 += pc[i0] * wb[c];
                        if (j1 < f && i1 < f) a1 += pc[i1] * wb[F.big_np + c];
                    }
                    col0[i0] = u[0][k] - a0;
                    if (j1 < f && i1 < f) col1[i1] = u[1][k] - a1;
                }
            }
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
    if (threadIdx.x == 0) s_task = -1;
    __syncthreads();
    while (true) {
        const unsigned long long tc = F.trace ? dev_clock_ns() : 0;
        if (threadIdx.x == 0 && s_task < 0) {
            int t;
            do {
                t = claim_slot(Q, spin_limit);
            } while (t == kSkip);
            if (t == -2) {
                atomicExch(&st->error, 1);
                t = -1;
            }
            s_task = t;
        }
        __syncthreads();
        const int item = s_task;
        __syncthreads();
        if (item < 0) break;
        const unsigned long long ts = F.trace ? dev_clock_ns() : 0;
        int t0, t1, par;   // one front per large item
        const TaskInfo ti = item_task(F.item_fwd, item, t1, t0, par);
        if ((int64_t)ti.f * ti.np <= F.big_panel)
            eliminate_front_big<T>(F, fronts, ti, pivot_tol, n_pos, n_neg, n_zero);
        else
            eliminate_front<T, kBT>(F, fronts, ti, threadIdx.x, pivot_tol, n_pos, n_neg, n_zero);
        __syncthreads();   // orders every thread's writes before the release below
        if (threadIdx.x == 0) {
            if (F.trace) trace_item(F, 4, item, tc, ts);
            s_task = (par >= 0 && complete_child(Q, par)) ? par : -1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (n_pos) atomicAdd(&st->n_pos, n_pos);
        if (n_neg) atomicAdd(&st->n_neg, n_neg);
        if (n_zero) atomicAdd(&st->n_zero, n_zero);
    }
}

// S = sum over blocks of the border fronts (lower triangle, fixed block
// order): block k goes to partial sum k mod 8 (in increasing k), and the
// eight partials are combined as ((p0 + p1) + (p2 + p3)) + ((p4 + p5) +
// (p6 + p7)).  A CTA takes 32 entries: warp u forms partial u of all 32
// (coalesced loads), warp 0 combines.
template <typename T>
__global__ void __launch_bounds__(256) k_schur_sum(int n_blocks, int nb,
                                                   const int64_t *__restrict__ boff,
                                                   const T *__restrict__ fronts,
                                                   double *__restrict__ S) {
    __shared__ double part[8][32];
    const int u = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int idx = blockIdx.x * 32 + lane;   // entry j * nb + i
    const bool in = idx < nb * nb;
    const int j = in ? idx / nb : 0, i = in ? idx - j * nb : 0;
    const bool lower = in && i >= j;
    double a = 0.0;
    if (lower) {
        const int64_t off = (int64_t)j * nb + i;
        for (int k = u; k < n_blocks; k += 8) a += (double)fronts[boff[k] + off];
    }
    part[u][lane] = a;
    __syncthreads();
    if (u == 0 && lower) {
        const double acc = ((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) +
                           ((part[4][lane] + part[5][lane]) + (part[6][lane] + part[7][lane]));
        S[(int64_t)j * nb + i] = acc;
        S[(int64_t)i * nb + j] = acc;
    }
}

// ---- dense LDL^T of the border block (FP64, blocked right-looking) -------
// One cooperative launch of G co-resident CTAs.  Per panel of kDB columns:
//  A. every CTA loads the kDB x kDB diagonal block and factors it in shared
//     memory (tiny; CTA 0 counts the inertia and writes it back), so no
//     barrier is needed before.  Column by column, the entries of the
//     trailing triangle are updated by 120 threads at once (one entry each,
//     one warp per SM sub-partition: on B300 an FP64 warp instruction holds
//     the sub-partition's FP64 pipe for its full width whatever its active
//     lanes, so the chain of pivots costs a few FP64 instructions each);
//  B. the rows below are solved for W = L21 D = A21 L11^-T, two rows per
//     warp (a half-warp per row, a lane per column: the forward substitution
//     is one FMA per step across the lanes), spread over the grid's warps,
//     and L21 = W D^-1 is stored;
//  C. after a grid barrier, the trailing matrix takes the rank-kDB update
//     A22 -= L21 D L21' in 32 x 32 tiles of its lower triangle, dealt to the
//     CTAs; a second barrier ends the panel.
// The grid barriers are bounded waits: a wait that runs out sets
// st->error and every CTA then leaves without waiting again.
constexpr int kDB = 16;     // panel width
constexpr int kDT = 256;    // threads per CTA
constexpr int kDTri = kDB * (kDB - 1) / 2;   // entries (r, j), 1 <= j <= r < kDB

__device__ __forceinline__ bool dense_grid_barrier(FactorStatus *st, int spin_limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int *err = &st->error;
        const int g = ld_acquire(reinterpret_cast<const int *>(&st->bar_gen));
        __threadfence();
        if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            st_release(reinterpret_cast<int *>(&st->bar_gen), g + 1);
        } else {
            int spins = 0;
            while (ld_acquire(reinterpret_cast<const int *>(&st->bar_gen)) == g && *err == 0) {
                if (++spins > spin_limit) {
                    atomicExch(&st->error, 3);
                    break;
                }
                __nanosleep(32);
            }
        }
    }
    __syncthreads();
    return *reinterpret_cast<volatile int *>(&st->error) == 0;
}

__global__ void __launch_bounds__(kDT) k_dense_ldlt(double *S, int n, FactorStatus *st,
                                                    double pivot_tol, int spin_limit) {
    __shared__ double A11[kDB][kDB + 1];
    __shared__ double dinv[kDB];
    __shared__ double Li[kDB][33], Wj[kDB][33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool ptol_zero = pivot_tol == 0.0;
    // this thread's entry (er, ej), 1 <= ej <= er < kDB, of the diagonal
    // block's trailing triangle (threads 0 .. kDTri - 1, row by row)
    int er = 0, ej = 0;
    if (tid < kDTri) {
        int r = 0;
        while ((r + 1) * (r + 2) / 2 <= tid) r++;
        er = r + 1;
        ej = tid - r * (r + 1) / 2 + 1;
    }
    int s_pos = 0, s_neg = 0, s_zero = 0;
    for (int k0 = 0; k0 < n; k0 += kDB) {
        const int k1 = min(k0 + kDB, n), pw = k1 - k0;
        // A: diagonal block (lower triangle), right-looking within the block
        for (int t = tid; t < kDB * kDB; t += kDT) {
            const int c = t / kDB, r = t - c * kDB;
            A11[r][c] = (r < pw && c < pw && r >= c) ? S[(int64_t)(k0 + c) * n + k0 + r] : 0.0;
        }
        __syncthreads();
        const bool act = tid < kDTri && er < pw;
        for (int c = 0; c < pw; c++) {
            if (tid < kDTri) {
                const double d = A11[c][c];
                const double di = pivot_reciprocal<double>(d);
                // u_r u_j / d_c with u the unscaled column (l d)
                if (act && ej > c) A11[er][ej] -= A11[er][c] * (A11[ej][c] * di);
                if (tid == 0) {
                    dinv[c] = di;
                    count_pivot<double>(d, pivot_tol, ptol_zero, s_pos, s_neg, s_zero);
                }
            }
            __syncthreads();
        }
        // the columns become L11 (unit lower)
        if (act) {
            const int c = ej - 1, r = er;   // every (r, c), 0 <= c < r < pw
            A11[r][c] *= dinv[c];
        }
        __syncthreads();
        // B: rows below the block, W = A21 L11^-T by forward substitution
        // (lane c of a half-warp holds w_c), then L21 = W D^-1
        {
            const int half = lane & 16, c = lane & 15;
            const int nwarps = gridDim.x * (kDT / 32);
            for (int gw = blockIdx.x * (kDT / 32) + warp; k1 + 2 * gw < n; gw += nwarps) {
                const int i = k1 + 2 * gw + (half >> 4);
                const bool ok = i < n && c < pw;
                double x = ok ? S[(int64_t)(k0 + c) * n + i] : 0.0;
                for (int c2 = 0; c2 + 1 < pw; c2++) {
                    const double xc2 = __shfl_sync(0xffffffffu, x, half | c2);
                    if (c > c2) x = fma(-xc2, A11[c][c2], x);
                }
                if (ok) S[(int64_t)(k0 + c) * n + i] = x * dinv[c];
            }
        }
        // CTA 0 stores the factored diagonal block once no CTA can still be
        // loading it (after the barrier; the last block has no reader left)
        const int R = n - k1;
        const bool last = R <= 0;
        if (!last && !dense_grid_barrier(st, spin_limit)) break;
        if (blockIdx.x == 0)
            for (int t = tid; t < pw * pw; t += kDT) {
                const int c = t / pw, r = t - c * pw;
                if (r >= c) S[(int64_t)(k0 + c) * n + k0 + r] = A11[r][c];
            }
        if (last) break;
        // C: trailing update of the lower triangle, 32 x 32 tiles
        const int T = (R + 31) / 32, ntiles = T * (T + 1) / 2;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            // tile -> (ti, tj), ti >= tj, tiles numbered row by row
            int ti = (int)((sqrtf(8.0f * (float)tile + 1.0f) - 1.0f) * 0.5f);
            while (ti * (ti + 1) / 2 > tile) ti--;
            while ((ti + 1) * (ti + 2) / 2 <= tile) ti++;
            const int tj = tile - ti * (ti + 1) / 2;
            const int i0 = k1 + 32 * ti, j0 = k1 + 32 * tj;
            __syncthreads();
            for (int t = tid; t < kDB * 32; t += kDT) {
                const int c = t >> 5, r = t & 31;
                const bool ok = c < pw;
                Li[c][r] = (ok && i0 + r < n) ? S[(int64_t)(k0 + c) * n + i0 + r] : 0.0;
                Wj[c][r] = (ok && j0 + r < n) ? S[(int64_t)(k0 + c) * n + j0 + r] * A11[c][c] : 0.0;
            }
            __syncthreads();
            // U -= L21 W' on the FP64 tensor pipe: the 32 x 32 tile is sixteen
            // 8 x 8 blocks, two per warp, each a chain of mma.m8n8k4 over the
            // panel's (zero-padded) kDB columns.  Fragments (PTX ISA, .f64
            // m8n8k4): A row = lane / 4, col = lane % 4; B row = lane % 4,
            // col = lane / 4; D row = lane / 4, cols 2 (lane % 4) + {0, 1}.
            const int g = lane >> 2, q = lane & 3;
            const int bi = warp >> 1;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int bj = 2 * (warp & 1) + h;
                double d0 = 0.0, d1 = 0.0;
#pragma unroll
                for (int kk = 0; kk < kDB; kk += 4) {
                    const double a = Li[kk + q][8 * bi + g];
                    const double b = Wj[kk + q][8 * bj + g];
                    asm volatile(
                        "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, "
                        "{%0, %1};"
                        : "+d"(d0), "+d"(d1)
                        : "d"(a), "d"(b));
                }
                const int i = i0 + 8 * bi + g;
                const int j = j0 + 8 * bj + 2 * q;
                if (i < n && j < n && i >= j) S[(int64_t)j * n + i] -= d0;
                if (i < n && j + 1 < n && i >= j + 1) S[(int64_t)(j + 1) * n + i] -= d1;
            }
        }
        if (!dense_grid_barrier(st, spin_limit)) break;
    }
    if (blockIdx.x == 0 && tid == 0) {
        atomicAdd(&st->n_pos, s_pos);
        atomicAdd(&st->n_neg, s_neg);
        atomicAdd(&st->n_zero, s_zero);
    }
}

// ---------------------------------------------------------------- solves
// f <= 32: lane i owns row i; its row of the L panel (np <= NP columns) is
// prefetched into registers, the children's update vectors are gathered in
// batches of four (all loads in flight, adds in child order), and the
// triangular solve runs on shuffles
template <typename T, int NP>
__device__ __forceinline__ void fwd_small(const DevFront &F, const T *__restrict__ L,
                                          T *__restrict__ v, const T *__restrict__ vec,
                                          const TaskInfo &ti, int lane, T *sv) {
    const int f = ti.f, np = ti.np;
    T Lr[NP];
#pragma unroll
    for (int c = 0; c < NP; c++) Lr[c] = (c < np && lane > c && lane < f) ? L[(int64_t)c * f + lane] : (T)0;
    const T dl = lane < np ? L[(int64_t)lane * f + lane] : (T)1;
    T vi = lane < np ? v[lane] : (T)0;   // D b, placed in the front's slots before the sweep
    sv[lane] = vi;
    __syncwarp();
    for (int q0 = ti.c0; q0 < ti.c1; q0 += 4) {
        int rr[4];
        T vv[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            rr[k] = -1;
            vv[k] = (T)0;
            if (q0 + k < ti.c1) {
                const ChildInfo c = child_info(F, q0 + k);
                if (lane < c.fc - c.npc) {
                    rr[k] = F.rel[c.rel_off + lane];
                    vv[k] = vec[c.vo + c.npc + lane];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (q0 + k < ti.c1) {
                if (rr[k] >= 0) sv[rr[k]] += vv[k];
                __syncwarp();
            }
        }
    }
    vi = sv[lane];
#pragma unroll
    for (int c = 0; c < NP; c++) {
        if (c < np) {
            const T xc = __shfl_sync(0xffffffffu, vi, c);
            vi -= Lr[c] * xc;
        }
    }
    if (lane < np) vi /= dl;
    if (lane < f) v[lane] = vi;
}

// Forward sweep of one front: D b on its pivot rows (placed in the front's
// vector slots before the sweep) plus the children's update vectors, then
// y = D^-1 L^-1 (.) on the pivot rows and the update vector -L21 y for the
// parent on the others.
template <typename T>
__device__ __forceinline__ void fwd_front(const DevFront &F, const T *__restrict__ fronts,
                                          T *__restrict__ vec, const TaskInfo &ti, int lane,
                                          T *sv) {
    const int f = ti.f, np = ti.np;
    const T *L = fronts + ti.front_off;
    T *v = vec + ti.vo;
    if (f <= 32) {
        if (np <= 8)
            fwd_small<T, 8>(F, L, v, vec, ti, lane, sv);
        else
            fwd_small<T, 32>(F, L, v, vec, ti, lane, sv);
        return;
    }
    // f > 32: the front's vector is staged in the warp's shared buffer; the
    // pivot block is solved in 32-row tiles (rows in registers, shuffles),
    // and the update rows take the mat-vec -L21 y with independent loads
    for (int i = lane; i < f; i += 32) sv[i] = i < np ? v[i] : (T)0;
    __syncwarp();
    // children four at a time: all their loads in flight, then the adds in
    // a fixed order (child by child within each 32-row chunk)
    for (int q0 = ti.c0; q0 < ti.c1; q0 += 4) {
        int nuk[4];
        const T *vck[4];
        const int32_t *relk[4];
        int numax = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            nuk[k] = 0;
            vck[k] = vec;
            relk[k] = F.rel;
            if (q0 + k < ti.c1) {
                const ChildInfo c = child_info(F, q0 + k);
                nuk[k] = c.fc - c.npc;
                vck[k] = vec + c.vo + c.npc;
                relk[k] = F.rel + c.rel_off;
                numax = max(numax, nuk[k]);
            }
        }
        for (int i0 = 0; i0 < numax; i0 += 32) {
            int rr[4];
            T vv[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = i0 + lane;
                rr[k] = i < nuk[k] ? relk[k][i] : -1;
                vv[k] = i < nuk[k] ? vck[k][i] : (T)0;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (rr[k] >= 0) sv[rr[k]] += vv[k];
                __syncwarp();
            }
        }
    }
    for (int k0 = 0; k0 < np; k0 += 32) {
        const int kn = min(32, np - k0);
        const int row = k0 + lane;
        T acc = (T)0;
        if (lane < kn) {
            acc = sv[row];
            for (int c0 = 0; c0 < k0; c0 += 8) {   // 8 loads in flight
                T l[8];
#pragma unroll
                for (int u = 0; u < 8; u++) l[u] = c0 + u < k0 ? L[(int64_t)(c0 + u) * f + row] : (T)0;
#pragma unroll
                for (int u = 0; u < 8; u++)
                    if (c0 + u < k0) acc -= l[u] * sv[c0 + u];
            }
        }
        T Lr[32];
#pragma unroll
        for (int c = 0; c < 32; c++)
            Lr[c] = (c < lane && lane < kn) ? L[(int64_t)(k0 + c) * f + row] : (T)0;
#pragma unroll
        for (int c = 0; c < 32; c++) {
            if (c < kn) {
                const T xc = __shfl_sync(0xffffffffu, acc, c);
                acc -= Lr[c] * xc;
            }
        }
        if (lane < kn) sv[row] = acc;
        __syncwarp();
    }
    // update rows, two 32-row chunks at a time: the loads of eight columns
    // for both chunks are in flight together, and every row's sum still
    // runs over the columns in order
    for (int i0 = np; i0 < f; i0 += 64) {
        T acc[2];
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int i = i0 + 32 * j + lane;
            acc[j] = i < f ? sv[i] : (T)0;
        }
        for (int c0 = 0; c0 < np; c0 += 8) {
            T l[8][2];
#pragma unroll
            for (int u = 0; u < 8; u++)
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    const int i = i0 + 32 * j + lane;
                    l[u][j] = (c0 + u < np && i < f) ? L[(int64_t)(c0 + u) * f + i] : (T)0;
                }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                if (c0 + u < np) {
                    const T sc = sv[c0 + u];
#pragma unroll
                    for (int j = 0; j < 2; j++) acc[j] -= l[u][j] * sc;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int i = i0 + 32 * j + lane;
            if (i < f) v[i] = acc[j];
        }
    }
    // diagonal: y = D^-1 (L^-1 b) on the pivot rows
    for (int c = lane; c < np; c += 32) v[c] = sv[c] / L[(int64_t)c * f + c];
}

// bottom-up over every task (border fronts included: they collect the
// block's contribution to the border right-hand side)
template <typename T>
__global__ void __launch_bounds__(kWT, sizeof(T) == 4 ? 8 : 5)
    k_solve_fwd(DevFront F, const T *__restrict__ fronts, T *__restrict__ vec, QueueView Q,
                FactorStatus *st, int spin_limit) {
    extern __shared__ unsigned char solve_smem[];
    const int lane = threadIdx.x & 31;
    T *sv = reinterpret_cast<T *>(solve_smem) + (threadIdx.x >> 5) * F.max_f;
    int item = -1;
    while (true) {
        const unsigned long long tc = F.trace ? dev_clock_ns() : 0;
        if (item < 0) item = warp_claim(Q, spin_limit, st, 2);
        if (item < 0) break;
        const unsigned long long ts = F.trace ? dev_clock_ns() : 0;
        int t0, t1, par;   // one record load starts the item
        TaskInfo ti = item_task(F.item_fwd, item, t1, t0, par);
        for (int task = t0; task < t1; task++) {
            const TaskInfo nx = task_info(F, task + 1 < t1 ? task + 1 : task);   // prefetch
            fwd_front<T>(F, fronts, vec, ti, lane, sv);
            __syncwarp();
            ti = nx;
        }
        if (F.trace && lane == 0) trace_item(F, 0, item, tc, ts);
        item = (par >= 0 && warp_complete_child(Q, par)) ? par : -1;
    }
}

// vec[vpos[r]] = scale[r] b[r] for every block row r (its pivot slot)
template <typename T>
__global__ void k_rhs_to_fronts(int64_t n, const int64_t *__restrict__ vpos,
                                const double *__restrict__ scale, const double *__restrict__ b,
                                T *__restrict__ vec) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t p = vpos[r];
    if (p >= 0) vec[p] = (T)(scale[r] * b[r]);
}

// Border right-hand side y = D b_border + sum_k (update vector of block k's
// border front), then the dense border solve with S = L_S D_S L_S' by one
// warp (column sweeps, warp-shuffle dot products).
// Border right-hand side over the whole GPU: CTA (c, g) sums, for the 32
// border rows of chunk c, the update vectors of the blocks k = g, g + kBG,
// ... (block order) into part[g][j].  The combination over g happens in a
// fixed order in the kernel that uses it, so the sum does not depend on
// scheduling.
constexpr int kBG = 16;     // block groups of the border gather
template <typename T>
__global__ void __launch_bounds__(256) k_border_gather(DevFront F, const T *__restrict__ vec, int n,
                                                       double *__restrict__ part) {
    __shared__ double red[8][33];
    const int j = 32 * blockIdx.x + (threadIdx.x & 31), sub = threadIdx.x >> 5;
    const int g = blockIdx.y;
    double a = 0.0;
    if (j < n)
        for (int k = g + kBG * sub; k < F.n_blocks; k += kBG * 8)
            a += (double)vec[F.border_vec_off[k] + j];
    red[sub][threadIdx.x & 31] = a;
    __syncthreads();
    if (sub == 0 && j < n) {
        double t = red[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < 8; q++) t += red[q][threadIdx.x];
        part[(size_t)g * n + j] = t;
    }
}

// y = D b_border + sum_g part[g] (fixed order, every CTA), then x = S^-1 y for
// this CTA's 16 border rows: one warp per two rows, lanes over the columns
// and a shuffle reduction (mixed precision: S^-1 formed from the FP64 factor)
template <typename T>
__global__ void __launch_bounds__(256) k_border_apply(DevFront F, const double *__restrict__ Sinv,
                                                      int n, const double *__restrict__ b,
                                                      const double *__restrict__ scale,
                                                      const double *__restrict__ part,
                                                      double *__restrict__ x) {
    extern __shared__ double yb[];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int64_t r = F.border_rows[j];
        double acc = scale[r] * b[r];
        for (int g = 0; g < kBG; g++) acc += part[(size_t)g * n + j];
        yb[j] = acc;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int jj = 0; jj < 2; jj++) {
        const int j = 16 * blockIdx.x + 2 * warp + jj;
        if (j >= n) break;
        double acc = 0.0;
        for (int k = lane; k < n; k += 32) acc += Sinv[(int64_t)k * n + j] * yb[k];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const int64_t r = F.border_rows[j];
            x[r] = scale[r] * acc;
            static_cast<T *>(F.xs)[r] = (T)acc;
        }
    }
}

constexpr int kBS = 1024;   // threads of the border solve
template <typename T>
__global__ void __launch_bounds__(kBS) k_border_solve(DevFront F, const T *__restrict__ vec,
                                                      const double *__restrict__ S,
                                                      const double *__restrict__ Sinv, int n,
                                                      const double *__restrict__ b,
                                                      const double *__restrict__ scale,
                                                      double *__restrict__ x,
                                                      double *__restrict__ y) {
    const int tid = threadIdx.x;
    // y = D b_border + sum_g part[g] (the gather's partials, fixed order)
    const double *part = y + n;
    for (int j = tid; j < n; j += kBS) {
        const int64_t r = F.border_rows[j];
        double acc = scale[r] * b[r];
        for (int g = 0; g < kBG; g++) acc += part[(size_t)g * n + j];
        y[j] = acc;
    }
    __syncthreads();
    block_ldlt_solve<kBS>(S, n, y);
    for (int j = tid; j < n; j += kBS) {
        const int64_t r = F.border_rows[j];
        x[r] = scale[r] * y[j];
        static_cast<T *>(F.xs)[r] = (T)y[j];
    }
}

// column j of S^-1 from the LDL^T factors of S (one CTA per column)
__global__ void __launch_bounds__(256) k_dense_inverse(const double *__restrict__ S, int n,
                                                       double *__restrict__ Sinv) {
    const int j = blockIdx.x;
    double *y = Sinv + (int64_t)j * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = i == j ? 1.0 : 0.0;
    __syncthreads();
    block_ldlt_solve<256>(S, n, y, j);   // L^-1 e_j is zero above row j
}

// f <= FB <= 32: lane c < np holds column c of the L panel (rows below c);
// every lane holds one row's value z (pivot rows: y, update rows: the final
// solution of ancestors and border).  Rows are finished from the last one up:
// row i's final value is broadcast once and each column lane adds its
// L[i][c] z_i, so pivot c's sum is complete when its turn comes.  One shuffle
// per front row.
template <typename T, int FB>
__device__ __forceinline__ void bwd_small(const T *__restrict__ L, const T *__restrict__ v,
                                          const int64_t *__restrict__ rows,
                                          const double *__restrict__ scale,
                                          double *__restrict__ x, T *__restrict__ xs, int f,
                                          int np, int lane) {
    T Lc[FB];
#pragma unroll
    for (int i = 0; i < FB; i++)
        Lc[i] = (lane < np && i > lane && i < f) ? L[(int64_t)lane * f + i] : (T)0;
    T z = (T)0;
    int64_t r = 0;
    if (lane < f) r = rows[lane];
    if (lane < np)
        z = v[lane];
    else if (lane < f)
        z = xs[r];   // the scaled solution, written by the row's pivot owner
    T acc = (T)0;
#pragma unroll
    for (int i = FB - 1; i >= 0; i--) {
        if (i < f) {
            if (lane == i && i < np) z -= acc;
            const T zi = __shfl_sync(0xffffffffu, z, i);
            acc += Lc[i] * zi;
        }
    }
    if (lane < np) {
        x[r] = scale[r] * (double)z;
        xs[r] = z;
    }
}

// Backward sweep of one (non-border) front: its update rows hold the final
// solution of ancestors and border, the pivot rows solve L11' x = y - L21' x2.
template <typename T>
__device__ __forceinline__ void bwd_front(const DevFront &F, const T *__restrict__ fronts,
                                          T *__restrict__ vec, const double *__restrict__ scale,
                                          double *__restrict__ x, const TaskInfo &ti, int lane,
                                          T *sv) {
    const int f = ti.f, np = ti.np;
    const T *L = fronts + ti.front_off;
    T *v = vec + ti.vo;
    const int64_t *rows = F.rows + ti.vo;
    T *xs = static_cast<T *>(F.xs);
    if (f <= 32) {
        if (f <= 16)
            bwd_small<T, 16>(L, v, rows, scale, x, xs, f, np, lane);
        else
            bwd_small<T, 32>(L, v, rows, scale, x, xs, f, np, lane);
        return;
    }
    // f > 32: stage [y (pivots); x (update rows)] in the warp's shared
    // buffer, then solve L' z = y in 32-row tiles from the last: the tile's
    // coupling to everything below it is one dot product per column (warp
    // reductions over independent loads), the tile itself a register solve
    for (int i = lane; i < f; i += 32) {
        if (i < np) {
            sv[i] = v[i];
        } else {
            sv[i] = xs[rows[i]];
        }
    }
    __syncwarp();
    for (int k0 = ((np - 1) >> 5) << 5; k0 >= 0; k0 -= 32) {
        const int kn = min(32, np - k0);
        T zi = lane < kn ? sv[k0 + lane] : (T)0;
        // eight column dot products at a time: their loads are independent
        for (int j0 = 0; j0 < kn; j0 += 8) {
            T pj[8];
#pragma unroll
            for (int u = 0; u < 8; u++) pj[u] = (T)0;
            // two 32-row chunks per round: their loads in flight together,
            // each lane's rows still summed in increasing order
            for (int i0 = k0 + kn; i0 < f; i0 += 64) {
                T l[2][8], xv[2];
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    const int i = i0 + 32 * j + lane;
                    xv[j] = i < f ? sv[i] : (T)0;
#pragma unroll
                    for (int u = 0; u < 8; u++)
                        l[j][u] = (i < f && j0 + u < kn) ? L[(int64_t)(k0 + j0 + u) * f + i] : (T)0;
                }
#pragma unroll
                for (int j = 0; j < 2; j++)
                    if (i0 + 32 * j + lane < f) {
#pragma unroll
                        for (int u = 0; u < 8; u++)
                            if (j0 + u < kn) pj[u] += l[j][u] * xv[j];
                    }
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                T p = pj[u];
                for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
                if (lane == j0 + u) zi -= p;
            }
        }
        // the tile, by columns: lane c holds column c of the tile's L and
        // subtracts L[r][c] z_r as each z_r (r > c) becomes final and is
        // broadcast (one shuffle per row instead of a reduction per column)
        T Lc[32];
#pragma unroll
        for (int r = 0; r < 32; r++)
            Lc[r] = (lane < r && r < kn) ? L[(int64_t)(k0 + lane) * f + k0 + r] : (T)0;
#pragma unroll
        for (int r = 31; r >= 0; r--) {
            if (r < kn) {
                const T zr = __shfl_sync(0xffffffffu, zi, r);
                if (lane < r) zi -= Lc[r] * zr;
            }
        }
        if (lane < kn) sv[k0 + lane] = zi;
        __syncwarp();
    }
    for (int c = lane; c < np; c += 32) {
        const int64_t r = rows[c];
        x[r] = scale[r] * (double)sv[c];
        xs[r] = sv[c];
    }
}

// top-down from the block roots (the border solution is already in x); a
// finished front pushes its children
template <typename T>
__global__ void __launch_bounds__(kWT, sizeof(T) == 4 ? 8 : 5) k_solve_bwd(DevFront F, const T *__restrict__ fronts,
                                                   T *__restrict__ vec, const double *__restrict__ scale,
                                                   double *__restrict__ x, QueueView Q,
                                                   FactorStatus *st, int spin_limit) {
    extern __shared__ unsigned char solve_smem[];
    const int lane = threadIdx.x & 31;
    T *sv = reinterpret_cast<T *>(solve_smem) + (threadIdx.x >> 5) * F.max_f;
    int item = -1;
    while (true) {
        const unsigned long long tc = F.trace ? dev_clock_ns() : 0;
        if (item < 0) item = warp_claim(Q, spin_limit, st, 3);
        if (item < 0) break;
        const unsigned long long ts = F.trace ? dev_clock_ns() : 0;
        int t0, t1, keep;   // one record load starts the item; keep: the child
                            // with the longest path below, run next by this warp
        TaskInfo ti = item_task(F.item_bwd, item, t0, t1, keep);
        for (int task = t1 - 1; task >= t0; task--) {
            const TaskInfo nx = task_info(F, task > t0 ? task - 1 : task);   // prefetch
            bwd_front<T>(F, fronts, vec, scale, x, ti, lane, sv);
            __syncwarp();
            ti = nx;
        }
        if (F.trace && lane == 0) trace_item(F, 1, item, tc, ts);
        push_children(Q, F, item, keep);
        item = keep;
    }
}

// ---- Ruiz equilibration: s_i <- s_i / sqrt(max_j |s_i K_ij s_j|) ---------
// Ruiz equilibration with power-of-two factors (s_i = 2^e_i), in integer
// exponent arithmetic.  The FP64 version kept B300's FP64 pipe 78% busy for a
// pass that only needs magnitudes; with powers of two the scaling is exact
// (D K D adds no rounding) and a sweep is integer work plus the loads.
// One sweep, entry-parallel: thread t takes the kRE stored entries
// [kRE t, kRE t + kRE) (vector loads; the entries of a row are consecutive)
// and forms, for each nonzero a_ij, the exponent of |a_ij| s_j (that of a_ij's
// leading bit plus e_j), keeping a running maximum per run of equal rows.  A
// run inside the chunk is the whole row: a plain store.  A run that touches
// either end of the chunk may continue in a neighbouring one: an atomic max.
// Maxima are stored offset by kRuizBias so that 0 means "no entry"; mx must
// be zero on entry and k_ruiz_finish re-zeroes it.
constexpr int kRE = 8;
constexpr int kRuizBias = 8192;
__device__ __forceinline__ void ruiz_flush(unsigned *mx, int r, int m, bool edge) {
    if (r < 0 || m == INT_MIN) return;
    const unsigned b = (unsigned)(m + kRuizBias);
    if (edge) atomicMax(&mx[r], b);
    else mx[r] = b;
}

// exponent of a normal FP64 value's leading bit, INT_MIN for zero, subnormal,
// infinite or NaN values (read from the high word: integer instructions)
__device__ __forceinline__ int exponent_of(int hi) {
    const int f = (hi >> 20) & 0x7ff;
    return (f == 0 || f == 0x7ff) ? INT_MIN : f - 1023;
}

__global__ void __launch_bounds__(256) k_ruiz_entries(int64_t nnz, const int32_t *__restrict__ row,
                                                      const int32_t *__restrict__ col,
                                                      const double *__restrict__ kval,
                                                      const int *__restrict__ e,
                                                      unsigned *__restrict__ mx) {
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t * kRE < nnz; t += nthr) {
        const int64_t e0 = t * kRE;
        int rr[kRE];
        int cc[kRE];
        int hh[kRE];
        int cnt = kRE;
        if (e0 + kRE <= nnz) {
            const int4 *r4 = reinterpret_cast<const int4 *>(row + e0);
            const int4 *c4 = reinterpret_cast<const int4 *>(col + e0);
            const int4 *v4 = reinterpret_cast<const int4 *>(kval + e0);   // (lo, hi) pairs
#pragma unroll
            for (int k = 0; k < kRE / 4; k++) {
                const int4 a = __ldg(r4 + k);
                rr[4 * k] = a.x;
                rr[4 * k + 1] = a.y;
                rr[4 * k + 2] = a.z;
                rr[4 * k + 3] = a.w;
                const int4 c = __ldg(c4 + k);
                cc[4 * k] = c.x;
                cc[4 * k + 1] = c.y;
                cc[4 * k + 2] = c.z;
                cc[4 * k + 3] = c.w;
            }
#pragma unroll
            for (int k = 0; k < kRE / 2; k++) {
                const int4 b = __ldg(v4 + k);
                hh[2 * k] = b.y;
                hh[2 * k + 1] = b.w;
            }
        } else {
            cnt = (int)(nnz - e0);
#pragma unroll
            for (int k = 0; k < kRE; k++) {
                rr[k] = k < cnt ? row[e0 + k] : -1;
                cc[k] = k < cnt ? col[e0 + k] : 0;
                hh[k] = k < cnt ? __double2hiint(kval[e0 + k]) : 0;
            }
        }
        int v[kRE];
#pragma unroll
        for (int k = 0; k < kRE; k++) {
            const int x = k < cnt ? exponent_of(hh[k]) : INT_MIN;
            v[k] = x == INT_MIN ? INT_MIN : x + e[cc[k]];
        }
        int cur = rr[0];
        int m = v[0];
        bool at_start = true;
#pragma unroll
        for (int k = 1; k < kRE; k++) {
            if (k >= cnt) break;
            if (rr[k] != cur) {
                ruiz_flush(mx, cur, m, at_start);
                at_start = false;
                cur = rr[k];
                m = INT_MIN;
            }
            m = max(m, v[k]);
        }
        ruiz_flush(mx, cur, m, true);
    }
}

// e_i <- e_i - floor(m_i / 2), m_i the exponent of max_j |s_i a_ij s_j|
// (Ruiz: s_i <- s_i / sqrt(row max), rounded to a power of two)
__global__ void k_ruiz_finish(int64_t n, int *__restrict__ e, unsigned *__restrict__ mx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned b = mx[i];
    mx[i] = 0u;
    if (b) {
        const int m = (int)b - kRuizBias + e[i];
        e[i] -= m >> 1;
    }
}

// scale_i = 2^e_i (built from the exponent bits)
__global__ void k_ruiz_scale(int64_t n, const int *__restrict__ e, double *__restrict__ scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) scale[i] = __hiloint2double((e[i] + 1023) << 20, 0);
}

// scaled original entries of every front, in task order
template <typename T>
__global__ void k_orig_vals(int64_t n_orig, const int64_t *__restrict__ nz,
                            const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                            const double *__restrict__ scale, const double *__restrict__ kval,
                            T *__restrict__ ovals) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_orig) return;
    const int64_t q = nz[p];
    ovals[p] = (T)(scale[row[q]] * kval[q] * scale[col[q]]);
}


int warp_grid() { return sm_count() * (2048 / kWT); }

}  // namespace

void launch_equilibrate(const DevModel &M, const double *kval, double *scale, double *tmp,
                        unsigned long long *mx, int iters, cudaStream_t s) {
    const int t = 256;
    const int64_t n = M.n_kkt;
    const int g = (int)((n + t - 1) / t);
    // entry sweep: resident warps over the stored entries
    const int resident = sm_count() * (2048 / t);
    const int64_t chunks = (M.nnz_kkt + kRE - 1) / kRE;
    const int ge = (int)std::min<int64_t>((chunks + t - 1) / t, (int64_t)resident);
    // exponents in tmp (n int32), row maxima in mx (n uint32, zeros)
    int *e = reinterpret_cast<int *>(tmp);
    unsigned *m32 = reinterpret_cast<unsigned *>(mx);
    cudaMemsetAsync(e, 0, sizeof(int) * (size_t)(n > 0 ? n : 1), s);
    for (int it = 0; it < iters; it++) {
        if (M.nnz_kkt)
            note_launch(), k_ruiz_entries<<<ge, t, 0, s>>>(M.nnz_kkt, M.kkt_row, M.kkt_col, kval, e, m32);
        note_launch(), k_ruiz_finish<<<g, t, 0, s>>>(n, e, m32);
    }
    note_launch(), k_ruiz_scale<<<g, t, 0, s>>>(n, e, scale);
}

template <typename T>
void launch_orig_vals(const DevFront &F, T *ovals, cudaStream_t s) {
    const int t = 256;
    if (F.n_orig > 0)
        note_launch(), k_orig_vals<T><<<(int)((F.n_orig + t - 1) / t), t, 0, s>>>(
            F.n_orig, F.orig_nz, F.kkt_row, F.kkt_col, F.scale, F.kval, ovals);
}
template void launch_orig_vals<float>(const DevFront &, float *, cudaStream_t);
template void launch_orig_vals<double>(const DevFront &, double *, cudaStream_t);

void launch_queue_reset(const DevFront &F, QueueSeeds seeds, const int32_t *pend, cudaStream_t s) {
    const int t = 256;
    const int n = F.n_items > 0 ? F.n_items : 1;
    note_launch(), k_queue_reset<<<(n + t - 1) / t, t, 0, s>>>(F.n_items, F.q_slots_a, F.q_slots_b, F.q_slots_c,
                                                seeds, F.q_pending, pend, F.q_ctr);
}

// SMs of the current device (cached per device ordinal)
int sm_count() {
    static int cache[64] = {};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
    if (dev >= 0 && dev < 64) cache[dev] = sms;
    return sms;
}

// Function attributes and occupancy are per device: the launch caches below
// are kept per device ordinal (beyond kMaxDev they are recomputed per call).
constexpr int kMaxDev = 64;
static int device_slot() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return -1;
    return dev;
}

// CTAs of `kernel` that fit on the device at once with `smem` bytes each
static int resident_grid(const void *kernel, int threads, size_t smem) {
    int dev = 0, sms = 148, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
    return sms * (occ > 0 ? occ : 1);
}

template <typename T>
void launch_factor(const DevFront &F, T *fronts, FactorStatus *st, double pivot_tol,
                   int spin_limit, cudaStream_t s) {
    // queues a, b, c: the three phases
    QueueSeeds seeds{{F.init_small, F.init_med, F.init_big},
                     {F.n_init_small, F.n_init_med, F.n_init_big}};
    launch_queue_reset(F, seeds, F.pend_factor, s);
    static int grids[kMaxDev][2][2] = {};   // [device][float, double][phase 1, 2]
    const size_t sm1 = sizeof(T) * (size_t)(kFT / 32) * 32 * 33;
    const size_t sm2 = sizeof(T) * (size_t)(med_threads<T>() / 32) * kMedF * (kMedF + 1);
    const int dev = device_slot();
    int gtmp[2] = {0, 0};
    int *g = dev >= 0 ? grids[dev][sizeof(T) == 4 ? 0 : 1] : gtmp;
    if (!g[0]) {
        for (const void *k : {(const void *)k_factor<float>, (const void *)k_factor<double>}) {
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 80 * 1024);
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        }
        for (const void *k : {(const void *)k_factor_med<float>, (const void *)k_factor_med<double>}) {
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024);
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        }
        g[0] = resident_grid((const void *)k_factor<T>, kFT, sm1);
        g[1] = resident_grid((const void *)k_factor_med<T>, med_threads<T>(), sm2);
    }
    const int n1 = F.n_items_small, n2 = F.n_items_med - F.n_items_small;
    if (n1 > 0) {
        const int grid = std::min(g[0], (n1 + kFT / 32 - 1) / (kFT / 32));
        note_launch(), k_factor<T><<<grid, kFT, sm1, s>>>(F, fronts, st, queue_a(F, n1), pivot_tol, spin_limit);
    }
    if (n2 > 0) {
        const int wpc = med_threads<T>() / 32;
        const int grid = std::min(g[1], (n2 + wpc - 1) / wpc);
        note_launch(), k_factor_med<T><<<grid, med_threads<T>(), sm2, s>>>(F, fronts, st, queue_b(F, n2), pivot_tol,
                                               spin_limit);
    }
    const int nbig = F.n_items - F.n_items_med;
    if (nbig > 0) {
        // shared panel sized to the largest np x f of this phase (capped at
        // creation to 12,288 elements, 96 KB in FP64); larger panels take the
        // global-memory path
        // plus the staged child->parent map of one child (at most max_f rows)
        const size_t sm3 = big_rel_offset<T>(F.big_panel, F.big_np) + sizeof(int) * (size_t)F.max_f;
        static int g3_all[kMaxDev][2] = {};
        static size_t g3_sm_all[kMaxDev][2] = {};
        int g3_tmp[2] = {0, 0};
        size_t g3_sm_tmp[2] = {0, 0};
        int *g3 = dev >= 0 ? g3_all[dev] : g3_tmp;
        size_t *g3_sm = dev >= 0 ? g3_sm_all[dev] : g3_sm_tmp;
        const int pi = sizeof(T) == 4 ? 0 : 1;
        if (g3_sm[pi] != sm3) {
            cudaFuncSetAttribute((const void *)k_factor_big<T>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
            g3[pi] = resident_grid((const void *)k_factor_big<T>, kBT, sm3);
            g3_sm[pi] = sm3;
        }
        const int grid = std::min(g3[pi], nbig);
        note_launch(), k_factor_big<T><<<grid, kBT, sm3, s>>>(F, fronts, st, queue_c(F, nbig), pivot_tol,
                                               spin_limit);
    }
}

template <typename T>
void launch_schur_sum(const DevFront &F, const T *fronts, double *S, cudaStream_t s) {
    const int nb = F.n_border;
    if (nb == 0) return;
    note_launch(), k_schur_sum<T><<<(nb * nb + 31) / 32, 256, 0, s>>>(F.n_blocks, nb, F.border_off, fronts, S);
}

int launch_reciprocal(int64_t n, const double *d, double *out, cudaStream_t s) {
    if (n > 0) note_launch(), k_reciprocal<<<(int)((n + 255) / 256), 256, 0, s>>>(n, d, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void launch_dense_inverse(const double *S, int n, double *Sinv, cudaStream_t s) {
    if (n > 0) note_launch(), k_dense_inverse<<<n, 256, 0, s>>>(S, n, Sinv);
}

cudaError_t launch_dense_ldlt(double *S, int n, FactorStatus *st, double pivot_tol,
                              cudaStream_t s, int spin_limit) {
    if (n <= 0) return cudaSuccess;
    // CTAs: enough for the first trailing update's tiles, at most one per SM
    // (all co-resident: the launch is cooperative)
    const int R = n - kDB > 0 ? n - kDB : 0, T = (R + 31) / 32;
    int grid = std::max(1, std::min(sm_count(), T * (T + 1) / 2));
    note_launch();
    void *args[] = {&S, &n, &st, &pivot_tol, &spin_limit};
    return cudaLaunchCooperativeKernel((const void *)k_dense_ldlt, dim3(grid), dim3(kDT), args, 0,
                                       s);
}

template <typename T>
void launch_solve(const DevFront &F, const T *fronts, T *vec, const double *S, const double *Sinv,
                  int nS, const double *scale, const double *b, double *x, double *border_work,
                  FactorStatus *st, int spin_limit, cudaStream_t s) {
    // queue a: forward sweep (all items), queue b: backward sweep (non-border)
    QueueSeeds seeds{{F.init_fwd, F.init_bwd, F.init_bwd}, {F.n_init_fwd, F.n_init_bwd, 0}};
    launch_queue_reset(F, seeds, F.nchild, s);
    int grid = warp_grid();
    const int need = (F.n_items + kWT / 32 - 1) / (kWT / 32);
    if (grid > need) grid = need;
    const size_t sm = sizeof(T) * (size_t)(kWT / 32) * F.max_f;
    // per-device shared-memory opt-in, set on the current device each call
    if (sm > 48 * 1024)
        for (const void *k : {(const void *)k_solve_fwd<T>, (const void *)k_solve_bwd<T>})
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    note_launch(), k_rhs_to_fronts<T><<<(int)((F.n_rows + 255) / 256), 256, 0, s>>>(F.n_rows, F.vpos_of_row,
                                                                     scale, b, vec);
    note_launch(), k_solve_fwd<T><<<grid, kWT, sm, s>>>(F, fronts, vec, queue_a(F, F.n_items), st, spin_limit);
    if (nS > 0) {
        // border_work: y (nS), then the gather's partials (kBG x nS)
        double *part = border_work + nS;
        note_launch(), k_border_gather<T><<<dim3((nS + 31) / 32, kBG), 256, 0, s>>>(F, vec, nS, part);
        if (Sinv)
            note_launch(), k_border_apply<T><<<(nS + 15) / 16, 256, sizeof(double) * (size_t)nS, s>>>(
                F, Sinv, nS, b, scale, part, x);
        else
            note_launch(), k_border_solve<T><<<1, kBS, 0, s>>>(F, vec, S, Sinv, nS, b, scale, x,
                                                               border_work);
    }
    const int nb = F.n_items - F.n_blocks;   // every item but the border fronts
    if (nb > 0)
        note_launch(), k_solve_bwd<T><<<grid, kWT, sm, s>>>(F, fronts, vec, scale, x, queue_b(F, nb), st,
                                             spin_limit);
}

#define INST(T)                                                                                    \
    template void launch_factor<T>(const DevFront &, T *, FactorStatus *, double, int,           \
                                   cudaStream_t);                                                \
    template void launch_schur_sum<T>(const DevFront &, const T *, double *, cudaStream_t);      \
    template void launch_solve<T>(const DevFront &, const T *, T *, const double *,               \
                                  const double *, int, const double *, const double *, double *,  \
                                  double *, FactorStatus *, int, cudaStream_t);
INST(float)
INST(double)

}  // namespace scopf
