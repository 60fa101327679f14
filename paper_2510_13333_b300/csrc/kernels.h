// Device kernels of the NCL / interior-point Newton step (launch wrappers).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <atomic>

namespace scopf {

// Every kernel launch of the library is counted here (scopf_launch_count).
extern std::atomic<long long> g_kernel_launches;
inline void note_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }


// A scalar kernel argument, given by value or -- for kernels replayed in a
// CUDA graph whose scalars change between replays -- read from device
// memory when the kernel runs (p != nullptr).
struct DScalar {
    double v = 0.0;
    const double *p = nullptr;
    DScalar() = default;
    DScalar(double x) : v(x) {}
    static DScalar at(const double *q) {
        DScalar d;
        d.p = q;
        return d;
    }
#ifdef __CUDACC__
    __device__ __forceinline__ double get() const { return p ? *p : v; }
#endif
};

// ---------------------------------------------------------------- model
struct DevModel {
    int64_t n, m, p, n_kkt, nnz;
    int64_t n_be, n_se, ev_branch0, ev_shunt0, ev_comp0, n_ev;
    const int32_t *be_x, *be_lam, *be_th;
    const double *be_par;
    const int32_t *se_v, *se_P, *se_Q;
    const double *se_G, *se_B;
    const int64_t *comp1, *comp2;
    const double *c_const;
    const int64_t *cf_ptr, *cf_idx;
    const double *cf_coef;
    const int64_t *kkt_ptr, *ctr_ptr;
    const int32_t *kkt_col;       // column of every stored entry (n_kkt < 2^31)
    const int32_t *kkt_row;       // row of every stored entry
    int64_t nnz_kkt;              // stored entries
    const int64_t *ctr_src;
    const double *ctr_coef;
    const int8_t *row_kind;
    const int64_t *row_index;
    const double *wl, *wu;        // relaxed bounds (+-inf where absent)
    const double *grad_scale;     // per border p_g^0: c1 part etc. (see objective)
    const double *c2, *c1;        // per generator
    int64_t border0;
    int ng;
    // KKT rows with more than kLongRow stored entries (the border rows, which
    // couple to every contingency block) are handled one warp per row
    const int8_t *is_long;
    const int64_t *long_rows;
    int64_t n_long;
};
constexpr int kLongRow = 48;

// mode: 0 = values only (flows, thermal values), 1 = values + derivatives
void launch_eval_elements(const DevModel &M, const double *w, const double *lam,
                          const double *yc, double *ev, int mode, cudaStream_t s);
void launch_constraints(const DevModel &M, const double *w, const double *ev, double *c,
                        cudaStream_t s);
void launch_gradient(const DevModel &M, const double *w, double *g, cudaStream_t s);
void launch_diag_terms(const DevModel &M, const double *w, const double *zl, const double *zu,
                       const double *sv, const double *zs, DScalar rho, DScalar delta_w,
                       double *diag, cudaStream_t s);
void launch_assemble(const DevModel &M, const double *ev, const double *diag, double *kval,
                     cudaStream_t s);
// gw[i] = g[i] + sum over dual columns of K(row of w_i, col) * (lam | yc)
void launch_dual_product(const DevModel &M, const double *kval, const double *g,
                         const double *lam, const double *yc, double *gw, cudaStream_t s);
struct RhsArgs {
    const double *w, *r, *t, *sv, *lam, *yc, *zs, *gw, *c, *lam_n, *nu0_n;
    DScalar rho, mu;
};
void launch_rhs(const DevModel &M, const RhsArgs &a, double *rhs, cudaStream_t s);
// y = b - K x  (FP64); K from kval
void launch_residual(const DevModel &M, const double *kval, const double *x, const double *b,
                     double *y, cudaStream_t s);

// ------------------------------------------------------------ reductions
// out[0] = max |x|, computed deterministically in two passes into scratch
void reduce_maxabs(const double *x, int64_t n, double *d_out, double *scratch, cudaStream_t s);
void reduce_sumabs(const double *x, int64_t n, double *d_out, double *scratch, cudaStream_t s);
// y += a * x
void launch_axpy(int64_t n, double a, const double *x, double *y, cudaStream_t s);

// ---- Krylov helpers (FGMRES refinement), vectors stored contiguously with
// stride n: V_j = V + j * n
constexpr int kMaxKrylov = 32;
constexpr int kDotBlocks = 296;
// partial[b * k + j] = block b's part of V_j' w, j < k
void launch_multi_dot(const double *V, int64_t n, int k, const double *w, double *partial,
                      cudaStream_t s);
// w -= sum_j c[j] V_j  (k <= kMaxKrylov)
void launch_multi_axpy(double *w, const double *V, int64_t n, int k, const double *c,
                       cudaStream_t s);
// y = a * x
void launch_scale_copy(int64_t n, double a, const double *x, double *y, cudaStream_t s);

// ---- FGMRES(m) with its small dense algebra on the device (no host round
// trip per Gram-Schmidt pass).  State layout (doubles), m <= kMaxKrylov:
// H (m+1) x m column-major, cs[m], sn[m], g[m+1], coef[kMaxKrylov] (first
// pass), coef2[kMaxKrylov] (second pass), sc[8] (0 beta, 1 h_{j+1,j},
// 2 |g_{j+1}|)
struct GmresLayout {
    int m;
    int H, cs, sn, g, c1, c2, sc, total;
};
GmresLayout gmres_layout(int m);

// Device-resident Krylov loop: control block in device memory (the graph's
// WHILE node repeats one captured Krylov step; see solve_impl)
struct KrylovCtl {
    int j;          // current column
    int it;         // preconditioner applications so far in the solve
    int max_it;     // refinement budget
    int jend;       // columns completed in this cycle
    double target;  // residual estimate at which the cycle stops
};
void launch_kry_start(KrylovCtl *c, int it, int max_it, double target, cudaStream_t s);

// Control block of the device-resident interior-point iteration: the
// scalars its kernels read at run time, the state of its inertia-correction,
// refinement and line-search loops, and the outcome the host reads back.
struct IpmCtl {
    // set by the host before the iteration
    double mu, rho, tau, th, theta_min, theta_max, pow_th, dw_last;
    int clear_filter, pad0;
    // inertia correction
    double delta, current, ic3;
    int tries, known_zero, lead_zero, pad1;
    // refinement
    double bnorm, bden, rel;
    int ref_it, ref_cycles;
    // line search
    double alpha[2];   // primal and dual step of the current trial
    double ph, gd, amin, pow_gd, tht, pht;
    int nback, accepted, ftype, trials, filt_n, pad2;
    // outcome
    int status;        // SCOPF_OK or the error of the direction
    int ok;            // the direction is usable: the step graph runs
    int stall;         // mixed precision: the refinement stalled
    int dir_done;      // the solve of the direction ran
};
void launch_kry_gather(int64_t n, const double *V, const KrylovCtl *c, double *out, cudaStream_t s);
void launch_kry_scatter(int64_t n, const double *in, double *Z, const KrylovCtl *c, cudaStream_t s);
void launch_kry_multi_dot(const double *V, int64_t n, const KrylovCtl *c, const double *w,
                          double *partial, cudaStream_t s);
void launch_kry_dot_finish(const double *partial, const KrylovCtl *c, double *out, cudaStream_t s);
void launch_kry_axpy(double *w, const double *V, int64_t n, const KrylovCtl *c, bool use_jend,
                     const double *coef, cudaStream_t s);
void launch_kry_scale_out(int64_t n, const double *den, const double *w, double *V,
                          const KrylovCtl *c, cudaStream_t s);
void launch_kry_column_next(double *st, int m, KrylovCtl *c, cudaGraphConditionalHandle loop,
                            cudaStream_t s);
void launch_kry_solve(double *st, int m, const KrylovCtl *c, cudaStream_t s);
// out[j] = sum over the kDotBlocks partials of V_j' w (fixed order); with
// take_sqrt the single result is replaced by its square root
void launch_dot_finish(const double *partial, int k, double *out, bool take_sqrt, cudaStream_t s);
// w -= sum_j c[j] V_j, coefficients in device memory (sign: +1 or -1)
void launch_multi_axpy_dev(double *w, const double *V, int64_t n, int k, const double *c,
                           double sign, cudaStream_t s);
// y = x / *den (y = 0 if *den == 0)
void launch_scale_inv(int64_t n, const double *den, const double *x, double *y, cudaStream_t s);
// new cycle: g = beta e1 (beta = sc[0])
void launch_gmres_init(double *st, int m, cudaStream_t s);
// column j: H(:, j) = coef + coef2, H(j+1, j) = sc[1]; previous Givens
// rotations, a new one, g updated; sc[2] = |g(j+1)|
void launch_gmres_column(double *st, int m, int j, cudaStream_t s);
// y = H(0:k, 0:k)^-1 g(0:k) by back substitution, stored (negated) in coef
void launch_gmres_solve(double *st, int m, int k, cudaStream_t s);
// base[i] = kval[pos[i]];  kval[pos[i]] = base[i] + shift
int sm_count();   // SMs of the current device
// out[i] = the FP64 pivot reciprocal the factorization uses, of d[i]
int launch_reciprocal(int64_t n, const double *d, double *out, cudaStream_t s);
void launch_count_zero_diag(int64_t n, const int64_t *idx, const double *base, int *count,
                            cudaStream_t s);
void launch_diag_gather(int64_t n, const int64_t *pos, const double *kval, double *base,
                        cudaStream_t s);
void launch_diag_set(int64_t n, const int64_t *pos, const double *base, double shift,
                     double *kval, cudaStream_t s);
// out[0] = max |a|, out[1] = max |b| (two deterministic reductions)
void reduce_maxabs2(const double *a, const double *b, int64_t n, double *d_out, double *scratch,
                    cudaStream_t s);
// y = K x (FP64)
void launch_spmv(const DevModel &M, const double *kval, const double *x, double *y,
                 cudaStream_t s);

// ----------------------------------------------------------- factorisation
struct DevFront {
    int n_tasks, n_blocks, n_border;
    int n_small;                  // tasks [0, n_small) are small fronts (one warp each)
    const int64_t *front_off;     // per task, element offset into fronts
    const int32_t *f, *npiv;      // per task
    const int32_t *child_ptr, *child; // per task: children task ids
    const int64_t *rel_off;       // per task (as a child): offset into rel
    const int32_t *rel;           // positions of a child's update rows in its parent front
    const int32_t *parent;        // per task (-1 for border tasks)
    const int64_t *rows_off;      // per task: offset into rows
    const int64_t *rows;          // KKT indices of every front row
    const int32_t *is_border;     // per task
    const int64_t *border_off;    // per block: element offset of the border front
    const int64_t *border_rows;   // n_border KKT indices (natural order)
    int64_t front_elems;          // size of the front buffer (elements)
    int64_t vec_elems;            // size of the per-front vector buffer
    const int64_t *vec_off;       // per task offset into the vector buffer
    const int64_t *border_vec_off; // per block: vec_off of its border task
    // original KKT entries of each front (lower triangle in elimination
    // order): entries [orig_ptr[t], orig_ptr[t+1]) with the stored-entry index
    // and the offset inside the front; each task loads its own before use
    const int64_t *orig_ptr;
    const int64_t *orig_nz;
    const int32_t *orig_off;
    const int32_t *kkt_row;       // row of every stored KKT entry
    const int32_t *kkt_col;
    const double *kval;           // assembled K (set before each factorization)
    const double *scale;          // Ruiz scaling
    const void *ovals;            // scaled original entries in task order (n_orig), in the
                                  // factor precision (float or double)
    void *xs;                     // per KKT row: the scaled solution in the factor
                                  // precision, written by the backward sweep and border
                                  // solve, read by the fronts whose update rows hold it
    int64_t n_orig;
    // work items: item i is tasks [item_ptr[i], item_ptr[i+1]) in postorder
    // (a subtree of small fronts, or one front).  Factorization phases:
    // items [0, n_items_small) tile-sized fronts, [n_items_small,
    // n_items_med) medium fronts and their ancestors, the rest large fronts
    // and theirs
    int n_items, n_items_small, n_items_med;
    int max_f;                    // largest front (rows), at least 32
    int big_panel;                // largest np x f of the large-front phase (elements, capped)
    int big_np;                   // largest np among those staged panels
    // packed records, 8 int32 each.  task_rec[t] (t <= n_tasks, the last a
    // sentinel): front_off (2 words), vec_off (2), f | npiv << 16,
    // first child slot, first original entry, parent.  child_rec[q] for
    // child slot q: front_off (2), vec_off (2), rel_off, f | npiv << 16,
    // task id, 0
    const int4 *task_rec, *child_rec;
    // vector slot of every KKT row's pivot (-1 for border rows): the forward
    // sweep finds D b there
    int64_t n_rows;
    const int64_t *vpos_of_row;
    // scheduler trace (NULL = off): 4 kinds x n_items x 4 uint64
    unsigned long long *trace;
    const int32_t *item_ptr, *item_parent, *item_child_ptr, *item_child;
    // per item, 3 int4 each: the record of the task a sweep starts the item
    // with (the first for the forward sweep, the last for the backward one)
    // together with the item's task range and successor, so that one load
    // starts an item: front_off (2 words), vec_off (2), f | npiv << 16, first
    // child slot, end child slot, then for the forward sweep t1, t0, parent
    // item, and for the backward sweep t0, t1, the child item run next; then
    // the task's original entries' range (2 words)
    const int4 *item_fwd, *item_bwd;
    const int32_t *item_cont;     // backward sweep: child item run next by the same warp (-1 none)
    // ready queues of items (three per run: the factorization phases, or
    // the forward and backward sweeps)
    int *q_slots_a, *q_slots_b, *q_slots_c;   // n_items each: item ids as they became ready
    int *q_ctr;                   // [a.claim, a.fill, b.claim, b.fill, c.claim, c.fill]
    int *q_pending;               // n_items: outstanding dependencies
    const int32_t *init_small, *init_med, *init_big, *init_fwd, *init_bwd;
    int n_init_small, n_init_med, n_init_big, n_init_fwd, n_init_bwd;
    const int32_t *pend_factor;   // dependencies counted by the factorization phases
    const int32_t *nchild;        // child items per item
};
// ovals[p] = scale[i] K_ij scale[j] for the p-th original front entry
template <typename T>
void launch_orig_vals(const DevFront &F, T *ovals, cudaStream_t s);

struct FactorStatus {             // device-side counters
    int n_pos, n_neg, n_zero, error, timeout_task;
    unsigned bar_count, bar_gen;     // grid barrier of the dense border factor
    int pad;
};

// Symmetric Ruiz equilibration of K (scale[i] > 0, `iters` sweeps).
// iters Ruiz sweeps of K into scale (tmp: ping-pong buffer; mx: n_kkt
// zeros on entry and on return)
void launch_equilibrate(const DevModel &M, const double *kval, double *scale, double *tmp,
                        unsigned long long *mx, int iters, cudaStream_t s);
template <typename T>
void launch_factor(const DevFront &F, T *fronts, FactorStatus *st, double pivot_tol,
                   int spin_limit, cudaStream_t s);
template <typename T>
void launch_schur_sum(const DevFront &F, const T *fronts, double *S, cudaStream_t s);
cudaError_t launch_dense_ldlt(double *S, int n, FactorStatus *st, double pivot_tol,
                              cudaStream_t s, int spin_limit = 1 << 22);
// Sinv = S^-1 from the LDL^T factors in S (one triangular solve pair per column)
void launch_dense_inverse(const double *S, int n, double *Sinv, cudaStream_t s);

// x = K^-1 b through the factors of D K D: x = D (DKD)^-1 D b
template <typename T>
// Sinv: explicit inverse of S (n x n, column-major) or NULL to solve with
// the LDL^T factors held in S
void launch_solve(const DevFront &F, const T *fronts, T *vec, const double *S, const double *Sinv,
                  int nS, const double *scale, const double *b, double *x, double *border_work,
                  FactorStatus *st, int spin_limit, cudaStream_t s);

}  // namespace scopf
