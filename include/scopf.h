/*
 * scopf.h -- C ABI of the B300 library for the Newton step of the NCL
 * augmented-Lagrangian / interior-point method on polar AC-SCOPF with
 * complementarity-modelled recourse (Pacaud, Nurkanovic, Pozharskiy,
 * Montoison, Shin: "An Augmented Lagrangian Method on GPU for
 * Security-Constrained AC Optimal Power Flow").
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: SCOPF_OK (0) or a negative
 *    SCOPF_ERR_* code; scopf_strerror() names it.  No C++ exception crosses
 *    this boundary.
 *  - "host" pointers are read during the call only and copied; the caller
 *    keeps ownership.  "device" pointers are CUDA global-memory pointers that
 *    the caller owns and keeps alive until the call has returned (all calls
 *    synchronise the handle's stream before returning, except where noted).
 *  - A handle is not thread-safe; use one handle per host thread / stream.
 *  - Floating point is IEEE FP64 unless stated otherwise.
 *
 * Vector layouts ("natural order")
 *  Variables w = [block 0 | block 1 | ... | block K | border u0], where the
 *  border u0 = (p_g^0 for every generator, v_b^0 for every PV bus in
 *  increasing bus id) holds the first-stage controls of Section II-B.
 *  Block 0 (base case): theta_b (b != ref), v_b (buses without generator),
 *  q_g^0, thermal slacks (per limited branch: from end, to end).
 *  Block k >= 1: theta_b (b != ref), v_b, p_g^k, q_g^k (generators in
 *  service), Delta^k, thermal slacks, pi_-, pi_+, sig_pmax, sig_pmin (per
 *  generator in service), nu_-, nu_+, sig_qmax, sig_qmin (per switch bus).
 *  Equality rows c = [block 0 | ... | block K]; per block: Pbal_b, Qbal_b
 *  (all buses), thermal rows (f, t per limited branch); k >= 1 adds droop,
 *  sig_pmax-def, sig_pmin-def (per generator), pvpq, sig_qmax-def,
 *  sig_qmin-def (per switch bus).  Complementarity pairs (p of them) are
 *  [block 1 | ... | block K]; per block (pi_-, sig_pmax), (pi_+, sig_pmin)
 *  per generator, then (nu_-, sig_qmax), (nu_+, sig_qmin) per switch bus.
 *  KKT vectors of eq. (newtonsystem) are ordered per block
 *  [dw_k ; dlam_k ; dyc_k] for k = 0..K, then du0.
 */
#ifndef SCOPF_H
#define SCOPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------- */
#define SCOPF_OK 0
#define SCOPF_ERR_INVALID_ARG -1
#define SCOPF_ERR_CUDA -2
#define SCOPF_ERR_NOT_FACTORED -3
#define SCOPF_ERR_WRONG_INERTIA -4
#define SCOPF_ERR_REFINE_STALL -5
#define SCOPF_ERR_INFEASIBLE -6
#define SCOPF_ERR_MAX_ITER -7
#define SCOPF_ERR_TIMEOUT -8
#define SCOPF_ERR_OOM -9
#define SCOPF_ERR_NUMERICAL -10

#define SCOPF_CTG_LINE 0
#define SCOPF_CTG_GEN 1

#define SCOPF_PREC_FP64 0   /* block factors and solves in FP64 */
#define SCOPF_PREC_MIXED 1  /* FP32 block factors and solves, FP64 Schur factor,
                               FP64 residual and refinement */

typedef struct scopf_handle scopf_handle;

/* Network (host arrays, copied by scopf_create).  Per unit on 100 MVA.
 * Buses: Pd, Qd (load), Gs, Bs (shunt), vmin, vmax.
 * Branches (pi-model, tap 1): from, to, r, x, b (total charging), rate
 *   (apparent-power limit; 0 = unlimited).
 * Generators: bus (at most one generator per bus), pmin, pmax, qmin, qmax,
 *   cost c2 ($/MW^2h), c1 ($/MWh), c0 ($/h).  ref_bus: angle reference. */
typedef struct {
    int32_t n_bus, n_branch, n_gen, ref_bus;
    const double *Pd, *Qd, *Gs, *Bs, *vmin, *vmax;
    const int32_t *br_from, *br_to;
    const double *br_r, *br_x, *br_b, *br_rate;
    const int32_t *gen_bus;
    const double *pmin, *pmax, *qmin, *qmax, *c2, *c1, *c0;
} scopf_network;

/* One contingency: loss of a line or a generator (Section II), with the set
 * of PV buses whose voltage control follows eq. (pvpq) (host array). */
typedef struct {
    int32_t kind;      /* SCOPF_CTG_LINE or SCOPF_CTG_GEN */
    int32_t element;   /* branch or generator index */
    int32_t n_switch;
    const int32_t *switch_buses;  /* sorted, each with an in-service generator */
} scopf_contingency;

/* Algorithm constants.  tol and mu_min follow Section V-A; the others are
 * the published defaults of the NCL (Montoison et al.) and interior-point
 * (Waechter & Biegler 2006) methods the paper builds on.
 * scopf_default_options fills every field. */
typedef struct {
    double tol, mu_min, mu_init, kappa_eps, kappa_mu, theta_mu, tau_min, s_max;
    double kappa_sigma, bound_relax, bound_push, bound_frac, slack_init, comp_init;
    double delta_w0, delta_w_min, delta_w_max, kappa_w_minus, kappa_w_plus, kappa_w_plus_bar;
    double gamma_theta, gamma_phi, delta_sw, s_theta, s_phi, eta_phi, gamma_alpha;
    double rho_init, rho_max, eta_init, omega_init;
    double refine_tol;        /* target |K dx - b|_inf / |b|_inf of kkt_solve */
    double pivot_tol;         /* |d| below this counts as a zero pivot */
    int32_t max_backtrack, max_outer, max_inner, max_refine;
    int32_t precision;        /* SCOPF_PREC_FP64 or SCOPF_PREC_MIXED */
    int32_t relax_max_nodes;  /* supernode amalgamation limit (nodes) */
    int32_t verbose;
    int32_t spin_limit;       /* bound on device-side dependency waits (polls) */
    int32_t host_only;        /* 1: scopf_create builds the model and the symbolic
                                 analysis only (no device memory is touched); the
                                 device entry points then return
                                 SCOPF_ERR_INVALID_ARG */
    int32_t cluster_max_tasks; /* a subtree of at most this many small fronts is
                                 one work item of the factorization and solve
                                 sweeps (run by one warp); >= 1 */
    int32_t relax_max_front;  /* relaxed amalgamation: a supernode absorbs a child
                                 while its front stays within this many rows
                                 (0 = off) */
    int32_t device_loop;      /* 1: the FGMRES Krylov steps of a refinement cycle
                                 run as one CUDA graph (a WHILE node repeating one
                                 captured step) with no host round trip per step;
                                 0: host-driven loop */
    int32_t fp64_switch_refine;  /* mixed precision: switch to FP64 factors for the
                                 rest of the solve once fp64_switch_streak Newton
                                 steps in a row needed at least this many
                                 refinement steps (0 = only when refinement
                                 stalls).  Default 6 */
    int32_t fp64_switch_streak;  /* default 5 */
    int32_t known_zero_pivot; /* 1: the inertia correction's first trial, delta_w = 0
                                 (IC-1 of Waechter & Biegler 2006), is taken as
                                 failed without factoring when the factorization
                                 must meet an exactly zero pivot: a primal row
                                 with no stored entry eliminated before it and a
                                 zero diagonal at delta_w = 0.  The outcome is
                                 the one factoring would give, so iterates are
                                 unchanged; 0: always factor at delta_w = 0 */
    int32_t dual_first;       /* 1: the condensed primal variant (Section IV-B,
                                 "signed Cholesky"): the symbolic order puts every
                                 block's dual rows (equality and complementarity
                                 rows) before its primal rows.  -C is diagonal, so
                                 the factorization first eliminates it exactly
                                 (pivots -C) and then factors the condensed matrix
                                 A + B' C^-1 B with positive pivots when K has the
                                 wanted inertia (Haynsworth).  0: node minimum
                                 degree over primal and dual rows together */
    int32_t fixed_mu;         /* 1: the interior-point loop keeps the barrier
                                 parameter at its starting value (mu_init, or the
                                 handle's mu for ncl_resume) and stops on the
                                 barrier error E_mu <= tol instead of E_0: the
                                 solution of the barrier problem at that mu, the
                                 smooth map scopf_adjoint differentiates */
    int32_t ipm_graph;        /* 1: each interior-point iteration, after the host's
                                 convergence test and barrier update, runs as two
                                 CUDA-graph launches with one host read-back: the
                                 inertia-correction trials, the refinement cycles
                                 (with their Krylov steps) and the filter
                                 line-search trials are WHILE nodes, the solve
                                 after a successful inertia correction and the
                                 elastic restoration IF nodes (Section IV-B; the
                                 decisions are those of the host loop).  If the
                                 graphs cannot be built the host loop runs (the
                                 reason in scopf_last_error).  Needs
                                 device_loop = 1.  0: host loop.  Default 1 */
} scopf_options;

/* Sizes of the handle's problem. */
typedef struct {
    int64_t n, m, p;          /* variables, equality rows, complementarity pairs */
    int64_t n_kkt;            /* rows of eq. (newtonsystem) = n + m + p */
    int64_t n_border;         /* first-stage variables u0 */
    int32_t n_blocks;         /* K + 1 */
    int64_t nnz_kkt;          /* stored nonzeros of the full symmetric KKT */
    int64_t nnz_L;            /* factor entries (supernodal, incl. explicit zeros) */
    int64_t n_supernodes;
    double factor_flops;      /* flops of one block factorisation (all blocks) */
    int64_t front_bytes;      /* device bytes of the frontal storage */
    int64_t n_elem_values;    /* model-evaluation value slots written per assembly */
    int64_t n_contrib;        /* (slot, coefficient) contributions gathered into K */
} scopf_sizes;

/* Primal-dual iterate (device pointers, FP64).  zl and zu have length n and
 * are read only where the bound is finite. */
typedef struct {
    double *w, *r, *t, *s, *lam, *yc, *zl, *zu, *zs;
} scopf_state;

/* Outcome of ncl_solve. */
typedef struct {
    int32_t status;           /* SCOPF_OK, SCOPF_ERR_INFEASIBLE, SCOPF_ERR_MAX_ITER, ... */
    int32_t outer_iters, inner_iters, factorizations, refine_steps;
    int32_t fp64_fallbacks;   /* mixed mode: Newton steps redone in FP64 */
    double objective, kkt_error, feas_rt, max_violation, rho, mu;
    double time_total_s, time_newton_s;
    double delta_w_last;      /* last nonzero inertia-correction delta_w */
    int64_t host_round_trips; /* stream synchronisations the host waited on
                                 (reductions read back, inertia, refinement
                                 cycles, line-search trials) during the solve */
    int32_t graph_iters;      /* interior-point iterations run as graph launches
                                 (option ipm_graph) */
    int32_t pad;
} scopf_result;

void scopf_default_options(scopf_options *opt);

/* Build the model of eq. (scopf) for the network and K contingencies, its
 * layouts, the KKT pattern and the symbolic analysis of every block, and
 * allocate device memory.  opt may be NULL (defaults). */
int scopf_create(const scopf_network *net, const scopf_contingency *ctg, int32_t K,
                 const scopf_options *opt, scopf_handle **out);
void scopf_destroy(scopf_handle *h);
const char *scopf_strerror(int status);
/* Text of the handle's last CUDA or internal error (owned by the handle,
 * valid until its next call; "" when none). */
const char *scopf_last_error(scopf_handle *h);

int scopf_get_sizes(scopf_handle *h, scopf_sizes *out);
/* Run the handle's kernels on this CUDA stream (cudaStream_t); NULL = legacy default. */
int scopf_set_stream(scopf_handle *h, void *stream);
int scopf_set_precision(scopf_handle *h, int32_t precision);

/* Symbolic analysis of block k (Section IV-B: static structure of the
 * pivot-free factorisation).  Host output arrays sized by the call with
 * NULL pointers first: *n_nodes, *n_block_nodes, *n_sn, *n_rows are always
 * written.  post[n_block_nodes]: node ids in elimination (post)order;
 * node_parent[n_block_nodes]: parent node id (-2 = border, -1 = none);
 * sn_start[n_sn+1]: supernode boundaries in postorder positions;
 * rows[n_rows]: KKT indices (global natural order) in elimination order,
 * block rows then border rows. */
int scopf_symbolic_block(scopf_handle *h, int32_t k, int32_t *n_nodes, int32_t *n_block_nodes,
                         int32_t *n_sn, int32_t *n_rows, int32_t *post, int32_t *node_parent,
                         int32_t *sn_start, int64_t *rows);

/* Model evaluation (Section II / eq. mpcc) at device w, lam: the objective
 * (host out), its gradient g[n], the constraint values c[m] (device).  Any
 * output pointer may be NULL. */
int scopf_eval(scopf_handle *h, const double *w, double *obj, double *g, double *c);

/* KKT assembly (eq. newtonsystem) at the iterate: A = H + barrier diagonal
 * + V0 coupling + delta_w I, B = [J; (0 W2 W1)], C = diag(1/rho, 1/rho +
 * s/zs).  lam_n, nu0_n: NCL multiplier estimates (device, m and p).  Also
 * forms the right-hand side for barrier parameter mu into rhs (device,
 * n_kkt; may be NULL).  The values are kept on the device for kkt_factor. */
int kkt_assemble(scopf_handle *h, const scopf_state *it, const double *lam_n,
                 const double *nu0_n, double rho, double mu, double delta_w, double *rhs);
/* Copy the assembled KKT matrix out (device, CSR in natural KKT order):
 * row_ptr[n_kkt+1], col[nnz] (int64) and val[nnz]; any may be NULL. */
int kkt_export(scopf_handle *h, int64_t *row_ptr, int64_t *col, double *val);

/* Pivot-free LDL^T of every block (three persistent launches, one per
 * front-size phase: tile-sized fronts, medium fronts, large fronts), Schur
 * complement onto u0 and its dense LDL^T.  inertia[0..2] = (#positive, #negative,
 * #zero-or-tiny pivots) over the whole KKT (host out).  precision overrides
 * the handle's setting for this factorisation (-1 = handle's). */
int kkt_factor(scopf_handle *h, int32_t precision, int32_t inertia[3]);

/* Solve K x = b with the last factorisation and FP64 iterative refinement
 * against the assembled (unregularised delta_w = 0 part excluded only when
 * delta_w was 0) matrix until |b - Kx|_inf <= refine_tol |b|_inf or
 * max_refine steps (-1 = options).  b, x: device, n_kkt, natural KKT order
 * (x may alias b).  rel_residual and steps (host out, may be NULL). */
int kkt_solve(scopf_handle *h, const double *b, double *x, int32_t max_refine,
              double *rel_residual, int32_t *steps);

/* One Newton step of the interior-point method on the NCL subproblem
 * (Section IV-B) at the iterate `it` (device, left unchanged): model
 * evaluation, KKT assembly with the barrier parameter mu, factorization
 * with inertia correction (delta_w starting from 0, the last successful
 * value dw_last guiding the first increase), Schur complement and border
 * factor, solve with iterative refinement (mixed mode falls back to FP64
 * factors if refinement stalls), recovery of the eliminated directions,
 * fraction-to-boundary step and one trial evaluation at the full step.
 * dir: device buffers for the direction (may be NULL: kept in the handle).
 * out (host, 6): alpha_primal, alpha_dual, theta at the trial point,
 * barrier objective at the trial point, delta_w used, preconditioner
 * applications (block solves: one per kkt solve plus its refinement steps).
 * inertia (host, 3): n and m + p (the inertia the correction reached), then
 * the number of factorizations it took. */
int scopf_newton_step(scopf_handle *h, const scopf_state *it, const double *lam_n,
                      const double *nu0_n, double rho, double mu, double dw_last,
                      scopf_state *dir, double out[6], int32_t inertia[3]);

/* Device-time breakdown (CUDA events on the handle's stream) of the
 * library's phases: 0 model evaluation + assembly, 1 front initialisation,
 * 2 block factorization (persistent kernel), 3 Schur sum + border factor,
 * 4 triangular solves, 5 refinement residuals, 6 IPM vector kernels.
 * enable = 1 starts (and zeroes) the timers, 0 stops them; ms_out[7] and
 * calls_out[7] (host, may be NULL) receive the accumulated totals. */
int scopf_timing(scopf_handle *h, int32_t enable, double *ms_out, int32_t *calls_out);

/* Scheduler trace.  The factorization and the triangular sweeps run work
 * items (a subtree of small fronts run by one warp, or one front) from ready
 * queues.  enable = 1 allocates a device buffer and makes every later sweep
 * record, per item, four uint64: the device clock (%globaltimer, ns) when
 * its worker started to look for it (or finished the item it continues
 * from), when it started it, when it finished it, and the SM it ran on;
 * 0 stops recording and frees the buffer.  Kinds: 0 forward sweep, 1
 * backward sweep, 2-4 factorization phases 1-3 (tile-sized fronts, medium
 * fronts and their ancestors, large fronts and theirs); each keeps the
 * record of its last run (zeros for items that did not run).
 * scopf_trace_read copies kind `kind` to out (host, 4 * n_items uint64).
 * scopf_trace_items describes the items: out (host, 6 * n_items int32) =
 * fronts in the item, parent item (-1 none), factorization phase (1-3),
 * largest front (rows), total pivots, block; returns n_items through
 * *n_items (out may be NULL). */
/* Number of kernels the library has launched in this process so far
 * (all handles; host only, no synchronization). */
int scopf_launch_count(int64_t *out);

int scopf_trace(scopf_handle *h, int32_t enable);
int scopf_trace_read(scopf_handle *h, int32_t kind, uint64_t *out);
int scopf_trace_items(scopf_handle *h, int32_t *n_items, int32_t *out);

/* Dense pivot-free LDL^T factorization and solve of a symmetric n x n
 * matrix: the factor of the first-stage Schur complement (border block) of
 * eq. (newtonsystem), available on its own.  S: device, column-major,
 * n*n, read only (a private copy is factored); b, x: device, n (x may not
 * alias S).  inertia (host, 3, may be NULL): signs of D.  stream: a
 * cudaStream_t or NULL.  Allocates its scratch (n*n + n doubles) with
 * cudaMalloc and frees it before returning.  A zero pivot (singular S) is
 * replaced by a tiny one and counted in inertia[2]; the call still returns
 * SCOPF_OK with a huge or non-finite x, so a caller that may pass a
 * singular S must pass inertia and check inertia[2] == 0. */
int scopf_dense_ldlt_solve(const double *S, int32_t n, const double *b, double *x,
                           int32_t inertia[3], void *stream);

/* The same factor + solve for callers that must not allocate device memory
 * during the call (e.g. an application whose device memory is reserved by
 * its own pool allocator, or a latency-critical loop that cannot take the
 * device-wide synchronisation of cudaMalloc/cudaFree).  The paper has no
 * counterpart: this is a deployment variant of scopf_dense_ldlt_solve.
 * Scratch is a static per-device array sized for n <= 768 (about 4.7 MB,
 * held by every GPU that loads the library until exit); n > 768 returns
 * SCOPF_ERR_INVALID_ARG.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress).
 * That address is cached per device ordinal for the life of the process: it
 * goes stale if the caller resets the device (cudaDeviceReset) and goes on
 * using the library.  Concurrent first calls from several host threads are
 * safe (the cache is atomic).  Each call synchronises its stream before
 * returning, so calls overlap on the GPU only when host threads call at
 * once; all calls on a device share the array, so such calls race and must
 * be ordered by the caller.  Zero pivots are reported as for
 * scopf_dense_ldlt_solve (check inertia[2]). */
int scopf_dense_ldlt_solve_noalloc(const double *S, int32_t n, const double *b, double *x,
                                   int32_t inertia[3], void *stream);

/* Arithmetic-throughput probe (measurement support for the roofline
 * fractions; the paper has no counterpart).  Launches one kernel on stream
 * (a cudaStream_t or NULL) that keeps every SM busy with independent chains
 * of kind 0: FP32 FMA, 1: FP64 FMA, 2: FP64 tensor MMA (mma.sync m8n8k4),
 * 3: FP64 FMA on one lane per warp (flops of the active lanes only),
 * 4: FP64 FMA on even warps and FP64 tensor MMA on odd warps at once (equal
 * flops per warp pair: whether the two share a pipe), iters iterations
 * each, and returns the launch's flop count in *flops (host, an FMA counted
 * as 2).  out: device, at least 8 bytes, written only in a
 * case that never occurs (it keeps the chains from being optimised away).
 * The caller times the launch (CUDA events on the same stream).  Does not
 * synchronise. */
int scopf_peak_probe(int32_t kind, int64_t iters, double *out, void *stream, double *flops);

/* One candidate of scopf_autotune. */
typedef struct {
    int32_t cluster_max_tasks, relax_max_nodes;
    double ms_per_step;       /* mean Newton step time from the common iterate */
    int32_t chosen;           /* 1 for the candidate written back into the options */
} scopf_tune_entry;

/* Autotuner of the supernodal tile shapes (the paper leaves them to cuDSS
 * and has no counterpart of this call): chooses cluster_max_tasks (small
 * fronts per warp work item) and relax_max_nodes (nodes an only-child chain
 * merges into one supernode) for this instance.  A short NCL run
 * (iterate_at interior-point iterations from the flat start, options *opt)
 * gives a common iterate; each candidate handle times `steps` Newton steps
 * (scopf_newton_step, after one untimed step) from it with CUDA events.
 * Candidates: item sizes 4, 8, 16, 32 at the given amalgamation limit, then
 * limits 4, 8, 16 at the best item size; a candidate replaces the best so
 * far only when it is more than 2% faster (shapes within the timing noise
 * keep the given ones, so the choice is repeatable).  On return opt holds
 * the chosen pair (every other field unchanged); entries
 * (host, capacity, may be NULL) receive the candidates in the order tried,
 * *n_entries their number.  Creates and destroys one handle per candidate on
 * the current device (device memory of two handles at a time). */
int scopf_autotune(const scopf_network *net, const scopf_contingency *ctg, int32_t K,
                   scopf_options *opt, int32_t iterate_at, int32_t steps, int32_t capacity,
                   scopf_tune_entry *entries, int32_t *n_entries);

/* The reciprocal the FP64 block factorization takes of its pivots (Newton's
 * method from a single-precision seed, within one unit in the last place of
 * 1/d), exposed so that it can be checked against the quotient: out[i] =
 * 1 / d[i] for n device values (stream-ordered, no synchronisation).  Not a
 * step of the paper's method. */
int scopf_pivot_reciprocal(const double *d, double *out, int64_t n, void *stream);

/* Full NCL solve (Section IV-A) from the flat start, or from warm (device
 * state, may be NULL).  The final iterate stays in the handle. */
int ncl_solve(scopf_handle *h, const scopf_state *warm, scopf_result *res);

/* Checkpoint / resume (the warm start between NCL outer iterations, Section
 * IV-A): continue the method from the handle's current iterate and NCL
 * parameters (lam_n, nu0_n, rho, mu, eta, omega).  These are left by the
 * handle's last ncl_solve / ncl_resume, or restored on any handle of the
 * same problem with scopf_load_state + scopf_set_ncl_params (which resets
 * eta and omega to their initial values).  The inner-iteration count and
 * limit start afresh.  SCOPF_ERR_INVALID_ARG if no parameters are set. */
int ncl_resume(scopf_handle *h, scopf_result *res);
/* Device views of the handle's current iterate (owned by the handle). */
int scopf_get_state(scopf_handle *h, scopf_state *out);
/* Copy the handle's iterate into caller-owned device buffers (dst fields
 * may be NULL to skip), or load it from src into the handle (src fields
 * must all be set).  Stream-ordered; synchronised before return. */
int scopf_copy_state(scopf_handle *h, const scopf_state *dst);
int scopf_load_state(scopf_handle *h, const scopf_state *src);
/* NCL multiplier estimates of the last solve (device views, m and p), rho. */
int scopf_get_ncl_params(scopf_handle *h, double **lam_n, double **nu0_n, double *rho);

/* Parameters of the instance that the adjoint differentiates: bus loads Pd,
 * Qd (n_bus, per unit) and linear cost coefficients c1 (n_gen), host arrays
 * copied into the handle (any may be NULL = unchanged).  The structure is
 * unchanged, so no symbolic work is redone; a later ncl_solve uses them. */
int scopf_set_params(scopf_handle *h, const double *Pd, const double *Qd, const double *c1);

/* Make the handle's current state (scopf_load_state) and these NCL
 * parameters (device lam_n: m, nu0_n: p; rho > 0, barrier mu > 0) the
 * solution that scopf_adjoint differentiates; ncl_solve sets them itself. */
int scopf_set_ncl_params(scopf_handle *h, const double *lam_n, const double *nu0_n, double rho,
                         double mu);

/* Adjoint of the converged solution (implicit function theorem on the
 * barrier KKT conditions of eq. (newtonsystem) at the final iterate):
 * gradients of J = seed_pg0' p_g^0 + seed_cost * objective with respect to
 * the bus loads Pd, Qd (n_bus each) and the linear cost coefficients c1
 * (n_gen), from one symmetric solve K a = dJ/dz.  K is refactored in FP64 at
 * the final iterate with the method's inertia correction, and the solve is
 * refined against the unshifted K.  seed_pg0: device, n_gen (NULL = zero);
 * outputs: device.  SCOPF_ERR_NOT_FACTORED if no solution is loaded. */
int scopf_adjoint(scopf_handle *h, const double *seed_pg0, double seed_cost,
                  double *grad_Pd, double *grad_Qd, double *grad_c1);

/* Iteration log of the handle's last ncl_solve (or scopf_screen).
 * which = 0: one record per interior-point iteration, 16 doubles: outer
 *   iteration, inner iteration (cumulative), mu, rho, scaled KKT error E_0
 *   before the step, constraint violation theta and barrier objective phi at
 *   the iterate, accepted primal and dual step lengths, delta_w, number of
 *   factorizations (inertia corrections and FP64 fallback included),
 *   refinement steps, precision of the factors that produced the step
 *   (SCOPF_PREC_*), 1 if the filter accepted the step (0: elastic reset),
 *   backtracking steps, wall time of the iteration in ms (host clock, from
 *   the right-hand side to the next iterate's norms read back).
 * which = 1: one record per NCL outer iteration, 8 doubles: outer iteration,
 *   rho, |r|_inf, |t|_inf, E_0, eta, omega, inner iterations so far.
 * *n_records and *record_len receive the log's size; out (host, capacity
 * records, may be NULL) receives the first min(n_records, capacity). */
int scopf_history(scopf_handle *h, int32_t which, int64_t capacity, double *out,
                  int64_t *n_records, int32_t *record_len);

/* Per-scenario infeasibility of the handle's current iterate: viol[k] =
 * |(r_k, t_k)|_inf over the constraint rows and complementarity pairs of
 * scenario k (k = 0 base case), the relaxations of eq. (nclsubpb).  viol:
 * host, n_blocks = K + 1.  A NaN entry of r or t reports as +inf. */
int scopf_block_violation(scopf_handle *h, double *viol);

/* Batched contingency screening (Section V-B, eqs. (screening), (feaspb)):
 * every scenario of the handle is checked for feasibility at the base-case
 * control u0 in one NCL solve.  u0 (host, n_border) boxes the first-stage
 * variables to [max(lo, u0 - eps), min(hi, u0 + eps)], widened to width eps
 * where u0 sits on a limit (eps > 0; a tiny eps decouples the scenarios into
 * the per-contingency systems); u0 = NULL leaves them free.  The outer loop
 * runs per block: while one scenario drives rho up, every scenario with
 * |(r_k, t_k)|_inf <= eta still takes its multiplier update.  The solve caps rho at rho_cap (the
 * handle's iteration limits apply); res receives its outcome, viol[k] (host, K + 1) the scenario's
 * |(r_k, t_k)|_inf at the end, and accepted[k] (host, K + 1) is 1 when
 * viol[k] <= accept_tol and the solve ended by convergence, by the rho cap
 * (SCOPF_ERR_INFEASIBLE) or by the outer-iteration limit, else 0.  The
 * handle's bounds and options are restored on return; its iterate is the
 * screening solve's final one.  Returns SCOPF_OK whenever the verdicts were
 * computed (res->status carries the solve's own status). */
int scopf_screen(scopf_handle *h, const double *u0, double eps, double rho_cap,
                 double accept_tol, scopf_result *res, double *viol, int32_t *accepted);

#ifdef __cplusplus
}
#endif
#endif /* SCOPF_H */
