// The library handle: host model, symbolic/frontal structure, device buffers.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "fronts_host.h"
#include "internal.h"
#include "kernels.h"

namespace scopf {

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
};

struct ScalarScratch {
    double *d = nullptr;      // device scalars
    double *partial = nullptr;
};

// CUDA-event timers of the library's phases on the handle's stream.  Each
// phase is also an NVTX range (start/end form, so phases may interleave),
// visible to a profiler whether or not the timers are on.
struct PhaseTimer {
    static constexpr int kPhases = 7;
    static constexpr const char *kNames[kPhases] = {"scopf assemble", "scopf front_init",
                                                    "scopf factor",   "scopf schur",
                                                    "scopf solve",    "scopf residual",
                                                    "scopf ipm"};
    nvtxRangeId_t range[kPhases] = {};
    bool on = false;
    double ms[kPhases] = {};
    int calls[kPhases] = {};
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    cudaEvent_t open[kPhases] = {};

    cudaEvent_t get() {
        if (pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    void begin(int ph, cudaStream_t s) {
        if (range[ph]) nvtxRangeEnd(range[ph]);
        range[ph] = nvtxRangeStartA(kNames[ph]);
        if (!on) return;
        open[ph] = get();
        cudaEventRecord(open[ph], s);
    }
    void end(int ph, cudaStream_t s) {
        if (range[ph]) {
            nvtxRangeEnd(range[ph]);
            range[ph] = 0;
        }
        if (!on || !open[ph]) return;
        cudaEvent_t e = get();
        cudaEventRecord(e, s);
        pending.push_back({ph, {open[ph], e}});
        open[ph] = nullptr;
    }
    // call after the stream has been synchronised
    void collect() {
        for (auto &pp : pending) {
            float t = 0;
            if (cudaEventElapsedTime(&t, pp.second.first, pp.second.second) == cudaSuccess) {
                ms[pp.first] += t;
                calls[pp.first]++;
            }
            pool.push_back(pp.second.first);
            pool.push_back(pp.second.second);
        }
        pending.clear();
    }
    void reset() {
        for (int i = 0; i < kPhases; i++) {
            ms[i] = 0;
            calls[i] = 0;
        }
    }
    ~PhaseTimer() {
        for (auto &pp : pending) {
            cudaEventDestroy(pp.second.first);
            cudaEventDestroy(pp.second.second);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

enum Phase { PH_ASSEMBLE = 0, PH_FRONT_INIT, PH_FACTOR, PH_SCHUR, PH_SOLVE, PH_RESIDUAL, PH_IPM };

}  // namespace scopf

struct scopf_handle {
    scopf::Model M;
    scopf_options opt;
    std::vector<scopf::BlockSymbolic> syms;
    scopf::HostFronts HF;
    bool host_only = false;
    cudaStream_t stream = nullptr;
    int precision = SCOPF_PREC_FP64;
    std::vector<void *> allocations;
    // device model and fronts
    scopf::DevModel dm{};
    scopf::DevFront df{};
    // work buffers
    double *ev = nullptr, *kval = nullptr, *diag = nullptr, *g = nullptr, *gw = nullptr;
    double *c = nullptr, *rhs = nullptr, *sol = nullptr, *res = nullptr, *dx = nullptr;
    double *wl = nullptr, *wu = nullptr;
    void *fronts = nullptr, *vec = nullptr;
    double *S = nullptr, *border_work = nullptr;
    double *Sinv = nullptr;                           // S^-1 (mixed-precision solves)
    bool sinv_stale = false;   // S was refactored since Sinv was formed (formed on first solve)
    double *scale = nullptr, *scale_tmp = nullptr;   // Ruiz equilibration of K
    unsigned long long *ruiz_mx = nullptr;          // per-row maxima of a Ruiz sweep (zeros)
    double *kv = nullptr, *kz = nullptr, *kpart = nullptr;  // FGMRES basis and scratch
    double *kst = nullptr;                                  // FGMRES small dense state
    // device-resident Krylov loop: control block, fixed step buffers (the
    // preconditioner's input and output, the new direction) and, per factor
    // precision, the instantiated graph whose WHILE node repeats the step
    scopf::KrylovCtl *kctl = nullptr;
    double *kry_buf = nullptr;
    struct KrylovGraph {
        cudaGraphExec_t exec = nullptr;
        long long body_kernels = 0;
        bool failed = false;
    } kgraph[2];
    bool kgraph_stale = false;   // a kernel argument captured in the graphs changed
    // device-resident interior-point iteration (option ipm_graph): control
    // block, filter entries, generator constant costs, and two graphs per
    // iteration -- the direction (one per factor precision) and the step
    scopf::IpmCtl *ipm_ctl = nullptr;
    double *ipm_filter = nullptr;
    double *gen_c0 = nullptr;
    struct IpmGraphs {
        cudaGraphExec_t dir[2] = {nullptr, nullptr};   // [mixed, FP64]
        cudaGraphExec_t step = nullptr;
        bool failed = false;
        const double *key_st = nullptr, *key_trial = nullptr;   // iterate buffers captured
        // kernels per launch of each part (the launch count)
        long long k_dir_pre[2] = {}, k_ic[2] = {}, k_solve[2] = {}, k_ref[2] = {}, k_kry[2] = {};
        long long k_step_pre = 0, k_step_if = 0, k_ls = 0, k_restore = 0;
    } ig;
    bool ig_stale = false;   // a kernel argument captured in the iteration graphs changed
    double *ovals = nullptr;                                // scaled front originals
    scopf::FactorStatus *fstat = nullptr;
    double *red_scratch = nullptr, *red_out = nullptr;
    bool assembled = false, factored = false;
    int factored_precision = SCOPF_PREC_FP64;
    double last_delta_w = 0.0, last_rho = 0.0;
    double assembled_delta_w = 0.0;           // delta_w of the last full assembly
    int64_t n_lower = 0, n_upper = 0;         // finite variable bounds
    double *ipm_part = nullptr;               // per-block partials of the IPM reductions
    int64_t n_pdiag = 0;                      // primal rows
    const int64_t *pdiag_pos = nullptr;       // their diagonal entries in kval
    double *pdiag_base = nullptr;             // those entries at the last assembly
    // primal rows whose pivot is their own diagonal entry (no stored entry of
    // the row is eliminated before it), as indices into pdiag_pos / pdiag_base
    int64_t n_lead = 0;
    const int64_t *lead_pdiag = nullptr;
    int *lead_zero = nullptr;                 // device count of those with a zero diagonal
    int lead_zero_host = 0;                   // that count, read back with the IPM norms
    bool lead_zero_valid = false;             // lead_zero_host describes the assembled K
    // iterate and NCL parameters owned by the handle
    scopf_state st{};
    double *lam_n = nullptr, *nu0_n = nullptr;
    double rho = 0.0;
    double mu_last = 0.0, dw_last = 0.0;   // barrier parameter and delta_w at the last solve's end
    double eta_last = 0.0, omega_last = 0.0;   // NCL tolerances at the last solve's end
    bool have_ncl = false;                 // rho, mu_last, lam_n, nu0_n, eta/omega_last are set
    bool has_solution = false;             // st, lam_n, nu0_n, rho, mu_last describe a solution
    bool inner_limit = false;              // the last solve stopped at max_inner
    long long n_solve_calls = 0;           // kkt solves (each: one preconditioner application + refinement)
    // iteration log of the last ncl_solve (records of kHistInner / kHistOuter doubles)
    std::vector<double> hist_inner, hist_outer;
    bool screen_blocks = false;            // NCL outer loop with the per-block screening rule
    // per-scenario ranges of r and t (c0, nrow, p0, ncomp) and their maxima
    int64_t *blk_rt = nullptr;
    double *blk_viol = nullptr;
    // adjoint index sets (built on first use): KKT row of every p_g^0, and
    // per bus the KKT rows of its P and Q balance in every block
    int64_t *adj_pg = nullptr, *adj_ptr = nullptr, *adj_rowsP = nullptr, *adj_rowsQ = nullptr;
    int64_t *adj_dpos = nullptr, adj_ndual = 0;   // diagonal entries of the dual rows
    double *adj_g = nullptr, *adj_a = nullptr;
    // IPM scratch (directions and trial point)
    scopf_state dir{}, trial{};
    double *tmp_n = nullptr, *tmp_m = nullptr, *tmp_p = nullptr, *tmp_kkt = nullptr;
    int64_t *d_il = nullptr, *d_iu = nullptr;
    // counters
    int n_factor = 0, n_refine = 0;
    bool force_fp64 = false;      // sticky FP64 fallback inside a solve
    long long n_known_zero = 0;   // delta_w = 0 trials taken as failed without factoring
    long long n_host_syncs = 0;   // stream synchronisations the host waited on
    unsigned long long *trace = nullptr;   // scheduler trace buffer (cudaMalloc'd)
    scopf::PhaseTimer timer;
    std::string last_error;
};

namespace scopf {
// a host wait on the handle's stream (counted: the host round trips of a solve)
inline cudaError_t host_sync(scopf_handle *h, cudaStream_t s) {
    h->n_host_syncs++;
    return cudaStreamSynchronize(s);
}
int ncl_solve_impl(scopf_handle *h, const scopf_state *warm, scopf_result *res,
                   bool resume = false);
int block_multiplier_update(scopf_handle *h, double rho, double thr);
constexpr int kHistInner = 16;   // fields of an inner-iteration record (scopf_history)
constexpr int kHistOuter = 8;    // fields of an outer-iteration record
void relaxed_bounds(const Model &M, double bound_relax, std::vector<double> &wl,
                    std::vector<double> &wu);
int ipm_partials();   // doubles of the IPM reduction partial buffer
int assemble_impl(scopf_handle *h, const scopf_state *it, const double *lam_n,
                  const double *nu0_n, double rho, double mu, double delta_w, double *rhs);
int factor_impl(scopf_handle *h, int precision, int inertia[3]);
int set_delta_w(scopf_handle *h, double delta_w);
// FP64 or mixed factorization of K(delta_w) with the inertia correction of
// the interior-point method (the first delta_w tried follows dw_last);
// delta_w used on return
int factor_inertia(scopf_handle *h, int precision, double dw_last, double &delta, int &tries);
int solve_impl(scopf_handle *h, const double *b, double *x, int max_refine, double *rel,
               int *steps);
// pieces of the factorization and the refinement, enqueued on h->stream
// (also captured into the device-resident iteration's graphs)
template <typename T>
cudaError_t factor_enqueue(scopf_handle *h);
template <typename T>
int solve_once(scopf_handle *h, const double *b, double *x);
template <typename T>
long long enqueue_krylov_step(scopf_handle *h, cudaGraphConditionalHandle loop);
int krylov_buffers(scopf_handle *h);
void assemble_enqueue(scopf_handle *h, const scopf_state *it, DScalar rho, double delta_w);
void ipm_graphs_release(scopf_handle *h);   // destroy the iteration graphs
double device_maxabs(scopf_handle *h, const double *x, int64_t n);
double device_sumabs(scopf_handle *h, const double *x, int64_t n);
}  // namespace scopf
