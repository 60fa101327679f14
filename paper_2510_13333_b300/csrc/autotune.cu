// Autotuner of the supernodal factorization's tile shapes: the work-item
// size of the tile-sized fronts (cluster_max_tasks: how many small fronts one
// warp runs as a subtree) and the supernode amalgamation limit
// (relax_max_nodes: how many nodes an only-child chain merges into one
// front).  Both are measured on the instance itself: a short NCL run gives
// a representative iterate, and every candidate handle times the Newton
// steps of the interior-point method (model, assembly, factorization with
// inertia correction, Schur border, refined solve, recovery) from that same
// iterate with CUDA events.  The iterate's vectors are in the natural order,
// which no symbolic option changes, so every candidate starts from the same
// point.  The symbolic options stay part of the bit-exact specification:
// the oracle reproduces the analysis for any value chosen.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "handle.h"

namespace {

struct Cand {
    int32_t cluster, relax;
};

// A candidate replaces the best so far only when its Newton step is faster
// by more than this fraction: repeated timings of one shape differ by well
// under 1%, and shapes within the noise would otherwise be picked at random
// from run to run (each shape rounds the factors differently, so the
// interior-point path would change with them).
constexpr double kMargin = 0.02;

// mean ms of `steps` Newton steps on h from the iterate of h0 (after one
// untimed step)
int time_steps(scopf_handle *h, scopf_handle *h0, int steps, double *ms) {
    int r = scopf_load_state(h, &h0->st);
    if (r != SCOPF_OK) return r;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double out[6];
    int32_t inertia[3];
    r = scopf_newton_step(h, &h->st, h0->lam_n, h0->nu0_n, h0->rho, h0->mu_last, h0->dw_last,
                          nullptr, out, inertia);
    if (r == SCOPF_OK) {
        cudaEventRecord(e0, h->stream);
        for (int i = 0; i < steps && r == SCOPF_OK; i++)
            r = scopf_newton_step(h, &h->st, h0->lam_n, h0->nu0_n, h0->rho, h0->mu_last,
                                  h0->dw_last, nullptr, out, inertia);
        cudaEventRecord(e1, h->stream);
        cudaEventSynchronize(e1);
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t / steps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
}

}  // namespace

extern "C" int scopf_autotune(const scopf_network *net, const scopf_contingency *ctg, int32_t K,
                              scopf_options *opt, int32_t iterate_at, int32_t steps,
                              int32_t capacity, scopf_tune_entry *entries, int32_t *n_entries) {
    if (!net || !opt || iterate_at < 1 || steps < 1) return SCOPF_ERR_INVALID_ARG;
    scopf_options base = *opt;
    base.host_only = 0;
    // the representative iterate: iterate_at interior-point iterations from
    // the flat start on the base options
    scopf_options o0 = base;
    o0.max_inner = iterate_at;
    scopf_handle *h0 = nullptr;
    int r = scopf_create(net, ctg, K, &o0, &h0);
    if (r != SCOPF_OK) return r;
    scopf_result res;
    r = ncl_solve(h0, nullptr, &res);
    if (r != SCOPF_OK && r != SCOPF_ERR_MAX_ITER) {
        scopf_destroy(h0);
        return r;
    }
    if (!h0->have_ncl) {
        scopf_destroy(h0);
        return SCOPF_ERR_NUMERICAL;
    }
    std::vector<Cand> tried;
    std::vector<double> cost;
    auto run = [&](Cand c, double *ms) -> int {
        for (size_t i = 0; i < tried.size(); i++)
            if (tried[i].cluster == c.cluster && tried[i].relax == c.relax) {
                *ms = cost[i];
                return SCOPF_OK;
            }
        scopf_options oc = base;
        oc.cluster_max_tasks = c.cluster;
        oc.relax_max_nodes = c.relax;
        scopf_handle *hc = nullptr;
        int rc = scopf_create(net, ctg, K, &oc, &hc);
        if (rc != SCOPF_OK) return rc;
        scopf_set_stream(hc, h0->stream);
        rc = time_steps(hc, h0, steps, ms);
        scopf_destroy(hc);
        if (rc != SCOPF_OK) return rc;
        tried.push_back(c);
        cost.push_back(*ms);
        return SCOPF_OK;
    };
    // 1. work-item size at the base amalgamation limit, 2. amalgamation
    // limit at the best item size
    Cand best{base.cluster_max_tasks, base.relax_max_nodes};
    double best_ms = 0;
    r = run(best, &best_ms);
    for (int32_t cl : {4, 8, 16, 32}) {
        if (r != SCOPF_OK) break;
        double ms;
        r = run({cl, base.relax_max_nodes}, &ms);
        if (r == SCOPF_OK && ms < best_ms * (1.0 - kMargin)) {
            best_ms = ms;
            best = {cl, base.relax_max_nodes};
        }
    }
    for (int32_t rx : {4, 8, 16}) {
        if (r != SCOPF_OK) break;
        double ms;
        r = run({best.cluster, rx}, &ms);
        if (r == SCOPF_OK && ms < best_ms * (1.0 - kMargin)) {
            best_ms = ms;
            best = {best.cluster, rx};
        }
    }
    scopf_destroy(h0);
    if (r != SCOPF_OK) return r;
    opt->cluster_max_tasks = best.cluster;
    opt->relax_max_nodes = best.relax;
    const int32_t n = (int32_t)tried.size();
    if (n_entries) *n_entries = n;
    for (int32_t i = 0; entries && i < n && i < capacity; i++) {
        entries[i].cluster_max_tasks = tried[i].cluster;
        entries[i].relax_max_nodes = tried[i].relax;
        entries[i].ms_per_step = cost[i];
        entries[i].chosen = tried[i].cluster == best.cluster && tried[i].relax == best.relax;
    }
    return SCOPF_OK;
}
