// Adjoint sensitivities of the converged SCOPF solution.
//
// At the final iterate z of the NCL subproblem, the reduced barrier KKT
// conditions F(z; p) = 0 of eq. (newtonsystem) hold up to the solver
// tolerance, with K = dF/dz the matrix the Newton steps factor (Section
// IV-B).  By the implicit function theorem dz/dp = -K^-1 dF/dp, so for
// J = seed_pg0' p_g^0 + seed_cost * phi(w) (phi: the base-case cost of eq.
// (scopf)) one symmetric solve K a = dJ/dz gives dJ/dp = dJ/dp|_explicit -
// a' dF/dp.  The loads enter the bus balance rows of c(w) with coefficient
// -1 in every scenario (dF/dPd_b = -1 on those rows, so dJ/dPd_b = sum of a
// over them); c1 enters the gradient of phi (d^2 phi / dp_g dc1_g = 100 /
// 1e4 with the cost scaling of the model) and phi itself (d phi / d c1_g =
// 100 p_g / 1e4).
//
// The matrix is the rho -> infinity limit of the final subproblem's K: the
// NCL relaxation adds -1/rho to the diagonal of the constraint and
// complementarity rows (C = diag(1/rho, 1/rho + s/zs)), and the outer loop
// drives r, t to zero by raising rho and updating lam_n, nu0_n, so the
// solution it returns moves with p as the problem with hard constraints
// does.  The subproblem's K, factored with the method's inertia correction
// (pivot-free LDL^T needs C > 0 and delta_w > 0 when variables that enter
// only linearly come before their rows), preconditions FGMRES on the limit
// matrix: a solves K_inf a = dJ/dz itself.
#include <cmath>
#include <vector>

#include "handle.h"

namespace scopf {

namespace {

constexpr int kAT = 256;

__global__ void k_adj_rhs(int ng, const int64_t *__restrict__ pg_row, const double *__restrict__ seed,
                          double seed_cost, const double *__restrict__ w, int64_t border0,
                          const double *__restrict__ c2, const double *__restrict__ c1,
                          double *__restrict__ g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    const double p = w[border0 + i] * 100.0;
    const double dphi = (2.0 * c2[i] * p + c1[i]) * 100.0 / 1.0e4;
    g[pg_row[i]] = (seed ? seed[i] : 0.0) + seed_cost * dphi;
}

// out[b] = sum of a over the rows of bus b, blocks in order
__global__ void k_bus_sum(int nb, const int64_t *__restrict__ ptr, const int64_t *__restrict__ rows,
                          const double *__restrict__ a, double *__restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double acc = 0.0;
    for (int64_t q = ptr[b]; q < ptr[b + 1]; q++) acc += a[rows[q]];
    out[b] = acc;
}

__global__ void k_add_at(int64_t n, const int64_t *__restrict__ pos, double v,
                         double *__restrict__ kval) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) kval[pos[i]] += v;
}

__global__ void k_adj_c1(int ng, const int64_t *__restrict__ pg_row, const double *__restrict__ a,
                         const double *__restrict__ w, int64_t border0, double seed_cost,
                         double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    out[i] = -0.01 * a[pg_row[i]] + seed_cost * 0.01 * w[border0 + i];
}

}  // namespace

// index sets of the adjoint (host model -> device, once per handle)
static int adjoint_setup(scopf_handle *h) {
    if (h->adj_pg) return SCOPF_OK;
    const Model &M = h->M;
    std::vector<int64_t> pg(M.ng), ptr(M.nb + 1, 0), rp, rq;
    for (int g = 0; g < M.ng; g++) pg[g] = M.kkt_of_w[M.border0 + g];
    std::vector<std::vector<int64_t>> P(M.nb), Q(M.nb);
    for (const Block &B : M.blocks)
        for (int b = 0; b < M.nb; b++) {
            P[b].push_back(M.kkt_of_c[B.c0 + B.rP[b]]);
            Q[b].push_back(M.kkt_of_c[B.c0 + B.rQ[b]]);
        }
    for (int b = 0; b < M.nb; b++) {
        ptr[b + 1] = ptr[b] + (int64_t)P[b].size();
        rp.insert(rp.end(), P[b].begin(), P[b].end());
        rq.insert(rq.end(), Q[b].begin(), Q[b].end());
    }
    auto up = [&](const std::vector<int64_t> &v, int64_t **out) {
        if (cudaMalloc(out, sizeof(int64_t) * std::max<size_t>(1, v.size())) != cudaSuccess)
            return SCOPF_ERR_OOM;
        h->allocations.push_back(*out);
        if (!v.empty() &&
            cudaMemcpy(*out, v.data(), sizeof(int64_t) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return SCOPF_ERR_CUDA;
        return SCOPF_OK;
    };
    // diagonal entries of the constraint and complementarity rows
    std::vector<int64_t> dpos;
    for (int64_t i = 0; i < M.n_kkt; i++) {
        if (M.row_kind[i] == 0) continue;
        for (int64_t q = M.kkt_ptr[i]; q < M.kkt_ptr[i + 1]; q++)
            if (M.kkt_col[q] == i) {
                dpos.push_back(q);
                break;
            }
    }
    h->adj_ndual = (int64_t)dpos.size();
    int r;
    if ((r = up(pg, &h->adj_pg)) || (r = up(ptr, &h->adj_ptr)) || (r = up(rp, &h->adj_rowsP)) ||
        (r = up(rq, &h->adj_rowsQ)) || (r = up(dpos, &h->adj_dpos)))
        return r;
    for (double **p : {&h->adj_g, &h->adj_a}) {
        if (cudaMalloc(p, sizeof(double) * std::max<int64_t>(1, M.n_kkt)) != cudaSuccess)
            return SCOPF_ERR_OOM;
        h->allocations.push_back(*p);
    }
    return SCOPF_OK;
}

}  // namespace scopf

extern "C" int scopf_set_params(scopf_handle *h, const double *Pd, const double *Qd,
                                const double *c1) {
    using namespace scopf;
    if (!h) return SCOPF_ERR_INVALID_ARG;
    Model &M = h->M;
    if (Pd || Qd) {
        for (const Block &B : M.blocks)
            for (int b = 0; b < M.nb; b++) {
                if (Pd) M.c_const[B.c0 + B.rP[b]] = -Pd[b];
                if (Qd) M.c_const[B.c0 + B.rQ[b]] = -Qd[b];
            }
        for (int b = 0; b < M.nb; b++) {
            if (Pd) M.Pd[b] = Pd[b];
            if (Qd) M.Qd[b] = Qd[b];
        }
    }
    if (c1)
        for (int g = 0; g < M.ng; g++) M.c1[g] = c1[g];
    h->has_solution = false;
    if (h->host_only) return SCOPF_OK;
    if (M.m && cudaMemcpy(const_cast<double *>(h->dm.c_const), M.c_const.data(),
                          sizeof(double) * M.m, cudaMemcpyHostToDevice) != cudaSuccess)
        return SCOPF_ERR_CUDA;
    if (M.ng && cudaMemcpy(const_cast<double *>(h->dm.c1), M.c1.data(), sizeof(double) * M.ng,
                           cudaMemcpyHostToDevice) != cudaSuccess)
        return SCOPF_ERR_CUDA;
    return SCOPF_OK;
}

extern "C" int scopf_set_ncl_params(scopf_handle *h, const double *lam_n, const double *nu0_n,
                                    double rho, double mu) {
    using namespace scopf;
    if (!h || h->host_only || !lam_n || (h->M.p && !nu0_n) || !(rho > 0) || !(mu > 0))
        return SCOPF_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    if (h->M.m)
        cudaMemcpyAsync(h->lam_n, lam_n, sizeof(double) * h->M.m, cudaMemcpyDeviceToDevice, s);
    if (h->M.p)
        cudaMemcpyAsync(h->nu0_n, nu0_n, sizeof(double) * h->M.p, cudaMemcpyDeviceToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return SCOPF_ERR_CUDA;
    h->rho = rho;
    h->mu_last = mu;
    h->dw_last = 0.0;
    h->eta_last = h->opt.eta_init;
    h->omega_last = h->opt.omega_init;
    h->have_ncl = true;
    h->has_solution = true;
    return SCOPF_OK;
}

extern "C" int scopf_adjoint(scopf_handle *h, const double *seed_pg0, double seed_cost,
                             double *grad_Pd, double *grad_Qd, double *grad_c1) {
    using namespace scopf;
    if (!h || h->host_only || !grad_Pd || !grad_Qd || !grad_c1) return SCOPF_ERR_INVALID_ARG;
    if (!h->has_solution) return SCOPF_ERR_NOT_FACTORED;
    int r = adjoint_setup(h);
    if (r != SCOPF_OK) return r;
    const Model &M = h->M;
    cudaStream_t s = h->stream;
    // K at the final iterate, delta_w = 0
    r = assemble_impl(h, &h->st, h->lam_n, h->nu0_n, h->rho, h->mu_last, 0.0, nullptr);
    if (r != SCOPF_OK) return r;
    double delta = 0.0;
    int tries = 0;
    r = factor_inertia(h, SCOPF_PREC_FP64, h->dw_last, delta, tries);
    if (r != SCOPF_OK) return r;
    // refine against K_inf (no delta_w shift, no -1/rho on the dual rows),
    // preconditioned by the factors just computed
    r = set_delta_w(h, 0.0);
    if (r != SCOPF_OK) return r;
    if (h->adj_ndual)
        note_launch(), k_add_at<<<(int)((h->adj_ndual + kAT - 1) / kAT), kAT, 0, s>>>(
            h->adj_ndual, h->adj_dpos, 1.0 / h->rho, h->kval);
    h->factored = true;
    cudaMemsetAsync(h->adj_g, 0, sizeof(double) * M.n_kkt, s);
    const DevModel &d = h->dm;
    note_launch(), k_adj_rhs<<<(M.ng + kAT - 1) / kAT, kAT, 0, s>>>(
        (int)M.ng, h->adj_pg, seed_pg0, seed_cost, h->st.w, M.border0, d.c2, d.c1, h->adj_g);
    double rel = 0;
    int steps = 0;
    r = solve_impl(h, h->adj_g, h->adj_a, std::max(h->opt.max_refine, 100), &rel, &steps);
    if (r != SCOPF_OK) return r;
    note_launch(), k_bus_sum<<<(M.nb + kAT - 1) / kAT, kAT, 0, s>>>((int)M.nb, h->adj_ptr,
                                                                     h->adj_rowsP, h->adj_a, grad_Pd);
    note_launch(), k_bus_sum<<<(M.nb + kAT - 1) / kAT, kAT, 0, s>>>((int)M.nb, h->adj_ptr,
                                                                     h->adj_rowsQ, h->adj_a, grad_Qd);
    note_launch(), k_adj_c1<<<(M.ng + kAT - 1) / kAT, kAT, 0, s>>>(
        (int)M.ng, h->adj_pg, h->adj_a, h->st.w, M.border0, seed_cost, grad_c1);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return SCOPF_ERR_CUDA;
    return SCOPF_OK;
}
