// Batched contingency screening (Section V-B).
//
// For a base-case control u0, contingency k is feasible when the system of
// eq. (screening) -- the scenario-k power flow, its operational limits and
// the complementarity recourse of eqs. (droopmpec), (pvpq), all at that u0
// -- has a solution.  NCL reaches the answer through eq. (feaspb): when no
// solution exists, rho grows without bound and (r_k, t_k) settle at a local
// minimiser of the infeasibility, whose size ranks the contingency.
//
// Here every candidate is screened in one NCL solve.  The handle holds the
// base case and the candidates as its scenarios; the first-stage variables
// are boxed to [u0 - eps, u0 + eps] (clipped to their own limits and kept
// nonempty), so the scenario blocks couple only through that box (not at
// all as eps -> 0), and the same kernels that run the SCOPF factor and solve
// them all at once.  The outer loop follows a per-block rule: while some
// block keeps |(r_k, t_k)|_inf above eta and drives rho up, every block
// within eta still takes its multiplier update, as it would in a solve of
// its own, so a feasible block ends near a feasible point and an infeasible
// one at the capped-penalty minimiser of its own infeasibility.  rho is capped at rho_cap; the
// handle's iteration limits apply.  Candidate k is accepted when
// |(r_k, t_k)|_inf <= accept_tol and the solve ended by convergence, by the
// rho cap or by the outer-iteration limit (not by the inner-iteration limit
// or a numerical failure).
#include <cmath>
#include <vector>

#include "handle.h"

namespace scopf {

namespace {

constexpr int kVT = 256;

// One CTA per scenario: max |r| over its constraint rows and |t| over its
// complementarity pairs (a NaN counts as infinite).
__global__ void __launch_bounds__(kVT) k_block_rt_max(const int64_t *__restrict__ rng,
                                                      const double *__restrict__ r,
                                                      const double *__restrict__ t,
                                                      double *__restrict__ out) {
    const int64_t c0 = rng[4 * blockIdx.x], nr = rng[4 * blockIdx.x + 1];
    const int64_t p0 = rng[4 * blockIdx.x + 2], np = rng[4 * blockIdx.x + 3];
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < nr; i += kVT) {
        const double a = fabs(r[c0 + i]);
        v = a == a ? fmax(v, a) : INFINITY;
    }
    for (int64_t i = threadIdx.x; i < np; i += kVT) {
        const double a = fabs(t[p0 + i]);
        v = a == a ? fmax(v, a) : INFINITY;
    }
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __shared__ double red[kVT / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kVT / 32; w++) v = fmax(v, red[w]);
        out[blockIdx.x] = v;
    }
}

// Lambda and nu0 updates (lam_n += rho r, nu0_n += rho t) of the blocks
// whose max |r_k|, |t_k| (viol[k]) is within thr.
__global__ void __launch_bounds__(kVT) k_block_multiplier_update(
    const int64_t *__restrict__ rng, const double *__restrict__ viol, double thr, double rho,
    const double *__restrict__ r, const double *__restrict__ t, double *__restrict__ lam_n,
    double *__restrict__ nu0_n) {
    if (!(viol[blockIdx.x] <= thr)) return;
    const int64_t c0 = rng[4 * blockIdx.x], nr = rng[4 * blockIdx.x + 1];
    const int64_t p0 = rng[4 * blockIdx.x + 2], np = rng[4 * blockIdx.x + 3];
    for (int64_t i = threadIdx.x; i < nr; i += kVT) lam_n[c0 + i] += rho * r[c0 + i];
    for (int64_t i = threadIdx.x; i < np; i += kVT) nu0_n[p0 + i] += rho * t[p0 + i];
}

int block_ranges(scopf_handle *h) {
    const Model &M = h->M;
    const int nblk = (int)M.blocks.size();
    if (!h->blk_rt) {
        std::vector<int64_t> rng(4 * nblk);
        for (int k = 0; k < nblk; k++) {
            const Block &B = M.blocks[k];
            rng[4 * k] = B.c0;
            rng[4 * k + 1] = B.nrow;
            rng[4 * k + 2] = B.p0;
            rng[4 * k + 3] = B.ncomp;
        }
        if (cudaMalloc(&h->blk_rt, sizeof(int64_t) * rng.size()) != cudaSuccess)
            return SCOPF_ERR_OOM;
        h->allocations.push_back(h->blk_rt);
        if (cudaMalloc(&h->blk_viol, sizeof(double) * nblk) != cudaSuccess) return SCOPF_ERR_OOM;
        h->allocations.push_back(h->blk_viol);
        if (cudaMemcpy(h->blk_rt, rng.data(), sizeof(int64_t) * rng.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return SCOPF_ERR_CUDA;
    }
    return SCOPF_OK;
}

int block_violation(scopf_handle *h, double *viol) {
    const int nblk = (int)h->M.blocks.size();
    cudaStream_t s = h->stream;
    const int r = block_ranges(h);
    if (r != SCOPF_OK) return r;
    note_launch(), k_block_rt_max<<<nblk, kVT, 0, s>>>(h->blk_rt, h->st.r, h->st.t, h->blk_viol);
    if (cudaMemcpyAsync(viol, h->blk_viol, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SCOPF_ERR_CUDA;
    return SCOPF_OK;
}

// Relaxed bounds of the model's current M.wl, M.wu to the device.
int upload_bounds(scopf_handle *h) {
    std::vector<double> wl, wu;
    relaxed_bounds(h->M, h->opt.bound_relax, wl, wu);
    const size_t bytes = sizeof(double) * wl.size();
    if (cudaMemcpy(h->wl, wl.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->wu, wu.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return SCOPF_ERR_CUDA;
    return SCOPF_OK;
}

}  // namespace

int block_multiplier_update(scopf_handle *h, double rho, double thr) {
    const int nblk = (int)h->M.blocks.size();
    cudaStream_t s = h->stream;
    const int r = block_ranges(h);
    if (r != SCOPF_OK) return r;
    note_launch(), k_block_rt_max<<<nblk, kVT, 0, s>>>(h->blk_rt, h->st.r, h->st.t, h->blk_viol);
    note_launch(), k_block_multiplier_update<<<nblk, kVT, 0, s>>>(
        h->blk_rt, h->blk_viol, thr, rho, h->st.r, h->st.t, h->lam_n, h->nu0_n);
    return cudaGetLastError() == cudaSuccess ? SCOPF_OK : SCOPF_ERR_CUDA;
}

}  // namespace scopf

extern "C" int scopf_block_violation(scopf_handle *h, double *viol) {
    using namespace scopf;
    if (!h || h->host_only || !viol) return SCOPF_ERR_INVALID_ARG;
    return block_violation(h, viol);
}

extern "C" int scopf_screen(scopf_handle *h, const double *u0, double eps, double rho_cap,
                            double accept_tol, scopf_result *res, double *viol,
                            int32_t *accepted) {
    using namespace scopf;
    if (!h || h->host_only || !res || !viol || !accepted || !(rho_cap > 0) ||
        !(accept_tol >= 0) || (u0 && !(eps > 0)))
        return SCOPF_ERR_INVALID_ARG;
    Model &M = h->M;
    const int64_t b0 = M.border0, nbr = M.nborder;
    const std::vector<double> wl0(M.wl), wu0(M.wu);
    if (u0) {
        for (int64_t j = 0; j < nbr; j++)
            if (!std::isfinite(u0[j])) return SCOPF_ERR_INVALID_ARG;
        for (int64_t j = 0; j < nbr; j++) {
            double lo = std::fmax(wl0[b0 + j], u0[j] - eps);
            double hi = std::fmin(wu0[b0 + j], u0[j] + eps);
            // u0 on (or past) a limit: keep an interval of width eps
            lo = std::fmin(lo, hi - eps);
            hi = std::fmax(hi, lo + eps);
            M.wl[b0 + j] = lo;
            M.wu[b0 + j] = hi;
        }
    }
    const scopf_options saved = h->opt;
    h->opt.rho_max = rho_cap;
    h->screen_blocks = true;
    int r = u0 ? upload_bounds(h) : SCOPF_OK;
    int status = SCOPF_ERR_CUDA;
    if (r == SCOPF_OK) {
        status = ncl_solve_impl(h, nullptr, res);
        res->status = status;
        r = status == SCOPF_ERR_CUDA || status == SCOPF_ERR_OOM ? status : block_violation(h, viol);
    }
    h->opt = saved;
    h->screen_blocks = false;
    M.wl = wl0;
    M.wu = wu0;
    if (u0) {
        const int r2 = upload_bounds(h);
        if (r == SCOPF_OK) r = r2;
        // the solution belongs to the boxed problem, not to the handle's SCOPF
        h->has_solution = false;
    }
    if (r != SCOPF_OK) return r;
    const bool ended = status == SCOPF_OK || status == SCOPF_ERR_INFEASIBLE ||
                       (status == SCOPF_ERR_MAX_ITER && !h->inner_limit);
    for (size_t k = 0; k < M.blocks.size(); k++) accepted[k] = ended && viol[k] <= accept_tol;
    return SCOPF_OK;
}
