// The library handle: host model, symbolic/frontal structure, device buffers.
#pragma once

#include <cuda_runtime.h>

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
    int *queue = nullptr, *done = nullptr;
    scopf::FactorStatus *fstat = nullptr;
    double *red_scratch = nullptr, *red_out = nullptr;
    int epoch = 0;
    bool assembled = false, factored = false;
    int factored_precision = SCOPF_PREC_FP64;
    double last_delta_w = 0.0, last_rho = 0.0;
    // iterate and NCL parameters owned by the handle
    scopf_state st{};
    double *lam_n = nullptr, *nu0_n = nullptr;
    double rho = 0.0;
    // IPM scratch (directions and trial point)
    scopf_state dir{}, trial{};
    double *tmp_n = nullptr, *tmp_m = nullptr, *tmp_p = nullptr, *tmp_kkt = nullptr;
    int64_t *d_il = nullptr, *d_iu = nullptr;
    // counters
    int n_factor = 0, n_refine = 0;
    std::string last_error;
};

namespace scopf {
int ncl_solve_impl(scopf_handle *h, const scopf_state *warm, scopf_result *res);
int assemble_impl(scopf_handle *h, const scopf_state *it, const double *lam_n,
                  const double *nu0_n, double rho, double mu, double delta_w, double *rhs);
int factor_impl(scopf_handle *h, int precision, int inertia[3]);
int solve_impl(scopf_handle *h, const double *b, double *x, int max_refine, double *rel,
               int *steps);
double device_maxabs(scopf_handle *h, const double *x, int64_t n);
double device_sumabs(scopf_handle *h, const double *x, int64_t n);
}  // namespace scopf
