// C ABI of the library (include/scopf.h): handle management, device
// uploads, and the assemble / factor / solve entry points of the Newton step
// of eq. (newtonsystem).
#include <atomic>
#include <chrono>
#include <cmath>
#include <thread>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "handle.h"

using namespace scopf;

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            h->last_error = cudaGetErrorString(e_);                                                \
            return SCOPF_ERR_CUDA;                                                                 \
        }                                                                                          \
    } while (0)

namespace scopf {
std::atomic<long long> g_kernel_launches{0};

// Bounds the interior-point method works with: every finite bound moved
// outwards by bound_relax * max(1, |bound|) (W&B 2006, Section 3.5).
void relaxed_bounds(const Model &M, double bound_relax, std::vector<double> &wl,
                    std::vector<double> &wu) {
    wl.resize(M.n);
    wu.resize(M.n);
    for (int64_t i = 0; i < M.n; i++) {
        wl[i] = std::isfinite(M.wl[i]) ? M.wl[i] - bound_relax * std::fmax(1.0, std::fabs(M.wl[i]))
                                       : -INFINITY;
        wu[i] = std::isfinite(M.wu[i]) ? M.wu[i] + bound_relax * std::fmax(1.0, std::fabs(M.wu[i]))
                                       : INFINITY;
    }
}
}  // namespace scopf

namespace {

template <typename T>
int upload(scopf_handle *h, const std::vector<T> &v, const T **out) {
    T *p = nullptr;
    size_t bytes = sizeof(T) * (v.empty() ? 1 : v.size());
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        h->last_error = cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SCOPF_ERR_OOM : SCOPF_ERR_CUDA;
    }
    h->allocations.push_back(p);
    if (!v.empty()) {
        e = cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            h->last_error = cudaGetErrorString(e);
            return SCOPF_ERR_CUDA;
        }
    }
    *out = p;
    return SCOPF_OK;
}

template <typename T>
int alloc(scopf_handle *h, size_t n, T **out) {
    T *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) {
        h->last_error = cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SCOPF_ERR_OOM : SCOPF_ERR_CUDA;
    }
    cudaMemset(p, 0, sizeof(T) * (n ? n : 1));
    h->allocations.push_back(p);
    *out = p;
    return SCOPF_OK;
}

#define TRY(x)                                                                                     \
    do {                                                                                           \
        int r_ = (x);                                                                              \
        if (r_ != SCOPF_OK) return r_;                                                             \
    } while (0)

int setup_device(scopf_handle *h) {
    Model &M = h->M;
    HostFronts &HF = h->HF;
    DevModel &d = h->dm;
    d.n = M.n;
    d.m = M.m;
    d.p = M.p;
    d.n_kkt = M.n_kkt;
    d.nnz = (int64_t)M.kkt_col.size();
    d.n_be = M.n_be;
    d.n_se = M.n_se;
    d.ev_branch0 = M.ev_branch0;
    d.ev_shunt0 = M.ev_shunt0;
    d.ev_comp0 = M.ev_comp0;
    d.n_ev = M.n_ev;
    d.border0 = M.border0;
    d.ng = M.ng;
    TRY(upload(h, M.be_x, &d.be_x));
    TRY(upload(h, M.be_lam, &d.be_lam));
    TRY(upload(h, M.be_th, &d.be_th));
    TRY(upload(h, M.be_par, &d.be_par));
    TRY(upload(h, M.se_v, &d.se_v));
    TRY(upload(h, M.se_P, &d.se_P));
    TRY(upload(h, M.se_Q, &d.se_Q));
    TRY(upload(h, M.se_G, &d.se_G));
    TRY(upload(h, M.se_B, &d.se_B));
    TRY(upload(h, M.comp1, &d.comp1));
    TRY(upload(h, M.comp2, &d.comp2));
    TRY(upload(h, M.c_const, &d.c_const));
    TRY(upload(h, M.cf_ptr, &d.cf_ptr));
    TRY(upload(h, M.cf_idx, &d.cf_idx));
    TRY(upload(h, M.cf_coef, &d.cf_coef));
    TRY(upload(h, M.kkt_ptr, &d.kkt_ptr));
    {
        if (M.n_kkt >= ((int64_t)1 << 31)) {
            h->last_error = "the KKT system has 2^31 rows or more";
            return SCOPF_ERR_INVALID_ARG;
        }
        const std::vector<int32_t> col32(M.kkt_col.begin(), M.kkt_col.end());
        TRY(upload(h, col32, &d.kkt_col));
    }
    TRY(upload(h, M.ctr_ptr, &d.ctr_ptr));
    {
        std::vector<int64_t> src(M.ctr.size());
        std::vector<double> coef(M.ctr.size());
        for (size_t i = 0; i < M.ctr.size(); i++) {
            src[i] = M.ctr[i].src;
            coef[i] = M.ctr[i].coef;
        }
        TRY(upload(h, src, &d.ctr_src));
        TRY(upload(h, coef, &d.ctr_coef));
        std::vector<int32_t> krow(M.kkt_col.size());
        for (int64_t r = 0; r < M.n_kkt; r++)
            for (int64_t q = M.kkt_ptr[r]; q < M.kkt_ptr[r + 1]; q++) krow[q] = (int32_t)r;
        TRY(upload(h, krow, &d.kkt_row));
        d.nnz_kkt = (int64_t)M.kkt_col.size();
    }
    TRY(upload(h, M.row_kind, &d.row_kind));
    {
        // stored position of the diagonal entry of every primal row (the
        // inertia correction delta_w shifts exactly these)
        std::vector<int64_t> pos;
        for (int64_t i = 0; i < M.n_kkt; i++) {
            if (M.row_kind[i] != 0) continue;
            for (int64_t q = M.kkt_ptr[i]; q < M.kkt_ptr[i + 1]; q++)
                if (M.kkt_col[q] == i) {
                    pos.push_back(q);
                    break;
                }
        }
        h->n_pdiag = (int64_t)pos.size();
        TRY(upload(h, pos, &h->pdiag_pos));
        TRY(alloc(h, pos.size(), &h->pdiag_base));
        // Rows that receive no update in the pivot-free elimination: a block
        // row none of whose stored neighbours is eliminated before it (block
        // rows never touch another block's rows; border rows go last).  Row
        // k of L is then empty and the pivot is the diagonal entry itself.
        std::vector<int64_t> elim(M.n_kkt, INT64_MAX);
        for (const BlockSymbolic &S : h->syms)
            for (int64_t i = 0; i < S.n_block_rows; i++) elim[S.rows[i]] = i;
        std::vector<int64_t> lead;
        for (int64_t i = 0, j = 0; i < M.n_kkt; i++) {
            if (M.row_kind[i] != 0) continue;
            bool has_diag = false, first = M.block_of_kkt[i] >= 0;
            for (int64_t q = M.kkt_ptr[i]; q < M.kkt_ptr[i + 1]; q++) {
                const int64_t c = M.kkt_col[q];
                if (c == i) has_diag = true;
                else if (elim[c] < elim[i]) first = false;
            }
            if (!has_diag) continue;
            if (first) lead.push_back(j);
            j++;
        }
        h->n_lead = (int64_t)lead.size();
        TRY(upload(h, lead, &h->lead_pdiag));
        TRY(alloc(h, 1, &h->lead_zero));
    }
    TRY(upload(h, M.row_index, &d.row_index));
    {
        std::vector<int8_t> is_long(M.n_kkt, 0);
        std::vector<int64_t> long_rows;
        for (int64_t r = 0; r < M.n_kkt; r++)
            if (M.kkt_ptr[r + 1] - M.kkt_ptr[r] > kLongRow) {
                is_long[r] = 1;
                long_rows.push_back(r);
            }
        TRY(upload(h, is_long, &d.is_long));
        TRY(upload(h, long_rows, &d.long_rows));
        d.n_long = (int64_t)long_rows.size();
    }
    {
        std::vector<double> wl, wu;
        relaxed_bounds(M, h->opt.bound_relax, wl, wu);
        const double *pl, *pu;
        TRY(upload(h, wl, &pl));
        TRY(upload(h, wu, &pu));
        d.wl = pl;
        d.wu = pu;
        h->wl = const_cast<double *>(pl);
        h->wu = const_cast<double *>(pu);
    }
    TRY(upload(h, M.c2, &d.c2));
    TRY(upload(h, M.c1, &d.c1));
    // fronts
    DevFront &F = h->df;
    F.n_tasks = HF.n_tasks;
    F.n_blocks = HF.n_blocks;
    F.n_border = HF.n_border;
    F.n_small = HF.n_small;
    TRY(upload(h, HF.front_off, &F.front_off));
    TRY(upload(h, HF.f, &F.f));
    TRY(upload(h, HF.npiv, &F.npiv));
    TRY(upload(h, HF.child_ptr, &F.child_ptr));
    TRY(upload(h, HF.child, &F.child));
    TRY(upload(h, HF.rel_off, &F.rel_off));
    TRY(upload(h, HF.rel, &F.rel));
    TRY(upload(h, HF.parent, &F.parent));
    TRY(upload(h, HF.rows_off, &F.rows_off));
    TRY(upload(h, HF.rows, &F.rows));
    TRY(upload(h, HF.is_border, &F.is_border));
    TRY(upload(h, HF.border_off, &F.border_off));
    TRY(upload(h, HF.border_rows, &F.border_rows));
    TRY(upload(h, HF.vec_off, &F.vec_off));
    TRY(upload(h, HF.border_vec_off, &F.border_vec_off));
    TRY(upload(h, HF.orig_ptr, &F.orig_ptr));
    TRY(upload(h, HF.orig_nz, &F.orig_nz));
    TRY(upload(h, HF.orig_off, &F.orig_off));
    F.kkt_row = d.kkt_row;
    F.kkt_col = d.kkt_col;
    F.front_elems = HF.front_elems;
    F.vec_elems = HF.vec_elems;
    // work buffers
    TRY(alloc(h, M.n_ev, &h->ev));
    TRY(alloc(h, M.kkt_col.size(), &h->kval));
    TRY(alloc(h, M.n_kkt, &h->diag));
    TRY(alloc(h, M.n, &h->g));
    TRY(alloc(h, M.n, &h->gw));
    TRY(alloc(h, M.m, &h->c));
    TRY(alloc(h, M.n_kkt, &h->rhs));
    TRY(alloc(h, M.n_kkt, &h->sol));
    TRY(alloc(h, M.n_kkt, &h->res));
    TRY(alloc(h, M.n_kkt, &h->dx));
    TRY(alloc(h, M.n_kkt, &h->scale));
    TRY(alloc(h, M.n_kkt, &h->scale_tmp));
    TRY(alloc(h, M.n_kkt, &h->ruiz_mx));
    F.kval = h->kval;
    F.scale = h->scale;
    {
        double *ov = nullptr;
        TRY(alloc(h, HF.orig_nz.size(), &ov));   // sized for FP64; FP32 uses half
        F.ovals = ov;
        double *xsb = nullptr;
        TRY(alloc(h, (size_t)M.n_kkt, &xsb));
        F.xs = xsb;
        h->ovals = ov;
        F.n_orig = (int64_t)HF.orig_nz.size();
    }
    double *fr = nullptr, *vv = nullptr;
    TRY(alloc(h, (size_t)HF.front_elems, &fr));
    TRY(alloc(h, (size_t)HF.vec_elems, &vv));
    h->fronts = fr;
    h->vec = vv;
    TRY(alloc(h, (size_t)M.nborder * M.nborder, &h->S));
    TRY(alloc(h, (size_t)M.nborder * M.nborder, &h->Sinv));
    TRY(alloc(h, (size_t)M.nborder * 17 + 1, &h->border_work));   // y + 16 gather partials
    {
        const size_t nt = HF.n_items > 0 ? (size_t)HF.n_items : 1;
        F.n_items = HF.n_items;
        F.max_f = 32;
        for (int t = 0; t < HF.n_tasks; t++) F.max_f = std::max(F.max_f, (int)HF.f[t]);
        // in-front offsets are 32-bit in the large-front kernel
        if ((int64_t)F.max_f * F.max_f >= ((int64_t)1 << 31)) {
            h->last_error = "a front has more than 46340 rows";
            return SCOPF_ERR_INVALID_ARG;
        }
        // the large-front kernel stages np x f panels up to 96 KB (FP64)
        F.big_panel = 1;
        F.big_np = 1;
        const int t3 = HF.n_items > HF.n_items_med ? HF.item_ptr[HF.n_items_med] : HF.n_tasks;
        for (int t = t3; t < HF.n_tasks; t++) {
            const int64_t pe = (int64_t)HF.f[t] * HF.npiv[t];
            if (pe <= 12288) {
                F.big_panel = std::max<int>(F.big_panel, (int)pe);
                F.big_np = std::max<int>(F.big_np, (int)HF.npiv[t]);
            }
        }
        F.n_items_small = HF.n_items_small;
        F.n_items_med = HF.n_items_med;
        TRY(upload(h, HF.item_ptr, &F.item_ptr));
        F.n_rows = (int64_t)HF.vpos_of_row.size();
        TRY(upload(h, HF.vpos_of_row, &F.vpos_of_row));
        {
            const int32_t *tr = nullptr, *cr = nullptr;
            TRY(upload(h, HF.task_rec, &tr));
            F.task_rec = reinterpret_cast<const int4 *>(tr);
            std::vector<int32_t> crv = HF.child_rec;
            if (crv.empty()) crv.assign(8, 0);
            TRY(upload(h, crv, &cr));
            F.child_rec = reinterpret_cast<const int4 *>(cr);
        }
        TRY(upload(h, HF.item_parent, &F.item_parent));
        {
            // the sweeps' item records (see DevFront::item_fwd)
            const int ni = HF.n_items;
            std::vector<int32_t> fw(12 * (size_t)(ni > 0 ? ni : 1), 0), bw(fw.size(), 0);
            for (int i = 0; i < ni; i++) {
                const int t0 = HF.item_ptr[i], t1 = HF.item_ptr[i + 1];
                for (int k = 0; k < 2; k++) {
                    const int t = k == 0 ? t0 : t1 - 1;
                    int32_t *r = (k == 0 ? fw.data() : bw.data()) + 12 * (size_t)i;
                    const int32_t *a = &HF.task_rec[8 * (size_t)t];
                    const int32_t *nx = &HF.task_rec[8 * (size_t)(t + 1)];
                    for (int w = 0; w < 5; w++) r[w] = a[w];
                    r[5] = a[5];    // first child slot
                    r[6] = nx[5];   // end child slot
                    if (k == 0) {
                        r[7] = t1;
                        r[8] = t0;
                        r[9] = HF.item_parent[i];
                    } else {
                        r[7] = t0;
                        r[8] = t1;
                        r[9] = HF.item_cont[i];
                    }
                    r[10] = a[6];   // original entries [o0, o1)
                    r[11] = nx[6];
                }
            }
            const int32_t *fwp = nullptr, *bwp = nullptr;
            TRY(upload(h, fw, &fwp));
            TRY(upload(h, bw, &bwp));
            F.item_fwd = reinterpret_cast<const int4 *>(fwp);
            F.item_bwd = reinterpret_cast<const int4 *>(bwp);
        }
        TRY(upload(h, HF.item_child_ptr, &F.item_child_ptr));
        TRY(upload(h, HF.item_child, &F.item_child));
        TRY(upload(h, HF.item_cont, &F.item_cont));
        TRY(alloc(h, nt, &F.q_slots_a));
        TRY(alloc(h, nt, &F.q_slots_b));
        TRY(alloc(h, nt, &F.q_slots_c));
        TRY(alloc(h, nt, &F.q_pending));
        TRY(alloc(h, 6, &F.q_ctr));
        TRY(upload(h, HF.init_small, &F.init_small));
        TRY(upload(h, HF.init_med, &F.init_med));
        TRY(upload(h, HF.init_big, &F.init_big));
        TRY(upload(h, HF.init_fwd, &F.init_fwd));
        TRY(upload(h, HF.init_bwd, &F.init_bwd));
        TRY(upload(h, HF.pend_factor, &F.pend_factor));
        TRY(upload(h, HF.nchild, &F.nchild));
        F.n_init_small = (int)HF.init_small.size();
        F.n_init_med = (int)HF.init_med.size();
        F.n_init_big = (int)HF.init_big.size();
        F.n_init_fwd = (int)HF.init_fwd.size();
        F.n_init_bwd = (int)HF.init_bwd.size();
    }
    TRY(alloc(h, 1, &h->fstat));
    TRY(alloc(h, 1024, &h->red_scratch));
    TRY(alloc(h, (size_t)ipm_partials(), &h->ipm_part));
    for (int64_t i = 0; i < M.n; i++) {
        if (std::isfinite(M.wl[i])) h->n_lower++;
        if (std::isfinite(M.wu[i])) h->n_upper++;
    }
    TRY(alloc(h, 16, &h->red_out));
    // iterate, NCL parameters, IPM scratch
    for (scopf_state *s : {&h->st, &h->dir, &h->trial}) {
        TRY(alloc(h, M.n, &s->w));
        TRY(alloc(h, M.m, &s->r));
        TRY(alloc(h, M.p, &s->t));
        TRY(alloc(h, M.p, &s->s));
        TRY(alloc(h, M.m, &s->lam));
        TRY(alloc(h, M.p, &s->yc));
        TRY(alloc(h, M.n, &s->zl));
        TRY(alloc(h, M.n, &s->zu));
        TRY(alloc(h, M.p, &s->zs));
    }
    TRY(alloc(h, M.m, &h->lam_n));
    TRY(alloc(h, M.p, &h->nu0_n));
    TRY(alloc(h, M.n, &h->tmp_n));
    TRY(alloc(h, M.m, &h->tmp_m));
    TRY(alloc(h, M.p, &h->tmp_p));
    TRY(alloc(h, M.n_kkt, &h->tmp_kkt));
    CK(cudaDeviceSynchronize());
    return SCOPF_OK;
}

}  // namespace

extern "C" {

void scopf_default_options(scopf_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->mu_min = 1e-7;
    o->mu_init = 1e-1;
    o->kappa_eps = 10.0;
    o->kappa_mu = 0.2;
    o->theta_mu = 1.5;
    o->tau_min = 0.99;
    o->s_max = 100.0;
    o->kappa_sigma = 1e10;
    o->bound_relax = 1e-8;
    o->bound_push = 1e-2;
    o->bound_frac = 1e-2;
    o->slack_init = 1e-1;
    o->comp_init = 1e-1;
    o->delta_w0 = 1e-4;
    o->delta_w_min = 1e-20;
    o->delta_w_max = 1e40;
    o->kappa_w_minus = 1.0 / 3.0;
    o->kappa_w_plus = 8.0;
    o->kappa_w_plus_bar = 100.0;
    o->gamma_theta = 1e-5;
    o->gamma_phi = 1e-8;
    o->delta_sw = 1.0;
    o->s_theta = 1.1;
    o->s_phi = 2.3;
    o->eta_phi = 1e-8;
    o->gamma_alpha = 0.05;
    o->rho_init = 1e2;
    o->rho_max = 1e12;
    o->eta_init = 1e-2;
    o->omega_init = 1e-2;
    o->refine_tol = 1e-10;
    o->pivot_tol = 0.0;
    o->max_backtrack = 40;
    o->max_outer = 40;
    o->max_inner = 3000;
    o->max_refine = 30;
    o->precision = SCOPF_PREC_FP64;
    o->relax_max_nodes = 8;
    o->verbose = 0;
    o->spin_limit = 1 << 24;
    o->host_only = 0;
    o->cluster_max_tasks = 16;
    o->relax_max_front = 0;
    o->device_loop = 1;
    o->fp64_switch_refine = 6;
    o->fp64_switch_streak = 5;
    o->known_zero_pivot = 1;
    o->dual_first = 0;
    o->fixed_mu = 0;
    o->ipm_graph = 1;
}

const char *scopf_last_error(scopf_handle *h) { return h ? h->last_error.c_str() : ""; }

const char *scopf_strerror(int s) {
    switch (s) {
        case SCOPF_OK: return "ok";
        case SCOPF_ERR_INVALID_ARG: return "invalid argument";
        case SCOPF_ERR_CUDA: return "CUDA error";
        case SCOPF_ERR_NOT_FACTORED: return "no valid factorization";
        case SCOPF_ERR_WRONG_INERTIA: return "wrong inertia after maximal correction";
        case SCOPF_ERR_REFINE_STALL: return "iterative refinement stalled";
        case SCOPF_ERR_INFEASIBLE: return "locally infeasible (penalty diverged)";
        case SCOPF_ERR_MAX_ITER: return "iteration limit";
        case SCOPF_ERR_TIMEOUT: return "device dependency wait timed out";
        case SCOPF_ERR_OOM: return "out of device memory";
        case SCOPF_ERR_NUMERICAL: return "numerical failure";
        default: return "unknown status";
    }
}

int scopf_create(const scopf_network *net, const scopf_contingency *ctg, int32_t K,
                 const scopf_options *opt, scopf_handle **out) {
    if (!out) return SCOPF_ERR_INVALID_ARG;
    *out = nullptr;
    scopf_handle *h = new (std::nothrow) scopf_handle();
    if (!h) return SCOPF_ERR_OOM;
    if (opt)
        h->opt = *opt;
    else
        scopf_default_options(&h->opt);
    h->precision = h->opt.precision;
    h->host_only = h->opt.host_only != 0;
    const auto tc = std::chrono::steady_clock::now();
    auto since = [&tc]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - tc).count();
    };
    std::string err = build_model(net, ctg, K, h->M);
    const double t_model = since();
    if (!err.empty()) {
        if (h->opt.verbose) std::fprintf(stderr, "scopf_create: %s\n", err.c_str());
        delete h;
        return SCOPF_ERR_INVALID_ARG;
    }
    // the blocks' symbolic analyses are independent (each reads the model and
    // writes its own result): spread them over the host's cores
    const size_t nblk = h->M.blocks.size();
    h->syms.resize(nblk);
    {
        std::vector<std::string> errs(nblk);
        const unsigned hw = std::thread::hardware_concurrency();
        const size_t nt = std::max<size_t>(1, std::min<size_t>(hw ? hw : 1, nblk));
        std::atomic<size_t> next{0};
        auto work = [&]() {
            for (size_t k; (k = next.fetch_add(1)) < nblk;)
                errs[k] = symbolic_block(h->M, (int)k, h->opt.relax_max_nodes,
                                         h->opt.relax_max_front, h->opt.dual_first != 0,
                                         h->syms[k]);
        };
        std::vector<std::thread> pool;
        for (size_t t = 1; t < nt; t++) pool.emplace_back(work);
        work();
        for (auto &th : pool) th.join();
        for (size_t k = 0; k < nblk; k++)
            if (!errs[k].empty()) {
                if (h->opt.verbose) std::fprintf(stderr, "scopf_create: %s\n", errs[k].c_str());
                delete h;
                return SCOPF_ERR_INVALID_ARG;
            }
    }
    const double t_symbolic = since();
    if (h->opt.cluster_max_tasks < 1) {
        delete h;
        return SCOPF_ERR_INVALID_ARG;
    }
    err = build_fronts(h->M, h->syms, h->opt.cluster_max_tasks, h->HF);
    const double t_fronts = since();
    if (h->opt.verbose)
        std::printf("scopf_create: model %.2f s, symbolic %.2f s, fronts %.2f s\n", t_model,
                    t_symbolic - t_model, t_fronts - t_symbolic);
    if (!err.empty()) {
        if (h->opt.verbose) std::fprintf(stderr, "scopf_create: %s\n", err.c_str());
        delete h;
        return SCOPF_ERR_INVALID_ARG;
    }
    if (!h->host_only) {
        int r = setup_device(h);
        if (r != SCOPF_OK) {
            if (h->opt.verbose) std::fprintf(stderr, "scopf_create: %s\n", h->last_error.c_str());
            scopf_destroy(h);
            return r;
        }
    }
    *out = h;
    return SCOPF_OK;
}

void scopf_destroy(scopf_handle *h) {
    if (!h) return;
    for (auto &g : h->kgraph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    ipm_graphs_release(h);
    for (void *p : h->allocations) cudaFree(p);
    if (h->trace) cudaFree(h->trace);
    delete h;
}

int scopf_get_sizes(scopf_handle *h, scopf_sizes *o) {
    if (!h || !o) return SCOPF_ERR_INVALID_ARG;
    o->n = h->M.n;
    o->m = h->M.m;
    o->p = h->M.p;
    o->n_kkt = h->M.n_kkt;
    o->n_border = h->M.nborder;
    o->n_blocks = (int32_t)h->M.blocks.size();
    o->nnz_kkt = (int64_t)h->M.kkt_col.size();
    o->nnz_L = h->HF.nnz_L;
    o->n_supernodes = h->HF.n_tasks - h->HF.n_blocks;
    o->factor_flops = h->HF.flops;
    o->front_bytes = h->HF.front_elems * 8;
    o->n_elem_values = h->M.n_ev;
    o->n_contrib = (int64_t)h->M.ctr.size();
    return SCOPF_OK;
}

int scopf_set_stream(scopf_handle *h, void *stream) {
    if (!h) return SCOPF_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)stream;
    return SCOPF_OK;
}

int scopf_set_precision(scopf_handle *h, int32_t precision) {
    if (!h || (precision != SCOPF_PREC_FP64 && precision != SCOPF_PREC_MIXED))
        return SCOPF_ERR_INVALID_ARG;
    h->precision = precision;
    return SCOPF_OK;
}

int scopf_symbolic_block(scopf_handle *h, int32_t k, int32_t *n_nodes, int32_t *n_block_nodes,
                         int32_t *n_sn, int32_t *n_rows, int32_t *post, int32_t *node_parent,
                         int32_t *sn_start, int64_t *rows) {
    if (!h || k < 0 || k >= (int32_t)h->syms.size()) return SCOPF_ERR_INVALID_ARG;
    const BlockSymbolic &S = h->syms[k];
    if (n_nodes) *n_nodes = S.n_nodes;
    if (n_block_nodes) *n_block_nodes = S.n_block_nodes;
    if (n_sn) *n_sn = (int32_t)S.sn_start.size() - 1;
    if (n_rows) *n_rows = (int32_t)S.rows.size();
    if (post)
        for (int i = 0; i < S.n_block_nodes; i++) post[i] = S.post[i];
    if (node_parent)
        for (int i = 0; i < S.n_block_nodes; i++) node_parent[i] = S.node_parent[i];
    if (sn_start)
        for (size_t i = 0; i < S.sn_start.size(); i++) sn_start[i] = S.sn_start[i];
    if (rows)
        for (size_t i = 0; i < S.rows.size(); i++) rows[i] = S.rows[i];
    return SCOPF_OK;
}

int scopf_eval(scopf_handle *h, const double *w, double *obj, double *g, double *c) {
    if (!h || h->host_only || !w) return SCOPF_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    const Model &M = h->M;
    if (c) {
        launch_eval_elements(h->dm, w, h->st.lam, h->st.yc, h->ev, 0, s);
        launch_constraints(h->dm, w, h->ev, c, s);
    }
    if (g) launch_gradient(h->dm, w, g, s);
    if (obj) {
        std::vector<double> p0(M.ng);
        CK(cudaMemcpyAsync(p0.data(), w + M.border0, sizeof(double) * M.ng, cudaMemcpyDeviceToHost, s));
        CK(host_sync(h, s));
        double f = 0;
        for (int i = 0; i < M.ng; i++) {
            const double p = 100.0 * p0[i];
            f += M.c2[i] * p * p + M.c1[i] * p + M.c0[i];
        }
        *obj = f / 1.0e4;
    }
    CK(host_sync(h, s));
    CK(cudaGetLastError());
    return SCOPF_OK;
}

int kkt_assemble(scopf_handle *h, const scopf_state *it, const double *lam_n, const double *nu0_n,
                 double rho, double mu, double delta_w, double *rhs) {
    if (!h || h->host_only || !it || !lam_n || (h->M.p && !nu0_n) || !(rho > 0))
        return SCOPF_ERR_INVALID_ARG;
    int r = assemble_impl(h, it, lam_n, nu0_n, rho, mu, delta_w, rhs);
    if (r != SCOPF_OK) return r;
    CK(host_sync(h, h->stream));
    h->timer.collect();
    return SCOPF_OK;
}

int scopf_launch_count(int64_t *out) {
    if (!out) return SCOPF_ERR_INVALID_ARG;
    *out = (int64_t)scopf::g_kernel_launches.load(std::memory_order_relaxed);
    return SCOPF_OK;
}

int scopf_trace(scopf_handle *h, int32_t enable) {
    if (!h || h->host_only) return SCOPF_ERR_INVALID_ARG;
    CK(host_sync(h, h->stream));
    h->kgraph_stale = true;   // the graphs captured the trace pointer
    h->ig_stale = true;
    if (h->trace) {
        cudaFree(h->trace);
        h->trace = nullptr;
    }
    if (enable) {
        const size_t bytes = sizeof(unsigned long long) * 20 * (size_t)std::max(1, h->HF.n_items);
        cudaError_t e = cudaMalloc(&h->trace, bytes);
        if (e != cudaSuccess) {
            h->trace = nullptr;
            h->last_error = cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? SCOPF_ERR_OOM : SCOPF_ERR_CUDA;
        }
        CK(cudaMemset(h->trace, 0, bytes));
    }
    h->df.trace = h->trace;
    return SCOPF_OK;
}

int scopf_trace_read(scopf_handle *h, int32_t kind, uint64_t *out) {
    if (!h || h->host_only || !h->trace || kind < 0 || kind > 4 || !out)
        return SCOPF_ERR_INVALID_ARG;
    const size_t n = 4 * (size_t)h->HF.n_items;
    CK(host_sync(h, h->stream));
    CK(cudaMemcpy(out, h->trace + (size_t)kind * n, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
    return SCOPF_OK;
}

int scopf_trace_items(scopf_handle *h, int32_t *n_items, int32_t *out) {
    if (!h || !n_items) return SCOPF_ERR_INVALID_ARG;
    const HostFronts &HF = h->HF;
    *n_items = HF.n_items;
    if (!out) return SCOPF_OK;
    for (int i = 0; i < HF.n_items; i++) {
        const int t0 = HF.item_ptr[i], t1 = HF.item_ptr[i + 1];
        int npv = 0, fmax = 0;
        for (int t = t0; t < t1; t++) {
            npv += HF.npiv[t];
            fmax = std::max(fmax, (int)HF.f[t]);
        }
        int32_t *o = out + 6 * (size_t)i;
        o[0] = t1 - t0;
        o[1] = HF.item_parent[i];
        o[2] = i < HF.n_items_small ? 1 : (i < HF.n_items_med ? 2 : 3);
        o[3] = fmax;
        o[4] = npv;
        o[5] = HF.block[t0];
    }
    return SCOPF_OK;
}

int scopf_timing(scopf_handle *h, int32_t enable, double *ms_out, int32_t *calls_out) {
    if (!h || h->host_only) return SCOPF_ERR_INVALID_ARG;
    CK(host_sync(h, h->stream));
    h->timer.collect();
    for (int i = 0; i < PhaseTimer::kPhases; i++) {
        if (ms_out) ms_out[i] = h->timer.ms[i];
        if (calls_out) calls_out[i] = h->timer.calls[i];
    }
    if (enable) h->timer.reset();
    h->timer.on = enable != 0;
    return SCOPF_OK;
}

int kkt_export(scopf_handle *h, int64_t *row_ptr, int64_t *col, double *val) {
    if (!h) return SCOPF_ERR_INVALID_ARG;
    const Model &M = h->M;
    if (row_ptr) std::memcpy(row_ptr, M.kkt_ptr.data(), sizeof(int64_t) * M.kkt_ptr.size());
    if (col) std::memcpy(col, M.kkt_col.data(), sizeof(int64_t) * M.kkt_col.size());
    if (val) {
        if (h->host_only || !h->assembled) return SCOPF_ERR_NOT_FACTORED;
        CK(cudaMemcpy(val, h->kval, sizeof(double) * M.kkt_col.size(), cudaMemcpyDeviceToHost));
    }
    return SCOPF_OK;
}

int kkt_factor(scopf_handle *h, int32_t precision, int32_t inertia[3]) {
    if (!h || h->host_only) return SCOPF_ERR_INVALID_ARG;
    if (!h->assembled) return SCOPF_ERR_NOT_FACTORED;
    int in[3] = {0, 0, 0};
    int r = factor_impl(h, precision < 0 ? h->precision : precision, in);
    if (inertia)
        for (int i = 0; i < 3; i++) inertia[i] = in[i];
    return r;
}

int kkt_solve(scopf_handle *h, const double *b, double *x, int32_t max_refine,
              double *rel_residual, int32_t *steps) {
    if (!h || h->host_only || !b || !x) return SCOPF_ERR_INVALID_ARG;
    if (!h->factored) return SCOPF_ERR_NOT_FACTORED;
    double rel = 0;
    int st = 0;
    int r = solve_impl(h, b, x, max_refine < 0 ? h->opt.max_refine : max_refine, &rel, &st);
    if (rel_residual) *rel_residual = rel;
    if (steps) *steps = st;
    return r;
}

int ncl_solve(scopf_handle *h, const scopf_state *warm, scopf_result *res) {
    if (!h || h->host_only || !res) return SCOPF_ERR_INVALID_ARG;
    return ncl_solve_impl(h, warm, res);
}

int scopf_get_state(scopf_handle *h, scopf_state *out) {
    if (!h || h->host_only || !out) return SCOPF_ERR_INVALID_ARG;
    *out = h->st;
    return SCOPF_OK;
}

static int copy_state(scopf_handle *h, const scopf_state *a, const scopf_state *b, bool skip_null) {
    const Model &M = h->M;
    double *const *pa[9] = {&a->w, &a->r, &a->t, &a->s, &a->lam, &a->yc, &a->zl, &a->zu, &a->zs};
    double *const *pb[9] = {&b->w, &b->r, &b->t, &b->s, &b->lam, &b->yc, &b->zl, &b->zu, &b->zs};
    const int64_t len[9] = {M.n, M.m, M.p, M.p, M.m, M.p, M.n, M.n, M.p};
    for (int i = 0; i < 9; i++) {
        if (!*pa[i] || !*pb[i]) {
            if (skip_null || len[i] == 0) continue;
            return SCOPF_ERR_INVALID_ARG;
        }
        if (len[i])
            CK(cudaMemcpyAsync(*pa[i], *pb[i], sizeof(double) * len[i], cudaMemcpyDeviceToDevice,
                               h->stream));
    }
    CK(host_sync(h, h->stream));
    return SCOPF_OK;
}

int scopf_copy_state(scopf_handle *h, const scopf_state *dst) {
    if (!h || h->host_only || !dst) return SCOPF_ERR_INVALID_ARG;
    return copy_state(h, dst, &h->st, true);
}

int scopf_load_state(scopf_handle *h, const scopf_state *src) {
    if (!h || h->host_only || !src) return SCOPF_ERR_INVALID_ARG;
    return copy_state(h, &h->st, src, false);
}

int scopf_get_ncl_params(scopf_handle *h, double **lam_n, double **nu0_n, double *rho) {
    if (!h || h->host_only) return SCOPF_ERR_INVALID_ARG;
    if (lam_n) *lam_n = h->lam_n;
    if (nu0_n) *nu0_n = h->nu0_n;
    if (rho) *rho = h->rho;
    return SCOPF_OK;
}

}  // extern "C"

// ----------------------------------------------------------- implementations
namespace scopf {

double device_maxabs(scopf_handle *h, const double *x, int64_t n) {
    if (n <= 0) return 0.0;
    reduce_maxabs(x, n, h->red_out, h->red_scratch, h->stream);
    double v = 0;
    cudaMemcpyAsync(&v, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    host_sync(h, h->stream);
    return v;
}

double device_sumabs(scopf_handle *h, const double *x, int64_t n) {
    if (n <= 0) return 0.0;
    reduce_sumabs(x, n, h->red_out, h->red_scratch, h->stream);
    double v = 0;
    cudaMemcpyAsync(&v, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    host_sync(h, h->stream);
    return v;
}

// The model evaluation and KKT assembly at `it` (no right-hand side),
// enqueued on h->stream; rho may be a device scalar
void assemble_enqueue(scopf_handle *h, const scopf_state *it, DScalar rho, double delta_w) {
    cudaStream_t s = h->stream;
    const DevModel &d = h->dm;
    launch_eval_elements(d, it->w, it->lam, it->yc, h->ev, 1, s);
    launch_constraints(d, it->w, h->ev, h->c, s);
    launch_gradient(d, it->w, h->g, s);
    launch_diag_terms(d, it->w, it->zl, it->zu, it->s, it->zs, rho, delta_w, h->diag, s);
    launch_assemble(d, h->ev, h->diag, h->kval, s);
    launch_diag_gather(h->n_pdiag, h->pdiag_pos, h->kval, h->pdiag_base, s);
    launch_dual_product(d, h->kval, h->g, it->lam, it->yc, h->gw, s);
}

int assemble_impl(scopf_handle *h, const scopf_state *it, const double *lam_n, const double *nu0_n,
                  double rho, double mu, double delta_w, double *rhs) {
    cudaStream_t s = h->stream;
    const DevModel &d = h->dm;
    h->timer.begin(PH_ASSEMBLE, s);
    assemble_enqueue(h, it, rho, delta_w);
    if (rhs) {
        RhsArgs a{it->w, it->r, it->t, it->s, it->lam, it->yc, it->zs, h->gw, h->c, lam_n, nu0_n,
                  rho, mu};
        launch_rhs(d, a, rhs, s);
    }
    h->timer.end(PH_ASSEMBLE, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->last_error = cudaGetErrorString(e);
        return SCOPF_ERR_CUDA;
    }
    h->assembled = true;
    h->factored = false;
    h->lead_zero_valid = false;
    h->last_delta_w = delta_w;
    h->assembled_delta_w = delta_w;
    h->last_rho = rho;
    return SCOPF_OK;
}

// K(delta) from the assembled K(delta_a): the primal diagonal entries
// become (assembled value) + (delta - delta_a); nothing else depends on
// delta_w
int set_delta_w(scopf_handle *h, double delta_w) {
    if (!h->assembled) return SCOPF_ERR_NOT_FACTORED;
    h->timer.begin(PH_ASSEMBLE, h->stream);
    launch_diag_set(h->n_pdiag, h->pdiag_pos, h->pdiag_base, delta_w - h->assembled_delta_w,
                    h->kval, h->stream);
    h->timer.end(PH_ASSEMBLE, h->stream);
    h->factored = false;
    h->last_delta_w = delta_w;
    return SCOPF_OK;
}

// The device work of one factorization of the assembled K (equilibration,
// block fronts, Schur sum, dense border factor), enqueued on h->stream; the
// inertia and status land in h->fstat.
template <typename T>
cudaError_t factor_enqueue(scopf_handle *h) {
    cudaStream_t s = h->stream;
    T *fr = reinterpret_cast<T *>(h->fronts);
    cudaError_t e = cudaMemsetAsync(h->fstat, 0, sizeof(FactorStatus), s);
    if (e != cudaSuccess) return e;
    h->timer.begin(PH_FRONT_INIT, s);
    // Ruiz equilibration with power-of-two scales.  Such a scaling is exact
    // in floating point: the factors of D K D are D-scaled copies of those of
    // K, rounding for rounding, so it changes no result except through the
    // floating-point range and a nonzero pivot tolerance (compared with the
    // scaled pivots).  FP64 fronts have range to spare and, with a zero
    // tolerance, skip it (scale 1).  FP32 fronts take one sweep: it already
    // bounds every scaled entry below 4 (|a_ij| is at most both its row's and
    // its column's maximum), the guard against FP32 overflow the scaling is
    // for.  A nonzero tolerance keeps the three sweeps it was defined with.
    const int sweeps = h->opt.pivot_tol != 0.0 ? 3 : (sizeof(T) == 4 ? 1 : 0);
    launch_equilibrate(h->dm, h->kval, h->scale, h->scale_tmp, h->ruiz_mx, sweeps, s);
    launch_orig_vals<T>(h->df, reinterpret_cast<T *>(h->ovals), s);
    h->timer.end(PH_FRONT_INIT, s);
    h->timer.begin(PH_FACTOR, s);
    launch_factor<T>(h->df, fr, h->fstat, h->opt.pivot_tol, h->opt.spin_limit, s);
    h->timer.end(PH_FACTOR, s);
    h->timer.begin(PH_SCHUR, s);
    launch_schur_sum<T>(h->df, fr, h->S, s);
    e = launch_dense_ldlt(h->S, (int)h->M.nborder, h->fstat, h->opt.pivot_tol, s,
                          h->opt.spin_limit);
    if (e != cudaSuccess) return e;
    // FP32 block factors: the border block is applied through S^-1 (a mat-vec
    // per solve instead of two sequential triangular solves); the refinement
    // corrects its rounding like that of the block factors.  S^-1 is formed
    // by the first solve with these factors, so factorizations rejected by
    // the inertia correction never pay for it.
    h->sinv_stale = sizeof(T) == 4;
    h->timer.end(PH_SCHUR, s);
    return cudaGetLastError();
}
template cudaError_t factor_enqueue<float>(scopf_handle *);
template cudaError_t factor_enqueue<double>(scopf_handle *);

template <typename T>
static int factor_t(scopf_handle *h, int inertia[3]) {
    cudaStream_t s = h->stream;
    CK(factor_enqueue<T>(h));
    FactorStatus fs;
    CK(cudaMemcpyAsync(&fs, h->fstat, sizeof(fs), cudaMemcpyDeviceToHost, s));
    CK(host_sync(h, s));
    h->timer.collect();
    CK(cudaGetLastError());
    inertia[0] = fs.n_pos;
    inertia[1] = fs.n_neg;
    inertia[2] = fs.n_zero;
    h->n_factor++;
    if (fs.error) {
        h->last_error = "dependency wait timed out in the factorization";
        return SCOPF_ERR_TIMEOUT;
    }
    h->factored = true;
    return SCOPF_OK;
}

int factor_impl(scopf_handle *h, int precision, int inertia[3]) {
    h->factored_precision = precision;
    if (precision == SCOPF_PREC_MIXED) return factor_t<float>(h, inertia);
    return factor_t<double>(h, inertia);
}

template <typename T>
int solve_once(scopf_handle *h, const double *b, double *x) {
    h->timer.begin(PH_SOLVE, h->stream);
    launch_solve<T>(h->df, reinterpret_cast<T *>(h->fronts), reinterpret_cast<T *>(h->vec), h->S,
                    sizeof(T) == 4 ? h->Sinv : nullptr, (int)h->M.nborder, h->scale, b, x,
                    h->border_work, h->fstat, h->opt.spin_limit, h->stream);
    h->timer.end(PH_SOLVE, h->stream);
    return SCOPF_OK;
}
template int solve_once<float>(scopf_handle *, const double *, double *);
template int solve_once<double>(scopf_handle *, const double *, double *);

// One Krylov step of the refinement's FGMRES cycle (the body of a WHILE
// node whose condition `loop` it sets), enqueued on h->stream -- a stream
// that is capturing into the WHILE node's body graph.  Returns the kernels
// it launched.
template <typename T>
long long enqueue_krylov_step(scopf_handle *h, cudaGraphConditionalHandle loop) {
    const int64_t n = h->M.n_kkt;
    constexpr int m = 16;
    const GmresLayout GL = gmres_layout(m);
    double *sc = h->kst + GL.sc;
    double *vb = h->kry_buf, *zb = vb + n, *wb = zb + n;
    cudaStream_t cs = h->stream;
    const long long k0 = g_kernel_launches.load();
    launch_kry_gather(n, h->kv, h->kctl, vb, cs);
    solve_once<T>(h, vb, zb);
    launch_kry_scatter(n, zb, h->kz, h->kctl, cs);
    launch_spmv(h->dm, h->kval, zb, wb, cs);
    for (double *coef : {h->kst + GL.c1, h->kst + GL.c2}) {   // classical Gram-Schmidt, twice
        launch_kry_multi_dot(h->kv, n, h->kctl, wb, h->kpart, cs);
        launch_kry_dot_finish(h->kpart, h->kctl, coef, cs);
        launch_kry_axpy(wb, h->kv, n, h->kctl, false, coef, cs);
    }
    launch_multi_dot(wb, n, 1, wb, h->kpart, cs);
    launch_dot_finish(h->kpart, 1, sc + 1, true, cs);
    launch_kry_scale_out(n, sc + 1, wb, h->kv, h->kctl, cs);
    launch_kry_column_next(h->kst, m, h->kctl, loop, cs);
    return g_kernel_launches.load() - k0;
}
template long long enqueue_krylov_step<float>(scopf_handle *, cudaGraphConditionalHandle);
template long long enqueue_krylov_step<double>(scopf_handle *, cudaGraphConditionalHandle);

// FGMRES work buffers and the Krylov control block (allocated on first use)
int krylov_buffers(scopf_handle *h) {
    const int64_t n = h->M.n_kkt;
    constexpr int m = 16;
    const GmresLayout GL = gmres_layout(m);
    if (!h->kv) {
        TRY(alloc(h, (size_t)(m + 1) * n, &h->kv));
        TRY(alloc(h, (size_t)m * n, &h->kz));
        TRY(alloc(h, (size_t)kDotBlocks * kMaxKrylov, &h->kpart));
        TRY(alloc(h, (size_t)GL.total, &h->kst));
    }
    if (!h->kctl) {
        TRY(alloc(h, 1, &h->kctl));
        TRY(alloc(h, (size_t)3 * n, &h->kry_buf));
    }
    return SCOPF_OK;
}

// One Krylov step of the FGMRES cycle below, captured once per factor
// precision into a CUDA graph whose WHILE node repeats it: the column j,
// the counts and the loop decision live in h->kctl, so the cycle runs with
// no host round trip per step.  The step is the host loop's, kernel for
// kernel (same arithmetic), except that the basis vector is copied into a
// fixed input buffer and the preconditioned vector and the new direction are
// formed in fixed buffers and copied out.
template <typename T>
static int build_krylov_graph(scopf_handle *h, scopf_handle::KrylovGraph &G) {
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    auto fail = [&](cudaError_t e) {
        if (cs) cudaStreamDestroy(cs);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        h->last_error = cudaGetErrorString(e);
        G.failed = true;
        return SCOPF_OK;   // the host-driven loop takes over
    };
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(e);
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return fail(e);
    cudaGraphConditionalHandle loop;
    if ((e = cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return fail(e);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = loop;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) return fail(e);
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return fail(e);
    cudaStream_t keep = h->stream;
    const bool timing = h->timer.on;
    h->stream = cs;
    h->timer.on = false;
    G.body_kernels = enqueue_krylov_step<T>(h, loop);
    g_kernel_launches -= G.body_kernels;   // counted when they run
    h->stream = keep;
    h->timer.on = timing;
    e = cudaStreamEndCapture(cs, &body);
    if (e != cudaSuccess) return fail(e);
    if ((e = cudaGraphInstantiate(&G.exec, g, 0)) != cudaSuccess) {
        G.exec = nullptr;
        return fail(e);
    }
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return SCOPF_OK;
}

// Solve K x = b.  First x = M^-1 b with the factors M of K (FP64 or FP32);
// if the FP64 residual is not yet below refine_tol, continue with restarted
// FGMRES in FP64 on the correction, right-preconditioned by M (GMRES-based
// iterative refinement: it converges where classical refinement with FP32
// factors stalls, for condition numbers up to about 1/u_fp32^2).  The
// preconditioner applications after the first count as refinement steps.
// Gram-Schmidt coefficients, the Hessenberg column, its Givens rotations and
// the small triangular solve stay on the device; the host reads one scalar
// per Krylov step (the residual estimate) and one pair per residual check.
int solve_impl(scopf_handle *h, const double *b, double *x, int max_refine, double *rel, int *steps) {
    cudaStream_t s = h->stream;
    const int64_t n = h->M.n_kkt;
    const bool mixed = h->factored_precision == SCOPF_PREC_MIXED;
    auto once = [&](const double *rhs, double *out) {
        return mixed ? solve_once<float>(h, rhs, out) : solve_once<double>(h, rhs, out);
    };
    if (mixed && h->sinv_stale) {   // before any solve (or graph) uses it
        h->timer.begin(PH_SCHUR, s);
        launch_dense_inverse(h->S, (int)h->M.nborder, h->Sinv, s);
        h->timer.end(PH_SCHUR, s);
        h->sinv_stale = false;
    }
    constexpr int m = 16;
    const GmresLayout GL = gmres_layout(m);
    TRY(krylov_buffers(h));
    double *sc = h->kst + GL.sc;
    // device-resident Krylov loop (one graph per factor precision)
    scopf_handle::KrylovGraph *G = nullptr;
    if (h->opt.device_loop) {
        if (h->kgraph_stale) {
            for (auto &g : h->kgraph) {
                if (g.exec) cudaGraphExecDestroy(g.exec);
                g = scopf_handle::KrylovGraph{};
            }
            h->kgraph_stale = false;
        }
        G = &h->kgraph[mixed ? 0 : 1];
        if (!G->exec && !G->failed) {
            if (mixed) build_krylov_graph<float>(h, *G);
            else build_krylov_graph<double>(h, *G);
        }
        if (!G->exec) G = nullptr;
    }
    KrylovCtl ctl{};
    // |b|_inf and |b - K x|_inf, the sweeps' status and the Krylov loop's
    // counts, in one round trip
    FactorStatus fs{};
    auto residual_check = [&](double &bn, double &rn) {
        h->timer.begin(PH_RESIDUAL, s);
        launch_residual(h->dm, h->kval, x, h->res, h->tmp_kkt, s);
        h->timer.end(PH_RESIDUAL, s);
        reduce_maxabs2(h->res, h->tmp_kkt, n, h->red_out, h->red_scratch, s);
        double v[2] = {0, 0};
        cudaMemcpyAsync(v, h->red_out, sizeof(v), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&fs, h->fstat, sizeof(fs), cudaMemcpyDeviceToHost, s);
        if (G) cudaMemcpyAsync(&ctl, h->kctl, sizeof(ctl), cudaMemcpyDeviceToHost, s);
        host_sync(h, s);
        bn = v[0];
        rn = v[1];
    };
    CK(cudaMemcpyAsync(h->res, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    once(h->res, x);
    double bnorm = 0, rn = 0;
    residual_check(bnorm, rn);
    const double bden = bnorm > 0 ? bnorm : 1.0;
    int it = 0;
    double r = rn / bden;
    while (true) {
        if (h->opt.verbose >= 2)
            std::printf("    refine: %d preconditioner applications, |b-Kx|/|b| = %.3e (%s)\n", it,
                        r, mixed ? "fp32 factors" : "fp64 factors");
        if (!(r > h->opt.refine_tol) || it >= max_refine || !std::isfinite(r)) break;
        // one FGMRES(m) cycle on K e = r (r = tmp_kkt, nonzero here)
        launch_multi_dot(h->tmp_kkt, n, 1, h->tmp_kkt, h->kpart, s);
        launch_dot_finish(h->kpart, 1, sc + 0, true, s);
        launch_gmres_init(h->kst, m, s);
        launch_scale_inv(n, sc + 0, h->tmp_kkt, h->kv, s);
        int jend = 0;
        const double target = h->opt.refine_tol * bnorm * 0.5;
        if (G) {
            launch_kry_start(h->kctl, it, max_refine, target, s);
            cudaError_t ge = cudaGraphLaunch(G->exec, s);
            if (ge != cudaSuccess) {
                h->last_error = cudaGetErrorString(ge);
                return SCOPF_ERR_CUDA;
            }
            launch_kry_solve(h->kst, m, h->kctl, s);
            launch_kry_axpy(x, h->kz, n, h->kctl, true, h->kst + GL.c1, s);
            residual_check(bnorm, rn);
            g_kernel_launches += G->body_kernels * ctl.jend;
            it = ctl.it;
            r = rn / bden;
            continue;
        }
        for (int j = 0; j < m && it < max_refine; j++) {
            double *vj = h->kv + (size_t)j * n, *zj = h->kz + (size_t)j * n;
            double *w = h->kv + (size_t)(j + 1) * n;
            once(vj, zj);
            it++;
            launch_spmv(h->dm, h->kval, zj, w, s);
            // classical Gram-Schmidt, twice
            launch_multi_dot(h->kv, n, j + 1, w, h->kpart, s);
            launch_dot_finish(h->kpart, j + 1, h->kst + GL.c1, false, s);
            launch_multi_axpy_dev(w, h->kv, n, j + 1, h->kst + GL.c1, 1.0, s);
            launch_multi_dot(h->kv, n, j + 1, w, h->kpart, s);
            launch_dot_finish(h->kpart, j + 1, h->kst + GL.c2, false, s);
            launch_multi_axpy_dev(w, h->kv, n, j + 1, h->kst + GL.c2, 1.0, s);
            launch_multi_dot(w, n, 1, w, h->kpart, s);
            launch_dot_finish(h->kpart, 1, sc + 1, true, s);
            launch_scale_inv(n, sc + 1, w, w, s);
            launch_gmres_column(h->kst, m, j, s);
            double gj = 0;
            cudaMemcpyAsync(&gj, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
            host_sync(h, s);
            jend = j + 1;
            if (!(gj > target)) break;
        }
        launch_gmres_solve(h->kst, m, jend, s);
        launch_multi_axpy_dev(x, h->kz, n, jend, h->kst + GL.c1, 1.0, s);
        residual_check(bnorm, rn);
        r = rn / bden;
    }
    h->n_refine += it;
    h->n_solve_calls++;
    // every exit follows a residual check, whose round trip also read the
    // sweeps' status after the last solve
    h->timer.collect();
    CK(cudaGetLastError());
    *rel = r;
    *steps = it;
    if (fs.error) return SCOPF_ERR_TIMEOUT;
    if (!std::isfinite(r)) return SCOPF_ERR_NUMERICAL;
    if (r > h->opt.refine_tol) return SCOPF_ERR_REFINE_STALL;
    return SCOPF_OK;
}

}  // namespace scopf


