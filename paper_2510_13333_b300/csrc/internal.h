// Internal declarations of the SCOPF / NCL Newton-step library.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/scopf.h"

namespace scopf {

// ---------------------------------------------------------------- layout
// One scenario block (k = 0 base case).  Local indices are -1 when the
// quantity is not a variable / row of the block.  Index maps follow the
// natural order documented in scopf.h.
struct Block {
    int k = 0, kind = -1, element = -1;
    std::vector<int> gens, branches, thermal, sw_bus, sw_gen;
    std::vector<int> th, v, p, q;               // per bus / per generator
    int delta = -1;
    std::vector<int> sth;                        // 2 per thermal branch
    std::vector<int> pim, pip, spu, spl;         // per in-service generator
    std::vector<int> num, nup, squ, sql;         // per switch bus
    std::vector<int> rP, rQ, rth;                // rows
    std::vector<int> rdroop, rspu, rspl, rpvpq, rsqu, rsql;
    std::vector<int> gen_pos;                    // generator -> position in gens (-1)
    std::vector<int> sw_of_gen;                  // generator -> switch position (-1)
    int nvar = 0, nrow = 0, ncomp = 0;
    int64_t w0 = 0, c0 = 0, p0 = 0;              // global offsets
    int64_t kkt0 = 0;                            // KKT offset of the block
    int64_t nkkt() const { return (int64_t)nvar + nrow + ncomp; }
    std::vector<double> alpha;                   // per generator (0 if out)
};

// Contribution of one stored KKT entry: coef * (src >= 0 ? ev[src] : 1).
struct Contrib {
    int64_t src;
    double coef;
};

// Per-branch-element value slots (structure of arrays, slot * n_be + e).
enum BranchSlot {
    BS_F = 0,          // 4 flows p_ij, q_ij, p_ji, q_ji
    BS_H = 4,          // 2 thermal values (p^2+q^2)/rate^2 (from, to)
    BS_DF = 6,         // 16: dF_a/dx_j, a*4+j, x = (th_f, th_t, v_f, v_t)
    BS_DH = 22,        // 8: dh_e/dx_j, e*4+j
    BS_HESS = 30,      // 10: weighted Hessian, upper triangle row-major
    BS_COUNT = 40
};

struct Model {
    // network copy
    int nb = 0, nl = 0, ng = 0, ref = 0, K = 0;
    std::vector<double> Pd, Qd, Gs, Bs, vmin, vmax, r, x, bch, rate, g, bs;
    std::vector<int> f, t, gbus;
    std::vector<double> pmin, pmax, qmin, qmax, c2, c1, c0;
    std::vector<int> gen_at, pv, pv_pos;
    std::vector<scopf_contingency> ctg;
    std::vector<std::vector<int>> ctg_sw;

    std::vector<Block> blocks;
    int64_t n = 0, m = 0, p = 0, border0 = 0, nborder = 0;
    int64_t n_kkt = 0, kkt_border0 = 0;

    // bounds (relaxation is applied by the solver), finite masks
    std::vector<double> wl, wu;
    std::vector<int64_t> comp1, comp2;   // w indices of the complementarity pairs
    std::vector<double> w_init;

    // ---- branch elements (one per in-service branch per scenario)
    int64_t n_be = 0;
    std::vector<int32_t> be_x;      // 4 per element: w index of th_f, th_t, v_f, v_t (-1 = theta_ref)
    std::vector<int32_t> be_lam;    // 4 per element: c rows Pf, Qf, Pt, Qt
    std::vector<int32_t> be_th;     // 2 per element: thermal c rows (-1)
    std::vector<double> be_par;     // 4 per element: g, b, bc, 1/rate^2 (0 = unlimited)
    // ---- bus shunt elements (one per bus per scenario): slots 5
    int64_t n_se = 0;
    std::vector<int32_t> se_v, se_P, se_Q;
    std::vector<double> se_G, se_B;
    // ---- value buffer layout
    int64_t ev_branch0 = 0, ev_shunt0 = 0, ev_comp0 = 0, n_ev = 0;

    // ---- KKT pattern (full symmetric CSR, natural KKT order)
    std::vector<int64_t> kkt_ptr, kkt_col;
    std::vector<int64_t> ctr_ptr;        // per stored entry
    std::vector<Contrib> ctr;
    std::vector<int64_t> diag_pos;       // per KKT row: stored index of (i,i)
    // KKT row type: 0 = w (with bound info), 1 = equality row, 2 = comp row
    std::vector<int8_t> row_kind;
    std::vector<int64_t> row_index;      // w index / c row / comp index
    // ---- constraint residual c: const + sum coef*ev[src] + sum coef*w[col]
    std::vector<double> c_const;
    std::vector<int64_t> cf_ptr;
    std::vector<int64_t> cf_idx;         // >= 0: ev index; < 0: -(w index) - 1
    std::vector<double> cf_coef;
    // KKT row of every w index / c row / comp index
    std::vector<int64_t> kkt_of_w, kkt_of_c, kkt_of_comp;
    std::vector<int32_t> block_of_kkt;   // -1 for border rows
};

std::string build_model(const scopf_network *net, const scopf_contingency *ctg, int32_t K,
                        Model &M);

// ------------------------------------------------------------- symbolic
struct BlockSymbolic {
    int n_nodes = 0, n_block_nodes = 0;
    std::vector<std::vector<int64_t>> node_rows;  // global KKT indices of each node
    std::vector<int> post;            // node ids in postorder
    std::vector<int> node_parent;     // per node id: parent node id, -2 border, -1 none
    std::vector<int> sn_start;        // n_sn + 1, postorder positions
    std::vector<std::vector<int>> sn_update_nodes;  // by postorder position order
    std::vector<int> sn_parent;       // -2 = border
    std::vector<int64_t> rows;        // KKT indices in elimination order (+ border)
    int64_t n_block_rows = 0;
};

std::string symbolic_block(const Model &M, int k, int relax_max_nodes, int relax_max_front,
                           bool dual_first, BlockSymbolic &S);

}  // namespace scopf
