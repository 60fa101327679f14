// Host-side construction of the SCOPF model (Section II, eq. scopf, in the
// vertical MPCC form of eq. mpcc): layouts, element tables, the KKT pattern
// of eq. (newtonsystem) and the per-entry contribution lists used by the
// device assembly kernel.
//
// Readings of the paper (all shared with the documentation of scopf.h):
//  * pi-model flows with tap 1 and no phase shift; theta_ref = 0;
//  * thermal row (p^2 + q^2)/rate^2 - 1 + sigma = 0, sigma >= 0;
//  * objective sum(c2 (100 p)^2 + c1 (100 p) + c0) / 1e4 over the base case;
//  * alpha_g = pmax_g / sum of pmax over generators in service in block k;
//  * PV buses outside the switch set keep q in bounds, v free in bounds.
#include <algorithm>
#include <thread>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace scopf {

static const double kObjScale = 1.0e4;
static const double kBaseMVA = 100.0;

namespace {

struct Tuple {
    int64_t row, col;
    int64_t src;
    double coef;
};

}  // namespace

std::string build_model(const scopf_network *net, const scopf_contingency *ctg, int32_t K,
                        Model &M) {
    if (!net || net->n_bus <= 0 || net->n_branch < 0 || net->n_gen <= 0 || K < 0)
        return "invalid network sizes";
    if (net->ref_bus < 0 || net->ref_bus >= net->n_bus) return "ref_bus out of range";
    if (K > 0 && !ctg) return "contingency array is NULL";
    M.nb = net->n_bus;
    M.nl = net->n_branch;
    M.ng = net->n_gen;
    M.ref = net->ref_bus;
    M.K = K;
    auto cp = [](const double *src, int n, std::vector<double> &dst) {
        dst.assign(src, src + n);
    };
    cp(net->Pd, M.nb, M.Pd);
    cp(net->Qd, M.nb, M.Qd);
    cp(net->Gs, M.nb, M.Gs);
    cp(net->Bs, M.nb, M.Bs);
    cp(net->vmin, M.nb, M.vmin);
    cp(net->vmax, M.nb, M.vmax);
    cp(net->br_r, M.nl, M.r);
    cp(net->br_x, M.nl, M.x);
    cp(net->br_b, M.nl, M.bch);
    cp(net->br_rate, M.nl, M.rate);
    M.f.assign(net->br_from, net->br_from + M.nl);
    M.t.assign(net->br_to, net->br_to + M.nl);
    M.gbus.assign(net->gen_bus, net->gen_bus + M.ng);
    cp(net->pmin, M.ng, M.pmin);
    cp(net->pmax, M.ng, M.pmax);
    cp(net->qmin, M.ng, M.qmin);
    cp(net->qmax, M.ng, M.qmax);
    cp(net->c2, M.ng, M.c2);
    cp(net->c1, M.ng, M.c1);
    cp(net->c0, M.ng, M.c0);
    for (int l = 0; l < M.nl; l++) {
        if (M.f[l] < 0 || M.f[l] >= M.nb || M.t[l] < 0 || M.t[l] >= M.nb || M.f[l] == M.t[l])
            return "branch endpoint out of range";
        double z2 = M.r[l] * M.r[l] + M.x[l] * M.x[l];
        if (!(z2 > 0)) return "branch with zero impedance";
        M.g.push_back(M.r[l] / z2);
        M.bs.push_back(-M.x[l] / z2);
    }
    M.gen_at.assign(M.nb, -1);
    for (int gi = 0; gi < M.ng; gi++) {
        int b = M.gbus[gi];
        if (b < 0 || b >= M.nb) return "generator bus out of range";
        if (M.gen_at[b] >= 0) return "at most one generator per bus is supported";
        M.gen_at[b] = gi;
    }
    M.pv_pos.assign(M.nb, -1);
    for (int b = 0; b < M.nb; b++)
        if (M.gen_at[b] >= 0) {
            M.pv_pos[b] = (int)M.pv.size();
            M.pv.push_back(b);
        }
    const int nb = M.nb, ng = M.ng, npv = (int)M.pv.size();
    M.ctg.assign(ctg, ctg + K);
    M.ctg_sw.resize(K);
    for (int k = 0; k < K; k++) {
        const auto &c = ctg[k];
        if (c.kind == SCOPF_CTG_LINE) {
            if (c.element < 0 || c.element >= M.nl) return "line contingency out of range";
        } else if (c.kind == SCOPF_CTG_GEN) {
            if (c.element < 0 || c.element >= ng) return "generator contingency out of range";
        } else {
            return "unknown contingency kind";
        }
        if (c.n_switch < 0 || (c.n_switch > 0 && !c.switch_buses)) return "bad switch set";
        M.ctg_sw[k].assign(c.switch_buses, c.switch_buses + c.n_switch);
        for (int i = 0; i < c.n_switch; i++) {
            int b = c.switch_buses[i];
            if (b < 0 || b >= nb || M.gen_at[b] < 0) return "switch bus without generator";
            if (c.kind == SCOPF_CTG_GEN && M.gen_at[b] == c.element)
                return "switch bus of an outaged generator";
            if (i > 0 && c.switch_buses[i - 1] >= b) return "switch buses not sorted";
        }
    }

    // ------------------------------------------------------------ blocks
    M.blocks.resize(K + 1);
    for (int k = 0; k <= K; k++) {
        Block &B = M.blocks[k];
        B.k = k;
        int nxt = 0;
        auto take = [&](int cnt, std::vector<int> &dst) {
            for (int i = 0; i < cnt; i++) dst.push_back(nxt++);
        };
        if (k > 0) {
            B.kind = M.ctg[k - 1].kind;
            B.element = M.ctg[k - 1].element;
        }
        for (int gi = 0; gi < ng; gi++)
            if (!(k > 0 && B.kind == SCOPF_CTG_GEN && B.element == gi)) B.gens.push_back(gi);
        for (int l = 0; l < M.nl; l++)
            if (!(k > 0 && B.kind == SCOPF_CTG_LINE && B.element == l)) {
                B.branches.push_back(l);
                if (M.rate[l] > 0) B.thermal.push_back(l);
            }
        if (k > 0) B.sw_bus = M.ctg_sw[k - 1];
        for (int b : B.sw_bus) B.sw_gen.push_back(M.gen_at[b]);
        B.gen_pos.assign(ng, -1);
        for (size_t i = 0; i < B.gens.size(); i++) B.gen_pos[B.gens[i]] = (int)i;
        B.sw_of_gen.assign(ng, -1);
        for (size_t i = 0; i < B.sw_gen.size(); i++) B.sw_of_gen[B.sw_gen[i]] = (int)i;
        // variables
        B.th.assign(nb, -1);
        for (int b = 0; b < nb; b++)
            if (b != M.ref) B.th[b] = nxt++;
        B.v.assign(nb, -1);
        for (int b = 0; b < nb; b++)
            if (k > 0 || M.gen_at[b] < 0) B.v[b] = nxt++;
        B.p.assign(ng, -1);
        B.q.assign(ng, -1);
        if (k > 0)
            for (int gi : B.gens) B.p[gi] = nxt++;
        for (int gi : B.gens) B.q[gi] = nxt++;
        if (k > 0) B.delta = nxt++;
        take(2 * (int)B.thermal.size(), B.sth);
        int ngk = k > 0 ? (int)B.gens.size() : 0;
        int nsw = k > 0 ? (int)B.sw_bus.size() : 0;
        take(ngk, B.pim);
        take(ngk, B.pip);
        take(ngk, B.spu);
        take(ngk, B.spl);
        take(nsw, B.num);
        take(nsw, B.nup);
        take(nsw, B.squ);
        take(nsw, B.sql);
        B.nvar = nxt;
        // rows
        nxt = 0;
        take(nb, B.rP);
        take(nb, B.rQ);
        take(2 * (int)B.thermal.size(), B.rth);
        take(ngk, B.rdroop);
        take(ngk, B.rspu);
        take(ngk, B.rspl);
        take(nsw, B.rpvpq);
        take(nsw, B.rsqu);
        take(nsw, B.rsql);
        B.nrow = nxt;
        B.ncomp = 2 * ngk + 2 * nsw;
        B.alpha.assign(ng, 0.0);
        double psum = 0;
        for (int gi : B.gens) psum += M.pmax[gi];
        for (int gi : B.gens) B.alpha[gi] = psum > 0 ? M.pmax[gi] / psum : 0.0;
    }
    int64_t ow = 0, oc = 0, op = 0, ok = 0;
    for (auto &B : M.blocks) {
        B.w0 = ow;
        B.c0 = oc;
        B.p0 = op;
        B.kkt0 = ok;
        ow += B.nvar;
        oc += B.nrow;
        op += B.ncomp;
        ok += B.nkkt();
    }
    M.border0 = ow;
    M.nborder = ng + npv;
    M.n = ow + M.nborder;
    M.m = oc;
    M.p = op;
    M.kkt_border0 = ok;
    M.n_kkt = ok + M.nborder;

    // global index helpers
    auto gw = [&](const Block &B, int local) -> int64_t { return local < 0 ? -1 : B.w0 + local; };
    auto gv = [&](const Block &B, int b) -> int64_t {
        if (B.k == 0 && M.gen_at[b] >= 0) return M.border0 + ng + M.pv_pos[b];
        return gw(B, B.v[b]);
    };
    auto gp = [&](const Block &B, int gi) -> int64_t {
        if (B.k == 0) return M.border0 + gi;
        return gw(B, B.p[gi]);
    };
    auto gc = [&](const Block &B, int local) -> int64_t { return B.c0 + local; };

    M.kkt_of_w.assign(M.n, -1);
    M.kkt_of_c.assign(M.m, -1);
    M.kkt_of_comp.assign(M.p, -1);
    M.block_of_kkt.assign(M.n_kkt, -1);
    M.row_kind.assign(M.n_kkt, 0);
    M.row_index.assign(M.n_kkt, 0);
    for (auto &B : M.blocks) {
        for (int i = 0; i < B.nvar; i++) {
            M.kkt_of_w[B.w0 + i] = B.kkt0 + i;
            M.row_kind[B.kkt0 + i] = 0;
            M.row_index[B.kkt0 + i] = B.w0 + i;
        }
        for (int i = 0; i < B.nrow; i++) {
            M.kkt_of_c[B.c0 + i] = B.kkt0 + B.nvar + i;
            M.row_kind[B.kkt0 + B.nvar + i] = 1;
            M.row_index[B.kkt0 + B.nvar + i] = B.c0 + i;
        }
        for (int i = 0; i < B.ncomp; i++) {
            M.kkt_of_comp[B.p0 + i] = B.kkt0 + B.nvar + B.nrow + i;
            M.row_kind[B.kkt0 + B.nvar + B.nrow + i] = 2;
            M.row_index[B.kkt0 + B.nvar + B.nrow + i] = B.p0 + i;
        }
        for (int64_t i = 0; i < B.nkkt(); i++) M.block_of_kkt[B.kkt0 + i] = B.k;
    }
    for (int64_t j = 0; j < M.nborder; j++) {
        M.kkt_of_w[M.border0 + j] = M.kkt_border0 + j;
        M.row_kind[M.kkt_border0 + j] = 0;
        M.row_index[M.kkt_border0 + j] = M.border0 + j;
    }

    // ------------------------------------------------ bounds, comp, start
    const double INF = INFINITY;
    M.wl.assign(M.n, -INF);
    M.wu.assign(M.n, INF);
    M.w_init.assign(M.n, 0.0);
    for (int gi = 0; gi < ng; gi++) {
        M.wl[M.border0 + gi] = M.pmin[gi];
        M.wu[M.border0 + gi] = M.pmax[gi];
        M.w_init[M.border0 + gi] = 0.5 * (M.pmin[gi] + M.pmax[gi]);
    }
    for (auto &B : M.blocks) {
        for (int b = 0; b < nb; b++) {
            int64_t iv = gv(B, b);
            M.wl[iv] = M.vmin[b];
            M.wu[iv] = M.vmax[b];
            M.w_init[iv] = 1.0;
        }
        for (int i : B.sth) {
            M.wl[B.w0 + i] = 0.0;
            M.w_init[B.w0 + i] = 1.0;
        }
        for (int gi : B.gens) {
            double qmid = 0.5 * (M.qmin[gi] + M.qmax[gi]);
            M.w_init[gw(B, B.q[gi])] = qmid;
            bool bounded_q = (B.k == 0) || (B.sw_of_gen[gi] < 0);
            if (bounded_q) {
                M.wl[gw(B, B.q[gi])] = M.qmin[gi];
                M.wu[gw(B, B.q[gi])] = M.qmax[gi];
            }
        }
        if (B.k > 0) {
            for (size_t i = 0; i < B.gens.size(); i++) {
                int gi = B.gens[i];
                double pmid = 0.5 * (M.pmin[gi] + M.pmax[gi]);
                M.w_init[gw(B, B.p[gi])] = pmid;
                M.w_init[gw(B, B.spu[i])] = M.pmax[gi] - pmid;
                M.w_init[gw(B, B.spl[i])] = pmid - M.pmin[gi];
            }
            for (size_t i = 0; i < B.sw_bus.size(); i++) {
                int gi = B.sw_gen[i];
                double qmid = 0.5 * (M.qmin[gi] + M.qmax[gi]);
                M.w_init[gw(B, B.squ[i])] = M.qmax[gi] - qmid;
                M.w_init[gw(B, B.sql[i])] = qmid - M.qmin[gi];
            }
            for (auto *vec : {&B.pim, &B.pip, &B.spu, &B.spl, &B.num, &B.nup, &B.squ, &B.sql})
                for (int i : *vec) M.wl[B.w0 + i] = 0.0;
        }
    }
    M.comp1.clear();
    M.comp2.clear();
    for (auto &B : M.blocks) {
        if (B.k == 0) continue;
        for (int i : B.pim) M.comp1.push_back(B.w0 + i);
        for (int i : B.pip) M.comp1.push_back(B.w0 + i);
        for (int i : B.num) M.comp1.push_back(B.w0 + i);
        for (int i : B.nup) M.comp1.push_back(B.w0 + i);
        for (int i : B.spu) M.comp2.push_back(B.w0 + i);
        for (int i : B.spl) M.comp2.push_back(B.w0 + i);
        for (int i : B.squ) M.comp2.push_back(B.w0 + i);
        for (int i : B.sql) M.comp2.push_back(B.w0 + i);
    }

    // ------------------------------------------------- element tables
    for (auto &B : M.blocks) M.n_be += (int64_t)B.branches.size();
    M.n_se = (int64_t)(K + 1) * nb;
    M.ev_branch0 = 0;
    M.ev_shunt0 = M.ev_branch0 + BS_COUNT * M.n_be;
    M.ev_comp0 = M.ev_shunt0 + 5 * M.n_se;
    M.n_ev = M.ev_comp0 + 3 * M.p;
    auto evb = [&](int slot, int64_t e) { return M.ev_branch0 + (int64_t)slot * M.n_be + e; };
    auto evs = [&](int slot, int64_t e) { return M.ev_shunt0 + (int64_t)slot * M.n_se + e; };
    auto evc = [&](int slot, int64_t q) { return M.ev_comp0 + (int64_t)slot * M.p + q; };

    std::vector<Tuple> tup;
    tup.reserve((size_t)M.n_be * 72 + (size_t)M.n_kkt * 4);
    // residual contributions: per c row
    // residual contributions (row, (source, coefficient)) in insertion order;
    // one flat list instead of a list per row (m small allocations)
    struct RowLists {
        std::vector<int64_t> row;
        std::vector<std::pair<int64_t, double>> val;
        struct Ref {
            RowLists *L;
            int64_t r;
            void push_back(const std::pair<int64_t, double> &p) {
                L->row.push_back(r);
                L->val.push_back(p);
            }
        };
        Ref operator[](int64_t r) { return Ref{this, r}; }
    } cfun;
    M.c_const.assign(M.m, 0.0);
    auto sym = [&](int64_t i, int64_t j, int64_t src, double coef) {
        tup.push_back({i, j, src, coef});
        if (i != j) tup.push_back({j, i, src, coef});
    };
    auto Kw = [&](int64_t wi) { return M.kkt_of_w[wi]; };
    auto Kc = [&](int64_t ci) { return M.kkt_of_c[ci]; };

    // diagonal of every KKT row (barrier / regularisation / -C terms)
    for (int64_t i = 0; i < M.n_kkt; i++) tup.push_back({i, i, -2, 0.0});

    int64_t e = 0;
    for (auto &B : M.blocks) {
        // branch elements
        std::vector<int> thpos(M.nl, -1);
        for (size_t j = 0; j < B.thermal.size(); j++) thpos[B.thermal[j]] = (int)j;
        for (int l : B.branches) {
            int fb = M.f[l], tb = M.t[l];
            int64_t X[4] = {gw(B, B.th[fb]), gw(B, B.th[tb]), gv(B, fb), gv(B, tb)};
            int64_t R[4] = {gc(B, B.rP[fb]), gc(B, B.rQ[fb]), gc(B, B.rP[tb]), gc(B, B.rQ[tb])};
            int j = thpos[l];
            int64_t TH[2] = {j >= 0 ? gc(B, B.rth[2 * j]) : -1, j >= 0 ? gc(B, B.rth[2 * j + 1]) : -1};
            for (int a = 0; a < 4; a++) M.be_x.push_back((int32_t)X[a]);
            for (int a = 0; a < 4; a++) M.be_lam.push_back((int32_t)R[a]);
            M.be_th.push_back((int32_t)TH[0]);
            M.be_th.push_back((int32_t)TH[1]);
            M.be_par.push_back(M.g[l]);
            M.be_par.push_back(M.bs[l]);
            M.be_par.push_back(M.bch[l]);
            M.be_par.push_back(j >= 0 ? 1.0 / (M.rate[l] * M.rate[l]) : 0.0);
            // balance rows carry -F
            for (int a = 0; a < 4; a++) {
                cfun[R[a]].push_back({evb(BS_F + a, e), -1.0});
                for (int xj = 0; xj < 4; xj++)
                    if (X[xj] >= 0) sym(Kc(R[a]), Kw(X[xj]), evb(BS_DF + 4 * a + xj, e), -1.0);
            }
            if (j >= 0) {
                for (int side = 0; side < 2; side++) {
                    int64_t row = TH[side];
                    int64_t sig = gw(B, B.sth[2 * j + side]);
                    cfun[row].push_back({evb(BS_H + side, e), 1.0});
                    cfun[row].push_back({-(sig + 1), 1.0});
                    M.c_const[row] = -1.0;
                    for (int xj = 0; xj < 4; xj++)
                        if (X[xj] >= 0) sym(Kc(row), Kw(X[xj]), evb(BS_DH + 4 * side + xj, e), 1.0);
                    sym(Kc(row), Kw(sig), -1, 1.0);
                }
            }
            int hs = 0;
            for (int a = 0; a < 4; a++)
                for (int b2 = a; b2 < 4; b2++, hs++)
                    if (X[a] >= 0 && X[b2] >= 0) {
                        if (X[a] == X[b2])
                            tup.push_back({Kw(X[a]), Kw(X[a]), evb(BS_HESS + hs, e), 1.0});
                        else
                            sym(Kw(X[a]), Kw(X[b2]), evb(BS_HESS + hs, e), 1.0);
                    }
            e++;
        }
        // bus: loads, shunts, generator injections
        for (int b = 0; b < nb; b++) {
            int64_t se = (int64_t)B.k * nb + b;
            int64_t iv = gv(B, b);
            int64_t rP = gc(B, B.rP[b]), rQ = gc(B, B.rQ[b]);
            M.se_v.push_back((int32_t)iv);
            M.se_P.push_back((int32_t)rP);
            M.se_Q.push_back((int32_t)rQ);
            M.se_G.push_back(M.Gs[b]);
            M.se_B.push_back(M.Bs[b]);
            M.c_const[rP] = -M.Pd[b];
            M.c_const[rQ] = -M.Qd[b];
            // slots: 0 -Gs v^2, 1 Bs v^2, 2 -2Gs v, 3 2Bs v, 4 hessian
            cfun[rP].push_back({evs(0, se), 1.0});
            cfun[rQ].push_back({evs(1, se), 1.0});
            sym(Kc(rP), Kw(iv), evs(2, se), 1.0);
            sym(Kc(rQ), Kw(iv), evs(3, se), 1.0);
            tup.push_back({Kw(iv), Kw(iv), evs(4, se), 1.0});
            int gi = M.gen_at[b];
            if (gi >= 0 && B.gen_pos[gi] >= 0) {
                int64_t ip = gp(B, gi), iq = gw(B, B.q[gi]);
                cfun[rP].push_back({-(ip + 1), 1.0});
                cfun[rQ].push_back({-(iq + 1), 1.0});
                sym(Kc(rP), Kw(ip), -1, 1.0);
                sym(Kc(rQ), Kw(iq), -1, 1.0);
            }
        }
        if (B.k > 0) {
            for (size_t i = 0; i < B.gens.size(); i++) {
                int gi = B.gens[i];
                int64_t pk = gw(B, B.p[gi]), p0 = M.border0 + gi;
                int64_t rd = gc(B, B.rdroop[i]), ru = gc(B, B.rspu[i]), rl = gc(B, B.rspl[i]);
                int64_t ipp = gw(B, B.pip[i]), ipm = gw(B, B.pim[i]);
                int64_t isu = gw(B, B.spu[i]), isl = gw(B, B.spl[i]);
                int64_t idl = gw(B, B.delta);
                // eq. (droopmpec): pi_+ - pi_- - p^k + p^0 + alpha Delta^k = 0
                std::pair<int64_t, double> dr[5] = {{ipp, 1.0}, {ipm, -1.0}, {pk, -1.0},
                                                    {p0, 1.0}, {idl, B.alpha[gi]}};
                for (auto &pr : dr) {
                    cfun[rd].push_back({-(pr.first + 1), pr.second});
                    sym(Kc(rd), Kw(pr.first), -1, pr.second);
                }
                std::pair<int64_t, double> du[2] = {{isu, 1.0}, {pk, 1.0}};
                for (auto &pr : du) {
                    cfun[ru].push_back({-(pr.first + 1), pr.second});
                    sym(Kc(ru), Kw(pr.first), -1, pr.second);
                }
                M.c_const[ru] = -M.pmax[gi];
                std::pair<int64_t, double> dl[2] = {{isl, 1.0}, {pk, -1.0}};
                for (auto &pr : dl) {
                    cfun[rl].push_back({-(pr.first + 1), pr.second});
                    sym(Kc(rl), Kw(pr.first), -1, pr.second);
                }
                M.c_const[rl] = M.pmin[gi];
            }
            for (size_t i = 0; i < B.sw_bus.size(); i++) {
                int b = B.sw_bus[i], gi = B.sw_gen[i];
                int64_t vk = gw(B, B.v[b]), v0 = M.border0 + ng + M.pv_pos[b];
                int64_t iq = gw(B, B.q[gi]);
                int64_t rv = gc(B, B.rpvpq[i]), ru = gc(B, B.rsqu[i]), rl = gc(B, B.rsql[i]);
                // eq. (pvpq): nu_+ - nu_- - v^k + v^0 = 0
                std::pair<int64_t, double> dv[4] = {{gw(B, B.nup[i]), 1.0}, {gw(B, B.num[i]), -1.0},
                                                    {vk, -1.0}, {v0, 1.0}};
                for (auto &pr : dv) {
                    cfun[rv].push_back({-(pr.first + 1), pr.second});
                    sym(Kc(rv), Kw(pr.first), -1, pr.second);
                }
                std::pair<int64_t, double> du[2] = {{gw(B, B.squ[i]), 1.0}, {iq, 1.0}};
                for (auto &pr : du) {
                    cfun[ru].push_back({-(pr.first + 1), pr.second});
                    sym(Kc(ru), Kw(pr.first), -1, pr.second);
                }
                M.c_const[ru] = -M.qmax[gi];
                std::pair<int64_t, double> dl[2] = {{gw(B, B.sql[i]), 1.0}, {iq, -1.0}};
                for (auto &pr : dl) {
                    cfun[rl].push_back({-(pr.first + 1), pr.second});
                    sym(Kc(rl), Kw(pr.first), -1, pr.second);
                }
                M.c_const[rl] = M.qmin[gi];
            }
        }
    }
    // objective Hessian on p_g^0 (constant 2 c2 * 100^2 / 1e4)
    for (int gi = 0; gi < ng; gi++) {
        int64_t k0 = Kw(M.border0 + gi);
        tup.push_back({k0, k0, -1, 2.0 * M.c2[gi] * kBaseMVA * kBaseMVA / kObjScale});
    }
    // complementarity rows: (comp, w1) = w2, (comp, w2) = w1, Hessian (w1, w2) = y_c
    for (int64_t qq = 0; qq < M.p; qq++) {
        int64_t kc = M.kkt_of_comp[qq];
        sym(kc, Kw(M.comp1[qq]), evc(0, qq), 1.0);
        sym(kc, Kw(M.comp2[qq]), evc(1, qq), 1.0);
        sym(Kw(M.comp1[qq]), Kw(M.comp2[qq]), evc(2, qq), 1.0);
    }

    // --------------------------------------------------- CSR + contributions
    // order the tuples by (row, col, src, coef): a counting sort by row, then
    // each row's few tuples sorted on (col, src, coef), rows spread over the
    // host's cores (the same order a global sort gives)
    {
        std::vector<int64_t> start(M.n_kkt + 1, 0);
        for (const Tuple &t : tup) start[t.row + 1]++;
        for (int64_t r = 0; r < M.n_kkt; r++) start[r + 1] += start[r];
        std::vector<Tuple> by_row(tup.size());
        {
            std::vector<int64_t> fill(start.begin(), start.end() - 1);
            for (const Tuple &t : tup) by_row[fill[t.row]++] = t;
        }
        tup.swap(by_row);
        auto less = [](const Tuple &a, const Tuple &b) {
            if (a.col != b.col) return a.col < b.col;
            if (a.src != b.src) return a.src < b.src;
            return a.coef < b.coef;
        };
        const unsigned hw = std::thread::hardware_concurrency();
        const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(hw ? hw : 1, M.n_kkt));
        std::vector<std::thread> pool;
        auto work = [&](int64_t t) {
            for (int64_t r = t; r < M.n_kkt; r += nt)
                std::sort(tup.begin() + start[r], tup.begin() + start[r + 1], less);
        };
        for (int64_t t = 1; t < nt; t++) pool.emplace_back(work, t);
        work(0);
        for (auto &th : pool) th.join();
    }
    M.kkt_ptr.assign(M.n_kkt + 1, 0);
    M.kkt_col.clear();
    M.ctr_ptr.clear();
    M.ctr.clear();
    M.kkt_col.reserve(tup.size());
    M.ctr_ptr.reserve(tup.size() + 1);
    M.ctr.reserve(tup.size());
    M.diag_pos.assign(M.n_kkt, -1);
    size_t i0 = 0;
    while (i0 < tup.size()) {
        size_t i1 = i0;
        while (i1 < tup.size() && tup[i1].row == tup[i0].row && tup[i1].col == tup[i0].col) i1++;
        int64_t row = tup[i0].row, col = tup[i0].col;
        M.kkt_ptr[row + 1]++;
        if (row == col) M.diag_pos[row] = (int64_t)M.kkt_col.size();
        M.kkt_col.push_back(col);
        M.ctr_ptr.push_back((int64_t)M.ctr.size());
        for (size_t q = i0; q < i1; q++)
            if (tup[q].src != -2) M.ctr.push_back({tup[q].src, tup[q].coef});
        i0 = i1;
    }
    M.ctr_ptr.push_back((int64_t)M.ctr.size());
    for (int64_t r0 = 0; r0 < M.n_kkt; r0++) M.kkt_ptr[r0 + 1] += M.kkt_ptr[r0];
    for (int64_t r0 = 0; r0 < M.n_kkt; r0++)
        if (M.diag_pos[r0] < 0) return "internal: missing KKT diagonal";
    // residual function CSR
    // (stable counting sort by row: each row keeps its insertion order)
    M.cf_ptr.assign(M.m + 1, 0);
    for (int64_t r : cfun.row) M.cf_ptr[r + 1]++;
    for (int64_t rr = 0; rr < M.m; rr++) M.cf_ptr[rr + 1] += M.cf_ptr[rr];
    M.cf_idx.assign(cfun.row.size(), 0);
    M.cf_coef.assign(cfun.row.size(), 0.0);
    {
        std::vector<int64_t> fill(M.cf_ptr.begin(), M.cf_ptr.end() - 1);
        for (size_t q = 0; q < cfun.row.size(); q++) {
            const int64_t at = fill[cfun.row[q]]++;
            M.cf_idx[at] = cfun.val[q].first;
            M.cf_coef[at] = cfun.val[q].second;
        }
    }
    return "";
}

}  // namespace scopf
