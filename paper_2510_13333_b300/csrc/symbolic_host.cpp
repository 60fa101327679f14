// Symbolic analysis of one block of the KKT matrix of eq. (newtonsystem).
//
// The pivot-free LDL^T that the NCL regularisation permits (Section IV-B)
// has a structure fixed once per instance.  The ordering is specified
// exactly so that it can be reproduced bit for bit:
//  1. node graph: each bus, limited branch, generator and Delta^k is one
//     node holding its primal and dual rows; the first-stage variables u0
//     are "border" nodes (p_g^0 per generator, v_b^0 per PV bus);
//  2. exact minimum degree on the elimination graph, ties to the smallest
//     node id, border nodes never eliminated (they are ordered last);
//  3. node elimination tree (parent = earliest-eliminated neighbour);
//  4. postorder, children in increasing node id;
//  5. supernodes: an only child directly below its parent joins the
//     parent's supernode while it has fewer than relax_max_nodes nodes;
//  6. rows: nodes in postorder (node rows in their fixed order), then border.
// Dual-first order (the condensed primal variant): every block node is split
// into its primal part (rows of w) and its dual part (equality and
// complementarity rows), each keeping its rows' order; ids: primal parts in
// node order, then dual parts in node order (empty parts dropped), then the
// border.  Minimum degree eliminates every dual node before any primal node
// (key: dual first, degree, id).  The -C block is diagonal, so the dual nodes
// are independent, and eliminating them leaves the pattern of A + B' C^-1 B.
#include <algorithm>
#include <functional>
#include <queue>
#include <set>
#include <tuple>
#include <unordered_map>

#include "internal.h"

namespace scopf {

std::string symbolic_block(const Model &M, int k, int relax_max_nodes, int relax_max_front,
                           bool dual_first, BlockSymbolic &S) {
    const Block &B = M.blocks[k];
    const int nb = M.nb, ng = M.ng, npv = (int)M.pv.size();
    auto Kw = [&](int64_t local) { return B.kkt0 + local; };
    auto Kc = [&](int64_t local) { return B.kkt0 + B.nvar + local; };
    auto Kp = [&](int64_t local) { return B.kkt0 + B.nvar + B.nrow + local; };
    std::vector<std::vector<int64_t>> &rows = S.node_rows;
    rows.clear();
    for (int b = 0; b < nb; b++) {
        std::vector<int64_t> r;
        if (B.th[b] >= 0) r.push_back(Kw(B.th[b]));
        if (B.v[b] >= 0) r.push_back(Kw(B.v[b]));
        r.push_back(Kc(B.rP[b]));
        r.push_back(Kc(B.rQ[b]));
        rows.push_back(r);
    }
    for (size_t j = 0; j < B.thermal.size(); j++)
        rows.push_back({Kw(B.sth[2 * j]), Kw(B.sth[2 * j + 1]), Kc(B.rth[2 * j]), Kc(B.rth[2 * j + 1])});
    const int ngk = k > 0 ? (int)B.gens.size() : 0;
    const int nsw = k > 0 ? (int)B.sw_bus.size() : 0;
    for (size_t i = 0; i < B.gens.size(); i++) {
        int gi = B.gens[i];
        if (k == 0) {
            rows.push_back({Kw(B.q[gi])});
            continue;
        }
        int si = B.sw_of_gen[gi];
        std::vector<int64_t> r = {Kw(B.p[gi]), Kw(B.q[gi]), Kw(B.pim[i]), Kw(B.pip[i]),
                                  Kw(B.spu[i]), Kw(B.spl[i])};
        if (si >= 0) {
            r.push_back(Kw(B.num[si]));
            r.push_back(Kw(B.nup[si]));
            r.push_back(Kw(B.squ[si]));
            r.push_back(Kw(B.sql[si]));
        }
        r.push_back(Kc(B.rdroop[i]));
        r.push_back(Kc(B.rspu[i]));
        r.push_back(Kc(B.rspl[i]));
        if (si >= 0) {
            r.push_back(Kc(B.rpvpq[si]));
            r.push_back(Kc(B.rsqu[si]));
            r.push_back(Kc(B.rsql[si]));
        }
        r.push_back(Kp(i));
        r.push_back(Kp(ngk + i));
        if (si >= 0) {
            r.push_back(Kp(2 * ngk + si));
            r.push_back(Kp(2 * ngk + nsw + si));
        }
        rows.push_back(r);
    }
    if (k > 0) rows.push_back({Kw(B.delta)});
    int dual_from = -1;   // dual-first: block nodes [dual_from, n_block) are dual parts
    if (dual_first) {
        const int64_t w_end = B.kkt0 + B.nvar;   // rows below are the block's w
        std::vector<std::vector<int64_t>> prim, dual;
        for (const auto &r : rows) {
            std::vector<int64_t> a, b;
            for (int64_t x : r) (x < w_end ? a : b).push_back(x);
            if (!a.empty()) prim.push_back(a);
            if (!b.empty()) dual.push_back(b);
        }
        rows = prim;
        dual_from = (int)rows.size();
        rows.insert(rows.end(), dual.begin(), dual.end());
    }
    const int n_block = (int)rows.size();
    for (int gi = 0; gi < ng; gi++) rows.push_back({M.kkt_border0 + gi});
    for (int q = 0; q < npv; q++) rows.push_back({M.kkt_border0 + ng + q});
    const int n_nodes = (int)rows.size();
    S.n_nodes = n_nodes;
    S.n_block_nodes = n_block;

    // node of every KKT row touched by this block
    std::unordered_map<int64_t, int> node_of;
    node_of.reserve((size_t)B.nkkt() * 2 + 1024);
    for (int v = 0; v < n_nodes; v++)
        for (int64_t x : rows[v]) node_of[x] = v;
    std::vector<std::set<int>> A(n_nodes);
    for (int v = 0; v < n_block; v++)
        for (int64_t x : rows[v])
            for (int64_t p = M.kkt_ptr[x]; p < M.kkt_ptr[x + 1]; p++) {
                auto it = node_of.find(M.kkt_col[p]);
                if (it == node_of.end()) continue;
                int u = it->second;
                if (u == v) continue;
                A[v].insert(u);
                A[u].insert(v);
            }

    // exact minimum degree (ties: smallest id); border nodes never eliminated;
    // dual-first: dual nodes before all others
    using QE = std::tuple<int, int, int>;   // (class, degree, id)
    auto cls = [&](int v) { return dual_from >= 0 && v >= dual_from ? 0 : 1; };
    std::priority_queue<QE, std::vector<QE>, std::greater<QE>> heap;
    for (int v = 0; v < n_block; v++) heap.push({cls(v), (int)A[v].size(), v});
    std::vector<char> alive(n_nodes, 1);
    std::vector<int> order;
    std::vector<std::set<int>> st(n_nodes);
    while (!heap.empty()) {
        QE top = heap.top();
        heap.pop();
        const int v = std::get<2>(top);
        if (!alive[v] || std::get<1>(top) != (int)A[v].size()) continue;
        alive[v] = 0;
        order.push_back(v);
        std::set<int> nbv = A[v];
        st[v] = nbv;
        for (int u : nbv) {
            A[u].insert(nbv.begin(), nbv.end());
            A[u].erase(u);
            A[u].erase(v);
            if (u < n_block) heap.push({cls(u), (int)A[u].size(), u});
        }
        A[v].clear();
    }
    if ((int)order.size() != n_block) return "internal: minimum degree incomplete";
    std::vector<int> pos(n_nodes, -1);
    for (int i = 0; i < n_block; i++) pos[order[i]] = i;
    S.node_parent.assign(n_block, -1);
    for (int v : order) {
        int best = -1;
        bool any = false;
        for (int u : st[v]) {
            any = true;
            if (u < n_block && (best < 0 || pos[u] < pos[best])) best = u;
        }
        S.node_parent[v] = best >= 0 ? best : (any ? -2 : -1);
    }
    // postorder, children in increasing id
    std::vector<std::vector<int>> children(n_block);
    std::vector<int> roots;
    for (int v = 0; v < n_block; v++) {
        if (S.node_parent[v] >= 0)
            children[S.node_parent[v]].push_back(v);
        else
            roots.push_back(v);
    }
    S.post.clear();
    for (int r0 : roots) {
        std::vector<std::pair<int, int>> stack = {{r0, 0}};
        while (!stack.empty()) {
            auto [v, i] = stack.back();
            stack.pop_back();
            if (i < (int)children[v].size()) {
                stack.push_back({v, i + 1});
                stack.push_back({children[v][i], 0});
            } else {
                S.post.push_back(v);
            }
        }
    }
    if ((int)S.post.size() != n_block) return "internal: postorder incomplete";
    std::vector<int> ppos(n_nodes, -1);
    for (int i = 0; i < n_block; i++) ppos[S.post[i]] = i;
    for (int v = n_block; v < n_nodes; v++) ppos[v] = v;  // border: after all block nodes
    // supernodes
    S.sn_start.assign(1, 0);
    int size = 1;
    for (int i = 1; i < n_block; i++) {
        int v = S.post[i], u = S.post[i - 1];
        bool chain = S.node_parent[u] == v && children[v].size() == 1;
        if (chain && size < relax_max_nodes) {
            size++;
        } else {
            S.sn_start.push_back(i);
            size = 1;
        }
    }
    S.sn_start.push_back(n_block);
    // update nodes (union of member structures minus members, by position,
    // border nodes last) and parent supernode (-2 = border) of every supernode
    auto link = [&]() {
        const int nsn = (int)S.sn_start.size() - 1;
        std::vector<int> sn_of(n_block);
        for (int s = 0; s < nsn; s++)
            for (int i = S.sn_start[s]; i < S.sn_start[s + 1]; i++) sn_of[i] = s;
        S.sn_update_nodes.assign(nsn, {});
        S.sn_parent.assign(nsn, -1);
        for (int s = 0; s < nsn; s++) {
            std::set<int> mem, u;
            for (int i = S.sn_start[s]; i < S.sn_start[s + 1]; i++) mem.insert(S.post[i]);
            for (int v : mem)
                for (int x : st[v])
                    if (!mem.count(x)) u.insert(x);
            std::vector<int> ul(u.begin(), u.end());
            std::sort(ul.begin(), ul.end(), [&](int a, int b) { return ppos[a] < ppos[b]; });
            S.sn_update_nodes[s] = ul;
            int first_block = -1;
            for (int x : ul)
                if (x < n_block) {
                    first_block = x;
                    break;
                }
            if (first_block >= 0)
                S.sn_parent[s] = sn_of[ppos[first_block]];
            else if (!ul.empty())
                S.sn_parent[s] = -2;
        }
    };
    link();
    if (relax_max_front > 0) {
        // relaxed amalgamation bounded by the front size: a supernode absorbs
        // a direct child c (children in increasing index) while its front
        // stays within relax_max_front rows after adding c's pivot rows; the
        // final supernode tree is postordered (roots and children in
        // increasing index), each supernode listing its absorbed children's
        // nodes (recursively, in order) before its own
        const int nsn = (int)S.sn_start.size() - 1;
        std::vector<std::vector<int>> members(nsn), kids(nsn), absorbed(nsn), tree_kids(nsn);
        std::vector<int> npiv(nsn, 0), front(nsn, 0), into(nsn, -1), rep(nsn);
        for (int s = 0; s < nsn; s++) {
            for (int i = S.sn_start[s]; i < S.sn_start[s + 1]; i++) {
                members[s].push_back(S.post[i]);
                npiv[s] += (int)rows[S.post[i]].size();
            }
            front[s] = npiv[s];
            for (int u : S.sn_update_nodes[s]) front[s] += (int)rows[u].size();
            if (S.sn_parent[s] >= 0) kids[S.sn_parent[s]].push_back(s);
        }
        for (int s = 0; s < nsn; s++)
            for (int c : kids[s])
                if (front[s] + npiv[c] <= relax_max_front) {
                    absorbed[s].push_back(c);
                    into[c] = s;
                    front[s] += npiv[c];
                    npiv[s] += npiv[c];
                }
        for (int s = nsn - 1; s >= 0; s--) rep[s] = into[s] >= 0 ? rep[into[s]] : s;
        std::vector<int> sroots;
        for (int s = 0; s < nsn; s++) {
            if (into[s] >= 0) continue;
            if (S.sn_parent[s] >= 0)
                tree_kids[rep[S.sn_parent[s]]].push_back(s);
            else
                sroots.push_back(s);
        }
        std::vector<int> order;
        for (int r0 : sroots) {
            std::vector<std::pair<int, int>> stack = {{r0, 0}};
            while (!stack.empty()) {
                auto [v, i] = stack.back();
                stack.pop_back();
                if (i < (int)tree_kids[v].size()) {
                    stack.push_back({v, i + 1});
                    stack.push_back({tree_kids[v][i], 0});
                } else {
                    order.push_back(v);
                }
            }
        }
        std::function<void(int, std::vector<int> &)> expand = [&](int s, std::vector<int> &out) {
            for (int c : absorbed[s]) expand(c, out);
            out.insert(out.end(), members[s].begin(), members[s].end());
        };
        std::vector<int> post;
        S.sn_start.assign(1, 0);
        for (int s : order) {
            expand(s, post);
            S.sn_start.push_back((int)post.size());
        }
        if ((int)post.size() != n_block) return "internal: relaxed supernodes lost nodes";
        S.post = post;
        for (int i = 0; i < n_block; i++) ppos[S.post[i]] = i;
        link();
    }
    S.rows.clear();
    for (int v : S.post) S.rows.insert(S.rows.end(), rows[v].begin(), rows[v].end());
    S.n_block_rows = (int64_t)S.rows.size();
    for (int v = n_block; v < n_nodes; v++) S.rows.insert(S.rows.end(), rows[v].begin(), rows[v].end());
    return "";
}

}  // namespace scopf
