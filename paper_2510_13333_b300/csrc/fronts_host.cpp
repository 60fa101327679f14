// Frontal structure of the multifrontal LDL^T, built once from the symbolic
// analysis of every block: front row lists, parent/child links, the
// child-to-parent index maps of the extend-add, the scatter map of the
// original KKT entries into the fronts, tree levels and the task order.
#include <algorithm>
#include <climits>
#include <numeric>

#include "fronts_host.h"

namespace scopf {

std::string build_fronts(const Model &M, const std::vector<BlockSymbolic> &syms, int cluster_cap,
                         HostFronts &H) {
    const int nblk = (int)M.blocks.size();
    const int nbor = (int)M.nborder;
    H = HostFronts();
    H.n_border = nbor;
    H.n_blocks = nblk;
    // elimination position of every KKT row inside its own block
    std::vector<int64_t> epos(M.n_kkt, -1);
    struct Sn {
        int block, local;
        int npiv, f, level;
        std::vector<int64_t> rows;   // KKT indices: pivot rows then update rows
        std::vector<int64_t> pos;    // elimination positions (sorted)
        int parent_task = -1;
        bool border = false;
    };
    std::vector<Sn> sn;
    std::vector<std::vector<int>> blk_tasks(nblk);
    std::vector<int> border_task(nblk, -1);
    for (int k = 0; k < nblk; k++) {
        const BlockSymbolic &S = syms[k];
        for (int64_t i = 0; i < S.n_block_rows; i++) epos[S.rows[i]] = i;
        const int nsn = (int)S.sn_start.size() - 1;
        std::vector<int64_t> node_first(S.n_nodes, -1);
        {
            int64_t acc = 0;
            for (int v : S.post) {
                node_first[v] = acc;
                acc += (int64_t)S.node_rows[v].size();
            }
        }
        int base = (int)sn.size();
        for (int s = 0; s < nsn; s++) {
            Sn x;
            x.block = k;
            x.local = s;
            for (int i = S.sn_start[s]; i < S.sn_start[s + 1]; i++) {
                int v = S.post[i];
                for (size_t q = 0; q < S.node_rows[v].size(); q++) {
                    x.rows.push_back(S.node_rows[v][q]);
                    x.pos.push_back(node_first[v] + (int64_t)q);
                }
            }
            x.npiv = (int)x.rows.size();
            for (int u : S.sn_update_nodes[s]) {
                if (u < S.n_block_nodes) {
                    for (size_t q = 0; q < S.node_rows[u].size(); q++) {
                        x.rows.push_back(S.node_rows[u][q]);
                        x.pos.push_back(node_first[u] + (int64_t)q);
                    }
                } else {
                    int64_t bi = S.node_rows[u][0] - M.kkt_border0;
                    x.rows.push_back(S.node_rows[u][0]);
                    x.pos.push_back(S.n_block_rows + bi);
                }
            }
            x.f = (int)x.rows.size();
            for (size_t q = 1; q < x.pos.size(); q++)
                if (x.pos[q] <= x.pos[q - 1]) return "internal: front rows not sorted";
            sn.push_back(std::move(x));
            blk_tasks[k].push_back(base + s);
        }
        Sn bt;
        bt.block = k;
        bt.local = nsn;
        bt.border = true;
        bt.npiv = 0;
        bt.f = nbor;
        for (int j = 0; j < nbor; j++) {
            bt.rows.push_back(M.kkt_border0 + j);
            bt.pos.push_back(S.n_block_rows + j);
        }
        border_task[k] = (int)sn.size();
        sn.push_back(std::move(bt));
        for (int s = 0; s < nsn; s++) {
            int ps = S.sn_parent[s];
            sn[base + s].parent_task = ps >= 0 ? base + ps : border_task[k];
        }
    }
    const int nt = (int)sn.size();
    // Factorization phases, each closed upwards (a front's ancestors are in
    // its phase or a later one): 2 = large fronts (f > 64, and the border
    // fronts) and their ancestors, one CTA per front; 1 = medium fronts
    // (32 < f <= 64) and their ancestors, one warp with a 64-row shared
    // front each; 0 = the rest (tile-sized fronts with tile-sized subtrees),
    // one warp with a 32-row shared tile each.
    std::vector<char> phase(nt, 0);
    for (int t = 0; t < nt; t++)
        phase[t] = (sn[t].f > 64 || sn[t].border) ? 2 : (sn[t].f > 32 ? 1 : 0);
    for (int t = 0; t < nt; t++) {   // children precede parents within a block
        const int p = sn[t].parent_task;
        if (p >= 0) phase[p] = std::max(phase[p], phase[t]);
    }
    std::vector<char> big(nt, 0);
    for (int t = 0; t < nt; t++) big[t] = phase[t] != 0;
    // Work items.  A maximal subtree of at most `cluster_cap` small fronts is
    // one item (a warp runs it in postorder with no scheduling in between);
    // the small fronts above such subtrees and every large front are items of
    // their own.  Small fronts have only small descendants, and a subtree
    // occupies the contiguous postorder range that ends at its root.
    // Only fronts of at most 32 rows (one warp tile) join subtrees: a larger
    // front costs as much as a whole small subtree, and a subtree runs
    // sequentially.
    std::vector<int> sz(nt, 1);
    std::vector<char> clus(nt, 0);   // the whole subtree is tile-sized
    for (int t = 0; t < nt; t++) clus[t] = !big[t] && sn[t].f <= 32;
    for (int t = 0; t < nt; t++) {
        const int p = sn[t].parent_task;
        if (p < 0) continue;
        if (!clus[t]) clus[p] = 0;
        if (!big[t] && !big[p]) sz[p] += sz[t];
    }
    std::vector<int> item_root(nt, -1);   // root task of each task's item
    for (int t = nt - 1; t >= 0; t--) {
        const int p = sn[t].parent_task;
        if (!clus[t] || sz[t] > cluster_cap)
            item_root[t] = t;
        else if (p >= 0 && clus[p] && sz[p] <= cluster_cap)
            item_root[t] = item_root[p];
        else
            item_root[t] = t;
    }
    // item heights (clusters and leaves 0) order the items: (phase, height,
    // block, root); tasks of an item follow in postorder
    std::vector<int> level(nt, 0);
    for (int t = 0; t < nt; t++) {
        const int p = sn[t].parent_task;
        if (item_root[t] == t && p >= 0)
            level[item_root[p]] = std::max(level[item_root[p]], level[t] + 1);
    }
    std::vector<int> order(nt);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const int ra = item_root[a], rb = item_root[b];
        if (phase[ra] != phase[rb]) return phase[ra] < phase[rb];
        if (level[ra] != level[rb]) return level[ra] < level[rb];
        if (sn[ra].block != sn[rb].block) return sn[ra].block < sn[rb].block;
        if (ra != rb) return ra < rb;
        return a < b;
    });
    for (int t = 0; t < nt; t++) level[t] = level[item_root[t]];
    std::vector<int> tid(nt);
    for (int i = 0; i < nt; i++) tid[order[i]] = i;
    H.n_tasks = nt;
    H.n_small = 0;
    for (int t = 0; t < nt; t++) H.n_small += big[t] ? 0 : 1;
    // items as contiguous task ranges
    H.item_ptr.clear();
    H.item_of_task.assign(nt, 0);
    for (int i = 0; i < nt; i++) {
        if (i == 0 || item_root[order[i]] != item_root[order[i - 1]]) H.item_ptr.push_back(i);
        H.item_of_task[i] = (int32_t)H.item_ptr.size() - 1;
    }
    H.item_ptr.push_back(nt);
    H.n_items = (int)H.item_ptr.size() - 1;
    H.n_items_small = H.n_small > 0 ? H.item_of_task[H.n_small - 1] + 1 : 0;
    {
        int n_med = 0;   // tasks of phases 0 and 1
        for (int t = 0; t < nt; t++) n_med += phase[t] < 2 ? 1 : 0;
        H.n_items_med = n_med > 0 ? H.item_of_task[n_med - 1] + 1 : 0;
    }
    H.front_off.resize(nt);
    H.vec_off.resize(nt);
    H.f.resize(nt);
    H.npiv.resize(nt);
    H.parent.resize(nt);
    H.is_border.resize(nt);
    H.rows_off.resize(nt);
    H.level.resize(nt);
    H.block.resize(nt);
    int64_t foff = 0, voff = 0, roff = 0;
    for (int i = 0; i < nt; i++) {
        const Sn &x = sn[order[i]];
        H.f[i] = x.f;
        H.npiv[i] = x.npiv;
        H.parent[i] = x.parent_task >= 0 ? tid[x.parent_task] : -1;
        H.is_border[i] = x.border ? 1 : 0;
        H.front_off[i] = foff;
        H.vec_off[i] = voff;
        H.rows_off[i] = roff;
        H.level[i] = level[order[i]];
        H.block[i] = x.block;
        foff += (int64_t)x.f * x.f;
        voff += x.f;
        roff += x.f;
        H.rows.insert(H.rows.end(), x.rows.begin(), x.rows.end());
        if (!x.border) {
            for (int c = 0; c < x.npiv; c++) {
                int64_t mrem = x.f - c - 1;
                H.flops += (double)mrem * (mrem + 1) + (double)mrem;
                H.nnz_L += (int64_t)(x.f - c);
            }
        }
    }
    H.rows_off.push_back(roff);
    H.front_elems = foff;
    H.vec_elems = voff;
    H.border_off.assign(nblk, 0);
    H.border_vec_off.assign(nblk, 0);
    for (int k = 0; k < nblk; k++) {
        H.border_off[k] = H.front_off[tid[border_task[k]]];
        H.border_vec_off[k] = H.vec_off[tid[border_task[k]]];
    }
    for (int j = 0; j < nbor; j++) H.border_rows.push_back(M.kkt_border0 + j);
    // children lists, relative maps.  Children are listed in the block's
    // postorder (their supernode index), not in task order: the extend-add
    // sums children in list order, so the arithmetic, and with it every
    // result, does not depend on how tasks are grouped or scheduled.
    std::vector<std::vector<int>> ch(nt);
    for (int i = 0; i < nt; i++)
        if (H.parent[i] >= 0) ch[H.parent[i]].push_back(i);
    for (auto &c : ch)
        std::sort(c.begin(), c.end(), [&](int a, int b) { return order[a] < order[b]; });
    H.child_ptr.assign(nt + 1, 0);
    for (int i = 0; i < nt; i++) {
        H.child_ptr[i + 1] = H.child_ptr[i] + (int)ch[i].size();
        for (int c : ch[i]) H.child.push_back(c);
    }
    // Ready-queue seeds, on items.  Factorization: phase 1 (small items)
    // starts from its leaves; phase 2 (large fronts, one item each) counts
    // only its own children (the small ones are complete when it starts).
    // Forward solve: all leaf items.  Backward solve: the items whose parent
    // is a border front (block roots); a finished item pushes its child items.
    const int ni = H.n_items;
    H.item_parent.assign(ni, -1);
    H.item_is_border.assign(ni, 0);
    std::vector<std::vector<int>> ich(ni);
    for (int i = 0; i < ni; i++) {
        const int root = H.item_ptr[i + 1] - 1;
        const int pt = H.parent[root];
        H.item_is_border[i] = H.is_border[root];
        if (pt >= 0) {
            H.item_parent[i] = H.item_of_task[pt];
            ich[H.item_parent[i]].push_back(i);
        }
    }
    H.item_child_ptr.assign(ni + 1, 0);
    H.item_child.clear();
    H.nchild.assign(ni, 0);
    H.pend_factor.assign(ni, 0);
    auto item_phase = [&](int i) {
        return i < H.n_items_small ? 0 : (i < H.n_items_med ? 1 : 2);
    };
    for (int i = 0; i < ni; i++) {
        H.item_child_ptr[i + 1] = H.item_child_ptr[i] + (int)ich[i].size();
        for (int c : ich[i]) H.item_child.push_back(c);
        H.nchild[i] = (int)ich[i].size();
        for (int c : ich[i])
            if (item_phase(i) == item_phase(c)) H.pend_factor[i]++;
    }
    for (int i = 0; i < ni; i++) {
        if (H.nchild[i] == 0) H.init_fwd.push_back(i);
        if (H.pend_factor[i] == 0) {
            if (item_phase(i) == 0) H.init_small.push_back(i);
            if (item_phase(i) == 1) H.init_med.push_back(i);
            if (item_phase(i) == 2) H.init_big.push_back(i);
        }
        const int pi = H.item_parent[i];
        if (!H.item_is_border[i] && (pi < 0 || H.item_is_border[pi])) H.init_bwd.push_back(i);
    }
    // Critical path first.  Estimated item cost (a few microseconds per
    // front, more for wide ones); rank_up = cost of the path from the item
    // to its root (bottom-up sweeps seed the longest paths first), rank_dn
    // = the longest path below it (the backward sweep continues with the
    // child that has the longest one).
    std::vector<double> cost(ni, 0.0), rank_up(ni, 0.0), rank_dn(ni, 0.0);
    for (int i = 0; i < ni; i++)
        for (int t = H.item_ptr[i]; t < H.item_ptr[i + 1]; t++)
            cost[i] += 4.0 + H.f[t] / 16.0 + (double)H.npiv[t] * H.f[t] / 256.0;
    for (int i = ni - 1; i >= 0; i--)   // parents have larger ids
        rank_up[i] = cost[i] + (H.item_parent[i] >= 0 ? rank_up[H.item_parent[i]] : 0.0);
    for (int i = 0; i < ni; i++) {
        double best = 0.0;
        for (int c : ich[i]) best = std::max(best, rank_dn[c]);
        rank_dn[i] = cost[i] + best;
    }
    H.item_cont.assign(ni, -1);
    for (int i = 0; i < ni; i++) {
        double best = -1.0;
        for (int c : ich[i])
            if (rank_dn[c] > best) {
                best = rank_dn[c];
                H.item_cont[i] = c;
            }
    }
    auto by = [](const std::vector<double> &r) {
        return [&r](int a, int b) { return r[a] != r[b] ? r[a] > r[b] : a < b; };
    };
    std::stable_sort(H.init_small.begin(), H.init_small.end(), by(rank_up));
    std::stable_sort(H.init_med.begin(), H.init_med.end(), by(rank_up));
    std::stable_sort(H.init_big.begin(), H.init_big.end(), by(rank_up));
    std::stable_sort(H.init_fwd.begin(), H.init_fwd.end(), by(rank_up));
    std::stable_sort(H.init_bwd.begin(), H.init_bwd.end(), by(rank_dn));
    H.rel_off.assign(nt, 0);
    for (int i = 0; i < nt; i++) {
        H.rel_off[i] = (int64_t)H.rel.size();
        const Sn &x = sn[order[i]];
        if (H.parent[i] < 0) continue;
        const Sn &p = sn[order[H.parent[i]]];
        for (int q = x.npiv; q < x.f; q++) {
            auto it = std::lower_bound(p.pos.begin(), p.pos.end(), x.pos[q]);
            if (it == p.pos.end() || *it != x.pos[q]) return "internal: update row not in parent front";
            H.rel.push_back((int32_t)(it - p.pos.begin()));
        }
    }
    // owner supernode (task) and pivot position of each block row
    std::vector<int32_t> owner(M.n_kkt, -1);
    for (int i = 0; i < nt; i++) {
        const Sn &x = sn[order[i]];
        if (x.border) continue;
        for (int c = 0; c < x.npiv; c++) owner[x.rows[c]] = i;
    }
    // scatter map of the original entries (lower triangle in elimination order)
    H.scatter.assign(M.kkt_col.size(), -1);
    for (int64_t i = 0; i < M.n_kkt; i++) {
        const bool ib = i >= M.kkt_border0;
        for (int64_t q = M.kkt_ptr[i]; q < M.kkt_ptr[i + 1]; q++) {
            const int64_t j = M.kkt_col[q];
            const bool jb = j >= M.kkt_border0;
            if (ib && jb) {
                // K_cc: block 0's border front
                int64_t bi = i - M.kkt_border0, bj = j - M.kkt_border0;
                if (bi >= bj) H.scatter[q] = H.border_off[0] + bj * nbor + bi;
                continue;
            }
            if (jb) continue;  // block row, border column: upper triangle
            // column j is a block row; row i is a block row of the same block or a border row
            const int t = owner[j];
            if (t < 0) return "internal: KKT row without owner";
            const Sn &x = sn[order[t]];
            const int64_t pj = epos[j];
            const int64_t pi = ib ? (int64_t)syms[x.block].n_block_rows + (i - M.kkt_border0) : epos[i];
            if (!ib && M.block_of_kkt[i] != x.block) return "internal: cross-block KKT entry";
            if (pi < pj) continue;
            auto itc = std::lower_bound(x.pos.begin(), x.pos.end(), pj);
            auto itr = std::lower_bound(x.pos.begin(), x.pos.end(), pi);
            if (itr == x.pos.end() || *itr != pi) return "internal: entry row not in front";
            const int64_t lc = itc - x.pos.begin(), lr = itr - x.pos.begin();
            H.scatter[q] = H.front_off[t] + lc * x.f + lr;
        }
    }
    // per-task lists of original entries (offset inside the task's front)
    {
        std::vector<int> task_of_front_start(0);
        std::vector<std::vector<std::pair<int64_t, int32_t>>> per(nt);
        for (size_t q = 0; q < H.scatter.size(); q++) {
            const int64_t off = H.scatter[q];
            if (off < 0) continue;
            // the front containing off: last task whose front_off <= off
            const int t = (int)(std::upper_bound(H.front_off.begin(), H.front_off.end(), off) -
                                H.front_off.begin()) - 1;
            per[t].push_back({(int64_t)q, (int32_t)(off - H.front_off[t])});
        }
        H.orig_ptr.assign(nt + 1, 0);
        for (int t = 0; t < nt; t++) {
            H.orig_ptr[t + 1] = H.orig_ptr[t] + (int64_t)per[t].size();
            for (auto &pr : per[t]) {
                H.orig_nz.push_back(pr.first);
                H.orig_off.push_back(pr.second);
            }
        }
    }
    H.max_level = 0;
    for (int i = 0; i < nt; i++) H.max_level = std::max(H.max_level, H.level[i]);
    // packed per-task and per-child records: one or two 16-byte loads give
    // everything a front needs to start
    if (H.orig_ptr[nt] >= (int64_t)INT32_MAX || (int64_t)H.rel.size() >= (int64_t)INT32_MAX)
        return "frontal structure too large for 32-bit record fields";
    auto lo = [](int64_t v) { return (int32_t)(uint32_t)(uint64_t)v; };
    auto hi = [](int64_t v) { return (int32_t)(uint32_t)((uint64_t)v >> 32); };
    H.task_rec.assign(8 * (size_t)(nt + 1), 0);
    for (int t = 0; t <= nt; t++) {
        int32_t *r = &H.task_rec[8 * (size_t)t];
        if (t < nt) {
            r[0] = lo(H.front_off[t]);
            r[1] = hi(H.front_off[t]);
            r[2] = lo(H.vec_off[t]);
            r[3] = hi(H.vec_off[t]);
            r[4] = H.f[t] | (H.npiv[t] << 16);
            r[7] = H.parent[t];
        } else {
            r[7] = -1;
        }
        r[5] = H.child_ptr[t];
        r[6] = (int32_t)H.orig_ptr[t];
    }
    H.vpos_of_row.assign(M.n_kkt, -1);
    for (int t = 0; t < nt; t++)
        for (int i = 0; i < H.npiv[t]; i++) H.vpos_of_row[H.rows[H.vec_off[t] + i]] = H.vec_off[t] + i;
    H.child_rec.assign(8 * H.child.size(), 0);
    for (size_t q = 0; q < H.child.size(); q++) {
        const int c = H.child[q];
        int32_t *r = &H.child_rec[8 * q];
        r[0] = lo(H.front_off[c]);
        r[1] = hi(H.front_off[c]);
        r[2] = lo(H.vec_off[c]);
        r[3] = hi(H.vec_off[c]);
        r[4] = (int32_t)H.rel_off[c];
        r[5] = H.f[c] | (H.npiv[c] << 16);
        r[6] = c;
    }
    return "";
}

}  // namespace scopf
