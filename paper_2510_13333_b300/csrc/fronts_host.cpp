// Frontal structure of the multifrontal LDL^T, built once from the symbolic
// analysis of every block: front row lists, parent/child links, the
// child-to-parent index maps of the extend-add, the scatter map of the
// original KKT entries into the fronts, tree levels and the task order.
#include <algorithm>
#include <numeric>

#include "fronts_host.h"

namespace scopf {

std::string build_fronts(const Model &M, const std::vector<BlockSymbolic> &syms, HostFronts &H) {
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
    // levels (children have smaller task ids within a block: postorder)
    std::vector<int> level(nt, 0);
    for (int t = 0; t < nt; t++)
        if (sn[t].parent_task >= 0)
            level[sn[t].parent_task] = std::max(level[sn[t].parent_task], level[t] + 1);
    // large fronts (f > kBigFront) and everything above them form the second
    // factorization phase (one CTA per front); the rest is one warp per front
    const int kBigFront = 64;
    std::vector<char> big(nt, 0);
    for (int t = 0; t < nt; t++)
        if (sn[t].f > kBigFront || sn[t].border) big[t] = 1;
    for (int t = 0; t < nt; t++)   // children precede parents within a block
        if (big[t] && sn[t].parent_task >= 0) big[sn[t].parent_task] = 1;
    // task order: (phase, level, block, local)
    std::vector<int> order(nt);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (big[a] != big[b]) return big[a] < big[b];
        if (level[a] != level[b]) return level[a] < level[b];
        if (sn[a].block != sn[b].block) return sn[a].block < sn[b].block;
        return sn[a].local < sn[b].local;
    });
    std::vector<int> tid(nt);
    for (int i = 0; i < nt; i++) tid[order[i]] = i;
    H.n_tasks = nt;
    H.n_small = 0;
    for (int t = 0; t < nt; t++) H.n_small += big[t] ? 0 : 1;
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
    // children lists in task order, relative maps
    std::vector<std::vector<int>> ch(nt);
    for (int i = 0; i < nt; i++)
        if (H.parent[i] >= 0) ch[H.parent[i]].push_back(i);
    H.child_ptr.assign(nt + 1, 0);
    for (int i = 0; i < nt; i++) {
        H.child_ptr[i + 1] = H.child_ptr[i] + (int)ch[i].size();
        for (int c : ch[i]) H.child.push_back(c);
    }
    // ready-queue seeds.  Factorization: phase 1 (small fronts) starts from
    // its leaves; phase 2 counts only its own children (the small ones are
    // complete when it starts).  Forward solve: all leaves.  Backward solve:
    // the non-border tasks whose parent is a border front (the block roots).
    H.nchild.assign(nt, 0);
    H.pend_factor.assign(nt, 0);
    for (int i = 0; i < nt; i++) {
        H.nchild[i] = (int)ch[i].size();
        for (int c : ch[i])
            if (!(i >= H.n_small && c < H.n_small)) H.pend_factor[i]++;
    }
    for (int i = 0; i < nt; i++) {
        if (H.nchild[i] == 0) H.init_fwd.push_back(i);
        if (i < H.n_small && H.pend_factor[i] == 0) H.init_small.push_back(i);
        if (i >= H.n_small && H.pend_factor[i] == 0) H.init_big.push_back(i);
        if (!H.is_border[i] && (H.parent[i] < 0 || H.is_border[H.parent[i]])) H.init_bwd.push_back(i);
    }
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
    return "";
}

}  // namespace scopf
