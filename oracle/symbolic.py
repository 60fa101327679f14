"""Symbolic analysis of the block-arrow KKT matrix (oracle).

The pivot-free factorisation of eq. (newtonsystem) (Section IV-B) allows the
whole symbolic analysis to be done once per structure.  The paper leaves the
ordering to cuDSS; here one deterministic algorithm is fixed, implemented
twice (here and in the CUDA library) and compared bit for bit:

1. Each scenario block is compressed to a *node graph* whose nodes keep the
   primal and dual rows of one physical element together:
     bus b      : theta_b (b != ref), v_b (if a variable of the block), Pbal_b, Qbal_b
     branch l   : (limited branches only) sigma_f, sigma_t, therm_f, therm_t
     generator g: base: q_g; contingency: p, q, pi_-, pi_+, sig_pmax, sig_pmin,
                  [nu_-, nu_+, sig_qmax, sig_qmin], droop, sig_pmax-row,
                  sig_pmin-row, [pvpq, sig_qmax-row, sig_qmin-row],
                  comp(pi_-), comp(pi_+), [comp(nu_-), comp(nu_+)]
                  (bracketed rows only for switch-set buses)
     Delta      : Delta^k (contingencies)
     border     : p_g^0 (every generator), v_b^0 (every PV bus) -- the
                  first-stage variables u0 = (p_g^0, v_PV^0) of Section II-B.
   Node ids: buses, then limited in-service branches, then in-service
   generators, then Delta, then border nodes (p^0 by generator, v^0 by PV bus).
   Two nodes are adjacent when a nonzero of the block's KKT matrix couples
   one of their rows.
2. Exact minimum degree on the elimination graph: repeatedly eliminate the
   non-border node of smallest current degree (ties: smallest node id); its
   neighbours become a clique.  Border nodes are never chosen: they come last.
3. Node elimination tree: parent(p) = the neighbour of p at its elimination
   with the earliest elimination position.  All border nodes form one final
   "border" supernode whose front collects the Schur-complement contribution.
4. Postorder of the tree (children visited in increasing node id).
5. Fundamental supernodes, then relaxed amalgamation of only-child chains
   while the merged supernode has at most ``relax_max_nodes`` nodes.
6. Relaxed amalgamation bounded by front size: supernodes in postorder
   (children first); each considers its children in increasing supernode
   index and absorbs child c when its front (pivot rows plus update rows)
   would stay within ``relax_max_front`` rows after adding c's pivot rows.
   c's update rows lie inside the parent's front, so the merged front is the
   parent's front plus c's pivot rows, and explicit zeros fill the rest of
   c's columns.  Only direct children are candidates: a grandchild that did
   not fit its own parent cannot fit the larger merged front.  The merged
   supernode eliminates its absorbed children (in increasing index, each in
   its own member order) and then its own nodes.
7. Postorder of the final supernode tree (roots and children in increasing
   supernode index); the node order is each supernode's member list in turn.
   Reordering independent subtrees changes no fill.
8. Rows: nodes in that order, each node's rows in the order of step 1, then
   the border rows.

Dual-first order (``dual_first=True``: the condensed primal variant).  Every
block node is split into its primal part (rows of w) and its dual part
(equality and complementarity rows), keeping the row order of step 1 within
each part.  Node ids: the primal parts in the original node order, then the
dual parts in the original node order (empty parts dropped), then the border
nodes.  Step 2 eliminates every dual node before any primal node (key: dual
before primal, then current degree, then node id).  The -C block of eq.
(newtonsystem) is diagonal, so dual nodes are never adjacent: eliminating
them all first leaves on the primal nodes exactly the pattern of the
condensed matrix A + B' C^-1 B, which the rest of the elimination factors
with positive pivots when it is positive definite ("signed Cholesky",
Section IV-B).  Steps 3-8 are unchanged.

Parity: integer, compared exactly with the CUDA implementation; pinned by
brute-force dense boolean elimination (fill and tree) and hand-checked
minimum-degree orders on path and grid graphs in the tests.
"""
from __future__ import annotations

import heapq

import numpy as np


class BlockGraph:
    """Node graph of one scenario block with the generic KKT rows of each node."""

    def __init__(self, node_rows, adj, n_block_nodes, dual_from=None):
        self.node_rows = node_rows          # list of arrays (generic KKT indices)
        self.adj = adj                      # list of sets of node ids
        self.n_block = n_block_nodes        # nodes [0, n_block) are eliminable
        self.n_nodes = len(node_rows)
        self.dual_from = dual_from          # dual-first order: nodes [dual_from, n_block) are dual


def block_graphs(model, dual_first: bool = False):
    """Build the node graph of every block of a ``SCOPFModel`` (with
    ``dual_first``, every block node split into its primal and dual parts)."""
    M = model
    n, m = M.n, M.m
    out = []
    for blk in M.blocks:
        rows = []
        # ---- bus nodes
        for b in range(M.nb):
            r = []
            if blk.th[b] >= 0:
                r.append(blk.gth[b])
            if blk.v[b] >= 0:
                r.append(blk.gv[b])
            r += [n + blk.grP[b], n + blk.grQ[b]]
            rows.append(r)
        # ---- limited branch nodes
        for j, l in enumerate(blk.thermal):
            rows.append([blk.gsth[j, 0], blk.gsth[j, 1], n + blk.grth[j, 0], n + blk.grth[j, 1]])
        # ---- generator nodes
        ngk = len(blk.gens) if blk.k > 0 else 0
        nsw = len(blk.switch) if blk.k > 0 else 0
        sw_of_gen = {int(g): si for si, g in enumerate(blk.sw_gen)} if blk.k > 0 else {}
        for gi, g in enumerate(blk.gens):
            if blk.k == 0:
                rows.append([blk.gq[g]])
                continue
            r = [blk.gp[g], blk.gq[g], blk.gpim[gi], blk.gpip[gi], blk.gspu[gi], blk.gspl[gi]]
            si = sw_of_gen.get(int(g), -1)
            if si >= 0:
                r += [blk.gnum[si], blk.gnup[si], blk.gsqu[si], blk.gsql[si]]
            r += [n + blk.grdroop[gi], n + blk.grspu[gi], n + blk.grspl[gi]]
            if si >= 0:
                r += [n + blk.grpvpq[si], n + blk.grsqu[si], n + blk.grsql[si]]
            base = n + m + blk.p0
            r += [base + gi, base + ngk + gi]
            if si >= 0:
                r += [base + 2 * ngk + si, base + 2 * ngk + nsw + si]
            rows.append(r)
        if blk.k > 0:
            rows.append([blk.gdelta])
        dual_from = None
        if dual_first:
            prim = [[x for x in r if x < n] for r in rows]
            dual = [[x for x in r if x >= n] for r in rows]
            rows = [r for r in prim if r]
            dual_from = len(rows)
            rows += [r for r in dual if r]
        n_block = len(rows)
        for g in range(M.ng):
            rows.append([M.border0 + g])
        for q in range(M.npv):
            rows.append([M.border0 + M.ng + q])
        out.append(BlockGraph([np.asarray(r, dtype=np.int64) for r in rows], None, n_block,
                              dual_from))
    return out


def attach_adjacency(graphs, K):
    """Node adjacency from the pattern of the reduced KKT matrix ``K`` (generic order)."""
    import scipy.sparse as sp
    Kc = sp.csr_matrix(K)
    owner_blk = np.full(Kc.shape[0], -1, dtype=np.int64)
    for gi, G in enumerate(graphs):
        node_of = {}
        for nid, r in enumerate(G.node_rows):
            for x in r.tolist():
                node_of[x] = nid
        G.node_of = node_of
    for gi, G in enumerate(graphs):
        adj = [set() for _ in range(G.n_nodes)]
        for nid in range(G.n_block):
            for x in G.node_rows[nid].tolist():
                for y in Kc.indices[Kc.indptr[x]:Kc.indptr[x + 1]].tolist():
                    other = G.node_of.get(y, -1)
                    if other >= 0 and other != nid:
                        adj[nid].add(other)
                        adj[other].add(nid)
        G.adj = adj
    return graphs


def min_degree(adj, n_block, dual_from=None):
    """Exact minimum degree with smallest-id tie-break; nodes >= n_block are
    never eliminated; with ``dual_from`` the nodes [dual_from, n_block) are
    all eliminated before the others.  Returns (order, struct) where
    struct[p] is the set of neighbours of p when it was eliminated."""
    n = len(adj)
    A = [set(a) for a in adj]
    cls = [0 if dual_from is not None and v >= dual_from else 1 for v in range(n)]
    heap = [(cls[v], len(A[v]), v) for v in range(n_block)]
    heapq.heapify(heap)
    alive = [True] * n
    order = []
    struct = [None] * n
    while heap:
        _, d, v = heapq.heappop(heap)
        if not alive[v] or d != len(A[v]):
            continue
        alive[v] = False
        order.append(v)
        nb = A[v]
        struct[v] = set(nb)
        for u in nb:
            A[u] |= nb
            A[u].discard(u)
            A[u].discard(v)
            if u < n_block:
                heapq.heappush(heap, (cls[u], len(A[u]), u))
        A[v] = set()
    return order, struct


class Symbolic:
    """Symbolic analysis of one block (see the module docstring)."""

    def __init__(self, G: BlockGraph, relax_max_nodes: int = 8, relax_max_front: int = 0):
        order, struct = min_degree(G.adj, G.n_block, G.dual_from)
        nb_nodes = G.n_block
        self.elim_order = order
        pos = np.full(G.n_nodes, -1, dtype=np.int64)
        pos[order] = np.arange(len(order))
        BORDER = -2
        parent = np.full(nb_nodes, -1, dtype=np.int64)
        for v in order:
            st = [u for u in struct[v]]
            inblk = [u for u in st if u < nb_nodes]
            if inblk:
                parent[v] = min(inblk, key=lambda u: pos[u])
            elif st:
                parent[v] = BORDER
            else:
                parent[v] = -1       # isolated from the border (not expected)
        # postorder, children in increasing node id; roots (border children
        # and isolated nodes) also in increasing id
        children = [[] for _ in range(nb_nodes)]
        roots = []
        for v in range(nb_nodes):
            if parent[v] >= 0:
                children[parent[v]].append(v)
            else:
                roots.append(v)
        post = []
        for r0 in roots:
            stack = [(r0, 0)]
            while stack:
                v, i = stack.pop()
                if i < len(children[v]):
                    stack.append((v, i + 1))
                    stack.append((children[v][i], 0))
                else:
                    post.append(v)
        self.post = np.array(post, dtype=np.int64)           # node ids in postorder
        ppos = np.full(G.n_nodes, -1, dtype=np.int64)
        ppos[self.post] = np.arange(nb_nodes)
        n_border = G.n_nodes - nb_nodes
        ppos[nb_nodes:] = nb_nodes + np.arange(n_border)
        self.ppos = ppos
        self.parent = parent
        self.struct = struct
        # ---- supernodes over the postorder
        cnt = np.array([len(struct[v]) for v in range(nb_nodes)], dtype=np.int64)
        nchild = np.array([len(c) for c in children], dtype=np.int64)
        starts = [0]
        size = 1
        for i in range(1, nb_nodes):
            v, u = self.post[i], self.post[i - 1]
            # an only child directly below its parent in the postorder joins the
            # parent's supernode (fundamental when cnt[u] == cnt[v] + 1, relaxed
            # otherwise) while the supernode stays within relax_max_nodes nodes
            chain = parent[u] == v and nchild[v] == 1
            if chain and size < relax_max_nodes:
                size += 1
            else:
                starts.append(i)
                size = 1
        starts.append(nb_nodes)
        self._supernode_links(np.array(starts, dtype=np.int64))
        if relax_max_front > 0:
            self._relax_by_front(G, relax_max_front)
        # ---- row permutation (generic KKT indices in elimination order)
        rows = [G.node_rows[v] for v in self.post.tolist()] + \
               [G.node_rows[v] for v in range(nb_nodes, G.n_nodes)]
        self.rows = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
        self.n_block_rows = int(sum(len(G.node_rows[v]) for v in range(nb_nodes)))

    def _supernode_links(self, sn_start):
        """Update nodes (union of the members' structures minus the members,
        sorted by position, border nodes last) and parent of every supernode
        (the supernode of the first in-block update node; -2 = border)."""
        nb_nodes = len(self.post)
        self.sn_start = sn_start
        nsn = len(sn_start) - 1
        sn_of = np.zeros(nb_nodes, dtype=np.int64)
        for s in range(nsn):
            sn_of[sn_start[s]:sn_start[s + 1]] = s
        self.sn_of_pos = sn_of
        ppos = self.ppos
        upd = []
        sn_parent = np.full(nsn, -1, dtype=np.int64)
        for s in range(nsn):
            members = self.post[sn_start[s]:sn_start[s + 1]]
            mset = set(members.tolist())
            u = set()
            for v in members.tolist():
                u |= self.struct[v]
            u -= mset
            ul = sorted(u, key=lambda x: ppos[x])
            upd.append(np.array(ul, dtype=np.int64))
            inb = [x for x in ul if x < nb_nodes]
            if inb:
                sn_parent[s] = sn_of[ppos[inb[0]]]
            elif ul:
                sn_parent[s] = -2
        self.sn_update_nodes = upd
        self.sn_parent = sn_parent
        self.n_sn = nsn

    def _relax_by_front(self, G, max_front):
        """Step 6 and 7 of the module docstring."""
        nsn = self.n_sn
        nrow = [len(r) for r in G.node_rows]
        members = [self.post[self.sn_start[s]:self.sn_start[s + 1]].tolist() for s in range(nsn)]
        npiv = [sum(nrow[v] for v in members[s]) for s in range(nsn)]
        front = [npiv[s] + sum(nrow[u] for u in self.sn_update_nodes[s].tolist()) for s in range(nsn)]
        kids = [[] for _ in range(nsn)]
        for s in range(nsn):
            if self.sn_parent[s] >= 0:
                kids[self.sn_parent[s]].append(s)
        absorbed = [[] for _ in range(nsn)]
        into = [-1] * nsn
        for s in range(nsn):                       # children before parents
            for c in kids[s]:                      # increasing index
                if front[s] + npiv[c] <= max_front:
                    absorbed[s].append(c)
                    into[c] = s
                    front[s] += npiv[c]
                    npiv[s] += npiv[c]

        def expand(s):
            out = []
            for c in absorbed[s]:
                out += expand(c)
            return out + members[s]

        rep_ = list(range(nsn))
        for s in range(nsn - 1, -1, -1):
            if into[s] >= 0:
                rep_[s] = rep_[into[s]]
        tree_kids = [[] for _ in range(nsn)]
        roots = []
        for s in range(nsn):
            if into[s] >= 0:
                continue
            if self.sn_parent[s] >= 0:
                tree_kids[rep_[self.sn_parent[s]]].append(s)
            else:
                roots.append(s)
        order = []
        for r0 in roots:
            stack = [(r0, 0)]
            while stack:
                v, i = stack.pop()
                if i < len(tree_kids[v]):
                    stack.append((v, i + 1))
                    stack.append((tree_kids[v][i], 0))
                else:
                    order.append(v)
        post, starts = [], [0]
        for s in order:
            post += expand(s)
            starts.append(len(post))
        nb_nodes = len(self.post)
        assert len(post) == nb_nodes
        self.post = np.array(post, dtype=np.int64)
        self.ppos[self.post] = np.arange(nb_nodes)
        self._supernode_links(np.array(starts, dtype=np.int64))


def structural_kkt(model, seed: int = 12345):
    """Reduced KKT matrix at a random interior point: every structurally
    nonzero entry is numerically nonzero (with probability one)."""
    from .ncl import NCLSolver, Params, State
    from .linsolve import DenseSolver
    rng = np.random.default_rng(seed)
    S = NCLSolver(model, DenseSolver())
    st = S.initial_state()
    n, m, p = model.n, model.m, model.p
    st.w = st.w + 1e-3 * rng.random(n)
    st.lam = rng.standard_normal(m)
    st.yc = rng.random(p) + 0.5
    st.s = rng.random(p) + 0.5
    st.zs = rng.random(p) + 0.5
    st.zl = rng.random(len(S.il)) + 0.5
    st.zu = rng.random(len(S.iu)) + 0.5
    prm = Params(rho=10.0, lam_n=np.zeros(m), nu0_n=np.zeros(p))
    H = model.hessian(st.w, st.lam)
    J = model.jacobian(st.w)
    return S.kkt_matrix(st, prm, H, J, 0.5)


def kkt_permutation(model, K=None, relax_max_nodes: int = 8, relax_max_front: int = 0,
                    dual_first: bool = False):
    """Global fill-reducing order of the reduced KKT matrix: each block's rows
    in its symbolic order, blocks 0..K in turn, then the border rows.  The
    node graphs come from the structural pattern (``structural_kkt``)."""
    Ks = structural_kkt(model)
    graphs = attach_adjacency(block_graphs(model, dual_first), Ks)
    syms = [Symbolic(G, relax_max_nodes, relax_max_front) for G in graphs]
    parts = [S.rows[:S.n_block_rows] for S in syms]
    border = np.arange(model.border0, model.border0 + model.nborder, dtype=np.int64)
    perm = np.concatenate(parts + [border])
    assert len(perm) == Ks.shape[0] and len(np.unique(perm)) == Ks.shape[0]
    return perm, syms
