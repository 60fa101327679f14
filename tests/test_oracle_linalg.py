"""Pins of the oracle's linear algebra: LDL^T, inertia, the reduced Newton
system of eq. (newtonsystem) against the unreduced Newton system, and the
symbolic analysis against brute force."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.linsolve import DenseSolver, SparseLDLSolver, dense_ldlt
from oracle.ncl import NCLSolver, Params, State
from oracle.scopf_model import SCOPFModel
from oracle import symbolic
from oracle.toys import ToyMPCC, ToyQP
from tests import helpers as H


def _sqd(n1, n2, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n1, n1))
    A = A @ A.T + n1 * np.eye(n1)
    C = rng.standard_normal((n2, n2))
    C = C @ C.T + n2 * np.eye(n2)
    B = rng.standard_normal((n2, n1))
    return np.block([[A, B.T], [B, -C]])


def test_dense_ldlt_reconstruction_and_inertia():
    K = _sqd(7, 5, 0)
    L, d = dense_ldlt(K)
    assert np.abs(L @ np.diag(d) @ L.T - K).max() <= 1e-13 * np.abs(K).max()
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.diag(L), 1)
    ev = np.linalg.eigvalsh(K)
    assert (d > 0).sum() == (ev > 0).sum() == 7
    assert (d < 0).sum() == (ev < 0).sum() == 5


def test_quasidefinite_any_permutation():
    """Vanderbei (1995): every symmetric permutation of a symmetric
    quasi-definite matrix has an LDL^T; all give the same solution."""
    K = _sqd(6, 4, 1)
    b = np.arange(10.0)
    x0 = np.linalg.solve(K, b)
    rng = np.random.default_rng(2)
    for _ in range(5):
        p = rng.permutation(10)
        L, d = dense_ldlt(K[np.ix_(p, p)])
        assert np.all(np.abs(d) > 1e-8)
        y = np.linalg.solve(L, b[p])
        z = np.linalg.solve(L.T, y / d)
        x = np.empty(10)
        x[p] = z
        np.testing.assert_allclose(x, x0, rtol=1e-10, atol=1e-12)


def test_sparse_ldlt_matches_dense():
    inst = H.small_instance()
    M = SCOPFModel(inst)
    K = symbolic.structural_kkt(M)
    perm, _ = symbolic.kkt_permutation(M)
    sps = SparseLDLSolver(perm_fn=lambda K: perm)
    inert = sps.factor(K)
    den = DenseSolver()
    assert inert == den.factor(K)
    L, D = sps.factors()
    Kp = K[perm][:, perm].toarray()
    assert np.abs((L @ sp.diags(D) @ L.T).toarray() - Kp).max() <= 1e-12 * np.abs(Kp).max()
    b = np.random.default_rng(0).standard_normal(K.shape[0])
    np.testing.assert_allclose(sps.solve(b), den.solve(b), rtol=1e-8, atol=1e-10)


# ----------------------------------------------------- reduced vs full Newton
def _kkt_map(S, st, prm, mu, n, m, p):
    """Full primal-dual KKT residual F of the barrier subproblem in the
    unknowns (w, r, t, s, lam, yc, zl, zu, zs), written out directly."""
    P = S.P

    def F(v):
        i = 0
        w = v[i:i + n]; i += n
        r = v[i:i + m]; i += m
        t = v[i:i + p]; i += p
        s = v[i:i + p]; i += p
        lam = v[i:i + m]; i += m
        yc = v[i:i + p]; i += p
        zl = v[i:i + len(S.il)]; i += len(S.il)
        zu = v[i:i + len(S.iu)]; i += len(S.iu)
        zs = v[i:i + p]; i += p
        gw = P.gradient(w) + P.jacobian(w).T @ lam
        gw[S.c1] += yc * w[S.c2]
        gw[S.c2] += yc * w[S.c1]
        gw[S.il] -= zl
        gw[S.iu] += zu
        return np.concatenate([
            gw,
            prm.lam_n + prm.rho * r - lam,
            prm.nu0_n + prm.rho * t - yc,
            yc - zs,
            P.constraints(w) - r,
            w[S.c1] * w[S.c2] - t + s,
            (w[S.il] - S.wl[S.il]) * zl - mu,
            (S.wu[S.iu] - w[S.iu]) * zu - mu,
            s * zs - mu])

    v0 = np.concatenate([st.w, st.r, st.t, st.s, st.lam, st.yc, st.zl, st.zu, st.zs])
    return F, v0


@pytest.mark.parametrize("prob", ["toy_quadratic", "toy_qp", "scopf_small"])
def test_reduced_newton_equals_full_newton(prob):
    if prob == "toy_quadratic":
        P = ToyMPCC("quadratic", x0=(0.7, 0.4))
    elif prob == "toy_qp":
        P = ToyQP(n=5, m=2, seed=3)
    else:
        P = SCOPFModel(H.small_instance(n_bus=8, n_gen=3, n_line=1, n_gen_ctg=1))
    S = NCLSolver(P, DenseSolver())
    st = H.random_interior_state(S, 4)
    n, m, p = S.n, S.m, S.p
    rng = np.random.default_rng(8)
    prm = Params(rho=37.0, lam_n=rng.standard_normal(m) * 0.3, nu0_n=rng.random(p) * 0.3)
    mu, delta_w = 0.03, 0.0
    res = S.residuals(st, prm)
    K = S.kkt_matrix(st, prm, P.hessian(st.w, st.lam), res["J"], delta_w)
    sol = np.linalg.solve(K.toarray(), S.reduced_rhs(st, prm, res, mu))
    d = S.recover(st, prm, res, mu, sol)
    red = np.concatenate([d.w, d.r, d.t, d.s, d.lam, d.yc, d.zl, d.zu, d.zs])
    # Newton direction of the unreduced system: -J_F^{-1} F, J_F by central differences
    F, v0 = _kkt_map(S, st, prm, mu, n, m, p)
    N = len(v0)
    JF = np.zeros((N, N))
    h = 1e-6
    for j in range(N):
        e = np.zeros(N)
        e[j] = h
        JF[:, j] = (F(v0 + e) - F(v0 - e)) / (2 * h)
    full = np.linalg.solve(JF, -F(v0))
    assert np.abs(red - full).max() <= 1e-6 * max(1.0, np.abs(full).max())


# ------------------------------------------------------------ symbolic
def test_min_degree_path_graph():
    adj = [{1}, {0, 2}, {1, 3}, {2, 4}, {3}]
    order, _ = symbolic.min_degree(adj, 5)
    assert order == [0, 1, 2, 3, 4]


def test_min_degree_grid_3x3():
    # node id = 3 * row + col; hand elimination: corners (degree 2, smallest
    # id first), then 1 (all degree 3, smallest id), then 3, 4, 5, 7
    adj = [set() for _ in range(9)]
    for r in range(3):
        for c in range(3):
            v = 3 * r + c
            for dr, dc in ((0, 1), (1, 0)):
                if r + dr < 3 and c + dc < 3:
                    u = 3 * (r + dr) + c + dc
                    adj[v].add(u)
                    adj[u].add(v)
    order, _ = symbolic.min_degree(adj, 9)
    assert order == [0, 2, 6, 8, 1, 3, 4, 5, 7]


def test_min_degree_border_last():
    adj = [{1, 3}, {0, 2}, {1, 3}, {0, 2}]
    order, struct = symbolic.min_degree(adj, 3)   # node 3 is a border node
    assert 3 not in order and sorted(order) == [0, 1, 2]


def test_symbolic_structure_brute_force():
    """Fill of the node graph by dense boolean elimination in the computed
    order equals the recorded structures; the node tree is the first
    eliminated neighbour; row order is a valid postorder of that tree."""
    inst = H.small_instance()
    M = SCOPFModel(inst)
    K = symbolic.structural_kkt(M)
    graphs = symbolic.attach_adjacency(symbolic.block_graphs(M), K)
    for G in graphs:
        Sy = symbolic.Symbolic(G)
        n = G.n_nodes
        A = np.zeros((n, n), dtype=bool)
        for v in range(n):
            for u in G.adj[v]:
                A[v, u] = A[u, v] = True
        alive = np.ones(n, dtype=bool)
        for v in Sy.elim_order:
            nb = np.flatnonzero(A[v] & alive)
            nb = nb[nb != v]
            assert set(nb.tolist()) == Sy.struct[v]
            A[np.ix_(nb, nb)] = True
            alive[v] = False
        pos = {v: i for i, v in enumerate(Sy.elim_order)}
        for v in Sy.elim_order:
            blk = [u for u in Sy.struct[v] if u < G.n_block]
            if blk:
                assert Sy.parent[v] == min(blk, key=pos.get)
        ppos = {v: i for i, v in enumerate(Sy.post.tolist())}
        for v in range(G.n_block):
            if Sy.parent[v] >= 0:
                assert ppos[v] < ppos[Sy.parent[v]]


def test_relaxed_amalgamation_star_by_hand():
    """Star: four one-row leaves around a one-row centre, no border.  Leaves
    (fronts of 2 rows: pivot + centre) are children of the centre (front 1).
    With a 3-row bound the centre absorbs leaves 0 and 1 (front 1 -> 2 -> 3)
    and rejects 2 and 3; the final tree {2}, {3} -> {0, 1, 4} is postordered
    children first, each supernode listing absorbed nodes before its own."""
    rows = [np.array([i]) for i in range(5)]
    adj = [{4}, {4}, {4}, {4}, {0, 1, 2, 3}]
    G = symbolic.BlockGraph(rows, adj, 5)
    S = symbolic.Symbolic(G, relax_max_nodes=8, relax_max_front=3)
    assert S.post.tolist() == [2, 3, 0, 1, 4]
    assert S.sn_start.tolist() == [0, 1, 2, 5]
    assert S.sn_parent.tolist() == [2, 2, -1]
    assert [u.tolist() for u in S.sn_update_nodes] == [[4], [4], []]
    S0 = symbolic.Symbolic(G, relax_max_nodes=8, relax_max_front=0)
    assert S0.post.tolist() == [0, 1, 2, 3, 4] and S0.sn_start.tolist() == [0, 1, 2, 3, 4, 5]


@pytest.mark.parametrize("max_front", [16, 32, 48])
def test_relaxed_amalgamation_invariants(max_front):
    """On every block of a small instance: the node order is a topological
    order of the elimination tree; every front holds its members' fill
    (brute-force elimination gives the structures); no final child fits its
    parent's front (greedy absorption is maximal); a front above the bound is
    an unmerged chain of only children."""
    inst = H.small_instance()
    M = SCOPFModel(inst)
    K = symbolic.structural_kkt(M)
    graphs = symbolic.attach_adjacency(symbolic.block_graphs(M), K)
    for G in graphs:
        S = symbolic.Symbolic(G, relax_max_nodes=8, relax_max_front=max_front)
        nb = G.n_block
        assert sorted(S.post.tolist()) == list(range(nb))
        ppos = {v: i for i, v in enumerate(S.post.tolist())}
        for v in range(nb):
            if S.parent[v] >= 0:
                assert ppos[v] < ppos[S.parent[v]]
        nrow = [len(r) for r in G.node_rows]
        nsn = S.n_sn
        npiv, front, members = [], [], []
        for s in range(nsn):
            mem = S.post[S.sn_start[s]:S.sn_start[s + 1]].tolist()
            members.append(mem)
            fill = set().union(*[S.struct[v] for v in mem]) - set(mem)
            assert fill == set(S.sn_update_nodes[s].tolist())
            npiv.append(sum(nrow[v] for v in mem))
            front.append(npiv[-1] + sum(nrow[u] for u in fill))
        for s in range(nsn):
            p = S.sn_parent[s]
            if p >= 0:
                assert p > s
                assert front[p] + npiv[s] > max_front
            if front[s] > max_front:
                mem = members[s]
                for a, b in zip(mem[:-1], mem[1:]):
                    assert S.parent[a] == b
                    assert sum(1 for v in range(nb) if S.parent[v] == b) == 1


def test_global_permutation_fill_matches_etree_counts():
    """nnz(L) of the scalar factor under the oracle permutation equals the
    count from brute-force dense symbolic elimination."""
    inst = H.small_instance(n_bus=8, n_gen=3, n_line=1, n_gen_ctg=1)
    M = SCOPFModel(inst)
    K = symbolic.structural_kkt(M)
    perm, _ = symbolic.kkt_permutation(M)
    sps = SparseLDLSolver(perm_fn=lambda K: perm)
    sps.factor(K)
    P = (K[perm][:, perm].toarray() != 0)
    n = P.shape[0]
    nnz = 0
    for k in range(n):
        rows = np.flatnonzero(P[k + 1:, k]) + k + 1
        nnz += len(rows)
        P[np.ix_(rows, rows)] = True
    assert nnz == sps.nnzL
