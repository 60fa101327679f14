"""Pins of the condensed primal variant (Section IV-B, the "signed
Cholesky" read as a Cholesky of A + B' C^-1 B): the condensed solve equals
the dense solve of the full Newton system; its inertia is Haynsworth's
In(-C) + In(Kc), checked against the eigenvalues of K; the pivot-free
LDL^T under the dual-first order eliminates -C first and leaves exactly the
condensed matrix, factored with positive pivots; the dual-first symbolic
structures are those of brute-force elimination; and the NCL method on the
condensed path converges to a certified solution."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import symbolic
from oracle.linsolve import CondensedSolver, DenseSolver, SparseLDLSolver
from oracle.ncl import NCLSolver, Params
from oracle.scopf_model import SCOPFModel
from oracle.toys import ToyQP
from tests import helpers as H


def _kkt(M, seed, rho=1e2, delta_w=0.0):
    S = NCLSolver(M, DenseSolver())
    st = H.random_interior_state(S, seed)
    rng = np.random.default_rng(seed + 1)
    prm = Params(rho=rho, lam_n=rng.standard_normal(M.m) * 0.1, nu0_n=rng.random(M.p) * 0.1)
    res = S.residuals(st, prm)
    K = S.kkt_matrix(st, prm, M.hessian(st.w, st.lam), res["J"], delta_w).tocsr()
    b = S.reduced_rhs(st, prm, res, 1e-2)
    return S, K, b


def _condensed_perm(M):
    perm, _ = symbolic.kkt_permutation(M, dual_first=True)
    return perm, perm[perm < M.n]


@pytest.mark.parametrize("delta_w", [1.0, 30.0])
def test_condensed_solve_equals_full_solve(delta_w):
    M = SCOPFModel(H.instance(0))
    _, pc = _condensed_perm(M)
    S, K, b = _kkt(M, 3, delta_w=delta_w)
    C = CondensedSolver(M.n, perm_fn=lambda Kc: pc)
    inertia = C.factor(K)
    assert inertia == (M.n, M.m + M.p, 0)
    x = C.solve(b)
    x_ref = np.linalg.solve(K.toarray(), b)
    assert np.abs(x - x_ref).max() <= 1e-9 * np.abs(x_ref).max()


def test_condensed_solve_on_a_convex_qp():
    P = ToyQP()
    S = NCLSolver(P, DenseSolver())
    st = H.random_interior_state(S, 2)
    prm = Params(rho=10.0, lam_n=np.zeros(P.m), nu0_n=np.zeros(P.p))
    res = S.residuals(st, prm)
    K = S.kkt_matrix(st, prm, P.hessian(st.w, st.lam), res["J"], 0.0)
    b = S.reduced_rhs(st, prm, res, 1e-1)
    C = CondensedSolver(P.n)
    assert C.factor(K) == (P.n, P.m + P.p, 0)
    assert np.allclose(C.solve(b), np.linalg.solve(K.toarray(), b), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("delta_w", [0.0, 1e-3, 0.1, 10.0])
def test_condensed_inertia_is_haynsworth(delta_w):
    """In(K) = (0, m + p, 0) + In(A + B' C^-1 B), against the signs of K's
    eigenvalues, both where the inertia is wrong (small delta_w) and right."""
    M = SCOPFModel(H.instance(0))
    _, pc = _condensed_perm(M)
    S, K, _ = _kkt(M, 5, delta_w=delta_w)
    ev = np.linalg.eigvalsh(K.toarray())
    expect = (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    assert CondensedSolver(M.n, perm_fn=lambda Kc: pc).factor(K) == expect


def test_dual_first_ldlt_leaves_the_condensed_matrix():
    """The pivot-free LDL^T of K under the dual-first order: the dual pivots
    are -C exactly (no updates reach them), and the factor's trailing primal
    block reproduces A + B' C^-1 B."""
    M = SCOPFModel(H.instance(0))
    perm, pc = _condensed_perm(M)
    S, K, _ = _kkt(M, 7, delta_w=1.0)
    L = SparseLDLSolver(perm_fn=lambda K_: perm)
    inertia = L.factor(K)
    Lf, D = L.factors()
    Kp = K[perm][:, perm]
    # every block lists its dual rows before its primal rows
    is_dual = perm >= M.n
    assert np.array_equal(D[is_dual], Kp.diagonal()[is_dual])
    prim = np.flatnonzero(~is_dual)
    dual = np.flatnonzero(is_dual)
    Lpp = Lf[prim][:, prim]
    Kc, _, _ = CondensedSolver(M.n).condense(K)
    Kc_p = Kc[pc][:, pc].toarray()
    rebuilt = (Lpp @ sp.diags(D[prim]) @ Lpp.T).toarray()
    assert np.abs(rebuilt - Kc_p).max() <= 1e-12 * np.abs(Kc_p).max()
    assert inertia == CondensedSolver(M.n, perm_fn=lambda Kc_: pc).factor(K)
    # the dual rows never couple: no entry of L between two dual rows
    assert Lf[dual][:, dual].nnz == len(dual)


def test_dual_first_structure_brute_force():
    """The dual-first symbolic analysis: every dual node is eliminated before
    every primal node, and the recorded structures are the fill of dense
    boolean elimination in that order."""
    M = SCOPFModel(H.small_instance())
    K = symbolic.structural_kkt(M)
    graphs = symbolic.attach_adjacency(symbolic.block_graphs(M, dual_first=True), K)
    for G in graphs:
        Sy = symbolic.Symbolic(G)
        nd = G.n_block - G.dual_from
        assert all(v >= G.dual_from for v in Sy.elim_order[:nd])
        assert all(v < G.dual_from for v in Sy.elim_order[nd:])
        for v in range(G.dual_from, G.n_block):       # dual nodes hold dual rows only
            assert np.all(G.node_rows[v] >= M.n)
            assert not any(G.dual_from <= u < G.n_block for u in G.adj[v])
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


def test_ncl_on_the_condensed_path():
    """The NCL method with the condensed solver on the 30-bus case converges
    to a point the error measure certifies, at the objective of the
    standard path."""
    M = SCOPFModel(H.instance(0))
    perm, pc = _condensed_perm(M)
    r = NCLSolver(M, CondensedSolver(M.n, perm_fn=lambda Kc: pc)).solve()
    assert r.status == "ok" and r.kkt_error <= 1e-6 and r.feas_rt <= 1e-6
    assert r.max_violation <= 1e-6
    perm0, _ = symbolic.kkt_permutation(M)
    r0 = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm0)).solve()
    assert abs(r.objective - r0.objective) <= 1e-6 * abs(r0.objective)
