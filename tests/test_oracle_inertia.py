"""Pins of the inertia-correction reading (Waechter & Biegler 2006, Alg. IC,
behind the IPM of Section IV-B): IC-1 tries delta_w = 0 at every iteration;
when the pivot-free LDL^T must meet an exactly zero pivot, the outcome of that
trial is taken without factoring.  The shortcut must change nothing: the same
delta_w at every iteration and bit-identical iterates as factoring every
IC-1 trial, and a certain zero pivot must really be one."""
from dataclasses import replace

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import symbolic
from oracle.linsolve import SparseLDLSolver
from oracle.ncl import NCLSolver, Options
from oracle.scopf_model import SCOPFModel
from oracle.toys import ToyQP
from tests import helpers as H


def _run(M, perm, known, max_inner=None):
    o = Options(known_zero_pivot=known)
    if max_inner is not None:
        o = replace(o, max_inner=max_inner)
    S = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm), o)
    return S, S.solve()


@pytest.mark.parametrize("idx,max_inner,fires", [(0, None, False), (1, 12, True)])
def test_known_zero_pivot_changes_nothing(idx, max_inner, fires):
    M = SCOPFModel(H.instance(idx))
    perm, _ = symbolic.kkt_permutation(M)
    Sa, ra = _run(M, perm, True, max_inner)
    Sb, rb = _run(M, perm, False, max_inner)
    # 118-bus: rows that enter only linearly are eliminated before every
    # row they touch, so the trial at 0 meets a zero pivot at every
    # iteration and the shortcut fires; the 30-bus case has no such row
    assert (Sa.n_known_zero > 0) == fires and Sb.n_known_zero == 0
    # ... saved exactly one factorization each time, and changed nothing else
    da = [h["delta_w"] for h in ra.history]
    db = [h["delta_w"] for h in rb.history]
    assert da == db
    ta = sum(h["tries"] for h in ra.history)
    tb = sum(h["tries"] for h in rb.history)
    assert tb - ta == Sa.n_known_zero
    for f in ("w", "r", "t", "s", "lam", "yc", "zl", "zu", "zs"):
        assert np.array_equal(getattr(ra.state, f), getattr(rb.state, f)), f
    assert ra.status == rb.status and ra.inner_iters == rb.inner_iters


def test_certain_zero_pivot_is_a_zero_pivot():
    """On random symmetric matrices with zero diagonals, whenever the
    structural test says a zero pivot is certain the plain LDL^T reports
    one; and a row whose zero diagonal does receive updates is not called
    certain."""
    rng = np.random.default_rng(3)
    hits = 0
    for trial in range(200):
        n = int(rng.integers(3, 9))
        A = sp.random(n, n, density=0.35, random_state=rng.integers(1 << 30)).toarray()
        A = A + A.T
        zero = rng.random(n) < 0.4
        d = np.where(zero, 0.0, rng.standard_normal(n) * 3)
        np.fill_diagonal(A, d)
        perm = rng.permutation(n)
        L = SparseLDLSolver(perm_fn=lambda K, p=perm: p)
        certain = L.zero_pivot_certain(sp.csr_matrix(A))
        _, _, iz = L.factor(sp.csr_matrix(A))
        if certain:
            hits += 1
            assert iz >= 1
        Ap = A[perm][:, perm]
        brute = any(Ap[k, k] == 0.0 and not np.any(Ap[k, :k] != 0.0) for k in range(n))
        assert certain == brute
    assert hits > 10
    # a zero diagonal with an entry to its left is updated: not certain
    K = np.array([[2.0, 1.0], [1.0, 0.0]])
    L = SparseLDLSolver()
    assert not L.zero_pivot_certain(sp.csr_matrix(K))
    assert L.factor(sp.csr_matrix(K)) == (1, 1, 0)


def test_no_shortcut_without_linear_only_rows():
    """A convex QP whose every variable has curvature: IC-1 succeeds at
    delta_w = 0 and the shortcut never fires."""
    P = ToyQP()
    S = NCLSolver(P, SparseLDLSolver())
    r = S.solve()
    assert r.status == "ok" and S.n_known_zero == 0
    assert all(h["delta_w"] == 0.0 for h in r.history)
