"""The per-entry parity checks catch what a check scaled by the largest
entry would not: an error planted in a small entry of K (the NCL block
-1/rho of an equality row) or of a solution vector (a small block)."""
import numpy as np
import scipy.sparse as sp
import pytest

from oracle.linsolve import DenseSolver
from oracle.ncl import NCLSolver, Params
from oracle.scopf_model import SCOPFModel
from tests import helpers as H


@pytest.fixture(scope="module")
def kkt():
    M = SCOPFModel(H.instance(0))
    S = NCLSolver(M, DenseSolver())
    st = H.random_interior_state(S, 4)
    prm = Params(rho=1e6, lam_n=np.zeros(M.m), nu0_n=np.zeros(M.p))
    res = S.residuals(st, prm)
    K = S.kkt_matrix(st, prm, M.hessian(st.w, st.lam), res["J"], 0.0).tocsr()
    return M, K


def test_kkt_check_catches_small_entry(kkt):
    M, K = kkt
    H.assert_kkt_close(K.copy(), K)
    i = M.n  # first equality row: its diagonal is -1/rho = -1e-6
    bad = K.tolil()
    bad[i, i] = K[i, i] * (1 + 1e-6)
    bad = bad.tocsr()
    # invisible to a tolerance scaled by the largest entry of K
    assert abs(bad - K).max() <= 1e-12 * abs(K).max()
    with pytest.raises(AssertionError):
        H.assert_kkt_close(bad, K)


def test_vector_check_catches_small_block(kkt):
    M, _ = kkt
    rng = np.random.default_rng(0)
    x = rng.standard_normal(M.n + M.m + M.p)
    blk = M.blocks[1]
    x[M.n + M.m + blk.p0:M.n + M.m + blk.p0 + blk.ncomp] *= 1e-6
    H.assert_entries_close("x", x.copy(), x, 1e-8, 1e-8 * H.group_scale(M, x))
    y = x.copy()
    y[M.n + M.m + blk.p0] += 1e-12
    assert np.abs(y - x).max() <= 1e-8 * np.abs(x).max()
    with pytest.raises(AssertionError):
        H.assert_entries_close("x", y, x, 1e-8, 1e-8 * H.group_scale(M, x))


def test_term_magnitude_bounds_entries(kkt):
    """sum |terms| >= |entry| for every stored KKT entry (triangle
    inequality), on the same pattern; and the term-scaled check still
    catches a planted error in an entry that is a single term."""
    M, K = kkt
    S = NCLSolver(M, DenseSolver())
    st = H.random_interior_state(S, 4)
    prm = Params(rho=1e6, lam_n=np.zeros(M.m), nu0_n=np.zeros(M.p))
    Kmag = H.kkt_magnitude(S, st, prm, 0.0)
    Kc = K.tocoo()
    mag = np.asarray(Kmag[Kc.row, Kc.col]).ravel()
    assert np.all(mag >= np.abs(Kc.data) * (1 - 1e-12))
    # entries with cancellation exist (the magnitude is far above the value)
    assert np.any(mag > 1e3 * np.abs(Kc.data) + 1e-300)
    H.assert_kkt_terms_close(K.copy(), K, Kmag)
    i = M.n
    bad = K.tolil()
    bad[i, i] = K[i, i] * (1 + 1e-9)
    with pytest.raises(AssertionError):
        H.assert_kkt_terms_close(bad.tocsr(), K, Kmag)


def test_rhs_magnitude_bounds_entries(kkt):
    M, _ = kkt
    S = NCLSolver(M, DenseSolver())
    st = H.random_interior_state(S, 4)
    prm = Params(rho=1e3, lam_n=np.zeros(M.m) + 0.1, nu0_n=np.zeros(M.p) + 0.1)
    res = S.residuals(st, prm)
    mu = 1e-2
    r = S.reduced_rhs(st, prm, res, mu)
    mag = H.rhs_magnitude(S, st, prm, mu)
    assert mag.shape == r.shape
    assert np.all(mag >= np.abs(r) * (1 - 1e-12))
