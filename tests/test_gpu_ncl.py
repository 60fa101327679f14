"""GPU full NCL solves against the oracle: final objective within 1e-6
relative, constraint violation <= 1e-6 (FP64 and mixed precision)."""
import numpy as np
import pytest

from oracle.linsolve import SparseLDLSolver
from oracle.ncl import NCLSolver
from oracle.scopf_model import SCOPFModel
from oracle import symbolic
from tests import helpers as H

pytestmark = pytest.mark.gpu

_ORACLE = {}


def oracle_solution(idx):
    if idx not in _ORACLE:
        inst = H.instance(idx)
        M = SCOPFModel(inst)
        perm, _ = symbolic.kkt_permutation(M)
        _ORACLE[idx] = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm)).solve()
    return _ORACLE[idx]


@pytest.mark.parametrize("idx,prec", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_ncl_solve_matches_oracle(cuda, idx, prec):
    import paper_2510_13333_b300 as P
    ref = oracle_solution(idx)
    assert ref.status == "ok"
    lib = P.SCOPF(H.instance(idx), precision=prec)
    res = lib.ncl_solve()
    assert res["call_status"] == 0, res
    assert abs(res["objective"] - ref.objective) <= 1e-6 * abs(ref.objective), (res, ref.objective)
    assert res["max_violation"] <= 1e-6
    assert res["kkt_error"] <= 1e-6 and res["feas_rt"] <= 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_iteration_log_consistent(cuda, prec):
    """The iteration log of a solve agrees with its result: one record per
    inner and outer iteration, factorizations and refinement steps summing
    to the result's counts, mu never increasing within an outer iteration,
    and the last outer record meeting the tolerance."""
    import paper_2510_13333_b300 as P
    lib = P.SCOPF(H.instance(0), precision=prec)
    res = lib.ncl_solve()
    assert res["call_status"] == 0
    names, inner = lib.history(0)
    onames, outer = lib.history(1)
    col = {n: i for i, n in enumerate(names)}
    ocol = {n: i for i, n in enumerate(onames)}
    assert inner.shape[0] == res["inner_iters"] and outer.shape[0] == res["outer_iters"]
    assert np.all(np.diff(inner[:, col["inner"]]) == 1)
    assert inner[:, col["factorizations"]].sum() == res["factorizations"]
    assert inner[:, col["refine_steps"]].sum() == res["refine_steps"]
    assert set(np.unique(inner[:, col["precision"]])) <= {0.0, 1.0}
    for o in np.unique(inner[:, col["outer"]]):
        mu = inner[inner[:, col["outer"]] == o, col["mu"]]
        assert np.all(np.diff(mu) <= 0)
    last = outer[-1]
    assert max(last[ocol["r_inf"]], last[ocol["t_inf"]]) <= 1e-6
    assert last[ocol["inner"]] == res["inner_iters"]
