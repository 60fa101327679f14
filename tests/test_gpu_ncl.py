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
