"""Edge cases of the SCOPF structure, GPU against the oracle: no
contingency at all (a base-case OPF with the border alone), generator
outages only, a single generator (border of two: p_g^0 and one v^0), a
five-bus network, full switch sets without thermal limits.  Host-side size
and symbolic checks run without a GPU."""
import warnings

import numpy as np
import pytest

from oracle.linsolve import SparseLDLSolver
from oracle.ncl import NCLSolver
from oracle.scopf_model import SCOPFModel
from oracle import symbolic
from tests import helpers as H

CASES = {
    "no_contingency": dict(n_line=0, n_gen_ctg=0),
    "gen_outages_only": dict(n_line=0, n_gen_ctg=2),
    "one_generator": dict(n_bus=5, n_gen=1, n_line=1, n_gen_ctg=0),
    "six_bus": dict(n_bus=6, n_gen=2, n_line=1, n_gen_ctg=0),
    "full_switch_no_thermal": dict(n_line=3, n_gen_ctg=1, switch="full", thermal=False),
}


def _inst(name):
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)
        return H.small_instance(**CASES[name])


@pytest.mark.parametrize("name", sorted(CASES))
def test_edge_sizes_and_symbolic(name):
    import paper_2510_13333_b300 as P
    inst = _inst(name)
    M = SCOPFModel(inst)
    lib = P.SCOPF(inst, host_only=1)
    assert lib.sizes.n_kkt == M.n + M.m + M.p
    assert lib.sizes.n_blocks == len(inst.ctgs) + 1
    assert lib.sizes.n_border == M.nborder
    _, syms = symbolic.kkt_permutation(M)
    for k, S in enumerate(syms):
        c = lib.scopf_symbolic_block(k)
        assert np.array_equal(c["post"], S.post) and np.array_equal(c["sn_start"], S.sn_start)


_ORACLE = {}


def _oracle(name):
    if name not in _ORACLE:
        M = SCOPFModel(_inst(name))
        perm, _ = symbolic.kkt_permutation(M)
        _ORACLE[name] = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm)).solve()
    return _ORACLE[name]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_edge_ncl_solve_matches_oracle(cuda, name, prec):
    import paper_2510_13333_b300 as P
    ref = _oracle(name)
    assert ref.status == "ok"
    lib = P.SCOPF(_inst(name), precision=prec)
    res = lib.ncl_solve()
    assert res["call_status"] == 0, res
    assert abs(res["objective"] - ref.objective) <= 1e-6 * abs(ref.objective), (res, ref.objective)
    assert res["max_violation"] <= 1e-6
