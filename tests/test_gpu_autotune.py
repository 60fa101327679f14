"""The supernode tile-shape autotuner (scopf_autotune) on the 118-bus x 32
case: every candidate is timed, the chosen shape is written back and is
within the 2% margin of the fastest (a shape replaces the best so far only
when more than 2% faster), and a solve with the chosen shapes still meets the
oracle's objective."""
import numpy as np
import pytest

from oracle import symbolic
from oracle.linsolve import SparseLDLSolver
from oracle.ncl import NCLSolver
from oracle.scopf_model import SCOPFModel
from tests import helpers as H

pytestmark = pytest.mark.gpu


def test_autotune_picks_fastest_and_solves(cuda):
    import paper_2510_13333_b300 as P
    inst = H.instance(1)
    opt, cands = P.autotune(inst, iterate_at=8, steps=2, precision=P.PREC_MIXED)
    assert 4 <= len(cands) <= 7
    ms = np.array([c["ms_per_step"] for c in cands])
    assert np.all(ms > 0)
    chosen = [c for c in cands if c["chosen"]]
    assert len(chosen) == 1 and chosen[0]["ms_per_step"] <= ms.min() / 0.98 + 1e-12
    assert (opt.cluster_max_tasks, opt.relax_max_nodes) == (chosen[0]["cluster_max_tasks"],
                                                            chosen[0]["relax_max_nodes"])
    lib = P.SCOPF(inst, options=opt)
    res = lib.ncl_solve()
    assert res["call_status"] == 0
    M = SCOPFModel(inst)
    perm, _ = symbolic.kkt_permutation(M, relax_max_nodes=opt.relax_max_nodes)
    ref = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm)).solve()
    assert abs(res["objective"] - ref.objective) <= 1e-6 * abs(ref.objective)
    assert res["max_violation"] <= 1e-6
