"""The device-resident interior-point iteration (option ipm_graph): after the
host's convergence test and barrier update, an iteration is two CUDA-graph
launches whose WHILE nodes run the inertia-correction trials, the refinement
cycles and the line-search trials.  Its decisions are the host loop's, taken
from the same partials combined in the same order, so it must take the very
same steps as the host loop (Section IV-B; W&B 2006 inertia correction and
filter line search), with one host read-back per iteration."""
import numpy as np
import pytest

from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("idx,prec,opts", [
    (0, 0, {}), (0, 1, {}), (1, 0, {}), (1, 1, {}),
    # the FP32 refinement stalls at the first step: the graph hands the step
    # to the host, which redoes the direction in FP64 and launches the step graph
    (0, 1, {"max_refine": 0}),
    # the refinement-cost switch to FP64, taken from the graph's read-back
    (0, 1, {"fp64_switch_refine": 1, "fp64_switch_streak": 1}),
])
def test_graph_iteration_takes_the_host_loops_steps(cuda, idx, prec, opts):
    import paper_2510_13333_b300 as P
    inst = H.instance(idx)
    host = P.SCOPF(inst, precision=prec, ipm_graph=0, **opts)
    rh = host.ncl_solve()
    assert rh["call_status"] == 0 and rh["graph_iters"] == 0
    _, hh = host.history(0)
    dev = P.SCOPF(inst, precision=prec, ipm_graph=1, **opts)
    rd = dev.ncl_solve()
    assert rd["call_status"] == 0, (rd, dev.last_error())
    assert rd["graph_iters"] == rd["inner_iters"] > 0, dev.last_error()
    _, hd = dev.history(0)
    assert rd["inner_iters"] == rh["inner_iters"] and rd["outer_iters"] == rh["outer_iters"]
    assert rd["factorizations"] == rh["factorizations"]
    assert rd["refine_steps"] == rh["refine_steps"]
    assert rd["fp64_fallbacks"] == rh["fp64_fallbacks"]
    cols = P.SCOPF.HISTORY_INNER
    for j, name in enumerate(cols):
        if name != "ms":   # wall time of the iteration
            np.testing.assert_array_equal(hd[:, j], hh[:, j], err_msg=name)
    assert rd["objective"] == rh["objective"]
    assert rd["max_violation"] == rh["max_violation"]
    # one read-back per iteration; the outer loop's assembly and the final
    # report add a few per outer iteration, an FP64 redo its own
    bound = rd["inner_iters"] + 3 * rd["outer_iters"] + 8 + 12 * rd["fp64_fallbacks"]
    assert rd["host_round_trips"] <= bound, (rd["host_round_trips"], bound)
    if not opts:
        assert rh["host_round_trips"] > 3 * rh["inner_iters"]
    if "max_refine" in opts or "fp64_switch_refine" in opts:
        assert rd["fp64_fallbacks"] == 1


def test_graph_iteration_full_size_fp64(cuda):
    """The same at the 500-bus x 256-contingency size (FP64 factors): the
    graph loop's 500-odd iterations take the host loop's steps."""
    import paper_2510_13333_b300 as P
    inst = H.instance(2)
    rh = P.SCOPF(inst, precision=P.PREC_FP64, ipm_graph=0)
    a = rh.ncl_solve()
    rd = P.SCOPF(inst, precision=P.PREC_FP64, ipm_graph=1)
    b = rd.ncl_solve()
    assert a["call_status"] == 0 and b["call_status"] == 0, rd.last_error()
    assert b["graph_iters"] == b["inner_iters"] == a["inner_iters"]
    assert b["objective"] == a["objective"]
    _, ha = rh.history(0)
    _, hb = rd.history(0)
    cols = P.SCOPF.HISTORY_INNER
    for j, name in enumerate(cols):
        if name != "ms":
            np.testing.assert_array_equal(hb[:, j], ha[:, j], err_msg=name)
