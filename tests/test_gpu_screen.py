"""GPU batched contingency screening (Section V-B) against the oracle's
batched screening on the same seeded workloads: the same verdicts, the
same per-scenario infeasibility |(r_k, t_k)|_inf, and the closed-form bound
on a capacity shortfall."""
import numpy as np
import pytest

import synthgrid
from oracle.screening import base_opf, screen_batch, sub_instance
from tests.test_oracle_screening import FIXED, _shortfall_instance

pytestmark = pytest.mark.gpu

ACCEPT_TOL = 1e-4
_ORACLE = {}


def oracle_batch(idx):
    if idx not in _ORACLE:
        inst, u0, _, _ = synthgrid.screening_batch(idx)
        _ORACLE[idx] = screen_batch(inst, u0, FIXED, accept_tol=ACCEPT_TOL)
    return _ORACLE[idx]


@pytest.mark.parametrize("idx,prec", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_screen_matches_oracle_batch(cuda, idx, prec):
    """Verdicts equal; an infeasible scenario's |(r_k, t_k)|_inf (the
    capped-penalty minimiser of its infeasibility) within 1e-3 relative, a
    feasible one's residual within accept_tol / 4 of the oracle's."""
    import paper_2510_13333_b300 as P
    acc_o, viol_o, res_o = oracle_batch(idx)
    inst, u0, _, _ = synthgrid.screening_batch(idx)
    lib = P.SCOPF(inst, precision=prec)
    acc, viol, res = lib.scopf_screen(u0, eps=FIXED, rho_cap=1e6, accept_tol=ACCEPT_TOL)
    assert res["status"] in (0, -6), res          # converged or rho at the cap
    assert list(acc) == list(acc_o), np.flatnonzero(acc != acc_o)
    bad = viol_o > ACCEPT_TOL
    assert np.all(np.abs(viol[bad] - viol_o[bad]) <= 1e-3 * viol_o[bad]), \
        np.max(np.abs(viol[bad] / viol_o[bad] - 1))
    assert np.all(np.abs(viol[~bad] - viol_o[~bad]) <= ACCEPT_TOL / 4)


def test_screen_shortfall_bound(cuda):
    """A generator outage the remaining capacity cannot cover stays
    infeasible with |r_k|_inf >= deficit / n_bus; the base case passes."""
    import paper_2510_13333_b300 as P
    inst, cand, deficit = _shortfall_instance()
    _, u0 = base_opf(inst)
    lib = P.SCOPF(sub_instance(inst, [cand]), precision=1)
    acc, viol, res = lib.scopf_screen(u0, eps=FIXED)
    assert acc[0] and not acc[1], viol
    assert viol[1] >= 0.99 * deficit / inst.net.n_bus


def test_screen_restores_handle(cuda):
    """After screening, the handle solves its own SCOPF as before (bounds
    and options restored), and bad arguments are refused."""
    import paper_2510_13333_b300 as P
    inst, u0, _, _ = synthgrid.screening_batch(0)
    lib = P.SCOPF(inst, precision=1)
    ref = lib.ncl_solve()
    lib.scopf_screen(u0, eps=FIXED)
    again = lib.ncl_solve()
    assert again["call_status"] == ref["call_status"]
    assert abs(again["objective"] - ref["objective"]) <= 1e-9 * abs(ref["objective"])
    assert again["outer_iters"] == ref["outer_iters"]
    with pytest.raises(P.ScopfError):
        lib.scopf_screen(u0, eps=0.0)
    bad = u0.copy()
    bad[0] = np.nan
    with pytest.raises(P.ScopfError):
        lib.scopf_screen(bad, eps=FIXED)
