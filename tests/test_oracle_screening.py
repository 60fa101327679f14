"""Oracle contingency screening (Section V-B): the batched solve against
per-candidate solves (the definition, eq. (screening) at a fixed u0), a
closed-form lower bound on the infeasibility of a capacity shortfall, and
acceptance of every contingency at a first stage the SCOPF itself found."""
import copy

import numpy as np
import pytest

import synthgrid
from oracle import symbolic
from oracle.linsolve import SparseLDLSolver
from oracle.ncl import NCLSolver
from oracle.scopf_model import SCOPFModel
from oracle.screening import base_opf, screen_batch, screen_candidate, sub_instance
from tests import helpers as H

FIXED = 1e-6    # first stage held within 1e-6 of u0: scenarios decouple


def test_batch_matches_single_candidate_solves():
    """Every candidate of the 30-bus screening workload: the batch's verdict
    equals the one of its own two-scenario solve, and |(r_k, t_k)|_inf of an
    infeasible one agrees to 2% (both end at the capped-penalty minimiser
    of the same infeasibility, eq. (feaspb))."""
    inst, u0, _, _ = synthgrid.screening_batch(0)
    acc, viol, res = screen_batch(inst, u0, FIXED)
    assert res.status in ("ok", "infeasible")
    assert acc[0], viol[0]
    n_rej = 0
    for k, cand in enumerate(inst.ctgs, start=1):
        ok, feas, status = screen_candidate(inst, cand, u0, eps=FIXED)
        assert acc[k] == ok, (k, viol[k], feas, status)
        v = max(viol[0], viol[k])      # the single solve reports base + candidate
        if feas > 1e-6:
            assert abs(v - feas) <= 2e-2 * feas, (k, v, feas)
        n_rej += not ok
    assert 0 < n_rej < len(inst.ctgs)   # the workload has both verdicts


def _shortfall_instance():
    """A generator outage the rest of the fleet cannot cover: the other
    generators' pmax sums to 85% of the load, the lost one carries 150%."""
    inst = H.small_instance(thermal=False)
    cand = inst.candidates.gens[0]
    g = cand.element
    net = copy.copy(inst.net)
    net.pmax = inst.net.pmax.copy()
    load = float(net.Pd.sum())
    others = np.arange(net.n_gen) != g
    net.pmax[others] *= 0.85 * load / net.pmax[others].sum()
    net.pmax[g] = 1.5 * load
    inst = copy.copy(inst)
    inst.net = net
    deficit = load - float(net.pmax[others].sum())
    return inst, cand, deficit


def test_capacity_shortfall_infeasibility_bound():
    """Summing the active-power balance rows of the outage scenario gives
    sum_b r_b = sum_g p_g - sum Pd - losses - sum Gs v^2 <= -deficit
    (losses and shunt conductances are nonnegative, p_g <= pmax), so no
    first stage makes the outage feasible and |r_k|_inf >= deficit / n_bus."""
    inst, cand, deficit = _shortfall_instance()
    res, u0 = base_opf(inst)
    assert res.status == "ok"
    acc, viol, res = screen_batch(sub_instance(inst, [cand]), u0, FIXED)
    assert acc[0] and not acc[1]
    assert viol[1] >= 0.99 * deficit / inst.net.n_bus, (viol[1], deficit)
    ok, feas, _ = screen_candidate(inst, cand, u0, eps=FIXED)
    assert not ok and feas >= 0.99 * deficit / inst.net.n_bus


def test_scopf_first_stage_screens_feasible():
    """At the u0 of a converged SCOPF, each of its contingencies has the
    solution the SCOPF found for it, so screening accepts all of them."""
    inst = H.instance(0)
    M = SCOPFModel(inst)
    perm, _ = symbolic.kkt_permutation(M)
    r = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm)).solve()
    assert r.status == "ok"
    u0 = r.state.w[M.border0:M.border0 + M.nborder]
    acc, viol, res = screen_batch(inst, u0, FIXED)
    assert acc.all(), viol
    assert viol.max() <= 1e-6


def test_box_keeps_limits_and_width():
    """The first-stage box: inside each variable's own limits, width eps
    where u0 sits on or beyond a limit, and centred on u0 elsewhere."""
    from oracle.screening import box_first_stage
    inst = H.instance(0)
    M = SCOPFModel(inst)
    b = slice(M.border0, M.border0 + M.nborder)
    lo, hi = M.wl[b].copy(), M.wu[b].copy()
    u0 = 0.5 * (lo + hi)
    u0[0] = hi[0] + 1.0       # beyond the upper limit
    u0[1] = lo[1]             # on the lower limit
    box_first_stage(M, u0, 1e-3)
    wl, wu = M.wl[b], M.wu[b]
    assert wl[0] == pytest.approx(hi[0] - 1e-3) and wu[0] == pytest.approx(hi[0])
    assert wl[1] == pytest.approx(lo[1]) and wu[1] == pytest.approx(lo[1] + 1e-3)
    assert np.allclose(wl[2:], u0[2:] - 1e-3) and np.allclose(wu[2:], u0[2:] + 1e-3)
