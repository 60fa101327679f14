"""Contingency screening with NCL (Section V-B), oracle version.

The paper computes a base-case solution u0 by solving the AC-OPF, then
solves the per-contingency system eq. (screening) with NCL at that u0; an
infeasible contingency makes rho diverge and NCL falls back to the
feasibility problem eq. (feaspb).  Only contingencies that are not
structurally infeasible enter the SCOPF.

With ``eps`` given, the first-stage variables are held at u0 by bounds
u0 +- eps (clipped to their own limits), as in the paper; the synthetic
workloads were screened this way, with eps = 1e-3 around a base point
computed with derated thermal limits and a narrowed voltage band, which
leaves the outages a recovery margin (``make_screened.py``).  With
eps = None u0 stays free and the candidate is solved together with the base
case as a two-scenario SCOPF.  The penalty is capped at ``rho_cap``: a
candidate is accepted when |(r, t)|_inf falls below ``accept_tol`` before
that cap.
"""
from __future__ import annotations

import numpy as np

from .linsolve import SparseLDLSolver
from .ncl import NCLSolver, Options
from .scopf_model import SCOPFModel
from . import symbolic


def _solver(model, opts):
    perm, _ = symbolic.kkt_permutation(model)
    return NCLSolver(model, SparseLDLSolver(perm_fn=lambda K: perm), opts)


def sub_instance(inst, ctgs):
    import copy
    sub = copy.copy(inst)
    sub.ctgs = list(ctgs)
    return sub


def base_opf(inst, opts: Options | None = None, derate: float | None = None,
             v_margin: float = 0.0):
    """AC-OPF of the base case alone (K = 0).  ``derate`` scales the thermal
    ratings and ``v_margin`` narrows the voltage band, which leaves recovery
    margin at the returned u0 for screening at a fixed first stage."""
    import copy
    sub = sub_instance(inst, [])
    if derate is not None or v_margin:
        sub.net = copy.copy(inst.net)
        if derate is not None:
            sub.net.rate = inst.net.rate * derate
        sub.net.vmin = inst.net.vmin + v_margin
        sub.net.vmax = inst.net.vmax - v_margin
    M = SCOPFModel(sub)
    res = _solver(M, opts or Options()).solve()
    u0 = res.state.w[M.border0:M.border0 + M.nborder].copy()
    return res, u0


def box_first_stage(M, u0, eps):
    """Hold the first-stage variables within eps of u0: bounds
    [max(lo, u0 - eps), min(hi, u0 + eps)], widened to width eps where u0
    sits on (or beyond) a limit."""
    b = np.arange(M.border0, M.border0 + M.nborder)
    lo, hi = M.wl[b].copy(), M.wu[b].copy()
    M.wl[b] = np.maximum(lo, u0 - eps)
    M.wu[b] = np.minimum(hi, u0 + eps)
    M.wl[b] = np.minimum(M.wl[b], M.wu[b] - eps)
    M.wu[b] = np.maximum(M.wu[b], M.wl[b] + eps)


def screen_candidate(inst, cand, u0, eps: float | None = None, rho_cap: float = 1e6,
                     accept_tol: float = 1e-4, opts: Options | None = None):
    """Feasibility of one contingency at the base control u0.

    Returns (accepted, |(r,t)|_inf, status)."""
    M = SCOPFModel(sub_instance(inst, [cand]))
    if eps is not None:
        box_first_stage(M, u0, eps)
    o = opts or Options()
    o = Options(**{**o.__dict__, "rho_max": rho_cap, "max_inner": 1000})
    res = _solver(M, o).solve()
    # structurally infeasible outages keep |(r, t)| far from zero as rho grows;
    # a residual below accept_tol (feasibility objective ~1e-8) is feasible up
    # to the complementarity floor sqrt(mu_min / rho) of the capped penalty
    ok = res.feas_rt <= accept_tol and res.status in ("ok", "infeasible", "max_outer")
    return ok, float(res.feas_rt), res.status


def block_violation(M, st):
    """|(r_k, t_k)|_inf of every scenario block (k = 0 base case)."""
    def inf(x):
        return float(np.max(np.abs(x))) if len(x) else 0.0
    return np.array([max(inf(st.r[b.c0:b.c0 + b.nrow]), inf(st.t[b.p0:b.p0 + b.ncomp]))
                     for b in M.blocks])


def screen_batch(inst, u0, eps: float = 1e-6, rho_cap: float = 1e6, accept_tol: float = 1e-4,
                 opts: Options | None = None):
    """All contingencies of ``inst`` screened at u0 in one NCL solve.

    The base case and every contingency are the scenarios of one model whose
    first stage is held within eps of u0; at a tiny eps the scenarios
    decouple into the per-contingency systems of eq. (screening).  The
    outer loop runs the per-block rule of ``NCLSolver.solve`` (a block that
    is feasible to eta takes its multiplier update even while another block
    drives rho up), so each block ends as it would alone: at a feasible
    point, or at the capped-penalty minimiser of its own infeasibility
    (eq. (feaspb)).  Scenario k is accepted when its |(r_k, t_k)|_inf <=
    accept_tol and the solve did not stop at the inner-iteration limit.

    Returns (accepted[K + 1], viol[K + 1], result)."""
    M = SCOPFModel(inst)
    box_first_stage(M, np.asarray(u0, dtype=float), eps)
    o = opts or Options()
    o = Options(**{**o.__dict__, "rho_max": rho_cap})
    blocks = [(b.c0, b.nrow, b.p0, b.ncomp) for b in M.blocks]
    res = _solver(M, o).solve(blocks=blocks)
    viol = block_violation(M, res.state)
    ended = res.status in ("ok", "infeasible", "max_outer")
    return ended & (viol <= accept_tol), viol, res
