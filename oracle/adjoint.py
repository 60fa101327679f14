"""Adjoint sensitivities of a converged NCL/SCOPF solution (oracle).

Test infrastructure: only tests and the benchmark's CPU baseline use it.

At the final iterate z = (w, lam, yc) of the last NCL subproblem the
reduced barrier KKT conditions F(z; p) = 0 hold (Section IV-B: the reduced
Newton system eq. (newtonsystem) is their linearization, K = dF/dz).  By the
implicit function theorem dz/dp = -K^-1 dF/dp, so for an output
J = seed_pg0' p_g^0 + seed_cost * phi(w) (phi: the base-case cost of
eq. (scopf), scaled as in ``SCOPFModel.objective``) one solve K a = dJ/dz gives

    dJ/dp = dJ/dp|explicit - a' dF/dp.

Parameters:
  * Pd_b, Qd_b enter the bus balance rows of c(w) in every scenario with
    coefficient -1, so dF/dPd_b = -1 on those rows: dJ/dPd_b = sum_k a[row].
  * c1_g enters dphi/dp_g^0 with d^2 phi / (dp_g^0 dc1_g) = BASE_MVA / 1e4
    and phi with dphi/dc1_g = BASE_MVA p_g^0 / 1e4.

K is taken in the rho -> infinity limit of the final subproblem: the NCL
relaxation contributes -1/rho to the diagonal of the constraint and
complementarity rows, and the outer loop drives r, t to zero, so the
solution it returns moves with p as the problem with hard constraints does
(C = diag(0, s/zs)).  The solve is a plain sparse LU of that matrix (no
regularization): the definition the GPU path must reproduce.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .scopf_model import BASE_MVA, OBJ_SCALE


def scopf_adjoint(solver, st, prm, seed_pg0=None, seed_cost=0.0):
    """Returns (grad_Pd, grad_Qd, grad_c1) at the solution (st, prm) of
    ``solver`` (an ``NCLSolver``)."""
    P = solver.P
    net = P.net
    n, m, p = solver.n, solver.m, solver.p
    H = P.hessian(st.w, st.lam)
    J = P.jacobian(st.w)
    hard = type(prm)(rho=np.inf, lam_n=prm.lam_n, nu0_n=prm.nu0_n)
    K = solver.kkt_matrix(st, hard, H, J, 0.0).tocsc()
    g = np.zeros(n + m + p)
    pg = P.border0 + np.arange(P.ng)
    pgv = st.w[pg] * BASE_MVA
    dphi = (2.0 * net.c2 * pgv + net.c1) * BASE_MVA / OBJ_SCALE
    g[pg] = (np.zeros(P.ng) if seed_pg0 is None else np.asarray(seed_pg0, dtype=float)) + \
        seed_cost * dphi
    a = spla.spsolve(K, g)
    gPd = np.zeros(net.n_bus)
    gQd = np.zeros(net.n_bus)
    for blk in P.blocks:
        gPd += a[n + blk.grP]
        gQd += a[n + blk.grQ]
    gc1 = -(BASE_MVA / OBJ_SCALE) * a[pg] + seed_cost * (BASE_MVA / OBJ_SCALE) * st.w[pg]
    return gPd, gQd, gc1


def polish_barrier(solver, st, mu, tol=1e-12, max_iter=15):
    """Newton's method on the barrier KKT conditions of the NCL subproblem
    with the relaxations r and t held at their values (Section IV-B,
    eq. kktncl at the barrier parameter mu):

        grad phi + J' lam + B_c' yc - zl + zu = 0,   yc - zs = 0,
        c(w) - r = 0,   W1 W2 e - t + s = 0,
        (w - l) zl = mu,   (u - w) zu = mu,   s zs = mu.

    Eliminating the bound multipliers and s as the method does gives the
    reduced matrix of eq. (newtonsystem) with C = diag(0, s/zs): the matrix
    ``scopf_adjoint`` solves with (its rho -> infinity limit).  So the
    solutions these steps converge to are the map whose derivative the
    adjoint computes, and a parameter change of size h moves them by O(h):
    from a nearby solution plain Newton steps (fraction to the boundary
    only) converge quadratically.  Returns (state, residual history); the
    residual is the infinity norm of the conditions above."""
    from .ncl import Params
    S = solver
    P = S.P
    n, m, p = S.n, S.m, S.p
    hard = Params(rho=np.inf, lam_n=np.zeros(m), nu0_n=np.zeros(p))
    st = st.copy()
    hist = []
    for _ in range(max_iter + 1):
        res = S.residuals(st, Params(rho=1.0, lam_n=st.lam, nu0_n=st.yc))
        sl, su = S.slacks(st)
        F = max(np.abs(res["gwz"]).max(), np.abs(res["gs"]).max() if p else 0.0,
                np.abs(res["pc"]).max(), np.abs(res["py"]).max() if p else 0.0,
                np.abs(sl * st.zl - mu).max() if len(sl) else 0.0,
                np.abs(su * st.zu - mu).max() if len(su) else 0.0,
                np.abs(st.s * st.zs - mu).max() if p else 0.0)
        hist.append(float(F))
        if F <= tol or len(hist) > max_iter:
            break
        K = S.kkt_matrix(st, hard, P.hessian(st.w, st.lam), res["J"], 0.0).tocsc()
        rw = res["gw"].copy()
        rw[S.il] -= mu / sl
        rw[S.iu] += mu / su
        b_y = -res["py"] - (mu / st.s - st.yc) * st.s / st.zs
        sol = spla.spsolve(K, np.concatenate([-rw, -res["pc"], b_y]))
        dw, dlam, dyc = sol[:n], sol[n:n + m], sol[n + m:]
        ds = (mu / st.s - st.yc - dyc) * st.s / st.zs
        dzl = mu / sl - st.zl - st.zl / sl * dw[S.il]
        dzu = mu / su - st.zu + st.zu / su * dw[S.iu]
        dzs = mu / st.s - st.zs - st.zs / st.s * ds
        # fraction to the boundary (tau = 0.99) on the positive quantities
        a = 1.0
        for x, dx in ((sl, dw[S.il]), (su, -dw[S.iu]), (st.s, ds), (st.zl, dzl), (st.zu, dzu),
                      (st.zs, dzs)):
            neg = dx < 0
            if np.any(neg):
                a = min(a, float(np.min(-0.99 * x[neg] / dx[neg])))
        st.w = st.w + a * dw
        st.lam = st.lam + a * dlam
        st.yc = st.yc + a * dyc
        st.s = st.s + a * ds
        st.zl = st.zl + a * dzl
        st.zu = st.zu + a * dzu
        st.zs = st.zs + a * dzs
    return st, hist
