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
