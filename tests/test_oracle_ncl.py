"""Pins of the oracle's NCL / interior-point solver: closed-form toys and
optimality certificates of the SCOPF solution (Sections II-IV)."""
import numpy as np
import pytest

from oracle.linsolve import DenseSolver, SparseLDLSolver
from oracle.ncl import NCLSolver, Options
from oracle.scopf_model import SCOPFModel
from oracle import symbolic
from oracle.toys import ToyInfeasible, ToyMPCC, ToyQP
from tests import helpers as H


def test_toy_mpcc_two_minima():
    """min (x-1)^2 + (y-1)^2, 0 <= x perp y >= 0: optimum 1 at (1,0) or (0,1)."""
    for x0 in ((0.5, 0.5), (0.9, 0.2), (0.2, 0.9)):
        r = NCLSolver(ToyMPCC("quadratic", x0=x0), DenseSolver()).solve()
        assert r.status == "ok"
        assert abs(r.objective - 1.0) <= 1e-5
        x, y = r.state.w
        assert min(abs(x - 1) + abs(y), abs(x) + abs(y - 1)) <= 1e-5


def test_toy_mpcc_degenerate_origin():
    """min x + y on the complementarity set: (0,0), where I_00 is nonempty and
    the rows (0 W2 W1) of B vanish; C keeps the Newton system nonsingular."""
    S = NCLSolver(ToyMPCC("linear"), DenseSolver())
    r = S.solve()
    assert r.status == "ok"
    assert np.abs(r.state.w).max() <= 1e-5
    # at the solution the complementarity row of B is ~0 (rank loss), yet the
    # reduced Newton matrix is nonsingular thanks to C (Section IV-B)
    st, prm = r.state, r.params
    res = S.residuals(st, prm)
    K = S.kkt_matrix(st, prm, S.P.hessian(st.w, st.lam), res["J"], 0.0).toarray()
    assert np.abs(K[2, :2]).max() <= 1e-5
    sv = np.linalg.svd(K, compute_uv=False)
    assert sv.min() >= 0.5 / prm.rho   # bounded below by the C block (1/rho + s/zs)


def test_toy_infeasible_feasibility_problem():
    """c(x) = x^2 + 1 = 0: rho diverges and the iterate approaches the
    minimiser x = 0, r = 1 of the feasibility problem (eq. feaspb)."""
    r = NCLSolver(ToyInfeasible(), DenseSolver()).solve()
    assert r.status == "infeasible"
    assert r.params.rho > 1e10
    assert abs(r.state.r[0] - 1.0) <= 1e-5
    assert abs(r.state.w[0]) <= 1e-3


def test_convex_qp_equals_kkt_solution():
    P = ToyQP(n=6, m=2, seed=0)
    r = NCLSolver(P, SparseLDLSolver()).solve()
    x, _ = P.exact()
    assert r.status == "ok"
    np.testing.assert_allclose(r.state.w, x, atol=1e-6)


@pytest.fixture(scope="module")
def cfg0_solution():
    inst = H.instance(0)
    M = SCOPFModel(inst)
    perm, _ = symbolic.kkt_permutation(M)
    S = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm))
    return inst, M, S, S.solve()


def test_cfg0_converges(cfg0_solution):
    inst, M, S, r = cfg0_solution
    assert r.status == "ok"
    assert r.kkt_error <= 1e-6
    assert r.feas_rt <= 1e-6
    assert r.max_violation <= 1e-6


def test_cfg0_multiplier_identities(cfg0_solution):
    """eq. (kktncl): lam = lam^(n) + rho r and nu0 = nu0^(n) + rho t."""
    inst, M, S, r = cfg0_solution
    st, prm = r.state, r.params
    scale = max(1.0, np.abs(st.lam).max())
    assert np.abs(prm.lam_n + prm.rho * st.r - st.lam).max() <= 1e-5 * scale
    assert np.abs(prm.nu0_n + prm.rho * st.t - st.yc).max() <= 1e-5 * scale


def test_cfg0_droop_clip_identity(cfg0_solution):
    """eq. (agc): p^k = min(max(p^0 + alpha Delta^k, pmin), pmax)."""
    inst, M, S, r = cfg0_solution
    w = r.state.w
    net = inst.net
    for blk in M.blocks[1:]:
        g = blk.gens
        a = M.alpha(blk)[g]
        target = np.clip(w[blk.gp0[g]] + a * w[blk.gdelta], net.pmin[g], net.pmax[g])
        # complementarity holds to products ~mu_min = 1e-7; at a biactive pair
        # each factor (pi, distance to the limit) is then ~sqrt(1e-7) ~ 3e-4
        assert np.abs(w[blk.gp[g]] - target).max() <= 2e-3


def test_cfg0_pvpq_logic(cfg0_solution):
    """eq. (pvpq): v^k = v^0 unless q^k sits at a limit; a drop (rise) of
    v^k needs q^k at its upper (lower) limit."""
    inst, M, S, r = cfg0_solution
    w = r.state.w
    net = inst.net
    for blk in M.blocks[1:]:
        for b, g in zip(blk.switch, blk.sw_gen):
            dv = w[blk.gv[b]] - w[blk.gv0[b]]
            q = w[blk.gq[g]]
            if dv < -1e-4:
                assert q >= net.qmax[g] - 1e-4
            elif dv > 1e-4:
                assert q <= net.qmin[g] + 1e-4
            if net.qmin[g] + 1e-3 < q < net.qmax[g] - 1e-3:
                assert abs(dv) <= 1e-4


def test_cfg0_complementarity_and_stationarity(cfg0_solution):
    """0 <= w1 perp w2 >= 0 at the solution; on the biactive set I_00 the
    MPCC multipliers (bound multipliers corrected by the coupling) are
    nonnegative (strong stationarity, eq. strongstationarity)."""
    inst, M, S, r = cfg0_solution
    st = r.state
    w1, w2 = st.w[S.c1], st.w[S.c2]
    assert np.all(w1 >= -1e-8) and np.all(w2 >= -1e-8)
    assert np.abs(w1 * w2).max() <= 1e-6
    zl = np.zeros(S.n)
    zl[S.il] = st.zl
    mu1 = zl[S.c1] - st.yc * w2
    mu2 = zl[S.c2] - st.yc * w1
    i00 = (w1 <= 1e-5) & (w2 <= 1e-5)
    assert np.all(mu1[i00] >= -1e-4) and np.all(mu2[i00] >= -1e-4)


def test_scopf_cost_not_below_opf():
    """Adding contingencies only restricts u0: the SCOPF optimum is not
    cheaper than the base-case OPF optimum (Table 2's objective grows with K)."""
    from oracle.screening import base_opf
    inst = H.instance(0)
    res, _ = base_opf(inst)
    M = SCOPFModel(inst)
    perm, _ = symbolic.kkt_permutation(M)
    r = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm)).solve()
    assert res.status == "ok" and r.status == "ok"
    assert r.objective >= res.objective - 1e-6
