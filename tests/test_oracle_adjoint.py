"""Pin of the oracle adjoint: directional derivatives of
J = seed' p_g^0 + objective with respect to the loads and the linear costs
match central finite differences of full oracle NCL solves on a small
instance (the sensitivity of the barrier solution differs from the exact
one by O(mu_final), and the difference quotients carry the solves'
tolerance divided by 2h; h = 1e-5)."""
import copy

import numpy as np
import pytest

from oracle.adjoint import scopf_adjoint
from oracle.linsolve import SparseLDLSolver
from oracle.ncl import NCLSolver
from oracle.scopf_model import SCOPFModel
from oracle import symbolic
from tests import helpers as H


def _solve(inst):
    M = SCOPFModel(inst)
    perm, _ = symbolic.kkt_permutation(M)
    S = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm))
    return M, S, S.solve()


@pytest.fixture(scope="module")
def base():
    inst = H.small_instance()
    M, S, r = _solve(inst)
    assert r.status == "ok"
    return inst, M, S, r


@pytest.mark.parametrize("param", ["Pd", "Qd", "c1"])
def test_adjoint_matches_finite_differences(base, param):
    inst, M, S, r = base
    rng = np.random.default_rng({"Pd": 1, "Qd": 2, "c1": 3}[param])
    seed = rng.standard_normal(M.ng)
    gPd, gQd, gc1 = scopf_adjoint(S, r.state, r.params, seed, 1.0)
    grad = {"Pd": gPd, "Qd": gQd, "c1": gc1}[param]
    d = rng.standard_normal(len(grad))
    d /= np.linalg.norm(d)
    h = 1e-5
    vals = []
    for sgn in (1.0, -1.0):
        inst2 = copy.deepcopy(inst)
        setattr(inst2.net, param, getattr(inst.net, param) + sgn * h * d)
        M2, S2, r2 = _solve(inst2)
        assert r2.status == "ok"
        vals.append(float(seed @ r2.state.w[M2.border0:M2.border0 + M2.ng]) + r2.objective)
    fd = (vals[0] - vals[1]) / (2 * h)
    # relative part: O(mu_final) bias of the barrier sensitivity; absolute
    # part: solver tolerance on J (about 1e-10) amplified by 1 / (2 h)
    assert abs(grad @ d - fd) <= 5e-4 * abs(fd) + 2e-5, (grad @ d, fd)


def test_adjoint_zero_seed_is_zero(base):
    inst, M, S, r = base
    gPd, gQd, gc1 = scopf_adjoint(S, r.state, r.params, np.zeros(M.ng), 0.0)
    assert not np.any(gPd) and not np.any(gQd) and not np.any(gc1)


def fd_protocol(inst, directions, h=1e-6, seed_rng=7):
    """The finite-difference protocol of the adjoint check: a solve to 1e-8
    (mu down to 1e-9), then Newton polishing (``polish_barrier``) at that
    final mu with r and t held, to a residual of 1e-12; per direction d
    (seeded N(0, 1), normalised) the same polish at loads Pd +- h d, from the
    base point.  J = seed' p_g^0 + objective.  Returns (oracle solver, base
    point, params, mu, seed, directions, central differences, one-sided
    differences, polish histories)."""
    from oracle.adjoint import polish_barrier
    from oracle.ncl import Options
    M = SCOPFModel(inst)
    perm, _ = symbolic.kkt_permutation(M)
    S = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm), Options(tol=1e-8, mu_min=1e-9))
    base = S.solve()
    assert base.status == "ok"
    st0, hist0 = polish_barrier(S, base.state, base.mu)
    assert hist0[-1] <= 1e-12, hist0
    rng = np.random.default_rng(seed_rng)
    seed = rng.standard_normal(M.ng)

    def J(Pd):
        inst2 = copy.deepcopy(inst)
        inst2.net.Pd = Pd
        S2 = NCLSolver(SCOPFModel(inst2), SparseLDLSolver(perm_fn=lambda K: perm))
        st, hist = polish_barrier(S2, st0, base.mu)
        assert hist[-1] <= 1e-12, hist
        return float(seed @ st.w[M.border0:M.border0 + M.ng]) + S2.P.objective(st.w), hist

    J0 = float(seed @ st0.w[M.border0:M.border0 + M.ng]) + M.objective(st0.w)
    D, fd, one, hists = [], [], [], []
    Pd0 = np.asarray(inst.net.Pd, dtype=float)
    for _ in range(directions):
        d = rng.standard_normal(len(Pd0))
        d /= np.linalg.norm(d)
        (jp, hp), (jm, hm) = J(Pd0 + h * d), J(Pd0 - h * d)
        D.append(d)
        fd.append((jp - jm) / (2 * h))
        one.append(((jp - J0) / h, (J0 - jm) / h))
        hists += [hp, hm]
    return S, st0, base.params, base.mu, seed, np.array(D), np.array(fd), np.array(one), hists


def test_adjoint_fixed_mu_finite_differences():
    """At the final mu, with r and t held, the barrier solution is a smooth
    function of the loads: central differences (h = 1e-6) of Newton-polished
    solutions agree with the adjoint to 1e-6 relative in every direction (J
    is exact to about 1e-13, so the quotient carries about 1e-7).  The polish
    converges quadratically (a few steps from the base point)."""
    S, st0, prm, mu, seed, D, fd, one, hists = fd_protocol(H.small_instance(), 8)
    gPd, _, _ = scopf_adjoint(S, st0, prm, seed, 1.0)
    adj = D @ gPd
    err = np.abs(adj - fd) / np.maximum(np.abs(fd), 1e-3)
    assert err.max() <= 1e-6, (adj, fd)
    assert max(len(hh) for hh in hists) <= 6
