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
