"""The ill-conditioning study (Section V-C: q_min close to q_max in eq. pvpq
makes the method ill-conditioned): on the 118-bus x 32 case the generators'
reactive bands are narrowed around the base-case reactive output of the
oracle's unstressed solution, and the library's solves in both precisions
are certified by the oracle at the points they return."""
import numpy as np
import pytest

from oracle import symbolic
from oracle.linsolve import SparseLDLSolver
from oracle.ncl import NCLSolver
from oracle.scopf_model import SCOPFModel
from tests import helpers as H
from tests.test_gpu_fullsize import certify

pytestmark = pytest.mark.gpu

_Q0 = {}


def narrowed(delta):
    """The 118-bus instance with every band [max(q_min, q* - delta w),
    min(q_max, q* + delta w)], w = (q_max - q_min) / 2, q* the base-case
    reactive output of the oracle's solution of the unstressed case."""
    if "q0" not in _Q0:
        M = SCOPFModel(H.instance(1))
        perm, _ = symbolic.kkt_permutation(M)
        r = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm)).solve()
        assert r.status == "ok"
        b0 = M.blocks[0]
        _Q0["q0"] = np.array([r.state.w[b0.gq[g]] for g in range(M.ng)])
    base = H.instance(1)
    inst = H.instance(1)
    half = 0.5 * (base.net.qmax - base.net.qmin)
    inst.net.qmin = np.maximum(base.net.qmin, _Q0["q0"] - delta * half)
    inst.net.qmax = np.minimum(base.net.qmax, _Q0["q0"] + delta * half)
    return inst


@pytest.mark.parametrize("delta", [0.1, 0.03])
@pytest.mark.parametrize("prec", [1, 0])
def test_narrow_reactive_bands_certified(cuda, delta, prec):
    import paper_2510_13333_b300 as P
    inst = narrowed(delta)
    assert np.all(inst.net.qmax - inst.net.qmin <= 2 * delta * 0.5 *
                  (H.instance(1).net.qmax - H.instance(1).net.qmin) + 1e-12)
    lib = P.SCOPF(inst, precision=prec)
    r = lib.ncl_solve()
    assert r["call_status"] == 0, r
    out = certify(inst, lib, r)
    print(f"delta {delta}, precision {prec}: {r['inner_iters']} IPM iterations, "
          f"{r['factorizations'] / r['inner_iters']:.2f} factorizations and "
          f"{r['refine_steps'] / r['inner_iters']:.1f} refinement steps per iteration, "
          f"certificate {out}")
