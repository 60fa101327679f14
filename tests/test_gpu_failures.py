"""Failure detection on the GPU without a fault: every device-side wait is
bounded and turns into a status the host reads, a refinement that cannot
reach its target says so, and the interior-point method's FP64 fallback
takes over from stalled FP32 refinement.  Nothing here traps, faults or
hangs: the waits run out because their limit is zero."""
import numpy as np
import pytest

from oracle.linsolve import SparseLDLSolver
from oracle.ncl import NCLSolver, Params
from oracle.scopf_model import SCOPFModel
from oracle import symbolic
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _assembled(lib, inst, torch, delta_w=1.0, mu=0.1):
    """Assemble K at the oracle's starting point of the 30-bus workload."""
    M = SCOPFModel(inst)
    perm, _ = symbolic.kkt_permutation(M)
    S = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm))
    st = S.initial_state()
    prm = Params(rho=S.o.rho_init, lam_n=np.zeros(M.m), nu0_n=np.zeros(M.p))
    d = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    b = lib.kkt_assemble(H.to_device_state(S, st, torch), d(prm.lam_n), d(prm.nu0_n), prm.rho,
                         mu, delta_w)
    return b


@pytest.mark.parametrize("prec", [0, 1])
def test_exhausted_waits_report_timeout(cuda, prec):
    """With a wait limit of zero, workers that find their queue slot still
    empty give up at once: the factorization and the solve end with
    SCOPF_ERR_TIMEOUT (-8) instead of waiting, and the context stays usable
    (a handle with the default limit then factors and solves normally)."""
    import torch
    import paper_2510_13333_b300 as P
    inst = H.instance(0)
    lib = P.SCOPF(inst, precision=prec, spin_limit=0)
    b = _assembled(lib, inst, torch)
    with pytest.raises(P.ScopfError) as e:
        lib.kkt_factor()
    assert e.value.status == -8
    torch.cuda.synchronize()
    ok = P.SCOPF(inst, precision=prec)
    b = _assembled(ok, inst, torch)
    ok.kkt_factor()
    x, rel, steps, st = ok.kkt_solve(b)
    assert st == 0 and rel <= 1e-10


def test_capped_refinement_reports_stall(cuda):
    """FP32 block factors alone leave a residual far above the 1e-10 target:
    with no refinement step allowed, kkt_solve says so (-5); with its
    default budget it reaches the target."""
    import torch
    import paper_2510_13333_b300 as P
    inst = H.instance(0)
    lib = P.SCOPF(inst, precision=P.PREC_MIXED)
    b = _assembled(lib, inst, torch)
    lib.kkt_factor()
    _, rel0, steps0, st0 = lib.kkt_solve(b, max_refine=0)
    assert st0 == -5 and steps0 == 0 and rel0 > 1e-10
    _, rel, steps, st = lib.kkt_solve(b)
    assert st == 0 and rel <= 1e-10 and steps > 0


def test_stalled_fp32_refinement_falls_back_to_fp64(cuda):
    """With refinement switched off, the first mixed-precision Newton step
    stalls; the method redoes it with FP64 factors and stays there (one
    fallback), and the solve converges to the FP64 solve's objective."""
    import paper_2510_13333_b300 as P
    inst = H.instance(0)
    mixed = P.SCOPF(inst, precision=P.PREC_MIXED, max_refine=0).ncl_solve()
    fp64 = P.SCOPF(inst, precision=P.PREC_FP64, max_refine=0).ncl_solve()
    assert mixed["call_status"] == 0 and fp64["call_status"] == 0
    assert mixed["fp64_fallbacks"] == 1 and fp64["fp64_fallbacks"] == 0
    assert abs(mixed["objective"] - fp64["objective"]) <= 1e-6 * abs(fp64["objective"])


def test_cost_switch_to_fp64(cuda):
    """With the refinement-cost switch set to one step, the first mixed
    Newton step that needs refinement moves the solve to FP64 factors (one
    switch), the solve converges to the FP64 solve's objective, and the
    iteration log shows FP32 factors only before the switch."""
    import paper_2510_13333_b300 as P
    inst = H.instance(0)
    lib = P.SCOPF(inst, precision=P.PREC_MIXED, fp64_switch_refine=1, fp64_switch_streak=1)
    r = lib.ncl_solve()
    ref = P.SCOPF(inst, precision=P.PREC_FP64).ncl_solve()
    assert r["call_status"] == 0 and r["fp64_fallbacks"] == 1
    assert abs(r["objective"] - ref["objective"]) <= 1e-6 * abs(ref["objective"])
    names, log = lib.history(0)
    prec = log[:, names.index("precision")]
    first64 = int(np.argmax(prec == 0))
    assert prec[first64] == 0 and np.all(prec[:first64] == 1) and np.all(prec[first64:] == 0)
