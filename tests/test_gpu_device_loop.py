"""The device-resident Krylov loop (a CUDA graph whose WHILE node repeats
one captured FGMRES step, option device_loop) against the host-driven loop:
the same kernels with the same arithmetic, so the refined solutions, the
step counts and whole NCL solves agree bit for bit."""
import numpy as np
import pytest

from tests import helpers as H
from tests.test_gpu_kkt import _case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_refined_solve_identical(cuda, prec):
    import torch
    import paper_2510_13333_b300 as P
    inst = H.instance(1)
    out = []
    for loop in (0, 1):
        M, S, st, prm, lib, dst, rhs, gen, K_or, rhs_or = _case(inst, 5, rho=1e4, delta_w=1e-2)
        lib2 = P.SCOPF(inst, precision=prec, device_loop=loop)
        t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
        b = lib2.kkt_assemble(dst, t(prm.lam_n), t(prm.nu0_n), prm.rho, 1e-2, 1e-2)
        lib2.kkt_factor(prec)
        lib2.scopf_timing(True)
        x, rel, steps, status = lib2.kkt_solve(b, max_refine=30)
        timed_solves = lib2.scopf_timing(False)["solve"][1]
        out.append((x.cpu().numpy(), rel, steps, status, timed_solves))
    (x0, r0, s0, st0, t0), (x1, r1, s1, st1, t1) = out
    assert st0 == st1 == 0 and s0 == s1 and r0 == r1
    assert np.array_equal(x0, x1)
    # the graph's preconditioner applications run outside the host's phase
    # timers: only the first solve of the call is timed when the graph runs
    # (FP32 factors always need refinement steps here; FP64 ones may not)
    assert t0 == 1 + s0
    if prec == 1:
        assert s0 > 0 and t1 == 1


def test_ncl_solve_identical(cuda):
    import paper_2510_13333_b300 as P
    inst = H.instance(1)
    res = [P.SCOPF(inst, precision=P.PREC_MIXED, device_loop=loop, ipm_graph=0).ncl_solve()
           for loop in (0, 1)]
    a, b = res
    assert a["call_status"] == b["call_status"] == 0
    for k in ("objective", "inner_iters", "factorizations", "refine_steps", "fp64_fallbacks"):
        assert a[k] == b[k], k
