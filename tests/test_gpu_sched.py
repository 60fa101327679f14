"""The device schedule of the block factorization and the triangular
sweeps, read back through the scheduler trace: every work item ran exactly
once, and no item started before the items it depends on had finished
(children before parents in the factorization and the forward sweep,
parents before children in the backward sweep).  Also the host-side item
structure (pure CPU)."""
import numpy as np
import pytest

from oracle.ncl import NCLSolver, Params
from oracle.scopf_model import SCOPFModel
from oracle.linsolve import DenseSolver
from tests import helpers as H


@pytest.mark.parametrize("cap", [1, 8, 32])
def test_items_partition_tasks_into_subtrees(cap):
    """Items (host side): parents have larger ids than children; the three
    factorization phases are contiguous and closed upwards; subtrees of
    several fronts only hold tile-sized fronts."""
    import paper_2510_13333_b300 as P
    h = P.SCOPF(H.instance(1), host_only=1, cluster_max_tasks=cap)
    it = h.scopf_trace_items()
    n = len(it)
    assert it[:, 0].min() >= 1 and it[:, 0].max() <= max(cap, 1) or cap == 1
    phase = it[:, 2]
    # phases are contiguous ranges of items, in order, and closed upwards
    assert np.all(np.diff(phase) >= 0) and set(phase.tolist()) <= {1, 2, 3}
    for i in range(n):
        p = it[i, 1]
        if p >= 0:
            assert p > i and phase[p] >= phase[i]
    # only phase-1 items group several fronts, all of them tile-sized
    assert np.all(it[phase > 1, 0] == 1)
    assert np.all(it[phase == 1, 3] <= 32)
    assert np.all(it[phase == 3, 3] > 0)
    if cap > 1:
        assert it[phase == 1, 0].max() > 1


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_schedule_respects_dependencies(cuda, prec):
    import torch
    import paper_2510_13333_b300 as P
    inst = H.instance(1)
    M = SCOPFModel(inst)
    S = NCLSolver(M, DenseSolver())
    st = H.random_interior_state(S, 5)
    rng = np.random.default_rng(6)
    prm = Params(rho=1e3, lam_n=rng.standard_normal(M.m) * 0.1, nu0_n=rng.random(M.p) * 0.1)
    lib = P.SCOPF(inst, cluster_max_tasks=8)
    dst = H.to_device_state(S, st, torch)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    rhs = lib.kkt_assemble(dst, t(prm.lam_n), t(prm.nu0_n), 1e3, 1e-2, 0.3)
    lib.scopf_trace(True)
    lib.kkt_factor(prec)
    lib.kkt_solve(rhs, max_refine=0, check=False)
    torch.cuda.synchronize()
    it = lib.scopf_trace_items()
    n = len(it)
    phase = it[:, 2]
    par = it[:, 1]
    tr = {k: lib.scopf_trace_read(k).astype(np.int64) for k in range(5)}
    lib.scopf_trace(False)
    # every item ran once in the factorization phase it belongs to (kinds
    # 2-4) and in the forward sweep (kind 0)
    for ph in (1, 2, 3):
        ran = tr[1 + ph][:, 1] > 0
        assert np.all(ran[phase == ph]) and not np.any(ran[phase != ph])
    assert np.all(tr[0][:, 1] > 0)
    ran_bwd = tr[1][:, 1] > 0
    for k in range(5):
        ok = tr[k][:, 1] > 0
        assert np.all(tr[k][ok, 0] <= tr[k][ok, 1]) and np.all(tr[k][ok, 1] <= tr[k][ok, 2])
    for i in range(n):
        p = par[i]
        if p < 0:
            continue
        assert phase[p] >= phase[i]
        # factorization: within a phase the parent starts after the child
        # finished (earlier phases end before later ones start)
        if phase[p] == phase[i]:
            k = 1 + phase[i]
            assert tr[k][p, 1] >= tr[k][i, 2]
        assert tr[0][p, 1] >= tr[0][i, 2]
        if ran_bwd[i] and ran_bwd[p]:
            assert tr[1][i, 1] >= tr[1][p, 2]
    # the backward sweep skips exactly the border fronts (one per block)
    assert n - ran_bwd.sum() == len(M.blocks)
