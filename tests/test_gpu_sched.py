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
    """Items (host side): parents have larger ids than children within a
    phase; phase-1 items come first; every block root item has no parent or
    a border item as parent."""
    import paper_2510_13333_b300 as P
    h = P.SCOPF(H.instance(1), host_only=1, cluster_max_tasks=cap)
    it = h.scopf_trace_items()
    n = len(it)
    assert it[:, 0].min() >= 1 and it[:, 0].max() <= max(cap, 1) or cap == 1
    small = it[:, 2] == 1
    # phase-1 items form a prefix
    assert not np.any(np.diff(small.astype(int)) > 0)
    for i in range(n):
        p = it[i, 1]
        if p >= 0:
            assert p > i
            if not small[i]:
                assert not small[p]
    if cap > 1:
        assert it[small, 0].max() > 1


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
    small = it[:, 2] == 1
    par = it[:, 1]
    tr = {k: lib.scopf_trace_read(k).astype(np.int64) for k in range(4)}
    lib.scopf_trace(False)
    # every item ran once in each sweep it belongs to
    assert np.all(tr[2][small, 1] > 0) and np.all(tr[2][~small, 1] == 0)
    assert np.all(tr[3][~small, 1] > 0) and np.all(tr[3][small, 1] == 0)
    assert np.all(tr[0][:, 1] > 0)
    ran_bwd = tr[1][:, 1] > 0
    for k in range(4):
        ok = tr[k][:, 1] > 0
        assert np.all(tr[k][ok, 0] <= tr[k][ok, 1]) and np.all(tr[k][ok, 1] <= tr[k][ok, 2])
    for i in range(n):
        p = par[i]
        if p < 0:
            continue
        # factorization: the parent starts after the child finished
        if small[i] and small[p]:
            assert tr[2][p, 1] >= tr[2][i, 2]
        if not small[i]:
            assert tr[3][p, 1] >= tr[3][i, 2]
        assert tr[0][p, 1] >= tr[0][i, 2]
        if ran_bwd[i] and ran_bwd[p]:
            assert tr[1][i, 1] >= tr[1][p, 2]
    # the backward sweep skips exactly the border fronts (one per block)
    assert n - ran_bwd.sum() == len(M.blocks)
