"""GPU parity of one Newton step's linear algebra against the oracle:
model values, KKT assembly of eq. (newtonsystem), inertia, solve."""
import numpy as np
import pytest

from oracle.linsolve import DenseSolver, SparseLDLSolver
from oracle.ncl import NCLSolver, Params
from oracle.scopf_model import SCOPFModel
from oracle import symbolic
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _case(inst, seed, rho, delta_w, mu=1e-2, lin=None, lam_scale=1.0, **opt):
    import torch
    import paper_2510_13333_b300 as P
    M = SCOPFModel(inst)
    S = NCLSolver(M, lin or DenseSolver())
    st = H.random_interior_state(S, seed)
    st.lam = st.lam * lam_scale   # large multipliers: negative curvature in H
    rng = np.random.default_rng(seed + 1)
    prm = Params(rho=rho, lam_n=rng.standard_normal(M.m) * 0.1, nu0_n=rng.random(M.p) * 0.1)
    lib = P.SCOPF(inst, **opt)
    dst = H.to_device_state(S, st, torch)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    rhs = lib.kkt_assemble(dst, t(prm.lam_n), t(prm.nu0_n), rho, mu, delta_w)
    gen = H.generic_of_natural(M)
    res = S.residuals(st, prm)
    K_or = S.kkt_matrix(st, prm, M.hessian(st.w, st.lam), res["J"], delta_w).tocsr()
    rhs_or = S.reduced_rhs(st, prm, res, mu)
    return M, S, st, prm, lib, dst, rhs, gen, K_or, rhs_or


@pytest.mark.parametrize("which", ["small", "cfg0"])
def test_model_values(cuda, which):
    import torch
    import paper_2510_13333_b300 as P
    inst = H.small_instance() if which == "small" else H.instance(0)
    M = SCOPFModel(inst)
    lib = P.SCOPF(inst)
    rng = np.random.default_rng(3)
    w = M.initial_point() + 0.03 * rng.standard_normal(M.n)
    obj, g, c = lib.scopf_eval(torch.tensor(w, device="cuda"))
    assert abs(obj - M.objective(w)) <= 1e-13 * max(1.0, abs(obj))
    np.testing.assert_allclose(g.cpu().numpy(), M.gradient(w), rtol=1e-13, atol=1e-13)
    c_or = M.constraints(w)
    np.testing.assert_allclose(c.cpu().numpy(), c_or, rtol=1e-12, atol=1e-12 * np.abs(c_or).max())


@pytest.mark.parametrize("which", ["small", "cfg0", "cfg1"])
def test_kkt_assembly_matches_oracle(cuda, which):
    inst = {"small": H.small_instance, "cfg0": lambda: H.instance(0),
            "cfg1": lambda: H.instance(1)}[which]()
    M, S, st, prm, lib, dst, rhs, gen, K_or, rhs_or = _case(inst, 11, rho=1e3, delta_w=0.3)
    K_lib = H.library_matrix(lib, lib.kkt_values(), gen)
    # per entry: 1e-12 relative plus 1e-14 x the sum of |terms| the entry adds
    # up (FP64 rounding of a sum in another order), so cancelling sums are
    # not held to a bound below their rounding and small entries are checked
    # on their own scale
    H.assert_kkt_terms_close(K_lib, K_or, H.kkt_magnitude(S, st, prm, 0.3))
    # same stored pattern (no entry of one missing from the other)
    assert K_lib.nnz >= K_or.count_nonzero()
    r = np.empty_like(rhs_or)
    r[gen] = rhs.cpu().numpy()
    H.assert_entries_close("rhs", r, rhs_or, 1e-12, 1e-14 * H.rhs_magnitude(S, st, prm, 1e-2))


@pytest.mark.parametrize("which,prec", [("small", 0), ("cfg0", 0), ("cfg0", 1), ("cfg1", 0),
                                        ("cfg1", 1)])
def test_factor_solve_matches_oracle(cuda, which, prec):
    inst = {"small": H.small_instance, "cfg0": lambda: H.instance(0),
            "cfg1": lambda: H.instance(1)}[which]()
    M, S, st, prm, lib, dst, rhs, gen, K_or, rhs_or = _case(inst, 5, rho=1e2, delta_w=1.0)
    perm, _ = symbolic.kkt_permutation(M)
    ora = SparseLDLSolver(perm_fn=lambda K: perm)
    inertia_or = ora.factor(K_or)
    inertia = lib.kkt_factor(prec)
    assert inertia == inertia_or
    x, rel, steps, status = lib.kkt_solve(rhs, max_refine=20)
    assert status == 0 and rel <= 1e-10, (rel, steps)
    x_or = ora.solve(rhs_or)
    xl = np.empty_like(x_or)
    xl[gen] = x.cpu().numpy()
    H.assert_entries_close("solution", xl, x_or, 1e-8, 1e-8 * H.group_scale(M, x_or))


def test_inertia_indefinite(cuda):
    """delta_w = 0 at a random point: A is indefinite; the pivot-free LDL^T
    must report the exact inertia (Sylvester) of K."""
    inst = H.instance(0)
    M, S, st, prm, lib, dst, rhs, gen, K_or, rhs_or = _case(inst, 9, rho=1e2, delta_w=0.0)
    ev = np.linalg.eigvalsh(K_or.toarray())
    expect = (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    assert lib.kkt_factor(0) == expect


@pytest.mark.parametrize("which,prec", [("cfg0", 0), ("cfg0", 1), ("cfg1", 0), ("cfg1", 1)])
def test_condensed_factor_solve_matches_oracle(cuda, which, prec):
    """The condensed primal variant (dual rows eliminated first): the
    library's factorization reports the oracle's inertia (which is
    Haynsworth's In(-C) + In(A + B' C^-1 B)), and the refined solve equals
    the oracle's condensed solve entry by entry."""
    from oracle.linsolve import CondensedSolver
    inst = {"cfg0": lambda: H.instance(0), "cfg1": lambda: H.instance(1)}[which]()
    M, S, st, prm, lib, dst, rhs, gen, K_or, rhs_or = _case(inst, 5, rho=1e2, delta_w=1.0,
                                                            dual_first=1)
    perm, _ = symbolic.kkt_permutation(M, dual_first=True)
    pc = perm[perm < M.n]
    ora = CondensedSolver(M.n, perm_fn=lambda Kc: pc)
    inertia_or = ora.factor(K_or)
    assert lib.kkt_factor(prec) == inertia_or
    x, rel, steps, status = lib.kkt_solve(rhs, max_refine=20)
    assert status == 0 and rel <= 1e-10, (rel, steps)
    x_or = ora.solve(rhs_or)
    xl = np.empty_like(x_or)
    xl[gen] = x.cpu().numpy()
    H.assert_entries_close("solution", xl, x_or, 1e-8, 1e-8 * H.group_scale(M, x_or))


def test_condensed_inertia_wrong_at_small_shift(cuda):
    """delta_w = 0 at a point with large multipliers (negative curvature):
    the condensed matrix is indefinite and the dual-first factorization
    reports K's exact (Sylvester) inertia."""
    inst = H.instance(0)
    M, S, st, prm, lib, dst, rhs, gen, K_or, rhs_or = _case(inst, 9, rho=1e2, delta_w=0.0,
                                                            lam_scale=30.0, dual_first=1)
    ev = np.linalg.eigvalsh(K_or.toarray())
    expect = (int((ev > 0).sum()), int((ev < 0).sum()), 0)
    assert expect != (M.n, M.m + M.p, 0)
    assert lib.kkt_factor(0) == expect


@pytest.mark.parametrize("prec", [0, 1])
def test_equilibration_changes_no_result(cuda, prec):
    """The factorization's Ruiz scales are powers of two, and scaling by a
    power of two is exact in floating point: FP64 factors without scaling
    (zero pivot tolerance) and FP32 factors after one sweep give bit for bit
    the solve of the same factorization after the three sweeps a nonzero
    pivot tolerance keeps (a tolerance below every pivot, so the inertia is
    the same)."""
    import paper_2510_13333_b300 as P
    inst = H.instance(1)
    out = []
    for tol in (0.0, 1e-300):
        M, S, st, prm, lib, dst, rhs, gen, K_or, rhs_or = _case(
            inst, 5, rho=1e3, delta_w=0.5, precision=prec, pivot_tol=tol)
        inertia = lib.kkt_factor()
        x, rel, steps, status = lib.kkt_solve(rhs)
        assert status == 0 and rel <= 1e-10
        out.append((inertia, x.cpu().numpy(), steps))
    (in0, x0, s0), (in1, x1, s1) = out
    assert in0 == in1 and s0 == s1
    assert np.array_equal(x0, x1)
