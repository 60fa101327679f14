"""Parity at the benchmark's full size: the 500-bus network with 256
contingencies (1.64M KKT rows), in the configuration bench.py times (FP32
block factors, the iterate after 30 interior-point iterations).  The
oracle's model and KKT assembly are vectorised and run at this size in
seconds, so every stored entry is compared; the factorization and solve are
checked through properties that hold at any size (the inertia the
correction settles on, the residual of the solve recomputed on the CPU);
and the converged solution is certified by the oracle's own error measure."""
import numpy as np
import pytest

from oracle.linsolve import DenseSolver
from oracle.ncl import NCLSolver, Params, State
from oracle.scopf_model import SCOPFModel
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _oracle_state(S, g):
    return State(w=g["w"], r=g["r"], t=g["t"], s=g["s"], lam=g["lam"], yc=g["yc"],
                 zl=g["zl"][S.il], zu=g["zu"][S.iu], zs=g["zs"])


@pytest.fixture(scope="module")
def bench_iterate():
    import torch
    import paper_2510_13333_b300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    inst = H.instance(2)
    lib = P.SCOPF(inst, precision=P.PREC_MIXED, max_inner=30)
    r = lib.ncl_solve()
    st = lib.get_state()
    lam_n, nu0_n, rho = lib.ncl_params_tensors()
    return inst, lib, st, lam_n, nu0_n, rho, r["mu"], r["delta_w_last"]


def test_fullsize_kkt_matches_oracle(bench_iterate):
    """Every stored entry of K (model values, barrier and NCL blocks,
    delta_w) and every right-hand-side entry at the bench iterate."""
    inst, lib, st, lam_n, nu0_n, rho, mu, dw = bench_iterate
    M = SCOPFModel(inst)
    S = NCLSolver(M, DenseSolver())
    g = {k: v.cpu().numpy() for k, v in st.items()}
    so = _oracle_state(S, g)
    prm = Params(rho=rho, lam_n=lam_n.cpu().numpy(), nu0_n=nu0_n.cpu().numpy())
    rhs = lib.kkt_assemble(st, lam_n, nu0_n, rho, mu, dw)
    res = S.residuals(so, prm)
    K_or = S.kkt_matrix(so, prm, M.hessian(so.w, so.lam), res["J"], dw).tocsr()
    rhs_or = S.reduced_rhs(so, prm, res, mu)
    gen = H.generic_of_natural(M)
    K_lib = H.library_matrix(lib, lib.kkt_values(), gen)
    H.assert_kkt_terms_close(K_lib, K_or, H.kkt_magnitude(S, so, prm, dw))
    r = np.empty_like(rhs_or)
    r[gen] = rhs.cpu().numpy()
    H.assert_entries_close("rhs", r, rhs_or, 1e-12, 1e-14 * H.rhs_magnitude(S, so, prm, mu))


def test_fullsize_step_inertia_and_solve(bench_iterate):
    """The Newton step's inertia correction settles on a delta_w at which the
    factorization reports the inertia (n, m + p, 0) of eq. (newtonsystem);
    the refined solve at that delta_w, multiplied back by K on the CPU in
    FP64, leaves a relative residual below 1e-9."""
    import paper_2510_13333_b300 as P
    inst, lib, st, lam_n, nu0_n, rho, mu, dw = bench_iterate
    out, tries = lib.scopf_newton_step(st, lam_n, nu0_n, rho, mu, dw)
    delta = out[4]
    s = lib.sizes
    rhs = lib.kkt_assemble(st, lam_n, nu0_n, rho, mu, delta)
    assert lib.kkt_factor(P.PREC_MIXED) == (int(s.n), int(s.m + s.p), 0)
    x, rel, steps, status = lib.kkt_solve(rhs)
    assert status == 0 and rel <= 1e-10
    import scipy.sparse as sp
    ptr, col = lib.kkt_pattern()
    K = sp.csr_matrix((lib.kkt_values(), col, ptr), shape=(len(ptr) - 1, len(ptr) - 1))
    b = rhs.cpu().numpy()
    res = K @ x.cpu().numpy() - b
    assert np.abs(res).max() <= 1e-9 * np.abs(b).max()


def certify(inst, lib, r, tol=1e-6):
    """The oracle's certificate of a GPU solution at the point it returned:
    scaled KKT error E_0, NCL relaxations |r|, |t|, violation of eq. (mpcc),
    objective recomputed, complementarity 0 <= w1 perp w2 >= 0, the
    multiplier identities of eq. (kktncl), and strong stationarity (the MPCC
    multipliers nonnegative on the biactive set I_00, eq.
    strongstationarity).  Returns the figures."""
    M = SCOPFModel(inst)
    S = NCLSolver(M, DenseSolver())
    g = {k: v.cpu().numpy() for k, v in lib.get_state().items()}
    so = _oracle_state(S, g)
    lam_n, nu0_n, rho = lib.ncl_params_tensors()
    prm = Params(rho=rho, lam_n=lam_n.cpu().numpy(), nu0_n=nu0_n.cpu().numpy())
    res = S.residuals(so, prm)
    out = {"E0": S.error(so, res, 0.0)[0],
           "rt": max(np.abs(so.r).max(), np.abs(so.t).max()),
           "viol": S.max_violation(so.w, M.constraints(so.w)),
           "obj_err": abs(M.objective(so.w) - r["objective"]) / abs(r["objective"])}
    assert out["E0"] <= tol and out["rt"] <= tol and out["viol"] <= tol, out
    assert out["obj_err"] <= 1e-12, out
    w1, w2 = so.w[S.c1], so.w[S.c2]
    assert np.all(w1 >= -1e-8) and np.all(w2 >= -1e-8)
    assert np.abs(w1 * w2).max() <= tol
    scale = max(1.0, np.abs(so.lam).max())
    assert np.abs(prm.lam_n + prm.rho * so.r - so.lam).max() <= 1e-5 * scale
    assert np.abs(prm.nu0_n + prm.rho * so.t - so.yc).max() <= 1e-5 * scale
    zl = np.zeros(S.n)
    zl[S.il] = so.zl
    mu1 = zl[S.c1] - so.yc * w2
    mu2 = zl[S.c2] - so.yc * w1
    i00 = (w1 <= 1e-5) & (w2 <= 1e-5)
    out["biactive"] = int(i00.sum())
    out["min_mpcc_multiplier"] = float(min(mu1[i00].min(), mu2[i00].min())) if i00.any() else 0.0
    assert out["min_mpcc_multiplier"] >= -1e-4, out
    return out


@pytest.mark.parametrize("prec", [1, 0])
def test_fullsize_solution_certified_by_oracle(prec):
    """A full NCL solve of the benchmark case in each precision, certified
    by the oracle at the returned point.  The two precisions may end at
    different stationary points of this non-convex problem (Section V-C):
    each is certified on its own."""
    import torch
    import paper_2510_13333_b300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    inst = H.instance(2)
    lib = P.SCOPF(inst, precision=prec)
    r = lib.ncl_solve()
    assert r["call_status"] == 0
    out = certify(inst, lib, r)
    print(f"precision {prec}: objective {r['objective']:.9f}, {r['inner_iters']} IPM "
          f"iterations, certificate {out}")
