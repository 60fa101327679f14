"""Pins of the oracle's SCOPF model (Section II) to facts outside itself."""
import numpy as np
import pytest

from oracle.scopf_model import SCOPFModel
from tests import helpers as H


def _point(M, seed=0, scale=0.05):
    rng = np.random.default_rng(seed)
    return M.initial_point() + scale * rng.standard_normal(M.n)


def test_balance_equals_complex_injection():
    """Polar balance rows equal -V conj(Y V) built from the bus admittance
    matrix with complex arithmetic (textbook identity), generation and load
    set to zero."""
    inst = H.small_instance()
    net = inst.net
    net.Pd[:] = 0.0
    net.Qd[:] = 0.0
    M = SCOPFModel(inst)
    w = _point(M, 1)
    blk = M.blocks[0]
    w[blk.gq[blk.gens]] = 0.0
    w[M.border0:M.border0 + M.ng] = 0.0
    c = M.constraints(w)
    nb = net.n_bus
    Y = np.zeros((nb, nb), dtype=complex)
    for l in range(net.n_branch):
        y = 1.0 / (net.r[l] + 1j * net.x[l])
        f, t = net.f[l], net.t[l]
        Y[f, f] += y + 0.5j * net.b[l]
        Y[t, t] += y + 0.5j * net.b[l]
        Y[f, t] -= y
        Y[t, f] -= y
    Y[np.diag_indices(nb)] += net.Gs + 1j * net.Bs
    th = np.where(blk.gth >= 0, w[np.maximum(blk.gth, 0)], 0.0)
    V = w[blk.gv] * np.exp(1j * th)
    S = V * np.conj(Y @ V)
    np.testing.assert_allclose(c[blk.grP], -S.real, atol=1e-13)
    np.testing.assert_allclose(c[blk.grQ], -S.imag, atol=1e-13)


def test_line_outage_removes_branch():
    inst = H.small_instance()
    M = SCOPFModel(inst)
    for blk in M.blocks[1:]:
        if blk.kind == 0:
            assert blk.element not in blk.branches
            assert len(blk.branches) == M.nl - 1
        else:
            assert blk.element not in blk.gens


def test_jacobian_finite_differences():
    inst = H.small_instance()
    M = SCOPFModel(inst)
    w = _point(M, 2)
    J = M.jacobian(w).toarray()
    h = 1e-6
    Jfd = np.zeros_like(J)
    for j in range(M.n):
        e = np.zeros(M.n)
        e[j] = h
        Jfd[:, j] = (M.constraints(w + e) - M.constraints(w - e)) / (2 * h)
    assert np.abs(J - Jfd).max() <= 1e-7 * max(1.0, np.abs(J).max())
    # no finite-difference entry outside the stored pattern
    pattern = M.jacobian(w + 0.01).toarray() != 0
    assert not np.any((np.abs(Jfd) > 1e-6) & ~pattern)


def test_hessian_finite_differences():
    inst = H.small_instance()
    M = SCOPFModel(inst)
    w = _point(M, 3)
    rng = np.random.default_rng(4)
    lam = rng.standard_normal(M.m)
    Hm = M.hessian(w, lam).toarray()
    h = 1e-6

    def glag(x):
        return M.gradient(x) + M.jacobian(x).T @ lam

    Hfd = np.zeros_like(Hm)
    for j in range(M.n):
        e = np.zeros(M.n)
        e[j] = h
        Hfd[:, j] = (glag(w + e) - glag(w - e)) / (2 * h)
    assert np.abs(Hm - Hfd).max() <= 1e-6 * max(1.0, np.abs(Hm).max())
    assert np.abs(Hm - Hm.T).max() <= 1e-12 * np.abs(Hm).max()


def test_gradient_finite_differences():
    inst = H.small_instance()
    M = SCOPFModel(inst)
    w = _point(M, 5)
    g = M.gradient(w)
    h = 1e-6
    for j in range(M.border0, M.n):
        e = np.zeros(M.n)
        e[j] = h
        fd = (M.objective(w + e) - M.objective(w - e)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-7 * max(1.0, abs(g[j]))


def test_sizes_per_contingency_same_order_as_paper():
    """Table 2 fits nvar = 3500 + 3725 K, ncon = 4583 + 4917 K for the
    500-bus case; the synthetic 500-bus formulation grows by the same order
    of magnitude per contingency (within a factor 2)."""
    import synthgrid
    c = dict(synthgrid.CONFIGS[2])
    c.pop("name"); c.pop("screen_as", None); c.pop("network_seed_of", None)
    c.update(n_line_ctg=1, n_gen_ctg=1)
    inst = synthgrid.make_instance(seed=1002, **c)
    M = SCOPFModel(inst)
    per_k_var = M.blocks[1].nvar
    per_k_con = M.blocks[1].nrow + M.blocks[1].ncomp
    assert 3725 / 2 <= per_k_var <= 3725 * 2
    assert 4917 / 2 <= per_k_con <= 4917 * 2


def test_droop_rows_are_agc_identity():
    """eq. (droopmpec): when both complementarity multipliers vanish the
    droop row states p^k = p^0 + alpha Delta^k (eq. agc without clipping)."""
    inst = H.small_instance()
    M = SCOPFModel(inst)
    w = M.initial_point()
    blk = M.blocks[1]
    w[blk.gpim] = 0.0
    w[blk.gpip] = 0.0
    w[blk.gdelta] = 0.37
    a = M.alpha(blk)[blk.gens]
    w[blk.gp[blk.gens]] = w[blk.gp0[blk.gens]] + a * 0.37
    c = M.constraints(w)
    assert np.abs(c[blk.grdroop]).max() <= 1e-14
    assert abs(a.sum() - 1.0) <= 1e-14
