"""Test helpers: map between the oracle's generic KKT order [w; lam; yc]
and the library's per-block natural order, and build matching states."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import synthgrid
from oracle.scopf_model import SCOPFModel


def instance(idx: int):
    return synthgrid.config_instance(idx)


def small_instance(seed=7, n_bus=14, n_gen=4, n_line=2, n_gen_ctg=1, thermal=True,
                   switch="random", shunts=True):
    inst = synthgrid.make_instance(n_bus=n_bus, mean_degree=2.7, n_gen=n_gen,
                                   n_line_ctg=n_line, n_gen_ctg=n_gen_ctg, thermal=thermal,
                                   switch=switch, seed=seed, load_scale=0.3)
    if shunts:
        inst.net.Gs = np.linspace(0.0, 0.05, inst.net.n_bus)
        inst.net.Bs = np.linspace(0.1, -0.05, inst.net.n_bus)
    return inst


def generic_of_natural(M: SCOPFModel) -> np.ndarray:
    """gen[i] = oracle generic KKT index of natural KKT index i."""
    n_kkt = M.n + M.m + M.p
    gen = np.zeros(n_kkt, dtype=np.int64)
    off = 0
    for blk in M.blocks:
        gen[off:off + blk.nvar] = blk.w0 + np.arange(blk.nvar)
        off += blk.nvar
        gen[off:off + blk.nrow] = M.n + blk.c0 + np.arange(blk.nrow)
        off += blk.nrow
        gen[off:off + blk.ncomp] = M.n + M.m + blk.p0 + np.arange(blk.ncomp)
        off += blk.ncomp
    gen[off:] = M.border0 + np.arange(M.nborder)
    assert off + M.nborder == n_kkt
    return gen


def random_interior_state(solver, seed=0):
    """An interior primal-dual point of the oracle NCL solver (strictly
    inside the relaxed bounds, positive multipliers)."""
    rng = np.random.default_rng(seed)
    st = solver.initial_state()
    n, m, p = solver.n, solver.m, solver.p
    w = st.w.copy()
    sl, su = solver.slacks(st)
    st.w = w
    st.lam = rng.standard_normal(m) * 0.5
    st.yc = rng.random(p) + 0.1
    st.s = rng.random(p) + 0.05
    st.zs = rng.random(p) + 0.1
    st.zl = rng.random(len(solver.il)) + 0.1
    st.zu = rng.random(len(solver.iu)) + 0.1
    st.r = rng.standard_normal(m) * 1e-2
    st.t = rng.random(p) * 1e-2
    return st


def to_device_state(solver, st, torch):
    n = solver.n
    zl = np.zeros(n)
    zu = np.zeros(n)
    zl[solver.il] = st.zl
    zu[solver.iu] = st.zu
    d = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    return dict(w=d(st.w), r=d(st.r), t=d(st.t), s=d(st.s), lam=d(st.lam), yc=d(st.yc),
                zl=d(zl), zu=d(zu), zs=d(st.zs))


def library_matrix(H, vals, gen):
    """Library KKT (natural order CSR) permuted into the oracle's generic order."""
    ptr, col = H.kkt_pattern()
    n = len(ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(ptr))
    return sp.csr_matrix((vals, (gen[rows], gen[col])), shape=(n, n))


def group_scale(M: SCOPFModel, v: np.ndarray) -> np.ndarray:
    """Per entry of a generic-order KKT vector [w; lam; yc]: max |v| over the
    entries of the same scenario block and the same kind (variables,
    equality rows, complementarity rows); the border variables form one
    group.  An absolute tolerance tied to this scale checks small blocks on
    their own scale instead of the largest entry of the whole vector."""
    sc = np.zeros(len(v))
    groups = []
    for blk in M.blocks:
        groups += [(blk.w0, blk.nvar), (M.n + blk.c0, blk.nrow), (M.n + M.m + blk.p0, blk.ncomp)]
    groups.append((M.border0, M.nborder))
    for a, k in groups:
        if k:
            sc[a:a + k] = np.abs(v[a:a + k]).max()
    return sc


def assert_entries_close(name, got, want, rtol, atol):
    """|got - want| <= rtol |want| + atol for every entry (atol may be a
    vector); the message names the worst entry."""
    got = np.asarray(got)
    want = np.asarray(want)
    err = np.abs(got - want)
    bound = rtol * np.abs(want) + atol
    bad = ~(err <= bound)
    if np.any(bad):
        ratio = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), np.inf)
        i = int(np.argmax(np.where(np.isnan(ratio), np.inf, ratio)))
        raise AssertionError(f"{name}: {int(bad.sum())} of {len(err)} entries outside "
                             f"rtol {rtol:g} + atol; worst index {i}: got {got[i]!r}, want "
                             f"{want[i]!r}, err/bound {ratio[i]:.3g}")


def assert_kkt_close(K_lib, K_or, rtol=1e-12, row_atol=1e-15):
    """Every stored entry of either matrix: |K_lib - K_or| <= rtol |K_or| +
    row_atol * (largest |entry| of the oracle's row).  Entries that are
    small next to their row (1/rho, the NCL block, small curvature) are
    checked on their own scale, not on that of the largest entry of K."""
    K_or = sp.csr_matrix(K_or)
    D = (sp.csr_matrix(K_lib) - K_or).tocoo()
    rowmax = np.asarray(abs(K_or).max(axis=1).todense()).ravel()
    want = np.asarray(K_or[D.row, D.col]).ravel()
    assert_entries_close("KKT entries", want + D.data, want, rtol, row_atol * rowmax[D.row])


# ---------------------------------------------------------------------------
# Rounding-error scale of every KKT entry.  An entry of K is a sum of terms
# (curvature of every flow at a bus weighted by its balance multipliers,
# thermal terms, barrier terms); two correct FP64 evaluations that add them
# in different orders, with different (correctly rounded to a few ulp)
# sin/cos, differ by at most a small multiple of u * sum |terms|, however far
# the sum cancels.  These helpers compute sum |terms| per entry by running the
# oracle model's formulas with every term replaced by its absolute value.

def _flow_parts_abs(M, w, blk, lines):
    """|F| bound (4, L), |dF/dx| (4, L, 4) and |d2F/dx2| (4, L, 4, 4) term
    magnitudes of the pi-model arc flows, x = (theta_i, theta_j, v_i, v_j)."""
    f, t, th, vi, vj = M._vals(w, blk, lines)
    A, B, al, be = M._coef(lines)
    c, s = np.abs(np.cos(th)), np.abs(np.sin(th))
    Ta = np.abs(al) * c + np.abs(be) * s          # bounds |T|, |T''| and their rounding
    Tpa = np.abs(al) * s + np.abs(be) * c         # bounds |T'|
    vi, vj = np.abs(vi), np.abs(vj)
    A, B = np.abs(A), np.abs(B)
    F = A * vi ** 2 + B * vj ** 2 + vi * vj * Ta
    L = len(lines)
    G = np.zeros((4, L, 4))
    G[:, :, 0] = vi * vj * Tpa
    G[:, :, 1] = vi * vj * Tpa
    G[:, :, 2] = 2 * A * vi + vj * Ta
    G[:, :, 3] = 2 * B * vj + vi * Ta
    H = np.zeros((4, L, 4, 4))
    for i, j in ((0, 0), (1, 1), (0, 1), (1, 0)):
        H[:, :, i, j] = vi * vj * Ta
    for i, j, v in ((0, 2, vj), (0, 3, vi), (1, 2, vj), (1, 3, vi)):
        H[:, :, i, j] = H[:, :, j, i] = v * Tpa
    H[:, :, 2, 2] = 2 * A
    H[:, :, 3, 3] = 2 * B
    H[:, :, 2, 3] = H[:, :, 3, 2] = Ta
    return F, G, H


def _coo_sum(R, C, V, shape):
    R = np.concatenate(R); C = np.concatenate(C); V = np.concatenate(V)
    keep = (R >= 0) & (C >= 0)
    return sp.csr_matrix((V[keep], (R[keep], C[keep])), shape=shape)


def hessian_magnitude(M: SCOPFModel, w, lam):
    """sum |terms| of every entry of grad^2 phi + sum_i lam_i grad^2 c_i."""
    from oracle.scopf_model import BASE_MVA, OBJ_SCALE
    net = M.net
    R, C, V = [], [], []

    def add(r, c, v):
        r = np.asarray(r).ravel(); c = np.asarray(c).ravel()
        R.append(r); C.append(c); V.append(np.broadcast_to(np.abs(v), r.shape).ravel())

    gp0 = M.border0 + np.arange(M.ng)
    add(gp0, gp0, 2 * net.c2 * BASE_MVA ** 2 / OBJ_SCALE)
    for blk in M.blocks:
        vb = blk.gv
        lP, lQ = np.abs(lam[blk.grP]), np.abs(lam[blk.grQ])
        add(vb, vb, 2 * np.abs(net.Gs) * lP + 2 * np.abs(net.Bs) * lQ)
        lines = blk.branches
        f, t = net.f[lines], net.t[lines]
        _, _, Hf = _flow_parts_abs(M, w, blk, lines)
        X = M._xidx(blk, lines)
        wgt = np.stack([lP[f], lQ[f], lP[t], lQ[t]])
        Hsum = np.einsum("al,alij->lij", wgt, Hf)
        if len(blk.thermal):
            th = blk.thermal
            pos = np.searchsorted(lines, th)
            Ft, Gt, Ht = _flow_parts_abs(M, w, blk, th)
            r2 = net.rate[th] ** 2
            for e, (ip, iq) in enumerate(((0, 1), (2, 3))):
                mu = np.abs(lam[blk.grth[:, e]]) * 2 / r2
                Hth = (np.einsum("li,lj->lij", Gt[ip], Gt[ip]) + Ft[ip][:, None, None] * Ht[ip]
                       + np.einsum("li,lj->lij", Gt[iq], Gt[iq]) + Ft[iq][:, None, None] * Ht[iq])
                Hsum[pos] += mu[:, None, None] * Hth
        for i in range(4):
            for j in range(4):
                add(X[:, i], X[:, j], Hsum[:, i, j])
    return _coo_sum(R, C, V, (M.n, M.n))


def jacobian_magnitude(M: SCOPFModel, w):
    """sum |terms| of every entry of J = dc/dw (linear coefficients count 1)."""
    net = M.net
    Jp = M.jacobian(w).tocsr()
    R, C, V = [], [], []

    def add(r, c, v):
        r = np.asarray(r).ravel(); c = np.asarray(c).ravel()
        R.append(r); C.append(c); V.append(np.broadcast_to(np.abs(v), r.shape).ravel())

    for blk in M.blocks:
        vb = blk.gv
        add(blk.grP, vb, 2 * np.abs(net.Gs * w[vb]))
        add(blk.grQ, vb, 2 * np.abs(net.Bs * w[vb]))
        lines = blk.branches
        _, G, _ = _flow_parts_abs(M, w, blk, lines)
        X = M._xidx(blk, lines)
        f, t = net.f[lines], net.t[lines]
        for a, rows in ((0, blk.grP[f]), (1, blk.grQ[f]), (2, blk.grP[t]), (3, blk.grQ[t])):
            for j in range(4):
                add(rows, X[:, j], G[a, :, j])
        if len(blk.thermal):
            th = blk.thermal
            Ft, Gt, _ = _flow_parts_abs(M, w, blk, th)
            Xt = M._xidx(blk, th)
            r2 = net.rate[th] ** 2
            for e, (ip, iq) in enumerate(((0, 1), (2, 3))):
                for j in range(4):
                    add(blk.grth[:, e], Xt[:, j], 2 * (Ft[ip] * Gt[ip, :, j] + Ft[iq] * Gt[iq, :, j]) / r2)
    Mag = _coo_sum(R, C, V, (M.m, M.n))
    # the remaining entries are single linear coefficients: their own size
    lin = abs(Jp).tocsr()
    return Mag.maximum(lin)


def kkt_magnitude(S, st, prm, delta_w):
    """sum |terms| of every entry of the reduced KKT matrix of eq.
    (newtonsystem) at the oracle state st (same order and blocks as
    NCLSolver.kkt_matrix)."""
    P = S.P
    Hm = hessian_magnitude(P, st.w, st.lam)
    Jm = jacobian_magnitude(P, st.w)
    # the rest of kkt_matrix has no cancelling sums: take it with absolute
    # values from the oracle itself, with H and J replaced by their magnitudes
    Kabs = abs(S.kkt_matrix(st, prm, Hm, Jm, delta_w)).tocsr()
    return Kabs


def assert_kkt_terms_close(K_lib, K_or, Kmag, rtol=1e-12, urel=1e-14):
    """|K_lib - K_or| <= rtol |K_or| + urel * (sum |terms| of the entry) for
    every stored entry of either matrix."""
    K_or = sp.csr_matrix(K_or)
    D = (sp.csr_matrix(K_lib) - K_or).tocoo()
    want = np.asarray(K_or[D.row, D.col]).ravel()
    mag = np.asarray(sp.csr_matrix(Kmag)[D.row, D.col]).ravel()
    assert_entries_close("KKT entries", want + D.data, want, rtol, urel * mag)


def constraints_magnitude(M: SCOPFModel, w):
    """sum |terms| of every equality row c_i(w)."""
    net = M.net
    c = M.constraints(w)
    J = M.jacobian(w).tocsr()
    # linear rows: sum |coef w| plus their constant, taken exactly
    mag = abs(J) @ np.abs(w) + np.abs(c - J @ w)
    for blk in M.blocks:
        P = np.abs(net.Pd) + np.abs(net.Gs) * w[blk.gv] ** 2
        Q = np.abs(net.Qd) + np.abs(net.Bs) * w[blk.gv] ** 2
        np.add.at(P, net.gbus[blk.gens], np.abs(w[blk.gp[blk.gens]]))
        np.add.at(Q, net.gbus[blk.gens], np.abs(w[blk.gq[blk.gens]]))
        lines = blk.branches
        F, _, _ = _flow_parts_abs(M, w, blk, lines)
        for a, ends, tgt in ((0, net.f, P), (1, net.f, Q), (2, net.t, P), (3, net.t, Q)):
            np.add.at(tgt, ends[lines], F[a])
        mag[blk.grP] = P
        mag[blk.grQ] = Q
        if len(blk.thermal):
            Ft, _, _ = _flow_parts_abs(M, w, blk, blk.thermal)
            r2 = net.rate[blk.thermal] ** 2
            for e, (ip, iq) in enumerate(((0, 1), (2, 3))):
                mag[blk.grth[:, e]] = (Ft[ip] ** 2 + Ft[iq] ** 2) / r2 + 1.0 + np.abs(w[blk.gsth[:, e]])
    return mag


def rhs_magnitude(S, st, prm, mu):
    """sum |terms| of every entry of the right-hand side (r1, r2) of eq.
    (newtonsystem) as NCLSolver.reduced_rhs forms it."""
    P = S.P
    n = S.n
    Jm = jacobian_magnitude(P, st.w)
    sl, su = S.slacks(st)
    r1 = np.abs(P.gradient(st.w)) + Jm.T @ np.abs(st.lam)
    np.add.at(r1, S.c1, np.abs(st.yc * st.w[S.c2]))
    np.add.at(r1, S.c2, np.abs(st.yc * st.w[S.c1]))
    r1[S.il] += mu / sl
    r1[S.iu] += mu / su
    rho = prm.rho
    gr = np.abs(prm.lam_n) + rho * np.abs(st.r) + np.abs(st.lam)
    r_lam = constraints_magnitude(P, st.w) + np.abs(st.r) + gr / rho
    gt = np.abs(prm.nu0_n) + rho * np.abs(st.t) + np.abs(st.yc)
    r_y = (np.abs(st.w[S.c1] * st.w[S.c2]) + np.abs(st.t) + np.abs(st.s) + gt / rho
           + (mu / st.s + np.abs(st.yc)) * st.s / st.zs)
    return np.concatenate([r1, r_lam, r_y])
