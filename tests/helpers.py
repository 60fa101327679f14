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
