"""The C-ABI library loads, exports every entry point of include/scopf.h, and
(host-only handle, no GPU) its symbolic analysis is bit-exact with the
oracle's."""
import ctypes

import numpy as np
import pytest

import paper_2510_13333_b300 as P
from oracle.scopf_model import SCOPFModel
from oracle import symbolic
from tests import helpers as H


def test_library_exports_header_symbols():
    names = P.exported_symbols()
    assert len(names) >= 15
    lib = ctypes.CDLL(P.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options_match_oracle():
    from oracle.ncl import Options
    o = P.default_options()
    ref = Options()
    for name in ("tol", "mu_min", "mu_init", "kappa_eps", "kappa_mu", "theta_mu", "tau_min",
                 "s_max", "kappa_sigma", "bound_relax", "bound_push", "bound_frac", "slack_init",
                 "comp_init", "delta_w0", "delta_w_min", "delta_w_max", "kappa_w_minus",
                 "kappa_w_plus", "kappa_w_plus_bar", "gamma_theta", "gamma_phi", "delta_sw",
                 "s_theta", "s_phi", "eta_phi", "gamma_alpha", "rho_init", "rho_max", "eta_init",
                 "omega_init", "max_backtrack", "max_outer", "max_inner"):
        assert getattr(o, name) == getattr(ref, name), name


def test_invalid_network_rejected():
    inst = H.small_instance()
    inst.net.f = inst.net.f.copy()
    inst.net.f[0] = inst.net.n_bus + 5
    with pytest.raises(P.ScopfError):
        P.SCOPF(inst, host_only=1)


@pytest.mark.parametrize("rmf,dual_first", [(0, 0), (32, 0), (0, 1), (32, 1)])
@pytest.mark.parametrize("which", ["small", "cfg0", "cfg1"])
def test_symbolic_bit_exact(which, rmf, dual_first):
    inst = {"small": H.small_instance, "cfg0": lambda: H.instance(0),
            "cfg1": lambda: H.instance(1)}[which]()
    M = SCOPFModel(inst)
    lib = P.SCOPF(inst, host_only=1, relax_max_front=rmf, dual_first=dual_first)
    assert lib.sizes.n_kkt == M.n + M.m + M.p
    assert lib.sizes.n == M.n and lib.sizes.m == M.m and lib.sizes.p == M.p
    gen = H.generic_of_natural(M)
    _, syms = symbolic.kkt_permutation(M, relax_max_front=rmf, dual_first=bool(dual_first))
    for k, S in enumerate(syms):
        c = lib.scopf_symbolic_block(k)
        assert np.array_equal(c["post"], S.post), k
        assert np.array_equal(c["node_parent"], S.parent), k
        assert np.array_equal(c["sn_start"], S.sn_start), k
        assert np.array_equal(gen[c["rows"]], S.rows), k


@pytest.mark.parametrize("rmn", [4, 16])
def test_symbolic_bit_exact_amalgamation_limits(rmn):
    """The autotuner's amalgamation limits (relax_max_nodes) keep the
    analysis bit-exact with the oracle's."""
    inst = H.instance(1)
    M = SCOPFModel(inst)
    lib = P.SCOPF(inst, host_only=1, relax_max_nodes=rmn)
    gen = H.generic_of_natural(M)
    _, syms = symbolic.kkt_permutation(M, relax_max_nodes=rmn)
    for k, S in enumerate(syms):
        c = lib.scopf_symbolic_block(k)
        assert np.array_equal(c["post"], S.post), k
        assert np.array_equal(c["sn_start"], S.sn_start), k
        assert np.array_equal(gen[c["rows"]], S.rows), k


def test_kkt_pattern_matches_oracle():
    inst = H.small_instance()
    M = SCOPFModel(inst)
    lib = P.SCOPF(inst, host_only=1)
    ptr, col = lib.kkt_pattern()
    gen = H.generic_of_natural(M)
    n = len(ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(ptr))
    lib_pat = set(zip(gen[rows].tolist(), gen[col].tolist()))
    K = symbolic.structural_kkt(M).tocoo()
    ora_pat = {(i, j) for i, j, v in zip(K.row.tolist(), K.col.tolist(), K.data.tolist()) if v != 0}
    assert ora_pat <= lib_pat
    # the library stores no structurally absent entry beyond zero-valued shunt terms
    assert len(lib_pat - ora_pat) <= 4 * inst.net.n_bus * (len(inst.ctgs) + 1)


def test_history_empty_before_a_solve():
    """The iteration log exists on a host-only handle and is empty until a
    solve has run; its record lengths match the documented fields."""
    import paper_2510_13333_b300 as P
    h = P.SCOPF(H.instance(0), host_only=1)
    names, rows = h.history(0)
    assert rows.shape == (0, 16) and len(names) == 16
    names, rows = h.history(1)
    assert rows.shape == (0, 8) and len(names) == 8


def test_symbolic_bit_exact_full_size_sampled_blocks():
    """The 500-bus x 256 workload of the benchmark: the symbolic analysis of
    the base case and of sampled contingency blocks equals the oracle's bit
    for bit (each block's analysis depends only on its own graph)."""
    inst = H.instance(2)
    M = SCOPFModel(inst)
    lib = P.SCOPF(inst, host_only=1)
    gen = H.generic_of_natural(M)
    graphs = symbolic.attach_adjacency(symbolic.block_graphs(M), symbolic.structural_kkt(M))
    for k in (0, 1, 37, 128, 221, len(graphs) - 1):
        S = symbolic.Symbolic(graphs[k])
        c = lib.scopf_symbolic_block(k)
        assert np.array_equal(c["post"], S.post), k
        assert np.array_equal(c["node_parent"], S.parent), k
        assert np.array_equal(c["sn_start"], S.sn_start), k
        assert np.array_equal(gen[c["rows"]], S.rows), k
