"""Python binding of the B300 SCOPF / NCL Newton-step library (ctypes).

Argument marshalling only: every step of the method runs in the CUDA
library ``libscopf_b300.so`` built from ``csrc/`` (see ``build.py``).  If the
library cannot be loaded, importing the entry points raises -- there is no
fallback.  PyTorch supplies device memory and the CUDA stream.

The function names follow the C ABI of ``include/scopf.h``:
``scopf_create``, ``kkt_assemble``, ``kkt_factor``, ``kkt_solve``,
``ncl_solve``, ``scopf_adjoint`` ...; ``SCOPF`` bundles them around a handle.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libscopf_b300.so")

c_i32, c_i64, c_dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
P_i32 = ctypes.POINTER(c_i32)
P_i64 = ctypes.POINTER(c_i64)
P_dbl = ctypes.POINTER(c_dbl)

PREC_FP64 = 0
PREC_MIXED = 1

STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "not factored",
          -4: "wrong inertia", -5: "refinement stalled", -6: "infeasible", -7: "max iter",
          -8: "timeout", -9: "out of memory", -10: "numerical failure"}


class ScopfError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)} ({status})")
        self.status = status


class Network(ctypes.Structure):
    _fields_ = [("n_bus", c_i32), ("n_branch", c_i32), ("n_gen", c_i32), ("ref_bus", c_i32),
                ("Pd", P_dbl), ("Qd", P_dbl), ("Gs", P_dbl), ("Bs", P_dbl), ("vmin", P_dbl),
                ("vmax", P_dbl), ("br_from", P_i32), ("br_to", P_i32), ("br_r", P_dbl),
                ("br_x", P_dbl), ("br_b", P_dbl), ("br_rate", P_dbl), ("gen_bus", P_i32),
                ("pmin", P_dbl), ("pmax", P_dbl), ("qmin", P_dbl), ("qmax", P_dbl), ("c2", P_dbl),
                ("c1", P_dbl), ("c0", P_dbl)]


class Contingency(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("element", c_i32), ("n_switch", c_i32),
                ("switch_buses", P_i32)]


_OPT_DOUBLES = ["tol", "mu_min", "mu_init", "kappa_eps", "kappa_mu", "theta_mu", "tau_min",
                "s_max", "kappa_sigma", "bound_relax", "bound_push", "bound_frac", "slack_init",
                "comp_init", "delta_w0", "delta_w_min", "delta_w_max", "kappa_w_minus",
                "kappa_w_plus", "kappa_w_plus_bar", "gamma_theta", "gamma_phi", "delta_sw",
                "s_theta", "s_phi", "eta_phi", "gamma_alpha", "rho_init", "rho_max", "eta_init",
                "omega_init", "refine_tol", "pivot_tol"]
_OPT_INTS = ["max_backtrack", "max_outer", "max_inner", "max_refine", "precision",
             "relax_max_nodes", "verbose", "spin_limit", "host_only", "cluster_max_tasks",
             "relax_max_front", "device_loop", "fp64_switch_refine", "fp64_switch_streak",
             "known_zero_pivot", "dual_first", "fixed_mu", "ipm_graph"]


class Options(ctypes.Structure):
    _fields_ = [(n, c_dbl) for n in _OPT_DOUBLES] + [(n, c_i32) for n in _OPT_INTS]


class TuneEntry(ctypes.Structure):
    _fields_ = [("cluster_max_tasks", c_i32), ("relax_max_nodes", c_i32),
                ("ms_per_step", c_dbl), ("chosen", c_i32)]


class Sizes(ctypes.Structure):
    _fields_ = [("n", c_i64), ("m", c_i64), ("p", c_i64), ("n_kkt", c_i64), ("n_border", c_i64),
                ("n_blocks", c_i32), ("nnz_kkt", c_i64), ("nnz_L", c_i64),
                ("n_supernodes", c_i64), ("factor_flops", c_dbl), ("front_bytes", c_i64),
                ("n_elem_values", c_i64), ("n_contrib", c_i64)]


_STATE_FIELDS = ["w", "r", "t", "s", "lam", "yc", "zl", "zu", "zs"]


class State(ctypes.Structure):
    _fields_ = [(n, P_dbl) for n in _STATE_FIELDS]


class Result(ctypes.Structure):
    _fields_ = [("status", c_i32), ("outer_iters", c_i32), ("inner_iters", c_i32),
                ("factorizations", c_i32), ("refine_steps", c_i32), ("fp64_fallbacks", c_i32),
                ("objective", c_dbl), ("kkt_error", c_dbl), ("feas_rt", c_dbl),
                ("max_violation", c_dbl), ("rho", c_dbl), ("mu", c_dbl),
                ("time_total_s", c_dbl), ("time_newton_s", c_dbl), ("delta_w_last", c_dbl),
                ("host_round_trips", c_i64), ("graph_iters", c_i32), ("pad", c_i32)]


_LIB = None
_CUDART = None


def _cudart():
    """The CUDA runtime already loaded by the library (for device copies of
    handle-owned buffers)."""
    global _CUDART
    if _CUDART is None:
        lib()
        import glob
        cands = glob.glob("/usr/local/cuda/lib64/libcudart.so*")
        _CUDART = ctypes.CDLL(cands[0] if cands else "libcudart.so")
        _CUDART.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        _CUDART.cudaMemcpy.restype = ctypes.c_int
    return _CUDART


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with "
                              "`python -m paper_2510_13333_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        H = ctypes.c_void_p
        sig = {
            "scopf_default_options": (None, [ctypes.POINTER(Options)]),
            "scopf_create": (c_i32, [ctypes.POINTER(Network), ctypes.POINTER(Contingency), c_i32,
                                     ctypes.POINTER(Options), ctypes.POINTER(H)]),
            "scopf_destroy": (None, [H]),
            "scopf_strerror": (ctypes.c_char_p, [c_i32]),
            "scopf_last_error": (ctypes.c_char_p, [H]),
            "scopf_get_sizes": (c_i32, [H, ctypes.POINTER(Sizes)]),
            "scopf_set_stream": (c_i32, [H, ctypes.c_void_p]),
            "scopf_set_precision": (c_i32, [H, c_i32]),
            "scopf_symbolic_block": (c_i32, [H, c_i32, P_i32, P_i32, P_i32, P_i32, P_i32, P_i32,
                                             P_i32, P_i64]),
            "scopf_eval": (c_i32, [H, P_dbl, P_dbl, P_dbl, P_dbl]),
            "kkt_assemble": (c_i32, [H, ctypes.POINTER(State), P_dbl, P_dbl, c_dbl, c_dbl, c_dbl,
                                     P_dbl]),
            "kkt_export": (c_i32, [H, P_i64, P_i64, P_dbl]),
            "kkt_factor": (c_i32, [H, c_i32, P_i32]),
            "kkt_solve": (c_i32, [H, P_dbl, P_dbl, c_i32, P_dbl, P_i32]),
            "ncl_solve": (c_i32, [H, ctypes.POINTER(State), ctypes.POINTER(Result)]),
            "ncl_resume": (c_i32, [H, ctypes.POINTER(Result)]),
            "scopf_get_state": (c_i32, [H, ctypes.POINTER(State)]),
            "scopf_copy_state": (c_i32, [H, ctypes.POINTER(State)]),
            "scopf_load_state": (c_i32, [H, ctypes.POINTER(State)]),
            "scopf_get_ncl_params": (c_i32, [H, ctypes.POINTER(P_dbl), ctypes.POINTER(P_dbl),
                                             P_dbl]),
            "scopf_adjoint": (c_i32, [H, P_dbl, c_dbl, P_dbl, P_dbl, P_dbl]),
            "scopf_set_params": (c_i32, [H, P_dbl, P_dbl, P_dbl]),
            "scopf_set_ncl_params": (c_i32, [H, P_dbl, P_dbl, c_dbl, c_dbl]),
            "scopf_block_violation": (c_i32, [H, P_dbl]),
            "scopf_history": (c_i32, [H, c_i32, c_i64, P_dbl, P_i64, P_i32]),
            "scopf_screen": (c_i32, [H, P_dbl, c_dbl, c_dbl, c_dbl, ctypes.POINTER(Result), P_dbl,
                                     P_i32]),
            "scopf_newton_step": (c_i32, [H, ctypes.POINTER(State), P_dbl, P_dbl, c_dbl, c_dbl,
                                          c_dbl, ctypes.POINTER(State), P_dbl, P_i32]),
            "scopf_timing": (c_i32, [H, c_i32, P_dbl, P_i32]),
            "scopf_trace": (c_i32, [H, c_i32]),
            "scopf_launch_count": (c_i32, [P_i64]),
            "scopf_trace_read": (c_i32, [H, c_i32, ctypes.POINTER(ctypes.c_uint64)]),
            "scopf_trace_items": (c_i32, [H, P_i32, P_i32]),
            "scopf_dense_ldlt_solve": (c_i32, [P_dbl, c_i32, P_dbl, P_dbl, P_i32, ctypes.c_void_p]),
            "scopf_dense_ldlt_solve_noalloc": (c_i32, [P_dbl, c_i32, P_dbl, P_dbl, P_i32,
                                                       ctypes.c_void_p]),
            "scopf_peak_probe": (c_i32, [c_i32, c_i64, P_dbl, ctypes.c_void_p, P_dbl]),
            "scopf_pivot_reciprocal": (c_i32, [P_dbl, P_dbl, c_i64, ctypes.c_void_p]),
            "scopf_autotune": (c_i32, [ctypes.POINTER(Network), ctypes.POINTER(Contingency),
                                       c_i32, ctypes.POINTER(Options), c_i32, c_i32, c_i32,
                                       ctypes.POINTER(TuneEntry), P_i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def exported_symbols():
    """Names declared by include/scopf.h that the library must export."""
    import re
    hdr = open(os.path.join(_HERE, "..", "include", "scopf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?(\w+)\(", hdr, re.M)))


def scopf_launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    n = ctypes.c_int64()
    _check("scopf_launch_count", lib().scopf_launch_count(ctypes.byref(n)))
    return n.value


def scopf_dense_ldlt_solve(S, b):
    """Dense pivot-free LDL^T solve of S x = b (torch float64 CUDA tensors,
    S column-major n x n, i.e. pass S.T.contiguous() for a row-major array).
    Returns (x, inertia)."""
    import torch
    n = b.numel()
    x = torch.empty_like(b)
    inert = np.zeros(3, dtype=np.int32)
    _check("scopf_dense_ldlt_solve", lib().scopf_dense_ldlt_solve(
        _dp(S), n, _dp(b), _dp(x), _hp(inert, c_i32),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return x, tuple(int(v) for v in inert)


def scopf_dense_ldlt_solve_noalloc(S, b, x=None):
    """As scopf_dense_ldlt_solve, through the entry point that allocates no
    device memory (static per-device scratch, n <= 768).  The output x may be
    passed in preallocated.  Returns (x, inertia, status)."""
    import torch
    n = b.numel()
    if x is None:
        x = torch.empty_like(b)
    inert = np.zeros(3, dtype=np.int32)
    st = lib().scopf_dense_ldlt_solve_noalloc(
        _dp(S), n, _dp(b), _dp(x), _hp(inert, c_i32),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return x, tuple(int(v) for v in inert), st


PEAK_KINDS = {0: "fp32_fma", 1: "fp64_fma", 2: "fp64_mma", 3: "fp64_fma_one_lane",
              4: "fp64_fma_and_mma"}


def scopf_peak_probe(kind: int, iters: int = 1 << 14, repeats: int = 5):
    """Measured arithmetic throughput (TFLOP/s) of one probe kind (0 FP32
    FMA, 1 FP64 FMA, 2 FP64 tensor MMA): the best of `repeats` launches,
    each timed with CUDA events on the current stream after one warm-up."""
    import torch
    s = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    fl = c_dbl()
    best = None
    for r in range(repeats + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _check("scopf_peak_probe", lib().scopf_peak_probe(kind, iters, _dp(out),
                                                          ctypes.c_void_p(s.cuda_stream),
                                                          ctypes.byref(fl)))
        e1.record(s)
        torch.cuda.synchronize()
        if r:
            t = fl.value / (e0.elapsed_time(e1) / 1e3) / 1e12
            best = t if best is None else max(best, t)
    return best


def scopf_pivot_reciprocal(d):
    """The FP64 factorization's pivot reciprocal of every entry of d (torch
    float64 CUDA tensor); returns a new tensor."""
    import torch
    out = torch.empty_like(d)
    _check("scopf_pivot_reciprocal", lib().scopf_pivot_reciprocal(
        _dp(d), _dp(out), d.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out


def default_options(**kw) -> Options:
    o = Options()
    lib().scopf_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _dp(t):
    """Device pointer of a torch tensor (float64), or NULL."""
    if t is None:
        return None
    import torch
    assert t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), P_dbl)


def _hp(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(fn, status):
    if status != 0:
        raise ScopfError(fn, status)


def _network_args(inst, keep):
    """scopf_network and scopf_contingency array of an instance (host arrays
    kept alive in `keep` for the duration of the call)."""
    net = inst.net

    def d(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return _hp(a, c_dbl)

    def i(a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        keep.append(a)
        return _hp(a, c_i32)

    N = Network(net.n_bus, net.n_branch, net.n_gen, int(net.ref_bus), d(net.Pd), d(net.Qd),
                d(net.Gs), d(net.Bs), d(net.vmin), d(net.vmax), i(net.f), i(net.t), d(net.r),
                d(net.x), d(net.b), d(net.rate), i(net.gbus), d(net.pmin), d(net.pmax),
                d(net.qmin), d(net.qmax), d(net.c2), d(net.c1), d(net.c0))
    K = len(inst.ctgs)
    C = (Contingency * max(1, K))()
    for k, c in enumerate(inst.ctgs):
        C[k] = Contingency(int(c.kind), int(c.element), len(c.switch_buses), i(c.switch_buses))
    return N, C, K


def autotune(inst, iterate_at: int = 10, steps: int = 3, options: Options | None = None,
             **opt_kw):
    """Run scopf_autotune on an instance: returns (the options with the
    chosen tile shapes, list of candidate dicts in the order tried)."""
    keep = []
    N, C, K = _network_args(inst, keep)
    o = options or default_options()
    for k, v in opt_kw.items():
        setattr(o, k, v)
    cap = 16
    E = (TuneEntry * cap)()
    n = c_i32()
    _check("scopf_autotune", lib().scopf_autotune(ctypes.byref(N), C, K, ctypes.byref(o),
                                                  iterate_at, steps, cap, E, ctypes.byref(n)))
    out = [{f: getattr(E[j], f) for f, _ in TuneEntry._fields_} for j in range(min(n.value, cap))]
    return o, out


class SCOPF:
    """A handle around one SCOPF instance (network + contingencies)."""

    def __init__(self, inst, options: Options | None = None, **opt_kw):
        L = lib()
        self._keep = []
        N, C, K = _network_args(inst, self._keep)
        o = options or default_options()
        for k, v in opt_kw.items():
            setattr(o, k, v)
        self.options = o
        self.host_only = bool(o.host_only)
        self.n_bus, self.n_gen = inst.net.n_bus, inst.net.n_gen
        h = ctypes.c_void_p()
        _check("scopf_create", L.scopf_create(ctypes.byref(N), C, K, ctypes.byref(o),
                                              ctypes.byref(h)))
        self.h = h
        s = Sizes()
        _check("scopf_get_sizes", L.scopf_get_sizes(h, ctypes.byref(s)))
        self.sizes = s
        self._keep = []
        if not self.host_only:
            import torch
            self.set_stream(torch.cuda.current_stream())

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                lib().scopf_destroy(h)
            except Exception:
                pass
            self.h = None

    # ------------------------------------------------------------ basics
    def set_stream(self, stream):
        _check("scopf_set_stream", lib().scopf_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    def set_precision(self, prec: int):
        _check("scopf_set_precision", lib().scopf_set_precision(self.h, prec))

    def scopf_symbolic_block(self, k: int):
        L = lib()
        nn, nbn, nsn, nr = c_i32(), c_i32(), c_i32(), c_i32()
        _check("scopf_symbolic_block", L.scopf_symbolic_block(
            self.h, k, ctypes.byref(nn), ctypes.byref(nbn), ctypes.byref(nsn), ctypes.byref(nr),
            None, None, None, None))
        post = np.zeros(nbn.value, dtype=np.int32)
        par = np.zeros(nbn.value, dtype=np.int32)
        sns = np.zeros(nsn.value + 1, dtype=np.int32)
        rows = np.zeros(nr.value, dtype=np.int64)
        _check("scopf_symbolic_block", L.scopf_symbolic_block(
            self.h, k, ctypes.byref(nn), ctypes.byref(nbn), ctypes.byref(nsn), ctypes.byref(nr),
            _hp(post, c_i32), _hp(par, c_i32), _hp(sns, c_i32), _hp(rows, c_i64)))
        return dict(n_nodes=nn.value, n_block_nodes=nbn.value, post=post, node_parent=par,
                    sn_start=sns, rows=rows)

    def kkt_pattern(self):
        s = self.sizes
        ptr = np.zeros(s.n_kkt + 1, dtype=np.int64)
        col = np.zeros(s.nnz_kkt, dtype=np.int64)
        _check("kkt_export", lib().kkt_export(self.h, _hp(ptr, c_i64), _hp(col, c_i64), None))
        return ptr, col

    # ------------------------------------------------------- device calls
    def new_state(self):
        import torch
        s = self.sizes
        n, m, p = s.n, s.m, s.p
        z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")
        return dict(w=z(n), r=z(m), t=z(p), s=z(p), lam=z(m), yc=z(p), zl=z(n), zu=z(n), zs=z(p))

    @staticmethod
    def _state(st):
        return State(*(_dp(st[f]) for f in _STATE_FIELDS))

    def scopf_eval(self, w, want_c=True, want_g=True):
        import torch
        s = self.sizes
        c = torch.empty(s.m, dtype=torch.float64, device="cuda") if want_c else None
        g = torch.empty(s.n, dtype=torch.float64, device="cuda") if want_g else None
        obj = c_dbl()
        _check("scopf_eval", lib().scopf_eval(self.h, _dp(w), ctypes.byref(obj), _dp(g), _dp(c)))
        return obj.value, g, c

    def kkt_assemble(self, st, lam_n, nu0_n, rho, mu, delta_w, want_rhs=True):
        import torch
        rhs = torch.empty(self.sizes.n_kkt, dtype=torch.float64, device="cuda") if want_rhs else None
        S = self._state(st)
        _check("kkt_assemble", lib().kkt_assemble(self.h, ctypes.byref(S), _dp(lam_n), _dp(nu0_n),
                                                  rho, mu, delta_w, _dp(rhs)))
        return rhs

    def kkt_values(self):
        v = np.zeros(self.sizes.nnz_kkt)
        _check("kkt_export", lib().kkt_export(self.h, None, None, _hp(v, c_dbl)))
        return v

    def kkt_factor(self, precision: int = -1):
        inertia = np.zeros(3, dtype=np.int32)
        _check("kkt_factor", lib().kkt_factor(self.h, precision, _hp(inertia, c_i32)))
        return tuple(int(x) for x in inertia)

    def kkt_solve(self, b, max_refine: int = -1, check: bool = True):
        import torch
        x = torch.empty_like(b)
        rel, steps = c_dbl(), c_i32()
        st = lib().kkt_solve(self.h, _dp(b), _dp(x), max_refine, ctypes.byref(rel), ctypes.byref(steps))
        if check and st not in (0, -5):
            raise ScopfError("kkt_solve", st)
        return x, rel.value, steps.value, st

    def ncl_solve(self, warm=None):
        R = Result()
        S = self._state(warm) if warm is not None else None
        st = lib().ncl_solve(self.h, ctypes.byref(S) if S is not None else None, ctypes.byref(R))
        out = {f: getattr(R, f) for f, _ in Result._fields_}
        out["call_status"] = st
        return out

    def ncl_resume(self):
        """Continue the NCL method from the handle's iterate and parameters
        (the last solve's end, or a checkpoint restored with load_state +
        set_ncl_params)."""
        R = Result()
        st = lib().ncl_resume(self.h, ctypes.byref(R))
        out = {f: getattr(R, f) for f, _ in Result._fields_}
        out["call_status"] = st
        return out

    def get_state(self):
        st = self.new_state()
        S = self._state(st)
        _check("scopf_copy_state", lib().scopf_copy_state(self.h, ctypes.byref(S)))
        return st

    def load_state(self, st):
        S = self._state(st)
        _check("scopf_load_state", lib().scopf_load_state(self.h, ctypes.byref(S)))

    def ncl_params(self):
        import torch
        s = self.sizes
        pl, pn, rho = P_dbl(), P_dbl(), c_dbl()
        _check("scopf_get_ncl_params", lib().scopf_get_ncl_params(self.h, ctypes.byref(pl),
                                                                  ctypes.byref(pn), ctypes.byref(rho)))
        return pl, pn, rho.value

    def scopf_newton_step(self, st, lam_n, nu0_n, rho, mu, dw_last=0.0, direction=None):
        """One Newton step at st (unchanged).  Returns (alpha_p, alpha_d,
        theta_trial, phi_trial, delta_w, _), inertia tries."""
        out = np.zeros(6)
        inert = np.zeros(3, dtype=np.int32)
        S = self._state(st)
        Dp = ctypes.byref(self._state(direction)) if direction is not None else None
        _check("scopf_newton_step", lib().scopf_newton_step(
            self.h, ctypes.byref(S), _dp(lam_n), _dp(nu0_n), rho, mu, dw_last, Dp,
            _hp(out, c_dbl), _hp(inert, c_i32)))
        return out, int(inert[2])

    PHASES = ("assemble", "front_init", "factor", "schur", "solve", "residual", "ipm")

    def scopf_timing(self, enable: bool):
        ms = np.zeros(7)
        calls = np.zeros(7, dtype=np.int32)
        _check("scopf_timing", lib().scopf_timing(self.h, int(enable), _hp(ms, c_dbl), _hp(calls, c_i32)))
        return {k: (float(ms[i]), int(calls[i])) for i, k in enumerate(self.PHASES)}

    def scopf_trace(self, enable: bool):
        """Start (True) or stop the scheduler trace (see scopf.h)."""
        _check("scopf_trace", lib().scopf_trace(self.h, 1 if enable else 0))

    def scopf_trace_read(self, kind: int):
        """(n_items, 4) uint64: claim start, claim end, finish (ns), SM."""
        n = c_i32()
        _check("scopf_trace_items", lib().scopf_trace_items(self.h, ctypes.byref(n), None))
        out = np.zeros((n.value, 4), dtype=np.uint64)
        _check("scopf_trace_read", lib().scopf_trace_read(
            self.h, kind, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return out

    def scopf_trace_items(self):
        """(n_items, 6) int32: fronts, parent item, phase-1 flag, largest
        front, pivots, block."""
        n = c_i32()
        _check("scopf_trace_items", lib().scopf_trace_items(self.h, ctypes.byref(n), None))
        out = np.zeros((n.value, 6), dtype=np.int32)
        _check("scopf_trace_items", lib().scopf_trace_items(self.h, ctypes.byref(n), _hp(out, c_i32)))
        return out

    def ncl_params_tensors(self):
        """Copies of the NCL multiplier estimates (lam_n, nu0_n) as torch tensors, and rho."""
        import torch
        pl, pn, rho = self.ncl_params()
        s = self.sizes
        lam_n = torch.empty(s.m, dtype=torch.float64, device="cuda")
        nu0_n = torch.empty(max(s.p, 1), dtype=torch.float64, device="cuda")[:s.p]
        cudart = _cudart()
        cudart.cudaMemcpy(ctypes.c_void_p(lam_n.data_ptr()), ctypes.cast(pl, ctypes.c_void_p),
                          ctypes.c_size_t(8 * s.m), 3)
        if s.p:
            cudart.cudaMemcpy(ctypes.c_void_p(nu0_n.data_ptr()), ctypes.cast(pn, ctypes.c_void_p),
                              ctypes.c_size_t(8 * s.p), 3)
        return lam_n, nu0_n, rho

    def set_params(self, Pd=None, Qd=None, c1=None):
        """Replace the bus loads and linear cost coefficients (host arrays)."""
        def h(a, n):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            assert a.shape == (n,)
            return a
        Pd, Qd, c1 = h(Pd, self.n_bus), h(Qd, self.n_bus), h(c1, self.n_gen)
        _check("scopf_set_params", lib().scopf_set_params(
            self.h, None if Pd is None else _hp(Pd, c_dbl), None if Qd is None else _hp(Qd, c_dbl),
            None if c1 is None else _hp(c1, c_dbl)))

    def set_ncl_params(self, lam_n, nu0_n, rho, mu):
        """Declare the loaded state a solution with these NCL parameters."""
        _check("scopf_set_ncl_params", lib().scopf_set_ncl_params(
            self.h, _dp(lam_n), _dp(nu0_n), float(rho), float(mu)))

    HISTORY_INNER = ("outer", "inner", "mu", "rho", "E0", "theta", "phi", "alpha_p", "alpha_d",
                     "delta_w", "factorizations", "refine_steps", "precision", "accepted",
                     "backtracks", "ms")
    HISTORY_OUTER = ("outer", "rho", "r_inf", "t_inf", "E0", "eta", "omega", "inner")

    def last_error(self) -> str:
        """Text of the handle's last CUDA or internal error ("" when none)."""
        return lib().scopf_last_error(self.h).decode()

    def history(self, which: int = 0):
        """Iteration log of the last solve: (field names, numpy array with one
        row per interior-point (which=0) or NCL outer (which=1) iteration)."""
        n, ln = ctypes.c_int64(), c_i32()
        _check("scopf_history", lib().scopf_history(self.h, which, 0, None, ctypes.byref(n),
                                                    ctypes.byref(ln)))
        out = np.zeros((n.value, ln.value))
        _check("scopf_history", lib().scopf_history(self.h, which, n.value, _hp(out, c_dbl),
                                                    ctypes.byref(n), ctypes.byref(ln)))
        return (self.HISTORY_INNER if which == 0 else self.HISTORY_OUTER), out

    def block_violation(self):
        """|(r_k, t_k)|_inf of the current iterate per scenario (numpy, K + 1)."""
        v = np.zeros(self.sizes.n_blocks)
        _check("scopf_block_violation", lib().scopf_block_violation(self.h, _hp(v, c_dbl)))
        return v

    def scopf_screen(self, u0=None, eps=1e-6, rho_cap=1e6, accept_tol=1e-4):
        """Screen every scenario at the base control u0 (numpy, n_border) in
        one solve (first stage held within eps of u0).  Returns (accepted bool[K + 1], |(r_k, t_k)|_inf[K + 1],
        result dict); entry 0 is the base case."""
        R = Result()
        nblk = self.sizes.n_blocks
        v = np.zeros(nblk)
        acc = np.zeros(nblk, dtype=np.int32)
        u = None
        if u0 is not None:
            u = np.ascontiguousarray(u0, dtype=np.float64)
            if u.shape != (self.sizes.n_border,):
                raise ValueError(f"u0 needs shape ({self.sizes.n_border},)")
        _check("scopf_screen", lib().scopf_screen(
            self.h, None if u is None else _hp(u, c_dbl), float(eps), float(rho_cap),
            float(accept_tol), ctypes.byref(R), _hp(v, c_dbl), _hp(acc, ctypes.c_int32)))
        out = {f: getattr(R, f) for f, _ in Result._fields_}
        return acc.astype(bool), v, out

    def scopf_adjoint(self, seed_pg0=None, seed_cost=0.0):
        """Gradients of seed_pg0' p_g^0 + seed_cost * objective with respect
        to (Pd, Qd, c1) at the converged solution (torch tensors)."""
        import torch
        net_nb, ng = self.n_bus, self.n_gen
        gP = torch.zeros(net_nb, dtype=torch.float64, device="cuda")
        gQ = torch.zeros(net_nb, dtype=torch.float64, device="cuda")
        gc = torch.zeros(ng, dtype=torch.float64, device="cuda")
        _check("scopf_adjoint", lib().scopf_adjoint(self.h, _dp(seed_pg0), float(seed_cost),
                                                    _dp(gP), _dp(gQ), _dp(gc)))
        return gP, gQ, gc


class SCOPFLayer:
    """Differentiable SCOPF solve: ``pg0, cost = SCOPFLayer.apply(model, Pd, Qd, c1)``.

    forward solves the NCL problem for the given loads and linear costs (the
    structure of ``model``, a :class:`SCOPF` handle, is kept); backward is one
    adjoint solve (scopf_adjoint) with the final factorization's matrix."""

    @staticmethod
    def apply(model, Pd, Qd, c1):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, Pd_, Qd_, c1_):
                ctx.devices = (Pd_.device, Qd_.device, c1_.device)
                model.set_params(Pd_.detach().cpu().numpy(), Qd_.detach().cpu().numpy(),
                                 c1_.detach().cpu().numpy())
                res = model.ncl_solve()
                if res["status"] != 0:
                    raise ScopfError("ncl_solve", res["status"])
                st = model.get_state()
                s = model.sizes
                b0 = int(s.n) - int(s.n_border)
                pg0 = st["w"][b0:b0 + model.n_gen].clone()
                return pg0.to(Pd_.device), torch.tensor(res["objective"], dtype=torch.float64,
                                                         device=Pd_.device)

            @staticmethod
            def backward(ctx, g_pg0, g_cost):
                seed = g_pg0.to("cuda", torch.float64).contiguous()
                gP, gQ, gc = model.scopf_adjoint(seed, float(g_cost))
                dP, dQ, dc = ctx.devices
                return gP.to(dP), gQ.to(dQ), gc.to(dc)

        return _Fn.apply(Pd, Qd, c1)
