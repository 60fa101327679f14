"""Linear solvers for the oracle's Newton systems.

DenseSolver     inertia by the signs of the eigenvalues of K (Sylvester's law
                of inertia: the definition, via LAPACK's symmetric
                eigensolver) and the solution by LAPACK's LU solve.  For the
                tiny systems of the toys and the 30-bus case.
SparseLDLSolver pivot-free LDL^T (D diagonal, "signed Cholesky", Section IV-B)
                of P K P' under a given fill-reducing permutation, by the
                plain left-looking column algorithm in ``ldlt.c``; inertia
                from the signs of D.  Pinned against DenseSolver.
dense_ldlt      pivot-free dense LDL^T written out in numpy (for the pins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp


class DenseSolver:
    def __init__(self, zero_tol: float = 0.0):
        self.zero_tol = zero_tol
        self.K = None

    def factor(self, K):
        Kd = K.toarray() if sp.issparse(K) else np.asarray(K)
        self.K = Kd
        ev = np.linalg.eigvalsh(Kd)
        tol = self.zero_tol * max(1.0, np.abs(ev).max())
        return int((ev > tol).sum()), int((ev < -tol).sum()), int((np.abs(ev) <= tol).sum())

    def solve(self, b):
        return np.linalg.solve(self.K, b)


def dense_ldlt(K):
    """K = L D L' with unit lower-triangular L and diagonal D, no pivoting.

    Column j: d_j = K_jj - sum_k L_jk^2 d_k;  L_ij = (K_ij - sum_k L_ik d_k L_jk) / d_j.
    """
    K = np.asarray(K, dtype=float)
    n = K.shape[0]
    L = np.eye(n)
    d = np.zeros(n)
    for j in range(n):
        d[j] = K[j, j] - np.sum(L[j, :j] ** 2 * d[:j])
        if j + 1 < n:
            L[j + 1:, j] = (K[j + 1:, j] - L[j + 1:, :j] @ (d[:j] * L[j, :j])) / d[j]
    return L, d


_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def build_c(force: bool = False) -> str:
    """Compile ``ldlt.c`` into ``_oracle_ldlt.so`` (plain gcc, -O2)."""
    src = os.path.join(_HERE, "ldlt.c")
    out = os.path.join(_HERE, "_oracle_ldlt.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", out, src, "-lm"])
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_c())
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_ldlt_symbolic.argtypes = [ctypes.c_int64, i64p, i64p, i64p, i64p]
        lib.oracle_ldlt_symbolic.restype = ctypes.c_int64
        lib.oracle_ldlt_numeric.argtypes = [ctypes.c_int64, i64p, i64p, dp, i64p, i64p,
                                            i64p, dp, dp, ctypes.c_double]
        lib.oracle_ldlt_numeric.restype = ctypes.c_int64
        lib.oracle_ldlt_solve.argtypes = [ctypes.c_int64, i64p, i64p, dp, dp, dp]
        lib.oracle_ldlt_solve.restype = None
        _LIB = lib
    return _LIB


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


class SparseLDLSolver:
    """Pivot-free sparse LDL^T of P K P' (P from ``perm``: new row i = old perm[i])."""

    def __init__(self, perm_fn=None, pivot_tol: float = 0.0):
        self.perm_fn = perm_fn
        self.pivot_tol = pivot_tol
        self.perm = None
        self.pattern_key = None

    def _order(self, K):
        n = K.shape[0]
        if self.perm is None or self.perm.shape[0] != n:
            self.perm = (np.asarray(self.perm_fn(K), dtype=np.int64) if self.perm_fn
                         else np.arange(n, dtype=np.int64))
        return self.perm

    def zero_pivot_certain(self, K) -> bool:
        """True when factor(K) must report an exactly zero pivot.

        A row of P K P' with no stored entry left of its diagonal gets no
        update in the elimination (row k of L is empty: its pattern is the
        union of the tree paths from those entries), so its pivot is its own
        diagonal entry.  If one such entry is 0.0, the pivot is 0.0 whatever
        the other values, and |d| <= pivot_tol counts it as zero.
        """
        K = sp.csr_matrix(K)
        perm = self._order(K)
        Kp = K[perm][:, perm]
        above = sp.triu(Kp, k=1, format="csc")   # column k: stored rows i < k
        above.sum_duplicates()
        no_update = np.diff(above.indptr) == 0
        return bool(np.any(no_update & (Kp.diagonal() == 0.0)))

    def factor(self, K):
        lib = _lib()
        K = sp.csr_matrix(K)
        n = K.shape[0]
        perm = self._order(K)
        iperm = np.empty(n, dtype=np.int64)
        iperm[perm] = np.arange(n)
        # upper triangle of the permuted matrix, stored by columns (CSC)
        Kp = K[perm][:, perm]
        U = sp.triu(Kp, format="csc")
        U.sum_duplicates()
        U.sort_indices()
        Ap = U.indptr.astype(np.int64)
        Ai = U.indices.astype(np.int64)
        Ax = U.data.astype(np.float64)
        parent = np.zeros(n, dtype=np.int64)
        Lnz = np.zeros(n, dtype=np.int64)
        Lp = np.zeros(n + 1, dtype=np.int64)
        lib.oracle_ldlt_symbolic(n, _p(Ap, ctypes.c_int64), _p(Ai, ctypes.c_int64),
                                 _p(parent, ctypes.c_int64), _p(Lnz, ctypes.c_int64))
        Lp[1:] = np.cumsum(Lnz)
        Li = np.zeros(max(1, Lp[-1]), dtype=np.int64)
        Lx = np.zeros(max(1, Lp[-1]))
        D = np.zeros(n)
        lib.oracle_ldlt_numeric(n, _p(Ap, ctypes.c_int64), _p(Ai, ctypes.c_int64),
                                _p(Ax, ctypes.c_double), _p(parent, ctypes.c_int64),
                                _p(Lp, ctypes.c_int64), _p(Li, ctypes.c_int64),
                                _p(Lx, ctypes.c_double), _p(D, ctypes.c_double), self.pivot_tol)
        self.n, self.iperm, self.Lp, self.Li, self.Lx, self.D = n, iperm, Lp, Li, Lx, D
        self.nnzL = int(Lp[-1])
        tol = self.pivot_tol
        return int((D > tol).sum()), int((D < -tol).sum()), int((np.abs(D) <= tol).sum())

    def solve(self, b):
        lib = _lib()
        x = np.ascontiguousarray(b[self.perm], dtype=np.float64)
        out = np.zeros(self.n)
        lib.oracle_ldlt_solve(self.n, _p(self.Lp, ctypes.c_int64), _p(self.Li, ctypes.c_int64),
                              _p(self.Lx, ctypes.c_double), _p(self.D, ctypes.c_double),
                              _p(x, ctypes.c_double))
        out[self.perm] = x
        return out

    def factors(self):
        """(L as CSC with unit diagonal, D) of the permuted matrix."""
        n = self.n
        L = sp.csc_matrix((self.Lx[:self.nnzL], self.Li[:self.nnzL], self.Lp), shape=(n, n))
        return (L + sp.eye(n)).tocsc(), self.D.copy()


class CondensedSolver:
    """The condensed primal variant of eq. (newtonsystem) (Section IV-B,
    "signed Cholesky" read as a Cholesky of the primal Schur complement).

    K = [[A, B'], [B, -C]] in the order [w; dual rows] with C diagonal and
    positive (the NCL block diag(1/rho, 1/rho + s/zs)).  Eliminating the dual
    rows gives the condensed matrix

        Kc = A + B' C^-1 B,     Kc dw = r1 + B' C^-1 r2,
        dy = C^-1 (B dw - r2),

    and Haynsworth's inertia formula In(K) = In(-C) + In(Kc) = (0, m+p, 0) +
    In(Kc): K has the inertia (n, m+p, 0) the interior-point method wants
    exactly when Kc is positive definite.  Kc is factored by the pivot-free
    LDL^T of ``SparseLDLSolver`` (all pivots positive = Cholesky) under the
    order ``perm_fn(Kc)`` (identity when None); ``factor`` returns the
    inertia of K.  ``n`` is the number of primal rows."""

    def __init__(self, n: int, perm_fn=None, pivot_tol: float = 0.0):
        self.n = n
        self.inner = SparseLDLSolver(perm_fn=perm_fn, pivot_tol=pivot_tol)

    def condense(self, K):
        K = sp.csr_matrix(K)
        n = self.n
        A = K[:n, :n]
        B = K[n:, :n]
        Kdd = K[n:, n:].tocoo()
        off = Kdd.row != Kdd.col
        if np.any(Kdd.data[off] != 0.0):
            raise ValueError("the dual-dual block is not diagonal")
        C = -K[n:, n:].diagonal()
        if np.any(C <= 0.0):
            raise ValueError("C must be positive")
        Kc = (A + B.T @ sp.diags(1.0 / C) @ B).tocsr()
        return Kc, B.tocsr(), C

    def factor(self, K):
        Kc, self.B, self.C = self.condense(K)
        ip, ineg, iz = self.inner.factor(Kc)
        return ip, ineg + len(self.C), iz

    def solve(self, b):
        n = self.n
        r1, r2 = b[:n], b[n:]
        dw = self.inner.solve(r1 + self.B.T @ (r2 / self.C))
        dy = (self.B @ dw - r2) / self.C
        return np.concatenate([dw, dy])
