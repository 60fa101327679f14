"""Small problems with closed-form answers, in the interface of ``ncl.NCLSolver``.

* ``ToyMPCC``: min (x-a)^2 + (y-b)^2 (quadratic) or min x + y (linear)
  subject to 0 <= x  perp  y >= 0 (eq. mpcc with no equality rows).
  (x-1)^2 + (y-1)^2 has two strongly stationary minima (1,0), (0,1), value 1;
  x + y has the unique solution (0,0), where I_00 is nonempty and the rows
  (0 W2 W1) of B vanish (Section IV-B).
* ``ToyInfeasible``: c(x) = x^2 + 1 = 0 has no solution; the NCL penalty
  diverges and the iterates approach the stationary point x = 0, r = 1 of
  the feasibility problem eq. (feaspb), objective |r|^2 = 1.
* ``ToyQP``: convex QP min 1/2 x'Qx + q'x s.t. Ax = b with inactive bounds;
  its solution is the solution of the KKT linear system.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class _Base:
    comp1 = np.zeros(0, dtype=np.int64)
    comp2 = np.zeros(0, dtype=np.int64)

    @property
    def p(self):
        return len(self.comp1)


class ToyMPCC(_Base):
    def __init__(self, kind="quadratic", a=1.0, b=1.0, x0=(0.5, 0.5)):
        self.kind, self.a, self.b = kind, a, b
        self.n, self.m = 2, 0
        self.wl = np.zeros(2)
        self.wu = np.full(2, np.inf)
        self.comp1 = np.array([0])
        self.comp2 = np.array([1])
        self.x0 = np.array(x0, dtype=float)

    def initial_point(self):
        return self.x0.copy()

    def objective(self, w):
        if self.kind == "linear":
            return float(w[0] + w[1])
        return float((w[0] - self.a) ** 2 + (w[1] - self.b) ** 2)

    def gradient(self, w):
        if self.kind == "linear":
            return np.ones(2)
        return np.array([2 * (w[0] - self.a), 2 * (w[1] - self.b)])

    def constraints(self, w):
        return np.zeros(0)

    def jacobian(self, w):
        return sp.csr_matrix((0, 2))

    def hessian(self, w, lam, obj_factor=1.0):
        if self.kind == "linear":
            return sp.csr_matrix((2, 2))
        return sp.csr_matrix(2.0 * obj_factor * np.eye(2))


class ToyInfeasible(_Base):
    n, m = 1, 1

    def __init__(self):
        self.wl = np.full(1, -np.inf)
        self.wu = np.full(1, np.inf)

    def initial_point(self):
        return np.array([0.7])

    def objective(self, w):
        return 0.0

    def gradient(self, w):
        return np.zeros(1)

    def constraints(self, w):
        return np.array([w[0] ** 2 + 1.0])

    def jacobian(self, w):
        return sp.csr_matrix(np.array([[2.0 * w[0]]]))

    def hessian(self, w, lam, obj_factor=1.0):
        return sp.csr_matrix(np.array([[2.0 * lam[0]]]))


class ToyQP(_Base):
    def __init__(self, n=6, m=2, seed=0):
        rng = np.random.default_rng(seed)
        M = rng.standard_normal((n, n))
        self.Q = M @ M.T + n * np.eye(n)
        self.q = rng.standard_normal(n)
        self.A = rng.standard_normal((m, n))
        self.b = rng.standard_normal(m)
        self.n, self.m = n, m
        self.wl = np.full(n, -100.0)
        self.wu = np.full(n, 100.0)

    def exact(self):
        n, m = self.n, self.m
        K = np.block([[self.Q, self.A.T], [self.A, np.zeros((m, m))]])
        sol = np.linalg.solve(K, np.concatenate([-self.q, self.b]))
        return sol[:n], sol[n:]

    def initial_point(self):
        return np.zeros(self.n)

    def objective(self, w):
        return float(0.5 * w @ self.Q @ w + self.q @ w)

    def gradient(self, w):
        return self.Q @ w + self.q

    def constraints(self, w):
        return self.A @ w - self.b

    def jacobian(self, w):
        return sp.csr_matrix(self.A)

    def hessian(self, w, lam, obj_factor=1.0):
        return sp.csr_matrix(obj_factor * self.Q)
