"""NCL outer loop and interior-point inner loop (oracle, FP64).

Section IV-A (eq. nclsubpb): the NCL subproblem at outer iteration n is

    min_{w,r,t}  phi(w) + lam_n' r + nu0_n' t + rho/2 (|r|^2 + |t|^2)
    s.t.         c(w) - r = 0,   W1 W2 e <= t,   bounds on w.

Section IV-B: with the slack s := t - W1 W2 e (s >= 0) the subproblem is
solved by a primal-dual interior-point method whose Newton system reduces to
eq. (newtonsystem)

    [ A   B' ] [dw]   [r1]       A = H + barrier diagonal + V0 coupling,
    [ B  -C  ] [dy] = [r2]       B = [J; (0 W2 W1)],
                                 C = diag(1/rho I, 1/rho I + V0^-1 S),

and the eliminated directions (dr, dt, ds, bound multipliers) are recovered
elementwise.  The paper fixes the subproblem, the multiplier identities
(lam = lam_n + rho r, nu0 = nu0_n + rho t) and the structure of the Newton
system; it defers the update rules and the IPM safeguards to MadNCL and
MadNLP.  Those are taken here from the published algorithms:

  * outer loop (bound-constrained augmented Lagrangian / NCL): accept the
    multiplier update when max(|r|, |t|) <= eta, then eta, omega /= 10;
    otherwise rho *= 10; declare infeasible once rho > rho_max;
  * inner loop: Waechter & Biegler (2006) -- monotone Fiacco-McCormick
    barrier update, fraction-to-boundary rule, filter line search,
    inertia correction by a primal regularisation delta_w;
  * the equality multiplier y_c of the complementarity rows and the bound
    multiplier z_s of s are kept as separate primal-dual variables (Ipopt
    style); C uses z_s (= V0) and the Hessian coupling uses y_c.

The derivation of the elimination (signs included) is written out in
``reduced_rhs`` and ``recover``; the test suite pins it against a dense solve
of the unreduced Newton system.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math
import time

import numpy as np
import scipy.sparse as sp


@dataclass
class Options:
    tol: float = 1e-6            # Section V-A
    mu_min: float = 1e-7         # Section V-A
    mu_init: float = 1e-1
    kappa_eps: float = 10.0
    kappa_mu: float = 0.2
    theta_mu: float = 1.5
    tau_min: float = 0.99
    s_max: float = 100.0
    kappa_sigma: float = 1e10
    bound_relax: float = 1e-8
    bound_push: float = 1e-2
    bound_frac: float = 1e-2
    slack_init: float = 1e-1      # initial s of the complementarity rows
    comp_init: float = 1e-1       # initial value of the w1 members (pi, nu)
    delta_w0: float = 1e-4
    delta_w_min: float = 1e-20
    delta_w_max: float = 1e40
    kappa_w_minus: float = 1.0 / 3.0
    kappa_w_plus: float = 8.0
    kappa_w_plus_bar: float = 100.0
    # IC-1 at every iteration, its outcome taken without factoring when the
    # pivot-free LDL^T must meet an exactly zero pivot (``newton_direction``)
    known_zero_pivot: bool = True
    # keep the barrier parameter at its starting value and stop the inner
    # loop on the barrier error E_mu instead of E_0 (solutions of the
    # barrier problem at a fixed mu: the smooth map the adjoint
    # differentiates)
    fixed_mu: bool = False
    gamma_theta: float = 1e-5
    gamma_phi: float = 1e-8
    delta_sw: float = 1.0
    s_theta: float = 1.1
    s_phi: float = 2.3
    eta_phi: float = 1e-8
    gamma_alpha: float = 0.05
    max_backtrack: int = 40
    rho_init: float = 1e2
    rho_max: float = 1e12
    eta_init: float = 1e-2
    omega_init: float = 1e-2
    max_outer: int = 40
    max_inner: int = 3000
    verbose: bool = False


@dataclass
class State:
    w: np.ndarray
    r: np.ndarray
    t: np.ndarray
    s: np.ndarray
    lam: np.ndarray
    yc: np.ndarray
    zl: np.ndarray
    zu: np.ndarray
    zs: np.ndarray

    def copy(self):
        return State(*(getattr(self, f).copy() for f in
                       ("w", "r", "t", "s", "lam", "yc", "zl", "zu", "zs")))


@dataclass
class Params:
    """NCL outer-iteration parameters (rho^(n), lam^(n), nu0^(n))."""
    rho: float
    lam_n: np.ndarray
    nu0_n: np.ndarray


@dataclass
class Result:
    status: str
    state: State
    params: Params
    objective: float
    outer_iters: int
    inner_iters: int
    kkt_error: float
    feas_rt: float
    max_violation: float
    mu: float
    history: list = field(default_factory=list)
    wall_s: float = 0.0


class NCLSolver:
    """Algorithm NCL with an interior-point inner solver on an MPCC problem.

    ``prob`` provides n, m, p, wl, wu, comp1, comp2, initial_point(),
    objective(w), gradient(w), constraints(w), jacobian(w) (CSR m x n) and
    hessian(w, lam) (CSR n x n).  ``linsolver`` is a factory with
    ``factor(K) -> (n_pos, n_neg, n_zero)`` and ``solve(b)``.
    """

    def __init__(self, prob, linsolver, opts: Options | None = None):
        self.P = prob
        self.lin = linsolver
        self.o = opts or Options()
        P = prob
        self.hl = np.isfinite(P.wl)
        self.hu = np.isfinite(P.wu)
        # bounds relaxed by bound_relax relative (Waechter & Biegler 2006,
        # Section 3.5) so that slacks never round to zero
        rf = self.o.bound_relax
        self.wl = np.where(self.hl, P.wl - rf * np.maximum(1.0, np.abs(np.where(self.hl, P.wl, 0.0))), P.wl)
        self.wu = np.where(self.hu, P.wu + rf * np.maximum(1.0, np.abs(np.where(self.hu, P.wu, 0.0))), P.wu)
        self.il = np.flatnonzero(self.hl)
        self.iu = np.flatnonzero(self.hu)
        self.c1 = np.asarray(P.comp1, dtype=np.int64)
        self.c2 = np.asarray(P.comp2, dtype=np.int64)
        self.n, self.m, self.p = P.n, P.m, P.p
        self.n_inner = 0
        self.history = []
        self.n_known_zero = 0      # IC-1 trials whose zero pivot was certain

    # ------------------------------------------------------------ helpers
    def project_start(self, w):
        """Bound push of Waechter & Biegler (2006), Section 3.6."""
        o = self.o
        w = w.copy()
        l, u = self.wl, self.wu
        both = self.hl & self.hu
        pl = np.where(self.hl, o.bound_push * np.maximum(1.0, np.abs(np.where(self.hl, l, 0.0))), 0.0)
        pu = np.where(self.hu, o.bound_push * np.maximum(1.0, np.abs(np.where(self.hu, u, 0.0))), 0.0)
        span = np.where(both, u - l, np.inf)
        pl = np.where(both, np.minimum(pl, o.bound_frac * span), pl)
        pu = np.where(both, np.minimum(pu, o.bound_frac * span), pu)
        w = np.where(self.hl, np.maximum(w, np.where(self.hl, l, 0.0) + pl), w)
        w = np.where(self.hu, np.minimum(w, np.where(self.hu, u, 0.0) - pu), w)
        return w

    def initial_state(self):
        o, P = self.o, self.P
        w = P.initial_point().copy()
        w[self.c1] = np.maximum(w[self.c1], o.comp_init)
        w = self.project_start(w)
        s = np.full(self.p, o.slack_init)
        t = w[self.c1] * w[self.c2] + s
        r = P.constraints(w)
        # multipliers from the identities of eq. (kktncl) at n = 0:
        # lam = lam_0 + rho r, nu0 = nu0_0 + rho t (lam_0 = nu0_0 = 0), z_s = nu0
        lam = o.rho_init * r
        yc = o.rho_init * t
        return State(w=w, r=r, t=t, s=s, lam=lam, yc=yc,
                     zl=np.ones(len(self.il)), zu=np.ones(len(self.iu)), zs=yc.copy())

    def slacks(self, st):
        return st.w[self.il] - self.wl[self.il], self.wu[self.iu] - st.w[self.iu]

    def comp_row(self, st):
        """W1 W2 e - t + s  (complementarity rows with their slack)."""
        return st.w[self.c1] * st.w[self.c2] - st.t + st.s

    def f_ncl(self, st, prm):
        return (self.P.objective(st.w) + prm.lam_n @ st.r + prm.nu0_n @ st.t
                + 0.5 * prm.rho * (st.r @ st.r + st.t @ st.t))

    # ------------------------------------------------- residuals / errors
    def residuals(self, st, prm, c=None, J=None, g=None):
        """Dual residuals (with bound multipliers) and primal residuals of the
        barrier KKT conditions (eq. kktncl with the slack s)."""
        P = self.P
        if c is None:
            c = P.constraints(st.w)
        if J is None:
            J = P.jacobian(st.w)
        if g is None:
            g = P.gradient(st.w)
        gw = g + J.T @ st.lam
        gw[self.c1] += st.yc * st.w[self.c2]
        gw[self.c2] += st.yc * st.w[self.c1]
        gwz = gw.copy()
        gwz[self.il] -= st.zl
        gwz[self.iu] += st.zu
        gr = prm.lam_n + prm.rho * st.r - st.lam
        gt = prm.nu0_n + prm.rho * st.t - st.yc
        gs = st.yc - st.zs
        pc = c - st.r
        py = self.comp_row(st)
        return dict(gw=gw, gwz=gwz, gr=gr, gt=gt, gs=gs, pc=pc, py=py, c=c, J=J, g=g)

    def error(self, st, res, mu):
        """Scaled optimality error E_mu (Waechter & Biegler 2006, eq. 5)."""
        o = self.o
        sl, su = self.slacks(st)
        nz = len(st.zl) + len(st.zu) + len(st.zs)
        zsum = np.abs(st.zl).sum() + np.abs(st.zu).sum() + np.abs(st.zs).sum()
        ysum = np.abs(st.lam).sum() + np.abs(st.yc).sum()
        sd = max(o.s_max, (ysum + zsum) / max(1, self.m + self.p + nz)) / o.s_max
        sc = max(o.s_max, zsum / max(1, nz)) / o.s_max
        dual = max(_inf(res["gwz"]), _inf(res["gr"]), _inf(res["gt"]), _inf(res["gs"]))
        prim = max(_inf(res["pc"]), _inf(res["py"]))
        comp = max(_inf(sl * st.zl - mu), _inf(su * st.zu - mu), _inf(st.s * st.zs - mu))
        return max(dual / sd, prim, comp / sc), dual, prim, comp

    # ------------------------------------------------ reduced Newton system
    def kkt_matrix(self, st, prm, H, J, delta_w):
        """Reduced KKT matrix of eq. (newtonsystem), order [dw; dlam; dyc]."""
        n, m, p = self.n, self.m, self.p
        sl, su = self.slacks(st)
        sig = np.zeros(n)
        sig[self.il] += st.zl / sl
        sig[self.iu] += st.zu / su
        # A = H + barrier diagonal + delta_w I + V0 coupling (H_12 + V0, H_21 + V0)
        Vc = sp.coo_matrix((np.concatenate([st.yc, st.yc]),
                            (np.concatenate([self.c1, self.c2]), np.concatenate([self.c2, self.c1]))),
                           shape=(n, n))
        A = (H + Vc + sp.diags(sig + delta_w)).tocsr()
        # B = [J; (0 W2 W1)]
        Bc = sp.coo_matrix((np.concatenate([st.w[self.c2], st.w[self.c1]]),
                            (np.concatenate([np.arange(p), np.arange(p)]),
                             np.concatenate([self.c1, self.c2]))), shape=(p, n))
        B = sp.vstack([J, Bc]).tocsr()
        # C = diag(1/rho I, 1/rho I + V0^-1 S)
        C = np.concatenate([np.full(m, 1.0 / prm.rho), 1.0 / prm.rho + st.s / st.zs])
        K = sp.bmat([[A, B.T], [B, -sp.diags(C)]], format="csr")
        return K

    def reduced_rhs(self, st, prm, res, mu):
        """Right-hand side (r1, r2) of eq. (newtonsystem).

        Linearising the barrier KKT conditions and eliminating
          dr  = (dlam - (lam_n + rho r - lam)) / rho,
          dt  = (dyc  - (nu0_n + rho t - yc)) / rho,
          ds  = (mu/s - yc - dyc) / (zs/s),
          dzl = mu/(w-l) - zl - (zl/(w-l)) dw,   dzu = mu/(u-w) - zu + (zu/(u-w)) dw,
        gives  r1 = -(grad phi + J'lam + B_c'yc - mu/(w-l) + mu/(u-w)),
               r2 = (-(c - r) - (lam_n + rho r - lam)/rho,
                     -(W1W2e - t + s) - (nu0_n + rho t - yc)/rho - (mu/s - yc) s/zs).
        """
        sl, su = self.slacks(st)
        rw = res["gw"].copy()
        rw[self.il] -= mu / sl
        rw[self.iu] += mu / su
        b_lam = -res["pc"] - res["gr"] / prm.rho
        b_y = -res["py"] - res["gt"] / prm.rho - (mu / st.s - st.yc) * st.s / st.zs
        return np.concatenate([-rw, b_lam, b_y])

    def recover(self, st, prm, res, mu, sol):
        """Eliminated directions (dr, dt, ds, dzl, dzu, dzs) from (dw, dlam, dyc)."""
        n, m = self.n, self.m
        dw, dlam, dyc = sol[:n], sol[n:n + m], sol[n + m:]
        sl, su = self.slacks(st)
        dr = (dlam - res["gr"]) / prm.rho
        dt = (dyc - res["gt"]) / prm.rho
        ds = (mu / st.s - st.yc - dyc) * st.s / st.zs
        dzl = mu / sl - st.zl - st.zl / sl * dw[self.il]
        dzu = mu / su - st.zu + st.zu / su * dw[self.iu]
        dzs = mu / st.s - st.zs - st.zs / st.s * ds
        return State(w=dw, r=dr, t=dt, s=ds, lam=dlam, yc=dyc, zl=dzl, zu=dzu, zs=dzs)

    def newton_direction(self, st, prm, res, mu, H, dw_last):
        """Factor with inertia correction (Waechter & Biegler 2006, Alg. IC).

        IC-1 tries delta_w = 0 at every iteration.  When the linear solver is
        a pivot-free LDL^T whose order gives some row no update and a zero
        diagonal (``zero_pivot_certain``), that factorization must report a
        zero pivot, so its outcome -- wrong inertia -- is known without
        computing it; the correction continues at IC-3 exactly as it would
        after factoring.  ``Options.known_zero_pivot = False`` factors anyway.
        """
        o = self.o
        n_pos, n_neg = self.n, self.m + self.p
        rhs = self.reduced_rhs(st, prm, res, mu)
        ic3 = o.delta_w0 if dw_last == 0.0 else max(o.delta_w_min, o.kappa_w_minus * dw_last)
        delta = 0.0
        certain = getattr(self.lin, "zero_pivot_certain", None)
        if o.known_zero_pivot and certain is not None:
            if certain(self.kkt_matrix(st, prm, H, res["J"], 0.0)):
                delta = ic3
                self.n_known_zero += 1
        tries = 0
        while True:
            K = self.kkt_matrix(st, prm, H, res["J"], delta)
            ip, ineg, iz = self.lin.factor(K)
            tries += 1
            if ip == n_pos and ineg == n_neg and iz == 0:
                break
            if delta == 0.0:
                delta = ic3
            else:
                delta *= o.kappa_w_plus if dw_last > 0.0 else o.kappa_w_plus_bar
            if delta > o.delta_w_max:
                raise RuntimeError("inertia correction failed")
        sol = self.lin.solve(rhs)
        return sol, delta, tries, K, rhs

    # ------------------------------------------------------- line search
    def frac_to_boundary(self, st, d, tau):
        sl, su = self.slacks(st)
        ap = 1.0
        for x, dx in ((sl, d.w[self.il]), (su, -d.w[self.iu]), (st.s, d.s)):
            neg = dx < 0
            if np.any(neg):
                ap = min(ap, float(np.min(-tau * x[neg] / dx[neg])))
        az = 1.0
        for z, dz in ((st.zl, d.zl), (st.zu, d.zu), (st.zs, d.zs)):
            neg = dz < 0
            if np.any(neg):
                az = min(az, float(np.min(-tau * z[neg] / dz[neg])))
        return ap, az

    def theta(self, st, c):
        return float(np.abs(c - st.r).sum() + np.abs(self.comp_row(st)).sum())

    def barrier_obj(self, st, prm, mu):
        sl, su = self.slacks(st)
        if np.any(sl <= 0) or np.any(su <= 0) or np.any(st.s <= 0):
            return math.inf
        return self.f_ncl(st, prm) - mu * (np.log(sl).sum() + np.log(su).sum() + np.log(st.s).sum())

    def barrier_dir_deriv(self, st, prm, res, mu, d):
        sl, su = self.slacks(st)
        return float(res["g"] @ d.w - mu * np.sum(d.w[self.il] / sl) + mu * np.sum(d.w[self.iu] / su)
                     + (prm.lam_n + prm.rho * st.r) @ d.r + (prm.nu0_n + prm.rho * st.t) @ d.t
                     - mu * np.sum(d.s / st.s))

    @staticmethod
    def step(st, d, a, az):
        return State(w=st.w + a * d.w, r=st.r + a * d.r, t=st.t + a * d.t, s=st.s + a * d.s,
                     lam=st.lam + a * d.lam, yc=st.yc + a * d.yc,
                     zl=st.zl + az * d.zl, zu=st.zu + az * d.zu, zs=st.zs + az * d.zs)

    def z_safeguard(self, st, mu):
        """Keep bound multipliers within kappa_sigma of mu/slack (W&B 2006, eq. 16)."""
        ks = self.o.kappa_sigma
        sl, su = self.slacks(st)
        st.zl = np.maximum(np.minimum(st.zl, ks * mu / sl), mu / (ks * sl))
        st.zu = np.maximum(np.minimum(st.zu, ks * mu / su), mu / (ks * su))
        st.zs = np.maximum(np.minimum(st.zs, ks * mu / st.s), mu / (ks * st.s))

    # ---------------------------------------------------------- inner loop
    def ipm(self, st, prm, mu, omega, dw_last):
        """Solve the NCL subproblem (eq. nclsubpb) to E_0 <= omega."""
        o, P = self.o, self.P
        res = self.residuals(st, prm)
        th0 = self.theta(st, res["c"])
        theta_max = 1e4 * max(1.0, th0)
        theta_min = 1e-4 * max(1.0, th0)
        filt = []
        while True:
            E0 = self.error(st, res, mu if o.fixed_mu else 0.0)[0]
            if E0 <= omega:
                return st, mu, dw_last, E0, "ok"
            if self.n_inner >= o.max_inner:
                return st, mu, dw_last, E0, "max_iter"
            Emu = self.error(st, res, mu)[0]
            while not o.fixed_mu and Emu <= o.kappa_eps * mu and mu > o.mu_min:
                mu = max(o.mu_min, min(o.kappa_mu * mu, mu ** o.theta_mu))
                filt = []
                Emu = self.error(st, res, mu)[0]
            tau = max(o.tau_min, 1.0 - mu)
            H = P.hessian(st.w, st.lam)
            try:
                sol, delta, tries, _, _ = self.newton_direction(st, prm, res, mu, H, dw_last)
            except RuntimeError:
                return st, mu, dw_last, E0, "numerical_failure"
            if not np.all(np.isfinite(sol)):
                return st, mu, dw_last, E0, "numerical_failure"
            if delta > 0.0:
                dw_last = delta
            d = self.recover(st, prm, res, mu, sol)
            ap, az = self.frac_to_boundary(st, d, tau)
            th = self.theta(st, res["c"])
            ph = self.barrier_obj(st, prm, mu)
            gd = self.barrier_dir_deriv(st, prm, res, mu, d)
            if gd < 0:
                amin = o.gamma_alpha * min(o.gamma_theta, o.gamma_phi * th / -gd,
                                           o.delta_sw * th ** o.s_theta / (-gd) ** o.s_phi)
            else:
                amin = o.gamma_alpha * o.gamma_theta
            a = ap
            accepted = False
            nback = 0
            while True:
                trial = self.step(st, d, a, az)
                ct = P.constraints(trial.w)
                tht = self.theta(trial, ct)
                pht = self.barrier_obj(trial, prm, mu)
                ok, ftype = False, False
                if tht <= theta_max and not any(tht >= tf and pht >= pf for tf, pf in filt):
                    switching = gd < 0 and a * (-gd) ** o.s_phi > o.delta_sw * th ** o.s_theta
                    if th <= theta_min and switching:
                        ok = pht <= ph + o.eta_phi * a * gd
                        ftype = ok
                    else:
                        ok = tht <= (1 - o.gamma_theta) * th or pht <= ph - o.gamma_phi * th
                if ok:
                    accepted = True
                    break
                nback += 1
                if a < amin or nback >= o.max_backtrack:
                    break
                a *= 0.5
            if not accepted:
                # elastic reset (NCL restoration): r and t absorb the violation
                trial = self.step(st, d, a, az)
                trial.r = P.constraints(trial.w)
                trial.t = trial.w[self.c1] * trial.w[self.c2] + trial.s
                filt = []
            elif not ftype:
                filt.append(((1 - o.gamma_theta) * th, ph - o.gamma_phi * th))
            self.z_safeguard(trial, mu)
            st = trial
            self.n_inner += 1
            res = self.residuals(st, prm)
            if o.verbose:
                print(f"  it {self.n_inner:4d} mu {mu:.1e} E0 {E0:.2e} th {th:.2e} a {a:.2e} "
                      f"dw {delta:.1e} tries {tries} {'R' if not accepted else ''}")
            self.history.append(dict(it=self.n_inner, mu=mu, E0=E0, alpha=a, delta_w=delta,
                                     tries=tries, backtracks=nback, restored=not accepted))

    # ---------------------------------------------------------- outer loop
    def solve(self, warm: State | None = None, params: Params | None = None, mu: float | None = None,
              blocks=None):
        """NCL outer loop.  ``blocks`` (a list of (c0, nrow, p0, ncomp) row
        ranges of r and t that no constraint couples, as for scenarios at a
        fixed first stage) switches on the per-block rule of batched
        screening: when max(|r|, |t|) > eta, every block whose own
        max(|r_k|, |t_k|) <= eta still takes its multiplier update -- as it
        would in a solve of its own -- before rho grows."""
        o = self.o
        t0 = time.perf_counter()
        st = warm.copy() if warm is not None else self.initial_state()
        prm = params or Params(rho=o.rho_init, lam_n=np.zeros(self.m), nu0_n=np.zeros(self.p))
        mu = o.mu_init if mu is None else mu
        eta, omega = o.eta_init, o.omega_init
        dw_last = 0.0
        status = "max_outer"
        E0 = math.inf
        feas = math.inf
        outer = 0
        for outer in range(1, o.max_outer + 1):
            st, mu, dw_last, E0, inner_status = self.ipm(st, prm, mu, max(omega, o.tol), dw_last)
            feas = max(_inf(st.r), _inf(st.t))
            if o.verbose:
                print(f"outer {outer} rho {prm.rho:.1e} |r,t| {feas:.2e} E0 {E0:.2e} eta {eta:.1e} "
                      f"omega {omega:.1e} inner {self.n_inner}")
            if inner_status != "ok":
                status = inner_status
                break
            if feas <= max(eta, o.tol):
                if feas <= o.tol and E0 <= o.tol:
                    status = "ok"
                    break
                # first-order multiplier update: lam_n + rho r, nu0_n + rho t
                prm = Params(rho=prm.rho, lam_n=prm.lam_n + prm.rho * st.r,
                             nu0_n=prm.nu0_n + prm.rho * st.t)
                eta = max(eta / 10.0, o.tol)
                omega = max(omega / 10.0, o.tol)
            else:
                lam_n, nu0_n = prm.lam_n, prm.nu0_n
                if blocks is not None:
                    lam_n, nu0_n = lam_n.copy(), nu0_n.copy()
                    for c0, nrow, p0, ncomp in blocks:
                        rk, tk = st.r[c0:c0 + nrow], st.t[p0:p0 + ncomp]
                        if max(_inf(rk), _inf(tk)) <= max(eta, o.tol):
                            lam_n[c0:c0 + nrow] += prm.rho * rk
                            nu0_n[p0:p0 + ncomp] += prm.rho * tk
                if prm.rho * 10.0 > o.rho_max:
                    status = "infeasible"
                    break
                prm = Params(rho=prm.rho * 10.0, lam_n=lam_n, nu0_n=nu0_n)
        res = self.residuals(st, prm)
        viol = self.max_violation(st.w, res["c"])
        return Result(status=status, state=st, params=prm, objective=self.P.objective(st.w),
                      outer_iters=outer, inner_iters=self.n_inner, kkt_error=E0, feas_rt=feas,
                      max_violation=viol, mu=mu, history=self.history,
                      wall_s=time.perf_counter() - t0)

    def max_violation(self, w, c):
        """Violation of eq. (mpcc): |c(w)|, bound and complementarity violations."""
        P = self.P
        v = _inf(c)
        if len(self.il):
            v = max(v, float(np.max(np.maximum(P.wl[self.il] - w[self.il], 0.0))))
        if len(self.iu):
            v = max(v, float(np.max(np.maximum(w[self.iu] - P.wu[self.iu], 0.0))))
        if self.p:
            v = max(v, float(np.max(np.abs(w[self.c1] * w[self.c2]))))
        return v


def _inf(x):
    return float(np.max(np.abs(x))) if len(x) else 0.0
