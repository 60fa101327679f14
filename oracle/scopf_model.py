"""Polar AC-SCOPF with complementarity-modelled recourse, as an MPCC.

Follows Section II (eq. agc, droopmpec, pvpq, scopf) and the vertical form of
Section III-A (eq. mpcc): every inequality gets a nonnegative slack, and the
two complementarity systems become pairs (w1, w2) >= 0 with w1 * w2 <= 0.

Readings where the paper is silent:
  * flows use the textbook pi-model (tap 1, no phase shift):
      S_ij = V_i conj(y (V_i - V_j) + j b_c/2 V_i),  y = 1/(r + jx) = g + jb;
  * bus balance: sum_g p_g - Pd - Gs v^2 - sum_arcs p_arc = 0 (and Q with +Bs v^2);
  * thermal limit per arc end: (p^2 + q^2)/rate^2 - 1 + sigma = 0, sigma >= 0;
  * theta_ref = 0 in every scenario (the reference angle is not a variable);
  * objective: base-case cost sum c2 (100 p)^2 + c1 (100 p) + c0, divided by 1e4;
  * alpha_g = pmax_g / sum of pmax over generators in service in contingency k;
  * generator outage removes the generator and its complementarity rows;
  * PV buses outside a contingency's switch set keep q within bounds and v free
    within [vmin, vmax]; buses in the set get the PV/PQ complementarity (eq. pvpq).

Variable / row layout (the "natural order", shared by convention with the
CUDA library -- both sides build it from the instance independently):

  w = [ block 0 | block 1 | ... | block K | border u0 ]
  border u0 = [ p_g^0 (all gens) | v_b^0 (PV buses, increasing bus id) ]

  block 0 (base) variables: theta_b (b != ref), v_b (non-PV buses), q_g^0,
                 sigma_th (per limited branch: from-end, to-end)
  block k >= 1 variables:   theta_b (b != ref), v_b (all), p_g^k, q_g^k (gens in
                 service), Delta^k, sigma_th (limited in-service branches, f/t),
                 pi_-, pi_+, sig_pmax, sig_pmin (per gen in service),
                 nu_-, nu_+, sig_qmax, sig_qmin (per switch bus)
  equality rows of block k: Pbal_b, Qbal_b (all buses), thermal (f, t per limited
                 branch); k >= 1 adds droop, sig_pmax-def, sig_pmin-def (per gen),
                 pvpq, sig_qmax-def, sig_qmin-def (per switch bus)
  complementarity pairs of block k >= 1 (in this order):
                 (pi_-, sig_pmax), (pi_+, sig_pmin) per gen, then
                 (nu_-, sig_qmax), (nu_+, sig_qmin) per switch bus.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

OBJ_SCALE = 1.0e4
BASE_MVA = 100.0
INF = np.inf


class Block:
    """Index maps of one scenario block (k = 0 is the base case)."""


class SCOPFModel:
    """Model functions of eq. (scopf) in the vertical MPCC form (eq. mpcc)."""

    def __init__(self, inst):
        self.inst = inst
        net = inst.net
        self.net = net
        nb, nl, ng = net.n_bus, net.n_branch, net.n_gen
        self.nb, self.nl, self.ng = nb, nl, ng
        if len(set(net.gbus.tolist())) != ng:
            raise ValueError("at most one generator per bus is supported")
        self.ref = int(net.ref_bus)
        self.gen_at = np.full(nb, -1, dtype=np.int64)
        self.gen_at[net.gbus] = np.arange(ng)
        self.pv = np.sort(net.gbus.astype(np.int64))
        self.npv = len(self.pv)
        self.pv_pos = np.full(nb, -1, dtype=np.int64)
        self.pv_pos[self.pv] = np.arange(self.npv)
        # branch admittances (pi-model, tap 1, no shift)
        z2 = net.r ** 2 + net.x ** 2
        self.g = net.r / z2
        self.bs = -net.x / z2
        self.bc = net.b
        self.limited = net.rate > 0
        self.blocks = [self._make_block(k) for k in range(inst.K + 1)]
        off_w, off_c, off_p = 0, 0, 0
        for blk in self.blocks:
            blk.w0, blk.c0, blk.p0 = off_w, off_c, off_p
            off_w += blk.nvar
            off_c += blk.nrow
            off_p += blk.ncomp
        self.border0 = off_w
        self.nborder = ng + self.npv
        self.n = off_w + self.nborder
        self.m = off_c
        self.p = off_p
        for blk in self.blocks:
            self._globalize(blk)
        self._bounds()
        self._comp_pairs()

    # ------------------------------------------------------------------ layout
    def _make_block(self, k):
        net, nb, ng = self.net, self.nb, self.ng
        blk = Block()
        blk.k = k
        if k == 0:
            blk.kind, blk.element = -1, -1
            blk.gens = np.arange(ng)
            blk.branches = np.arange(self.nl)
            blk.switch = np.zeros(0, dtype=np.int64)
        else:
            c = self.inst.ctgs[k - 1]
            blk.kind, blk.element = c.kind, c.element
            blk.gens = np.array([g for g in range(ng) if not (c.kind == 1 and g == c.element)],
                                dtype=np.int64)
            blk.branches = np.array([l for l in range(self.nl) if not (c.kind == 0 and l == c.element)],
                                    dtype=np.int64)
            blk.switch = np.asarray(c.switch_buses, dtype=np.int64)
        blk.thermal = blk.branches[self.limited[blk.branches]]
        nxt = [0]

        def take(cnt):
            a = np.arange(nxt[0], nxt[0] + cnt)
            nxt[0] += cnt
            return a

        # local variable indices (-1 = not a variable of this block)
        blk.th = np.full(nb, -1, dtype=np.int64)
        nonref = np.array([b for b in range(nb) if b != self.ref], dtype=np.int64)
        blk.th[nonref] = take(nb - 1)
        blk.v = np.full(nb, -1, dtype=np.int64)
        if k == 0:
            nonpv = np.array([b for b in range(nb) if self.gen_at[b] < 0], dtype=np.int64)
            blk.v[nonpv] = take(len(nonpv))
        else:
            blk.v[:] = take(nb)
        blk.p = np.full(ng, -1, dtype=np.int64)
        blk.q = np.full(ng, -1, dtype=np.int64)
        if k > 0:
            blk.p[blk.gens] = take(len(blk.gens))
        blk.q[blk.gens] = take(len(blk.gens))
        blk.delta = take(1)[0] if k > 0 else -1
        nth = len(blk.thermal)
        blk.sth = take(2 * nth).reshape(nth, 2) if nth else np.zeros((0, 2), dtype=np.int64)
        ngk, nsw = (len(blk.gens), len(blk.switch)) if k > 0 else (0, 0)
        blk.pim, blk.pip = take(ngk), take(ngk)
        blk.spu, blk.spl = take(ngk), take(ngk)
        blk.num, blk.nup = take(nsw), take(nsw)
        blk.squ, blk.sql = take(nsw), take(nsw)
        blk.nvar = nxt[0]
        # local rows
        nxt[0] = 0
        blk.rP, blk.rQ = take(nb), take(nb)
        blk.rth = take(2 * nth).reshape(nth, 2) if nth else np.zeros((0, 2), dtype=np.int64)
        blk.rdroop, blk.rspu, blk.rspl = take(ngk), take(ngk), take(ngk)
        blk.rpvpq, blk.rsqu, blk.rsql = take(nsw), take(nsw), take(nsw)
        blk.nrow = nxt[0]
        blk.ncomp = 2 * ngk + 2 * nsw
        blk.sw_gen = self.gen_at[blk.switch] if nsw else np.zeros(0, dtype=np.int64)
        return blk

    def _globalize(self, blk):
        """Global w indices of every quantity block k touches."""
        b0 = blk.w0
        g = lambda a: np.where(a >= 0, a + b0, -1)
        blk.gth = g(blk.th)
        blk.gv = g(blk.v)
        blk.gp = g(blk.p)
        blk.gq = g(blk.q)
        if blk.k == 0:
            # base-case p_g and PV voltages are the border u0
            blk.gp = self.border0 + np.arange(self.ng)
            blk.gv = blk.gv.copy()
            blk.gv[self.pv] = self.border0 + self.ng + np.arange(self.npv)
        blk.gdelta = blk.delta + b0 if blk.delta >= 0 else -1
        blk.gsth = blk.sth + b0
        for nm in ("pim", "pip", "spu", "spl", "num", "nup", "squ", "sql"):
            setattr(blk, "g" + nm, getattr(blk, nm) + b0)
        for nm in ("rP", "rQ", "rth", "rdroop", "rspu", "rspl", "rpvpq", "rsqu", "rsql"):
            setattr(blk, "g" + nm, getattr(blk, nm) + blk.c0)
        # border indices this contingency couples to
        blk.gp0 = self.border0 + np.arange(self.ng)
        blk.gv0 = self.border0 + self.ng + self.pv_pos

    def _bounds(self):
        net = self.net
        wl = np.full(self.n, -INF)
        wu = np.full(self.n, INF)
        for blk in self.blocks:
            vb = blk.gv >= 0
            # voltage bounds on every voltage variable (base PV voltages are border)
            wl[blk.gv[vb]] = net.vmin[vb]
            wu[blk.gv[vb]] = net.vmax[vb]
            wl[blk.gsth.ravel()] = 0.0
            if blk.k == 0:
                wl[blk.gp[blk.gens]] = net.pmin
                wu[blk.gp[blk.gens]] = net.pmax
                wl[blk.gq[blk.gens]] = net.qmin
                wu[blk.gq[blk.gens]] = net.qmax
            else:
                for nm in ("pim", "pip", "spu", "spl", "num", "nup", "squ", "sql"):
                    wl[getattr(blk, "g" + nm)] = 0.0
                on_switch = np.zeros(self.ng, dtype=bool)
                on_switch[blk.sw_gen] = True
                plain = blk.gens[~on_switch[blk.gens]]
                wl[blk.gq[plain]] = net.qmin[plain]
                wu[blk.gq[plain]] = net.qmax[plain]
        self.wl, self.wu = wl, wu

    def _comp_pairs(self):
        c1, c2 = [], []
        for blk in self.blocks[1:]:
            c1 += [blk.gpim, blk.gpip, blk.gnum, blk.gnup]
            c2 += [blk.gspu, blk.gspl, blk.gsqu, blk.gsql]
        self.comp1 = np.concatenate(c1) if c1 else np.zeros(0, dtype=np.int64)
        self.comp2 = np.concatenate(c2) if c2 else np.zeros(0, dtype=np.int64)

    # ---------------------------------------------------------- start point
    def initial_point(self):
        """Flat start: theta = 0, v = 1, p at mid-range, q = 0, slacks consistent."""
        net = self.net
        w = np.zeros(self.n)
        pmid = 0.5 * (net.pmin + net.pmax)
        qmid = 0.5 * (net.qmin + net.qmax)
        w[self.border0:self.border0 + self.ng] = pmid
        for blk in self.blocks:
            w[blk.gv[blk.gv >= 0]] = 1.0
            w[blk.gq[blk.gens]] = qmid[blk.gens]
            w[blk.gsth.ravel()] = 1.0
            if blk.k > 0:
                w[blk.gp[blk.gens]] = pmid[blk.gens]
                w[blk.gspu] = net.pmax[blk.gens] - pmid[blk.gens]
                w[blk.gspl] = pmid[blk.gens] - net.pmin[blk.gens]
                sg = blk.sw_gen
                w[blk.gsqu] = net.qmax[sg] - qmid[sg]
                w[blk.gsql] = qmid[sg] - net.qmin[sg]
        return w

    # ------------------------------------------------------- pi-model flows
    # Each arc flow has the form F = A vi^2 + B vj^2 + vi vj (al cos(ti-tj) + be sin(ti-tj)):
    #   p_ij: A = g,         B = 0, al = -g, be = -b
    #   q_ij: A = -(b+bc/2), B = 0, al =  b, be = -g
    #   p_ji: A = 0, B = g,         al = -g, be =  b
    #   q_ji: A = 0, B = -(b+bc/2), al =  b, be =  g
    def _coef(self, lines):
        g, b, bc = self.g[lines], self.bs[lines], self.bc[lines]
        z = np.zeros_like(g)
        sh = -(b + 0.5 * bc)
        A = np.stack([g, sh, z, z])
        B = np.stack([z, z, g, sh])
        al = np.stack([-g, b, -g, b])
        be = np.stack([-b, -g, b, g])
        return A, B, al, be

    def _vals(self, w, blk, lines):
        net = self.net
        f, t = net.f[lines], net.t[lines]
        thi = np.where(blk.gth[f] >= 0, w[np.maximum(blk.gth[f], 0)], 0.0)
        thj = np.where(blk.gth[t] >= 0, w[np.maximum(blk.gth[t], 0)], 0.0)
        vi, vj = w[blk.gv[f]], w[blk.gv[t]]
        return f, t, thi - thj, vi, vj

    def flows(self, w, blk, lines):
        """(4, L) array of p_ij, q_ij, p_ji, q_ji."""
        f, t, th, vi, vj = self._vals(w, blk, lines)
        A, B, al, be = self._coef(lines)
        T = al * np.cos(th) + be * np.sin(th)
        return A * vi ** 2 + B * vj ** 2 + vi * vj * T

    def flow_derivs(self, w, blk, lines):
        """Gradients (4, L, 4) and Hessians (4, L, 4, 4) of the four arc flows
        w.r.t. x = (theta_i, theta_j, v_i, v_j)."""
        f, t, th, vi, vj = self._vals(w, blk, lines)
        A, B, al, be = self._coef(lines)
        c, s = np.cos(th), np.sin(th)
        T = al * c + be * s
        Tp = -al * s + be * c
        Tpp = -T
        L = len(lines)
        G = np.zeros((4, L, 4))
        G[:, :, 0] = vi * vj * Tp
        G[:, :, 1] = -vi * vj * Tp
        G[:, :, 2] = 2 * A * vi + vj * T
        G[:, :, 3] = 2 * B * vj + vi * T
        H = np.zeros((4, L, 4, 4))
        H[:, :, 0, 0] = vi * vj * Tpp
        H[:, :, 1, 1] = vi * vj * Tpp
        H[:, :, 0, 1] = H[:, :, 1, 0] = -vi * vj * Tpp
        H[:, :, 0, 2] = H[:, :, 2, 0] = vj * Tp
        H[:, :, 0, 3] = H[:, :, 3, 0] = vi * Tp
        H[:, :, 1, 2] = H[:, :, 2, 1] = -vj * Tp
        H[:, :, 1, 3] = H[:, :, 3, 1] = -vi * Tp
        H[:, :, 2, 2] = 2 * A
        H[:, :, 3, 3] = 2 * B
        H[:, :, 2, 3] = H[:, :, 3, 2] = T
        return G, H

    def _xidx(self, blk, lines):
        f, t = self.net.f[lines], self.net.t[lines]
        return np.stack([blk.gth[f], blk.gth[t], blk.gv[f], blk.gv[t]], axis=1)  # (L,4), -1 = const

    # ------------------------------------------------------------ functions
    def objective(self, w):
        net = self.net
        p = w[self.border0:self.border0 + self.ng] * BASE_MVA
        return float(np.sum(net.c2 * p ** 2 + net.c1 * p + net.c0)) / OBJ_SCALE

    def gradient(self, w):
        net = self.net
        gr = np.zeros(self.n)
        p = w[self.border0:self.border0 + self.ng] * BASE_MVA
        gr[self.border0:self.border0 + self.ng] = (2 * net.c2 * p + net.c1) * BASE_MVA / OBJ_SCALE
        return gr

    def alpha(self, blk):
        net = self.net
        a = np.zeros(self.ng)
        a[blk.gens] = net.pmax[blk.gens] / net.pmax[blk.gens].sum()
        return a

    def constraints(self, w):
        """c(w), all equality rows of eq. (mpcc) (complementarity excluded)."""
        net = self.net
        c = np.zeros(self.m)
        for blk in self.blocks:
            P = -net.Pd - net.Gs * w[blk.gv] ** 2
            Q = -net.Qd + net.Bs * w[blk.gv] ** 2
            np.add.at(P, net.gbus[blk.gens], w[blk.gp[blk.gens]])
            np.add.at(Q, net.gbus[blk.gens], w[blk.gq[blk.gens]])
            lines = blk.branches
            F = self.flows(w, blk, lines)
            np.add.at(P, net.f[lines], -F[0])
            np.add.at(Q, net.f[lines], -F[1])
            np.add.at(P, net.t[lines], -F[2])
            np.add.at(Q, net.t[lines], -F[3])
            c[blk.grP] = P
            c[blk.grQ] = Q
            if len(blk.thermal):
                Ft = self.flows(w, blk, blk.thermal)
                r2 = net.rate[blk.thermal] ** 2
                c[blk.grth[:, 0]] = (Ft[0] ** 2 + Ft[1] ** 2) / r2 - 1.0 + w[blk.gsth[:, 0]]
                c[blk.grth[:, 1]] = (Ft[2] ** 2 + Ft[3] ** 2) / r2 - 1.0 + w[blk.gsth[:, 1]]
            if blk.k > 0:
                gk = blk.gens
                a = self.alpha(blk)[gk]
                pk = w[blk.gp[gk]]
                p0 = w[blk.gp0[gk]]
                # eq. (droopmpec): pi_+ - pi_- = p^k - (p^0 + alpha Delta^k)
                c[blk.grdroop] = w[blk.gpip] - w[blk.gpim] - pk + p0 + a * w[blk.gdelta]
                c[blk.grspu] = w[blk.gspu] + pk - net.pmax[gk]
                c[blk.grspl] = w[blk.gspl] - pk + net.pmin[gk]
                sb, sg = blk.switch, blk.sw_gen
                # eq. (pvpq): nu_+ - nu_- = v^k - v^0
                c[blk.grpvpq] = w[blk.gnup] - w[blk.gnum] - w[blk.gv[sb]] + w[blk.gv0[sb]]
                c[blk.grsqu] = w[blk.gsqu] + w[blk.gq[sg]] - net.qmax[sg]
                c[blk.grsql] = w[blk.gsql] - w[blk.gq[sg]] + net.qmin[sg]
        return c

    def jacobian(self, w):
        """J = dc/dw as scipy CSR (m x n)."""
        net = self.net
        R, C, V = [], [], []

        def add(r, cidx, v):
            r = np.asarray(r).ravel()
            cidx = np.asarray(cidx).ravel()
            v = np.broadcast_to(np.asarray(v, dtype=float), r.shape).ravel()
            keep = cidx >= 0
            R.append(r[keep]); C.append(cidx[keep]); V.append(v[keep])

        for blk in self.blocks:
            vb = blk.gv
            add(blk.grP, vb, -2 * net.Gs * w[vb])
            add(blk.grQ, vb, 2 * net.Bs * w[vb])
            gk = blk.gens
            add(blk.grP[net.gbus[gk]], blk.gp[gk], 1.0)
            add(blk.grQ[net.gbus[gk]], blk.gq[gk], 1.0)
            lines = blk.branches
            G, _ = self.flow_derivs(w, blk, lines)
            X = self._xidx(blk, lines)
            f, t = net.f[lines], net.t[lines]
            for a, rows in ((0, blk.grP[f]), (1, blk.grQ[f]), (2, blk.grP[t]), (3, blk.grQ[t])):
                for j in range(4):
                    add(rows, X[:, j], -G[a, :, j])
            if len(blk.thermal):
                th = blk.thermal
                Ft = self.flows(w, blk, th)
                Gt, _ = self.flow_derivs(w, blk, th)
                Xt = self._xidx(blk, th)
                r2 = net.rate[th] ** 2
                for e, (ip, iq) in enumerate(((0, 1), (2, 3))):
                    rows = blk.grth[:, e]
                    for j in range(4):
                        add(rows, Xt[:, j], 2 * (Ft[ip] * Gt[ip, :, j] + Ft[iq] * Gt[iq, :, j]) / r2)
                    add(rows, blk.gsth[:, e], 1.0)
            if blk.k > 0:
                a = self.alpha(blk)[gk]
                add(blk.grdroop, blk.gpip, 1.0)
                add(blk.grdroop, blk.gpim, -1.0)
                add(blk.grdroop, blk.gp[gk], -1.0)
                add(blk.grdroop, blk.gp0[gk], 1.0)
                add(blk.grdroop, np.full(len(gk), blk.gdelta), a)
                add(blk.grspu, blk.gspu, 1.0)
                add(blk.grspu, blk.gp[gk], 1.0)
                add(blk.grspl, blk.gspl, 1.0)
                add(blk.grspl, blk.gp[gk], -1.0)
                sb, sg = blk.switch, blk.sw_gen
                add(blk.grpvpq, blk.gnup, 1.0)
                add(blk.grpvpq, blk.gnum, -1.0)
                add(blk.grpvpq, blk.gv[sb], -1.0)
                add(blk.grpvpq, blk.gv0[sb], 1.0)
                add(blk.grsqu, blk.gsqu, 1.0)
                add(blk.grsqu, blk.gq[sg], 1.0)
                add(blk.grsql, blk.gsql, 1.0)
                add(blk.grsql, blk.gq[sg], -1.0)
        R = np.concatenate(R); C = np.concatenate(C); V = np.concatenate(V)
        return sp.csr_matrix((V, (R, C)), shape=(self.m, self.n))

    def hessian(self, w, lam, obj_factor=1.0):
        """obj_factor * grad^2 phi + sum_i lam_i grad^2 c_i, full symmetric CSR (n x n)."""
        net = self.net
        R, C, V = [], [], []

        def add(r, cidx, v):
            r = np.asarray(r).ravel(); cidx = np.asarray(cidx).ravel()
            v = np.broadcast_to(np.asarray(v, dtype=float), r.shape).ravel()
            keep = (r >= 0) & (cidx >= 0)
            R.append(r[keep]); C.append(cidx[keep]); V.append(v[keep])

        gp0 = self.border0 + np.arange(self.ng)
        add(gp0, gp0, obj_factor * 2 * net.c2 * BASE_MVA ** 2 / OBJ_SCALE)
        for blk in self.blocks:
            vb = blk.gv
            lP, lQ = lam[blk.grP], lam[blk.grQ]
            add(vb, vb, -2 * net.Gs * lP + 2 * net.Bs * lQ)
            lines = blk.branches
            f, t = net.f[lines], net.t[lines]
            _, Hf = self.flow_derivs(w, blk, lines)
            X = self._xidx(blk, lines)
            # balance rows carry the arc flows with a minus sign
            wgt = np.stack([-lP[f], -lQ[f], -lP[t], -lQ[t]])  # (4, L)
            Hsum = np.einsum("al,alij->lij", wgt, Hf)
            if len(blk.thermal):
                th = blk.thermal
                pos = np.searchsorted(lines, th)
                Ft = self.flows(w, blk, th)
                Gt, Ht = self.flow_derivs(w, blk, th)
                r2 = net.rate[th] ** 2
                for e, (ip, iq) in enumerate(((0, 1), (2, 3))):
                    mu = lam[blk.grth[:, e]] * 2 / r2
                    Hth = (np.einsum("li,lj->lij", Gt[ip], Gt[ip]) + Ft[ip][:, None, None] * Ht[ip]
                           + np.einsum("li,lj->lij", Gt[iq], Gt[iq]) + Ft[iq][:, None, None] * Ht[iq])
                    Hsum[pos] += mu[:, None, None] * Hth
            for i in range(4):
                for j in range(4):
                    add(X[:, i], X[:, j], Hsum[:, i, j])
        R = np.concatenate(R); C = np.concatenate(C); V = np.concatenate(V)
        return sp.csr_matrix((V, (R, C)), shape=(self.n, self.n))

    # ------------------------------------------------------- summaries
    def nvar_ncon(self):
        """(number of variables, number of constraints incl. complementarity)."""
        return self.n, self.m + self.p
