"""Seeded synthetic AC transmission networks and contingency lists.

This module only *makes inputs*: buses, branches, generators, contingencies,
PV/PQ switch sets and thermal ratings.  It holds none of the arithmetic of the
solution method (no power-flow equations in polar form, no optimisation, no
linear algebra of the Newton step).  Both the CPU oracle and the CUDA library
consume its output; neither is imported here.

The paper measures on MATPOWER cases (Section V).  Those cases are not
available, so every workload is a seeded synthetic stand-in with the sizes the
paper's cases have (see ``CONFIGS``).  All random draws come from the
SplitMix64 generator below (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so an instance depends only on
its seed.

Units are per unit on a 100 MVA base.  Generator cost coefficients are in
MATPOWER's convention ($/MW^2h, $/MWh).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

_MASK64 = (1 << 64) - 1

CTG_LINE = 0
CTG_GEN = 1


class SplitMix64:
    """SplitMix64 (Steele et al. 2014): state += golden gamma, then mix."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        # 53 high bits -> [0, 1)
        return a + (b - a) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def randbelow(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("randbelow needs n > 0")
        limit = (_MASK64 + 1) - ((_MASK64 + 1) % n)
        while True:
            v = self.next_u64()
            if v < limit:
                return v % n

    def shuffle(self, items: list) -> list:
        """Fisher-Yates, in place; returns the list."""
        for i in range(len(items) - 1, 0, -1):
            j = self.randbelow(i + 1)
            items[i], items[j] = items[j], items[i]
        return items


@dataclass
class Contingency:
    kind: int              # CTG_LINE or CTG_GEN
    element: int           # branch index or generator index
    switch_buses: np.ndarray  # sorted bus ids with PV/PQ complementarity


@dataclass
class Network:
    # buses
    Pd: np.ndarray
    Qd: np.ndarray
    Gs: np.ndarray
    Bs: np.ndarray
    vmin: np.ndarray
    vmax: np.ndarray
    # branches
    f: np.ndarray
    t: np.ndarray
    r: np.ndarray
    x: np.ndarray
    b: np.ndarray
    rate: np.ndarray       # MVA/100; 0 means "no thermal limit"
    # generators
    gbus: np.ndarray
    pmin: np.ndarray
    pmax: np.ndarray
    qmin: np.ndarray
    qmax: np.ndarray
    c2: np.ndarray
    c1: np.ndarray
    c0: np.ndarray
    ref_bus: int
    xy: np.ndarray = field(default=None)  # bus coordinates (generation only)

    @property
    def n_bus(self) -> int:
        return len(self.Pd)

    @property
    def n_branch(self) -> int:
        return len(self.f)

    @property
    def n_gen(self) -> int:
        return len(self.gbus)


@dataclass
class Instance:
    name: str
    net: Network
    ctgs: List[Contingency]
    seed: int
    recipe: dict

    @property
    def K(self) -> int:
        return len(self.ctgs)


# ----------------------------------------------------------------------------
# graph helpers
# ----------------------------------------------------------------------------

def _find(parent, a):
    while parent[a] != a:
        parent[a] = parent[parent[a]]
        a = parent[a]
    return a


def bridges(n: int, f: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Boolean mask of bridge edges (Tarjan's low-link, iterative DFS)."""
    adj = [[] for _ in range(n)]
    for e, (a, b) in enumerate(zip(f.tolist(), t.tolist())):
        adj[a].append((b, e))
        adj[b].append((a, e))
    disc = [-1] * n
    low = [0] * n
    is_bridge = np.zeros(len(f), dtype=bool)
    timer = 0
    for root in range(n):
        if disc[root] != -1:
            continue
        disc[root] = low[root] = timer
        timer += 1
        stack = [(root, -1, iter(adj[root]))]
        while stack:
            v, pe, it = stack[-1]
            advanced = False
            for (w, e) in it:
                if e == pe:
                    continue
                if disc[w] == -1:
                    disc[w] = low[w] = timer
                    timer += 1
                    stack.append((w, e, iter(adj[w])))
                    advanced = True
                    break
                low[v] = min(low[v], disc[w])
            if not advanced:
                stack.pop()
                if stack:
                    u = stack[-1][0]
                    low[u] = min(low[u], low[v])
                    if low[v] > disc[u]:
                        is_bridge[pe] = True
    return is_bridge


def _connected(n, f, t, skip=-1):
    parent = list(range(n))
    for e, (a, b) in enumerate(zip(f.tolist(), t.tolist())):
        if e == skip:
            continue
        ra, rb = _find(parent, a), _find(parent, b)
        if ra != rb:
            parent[ra] = rb
    r0 = _find(parent, 0)
    return all(_find(parent, i) == r0 for i in range(n))


# ----------------------------------------------------------------------------
# network generation
# ----------------------------------------------------------------------------

def make_network(rng: SplitMix64, n_bus: int, mean_degree: float, n_gen: int,
                 knn: int = 6) -> Network:
    """Geometric synthetic grid.

    Buses are uniform in the unit square.  A random spanning tree is drawn
    over the k-nearest-neighbour graph (Kruskal on a random edge order), then
    further k-NN edges are added in random order until the branch count is
    round(mean_degree * n_bus / 2).  Real grids are near-planar with small
    separators; uniformly random extra edges would give an expander instead.
    """
    xy = np.array([[rng.uniform(), rng.uniform()] for _ in range(n_bus)])
    d2 = ((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    cand = set()
    k = min(knn, n_bus - 1)   # never the bus itself (its distance is inf)
    for i in range(n_bus):
        nbrs = np.argsort(d2[i], kind="stable")[:k]
        for j in nbrs.tolist():
            cand.add((min(i, j), max(i, j)))
    cand = sorted(cand)
    order = rng.shuffle(list(range(len(cand))))
    parent = list(range(n_bus))
    tree, rest = [], []
    for idx in order:
        a, b = cand[idx]
        ra, rb = _find(parent, a), _find(parent, b)
        if ra != rb:
            parent[ra] = rb
            tree.append((a, b))
        else:
            rest.append((a, b))
    # join leftover components (rare) by their closest bus pair
    while True:
        roots = sorted({_find(parent, i) for i in range(n_bus)})
        if len(roots) == 1:
            break
        comp0 = [i for i in range(n_bus) if _find(parent, i) == roots[0]]
        other = [i for i in range(n_bus) if _find(parent, i) != roots[0]]
        sub = d2[np.ix_(comp0, other)]
        a_i, b_i = np.unravel_index(np.argmin(sub), sub.shape)
        a, b = comp0[a_i], other[b_i]
        parent[_find(parent, a)] = _find(parent, b)
        tree.append((min(a, b), max(a, b)))
    n_branch = max(len(tree), int(round(mean_degree * n_bus / 2.0)))
    edges = list(tree)
    for e in rest:
        if len(edges) >= n_branch:
            break
        edges.append(e)
    edges.sort()
    n_l = len(edges)
    f = np.array([e[0] for e in edges], dtype=np.int32)
    t = np.array([e[1] for e in edges], dtype=np.int32)
    r = np.array([rng.uniform(0.002, 0.05) for _ in range(n_l)])
    x = np.array([rng.uniform(0.02, 0.3) for _ in range(n_l)])
    b = np.array([rng.uniform(0.0, 0.05) for _ in range(n_l)])

    gen_buses = sorted(rng.shuffle(list(range(n_bus)))[:n_gen])
    gbus = np.array(gen_buses, dtype=np.int32)
    is_gen = np.zeros(n_bus, dtype=bool)
    is_gen[gbus] = True
    Pd = np.array([0.0 if is_gen[i] else rng.uniform(0.2, 1.0) for i in range(n_bus)])
    Qd = 0.3 * Pd
    w = np.array([rng.uniform(0.5, 1.5) for _ in range(n_gen)])
    pmax = 1.6 * Pd.sum() * w / w.sum()
    pmin = np.zeros(n_gen)
    qmax = 0.5 * pmax
    qmin = -0.5 * pmax
    c2 = np.array([rng.uniform(0.005, 0.05) for _ in range(n_gen)])
    c1 = np.array([rng.uniform(10.0, 40.0) for _ in range(n_gen)])
    c0 = np.zeros(n_gen)
    ref_bus = int(gbus[int(np.argmax(pmax))])
    return Network(Pd=Pd, Qd=Qd, Gs=np.zeros(n_bus), Bs=np.zeros(n_bus),
                   vmin=np.full(n_bus, 0.94), vmax=np.full(n_bus, 1.06),
                   f=f, t=t, r=r, x=x, b=b, rate=np.zeros(n_l),
                   gbus=gbus, pmin=pmin, pmax=pmax, qmin=qmin, qmax=qmax,
                   c2=c2, c1=c1, c0=c0, ref_bus=ref_bus, xy=xy)


def _dc_flows(net: Network, skip_branch: int = -1, out_gen: int = -1) -> np.ndarray:
    """Lossless DC flows (B theta = P) at a dispatch proportional to pmax.

    Used only to size the synthetic thermal ratings; the solution method
    never sees it.  A generator outage shifts its output to the others in
    proportion to pmax.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n = net.n_bus
    scale = net.Pd.sum() / net.pmax.sum()
    pg = net.pmax * scale
    if out_gen >= 0:
        lost = pg[out_gen]
        mask = np.ones(net.n_gen, dtype=bool)
        mask[out_gen] = False
        pg = np.where(mask, pg + lost * net.pmax / net.pmax[mask].sum(), 0.0)
    P = -net.Pd.copy()
    np.add.at(P, net.gbus, pg)
    on = np.ones(net.n_branch, dtype=bool)
    if skip_branch >= 0:
        on[skip_branch] = False
    y = 1.0 / net.x[on]
    a, c = net.f[on], net.t[on]
    B = sp.coo_matrix((np.concatenate([y, y, -y, -y]),
                       (np.concatenate([a, c, a, c]), np.concatenate([a, c, c, a]))),
                      shape=(n, n)).tocsc()
    keep = np.array([i for i in range(n) if i != net.ref_bus])
    th = np.zeros(n)
    th[keep] = spla.splu(B[keep][:, keep].tocsc()).solve(P[keep])
    fl = (th[net.f] - th[net.t]) / net.x
    if skip_branch >= 0:
        fl[skip_branch] = 0.0
    return fl


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

CONFIGS = {
    # name: (n_bus, mean_degree, n_gen, n_line_ctg, n_gen_ctg, thermal, switch)
    0: dict(name="syn30_k4", n_bus=30, mean_degree=2.7, n_gen=6, n_line_ctg=4,
            n_gen_ctg=0, thermal=False, switch="full"),
    1: dict(name="syn118_k32", n_bus=118, mean_degree=2.7, n_gen=19, n_line_ctg=28,
            n_gen_ctg=4, thermal=True, switch="full"),
    2: dict(name="syn500_k256", n_bus=500, mean_degree=2.8, n_gen=90, n_line_ctg=220,
            n_gen_ctg=36, thermal=True, switch="random"),
    3: dict(name="syn500_k64", n_bus=500, mean_degree=2.8, n_gen=90, n_line_ctg=55,
            n_gen_ctg=9, thermal=True, switch="random", network_seed_of=2,
            screen_as="syn500_k256"),
    4: dict(name="syn2000_k128", n_bus=2000, mean_degree=2.7, n_gen=360, n_line_ctg=100,
            n_gen_ctg=28, thermal=True, switch="random"),
}

RATING_MARGIN = 1.2
RATING_PF = 1.0440306508910551   # |S| / |P| at the loads' Q = 0.3 P
RATING_ADD = 0.25                # p.u., room for line charging and I^2 x
RATING_FLOOR = 0.5
_SCREEN_DIR = __import__("os").path.join(__import__("os").path.dirname(__file__), "screened")


@dataclass
class Candidates:
    """All single-outage candidates of a network, in seeded order, each with
    its PV/PQ switch set drawn in that order."""
    lines: List[Contingency]
    gens: List[Contingency]


def make_candidates(net: Network, rng: SplitMix64, switch: str) -> Candidates:
    br = bridges(net.n_bus, net.f, net.t)
    lines = [e for e in range(net.n_branch) if not br[e]]
    rng.shuffle(lines)
    gens = rng.shuffle(list(range(net.n_gen)))

    def sw_set(kind, el):
        pv = sorted({int(net.gbus[g]) for g in range(net.n_gen)
                     if not (kind == CTG_GEN and g == el)})
        if switch == "full":
            return np.array(pv, dtype=np.int32)
        frac = rng.uniform(0.5, 1.0)
        cnt = max(1, int(round(frac * len(pv))))
        return np.array(sorted(rng.shuffle(list(pv))[:cnt]), dtype=np.int32)

    return Candidates(lines=[Contingency(CTG_LINE, e, sw_set(CTG_LINE, e)) for e in lines],
                      gens=[Contingency(CTG_GEN, g, sw_set(CTG_GEN, g)) for g in gens])


def set_ratings(net: Network, cands: Candidates) -> None:
    """RATING_MARGIN times the largest DC flow of each branch over the base
    case and every candidate outage (pmax-proportional dispatch), converted
    to apparent power at the loads' power factor, plus RATING_ADD for the
    reactive flows a lossless DC model does not see, floored at RATING_FLOOR.
    """
    worst = np.abs(_dc_flows(net))
    for c in cands.lines:
        worst = np.maximum(worst, np.abs(_dc_flows(net, skip_branch=c.element)))
    for c in cands.gens:
        worst = np.maximum(worst, np.abs(_dc_flows(net, out_gen=c.element)))
    net.rate = np.maximum(RATING_MARGIN * RATING_PF * worst + RATING_ADD, RATING_FLOOR)


def make_instance(n_bus: int, mean_degree: float, n_gen: int, n_line_ctg: int,
                  n_gen_ctg: int, thermal: bool, switch: str, seed: int,
                  name: str = "custom", accepted: dict | None = None,
                  load_scale: float = 1.0) -> Instance:
    """Network + contingency list.

    * line outages: non-bridge branches (the grid stays connected), in a
      seeded random order; generator outages: generators in a seeded order;
    * PV/PQ switch set of a candidate: all in-service generator buses
      ("full") or a seeded subset with 50-100% of them ("random");
    * thermal ratings (when ``thermal``): see ``set_ratings``;
    * ``accepted`` (from the screening file) lists, per kind, the candidate
      elements found feasible at the base-case optimum (Section V-B); the
      instance takes the first ``n_line_ctg`` / ``n_gen_ctg`` of them.
      Without it the first candidates are taken unscreened.
    * ``load_scale`` multiplies every load (recorded by the screening when
      the base case needed it).
    """
    rng = SplitMix64(seed)
    net = make_network(rng, n_bus, mean_degree, n_gen)
    net.Pd = net.Pd * load_scale
    net.Qd = net.Qd * load_scale
    cands = make_candidates(net, rng, switch)
    if thermal:
        set_ratings(net, cands)
    if accepted is None:
        lines = cands.lines[:n_line_ctg]
        gens = cands.gens[:n_gen_ctg]
    else:
        okl, okg = set(accepted["lines"]), set(accepted["gens"])
        lines = [c for c in cands.lines if c.element in okl][:n_line_ctg]
        gens = [c for c in cands.gens if c.element in okg][:n_gen_ctg]
    if len(lines) < n_line_ctg or len(gens) < n_gen_ctg:
        raise ValueError("not enough (screened) candidates for the requested outages")
    recipe = dict(n_bus=n_bus, mean_degree=mean_degree, n_gen=n_gen,
                  n_line_ctg=n_line_ctg, n_gen_ctg=n_gen_ctg, thermal=thermal,
                  switch=switch, seed=seed, rating_margin=RATING_MARGIN,
                  rating_pf=RATING_PF, rating_add=RATING_ADD,
                  rating_floor=RATING_FLOOR, load_scale=load_scale,
                  screened=accepted is not None)
    inst = Instance(name=name, net=net, ctgs=lines + gens, seed=seed, recipe=recipe)
    inst.candidates = cands
    return inst


def screening_file(idx: int) -> str:
    c = CONFIGS[idx]
    return __import__("os").path.join(_SCREEN_DIR, f"{c.get('screen_as', c['name'])}.json")


def config_instance(idx: int, screened: bool = True) -> Instance:
    """Workload ``idx`` (0..4), seed = 1000 + idx (config 3 reuses the
    network and candidates of config 2).  ``screened`` reads the stored
    list of feasible candidates written by the oracle's screening script."""
    import json
    import os
    c = dict(CONFIGS[idx])
    name = c.pop("name")
    seed_of = c.pop("network_seed_of", idx)
    c.pop("screen_as", None)
    accepted, scale = None, 1.0
    if screened:
        path = screening_file(idx)
        if not os.path.exists(path):
            raise FileNotFoundError(f"screening file {path} missing")
        with open(path) as fh:
            data = json.load(fh)
        accepted = dict(lines=data["accepted_lines"], gens=data["accepted_gens"])
        scale = data.get("load_scale", 1.0)
    return make_instance(seed=1000 + seed_of, name=name, accepted=accepted,
                         load_scale=scale, **c)


def screening_batch(idx: int):
    """The candidates the oracle's screening of workload ``idx`` examined,
    as one instance (base case + every examined outage as a scenario, line
    outages then generator outages, each in candidate order), with the
    stored base control u0, box half-width eps and the oracle's verdicts
    (True = accepted) in scenario order."""
    import json
    with open(screening_file(idx)) as fh:
        data = json.load(fh)
    c = dict(CONFIGS[idx])
    name = c.pop("name")
    seed_of = c.pop("network_seed_of", idx)
    c.pop("screen_as", None)
    inst = make_instance(seed=1000 + seed_of, name=name, load_scale=data.get("load_scale", 1.0),
                         **c)
    acc = {"line": set(data["accepted_lines"]), "gen": set(data["accepted_gens"])}
    rej = {"line": set(), "gen": set()}
    for r in data["rejected"]:
        rej[r["kind"]].add(int(r["element"]))
    ctgs, verdict = [], []
    for kind, cands in (("line", inst.candidates.lines), ("gen", inst.candidates.gens)):
        for cand in cands:
            if cand.element in acc[kind] or cand.element in rej[kind]:
                ctgs.append(cand)
                verdict.append(cand.element in acc[kind])
    inst.ctgs = ctgs
    inst.recipe = dict(inst.recipe, screening_batch=True)
    return inst, np.asarray(data["u0"]), float(data["fix_eps"]), verdict
