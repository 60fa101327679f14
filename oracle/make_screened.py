"""Write the screened contingency lists of the synthetic workloads.

Runs the oracle's screening (``oracle.screening``, Section V-B of the paper)
over the seeded candidate outages of each workload network and stores, in
``synthgrid/screened/<name>.json``, the candidates accepted in candidate
order (stopping once enough are found), the load scale used and the base
control u0.  ``synthgrid.config_instance`` reads these files.

    python -m oracle.make_screened 0 1 2 4        # workloads to screen
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

import synthgrid


def _screen_one(args):
    idx, load_scale, kind, pos, u0 = args
    from oracle.screening import screen_candidate
    inst = _unscreened(idx, load_scale)
    cand = (inst.candidates.lines if kind == "line" else inst.candidates.gens)[pos]
    ok, feas, status = screen_candidate(inst, cand, np.asarray(u0), eps=FIX_EPS)
    return kind, pos, cand.element, ok, feas, status


# Screening at a fixed first stage (Section V-B) taken from a base-case OPF
# with derated limits: every accepted outage is feasible at the same u0, so
# the SCOPF over all of them is feasible.
DERATE = 0.75       # thermal ratings of the base point
V_MARGIN = 0.01     # voltage band of the base point narrowed by this much
FIX_EPS = 1e-3      # u0 held within +-FIX_EPS of the base point


_CACHE = {}


def _unscreened(idx, load_scale):
    key = (idx, load_scale)
    if key not in _CACHE:
        c = dict(synthgrid.CONFIGS[idx])
        name = c.pop("name")
        c.pop("network_seed_of", None)
        c.pop("screen_as", None)
        _CACHE[key] = synthgrid.make_instance(seed=1000 + idx, name=name,
                                              load_scale=load_scale, **c)
    return _CACHE[key]


def screen_config(idx: int, workers: int) -> dict:
    from oracle.screening import base_opf
    c = synthgrid.CONFIGS[idx]
    scale = 1.0
    while True:
        inst = _unscreened(idx, scale)
        res, u0 = base_opf(inst)
        print(f"[{c['name']}] base OPF status {res.status} obj {res.objective:.6f} "
              f"scale {scale:.3f} ({res.wall_s:.1f}s)", flush=True)
        if res.status == "ok":
            break
        scale *= 0.9
    derate, vm = DERATE, V_MARGIN
    for derate, vm in ((DERATE, V_MARGIN), (0.85, 0.005), (1.0, 0.0)):
        resc, u0c = base_opf(inst, derate=derate, v_margin=vm)
        print(f"[{c['name']}] derated base point (rating x{derate}, v margin {vm}): "
              f"{resc.status} obj {resc.objective:.6f}", flush=True)
        if resc.status == "ok":
            u0 = u0c
            break
    out = dict(name=c["name"], load_scale=scale, base_objective=res.objective,
               derate=derate, v_margin=vm, fix_eps=FIX_EPS,
               u0=u0.tolist(), accepted_lines=[], accepted_gens=[], rejected=[])
    need = {"line": c["n_line_ctg"], "gen": c["n_gen_ctg"]}
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for kind in ("line", "gen"):
            cands = inst.candidates.lines if kind == "line" else inst.candidates.gens
            pos = 0
            acc = out["accepted_lines"] if kind == "line" else out["accepted_gens"]
            while len(acc) < need[kind] and pos < len(cands):
                batch = list(range(pos, min(len(cands), pos + max(workers, need[kind] - len(acc)))))
                pos = batch[-1] + 1
                results = pool.map(_screen_one, [(idx, scale, kind, p, u0.tolist()) for p in batch])
                for kind_, p, el, ok, feas, status in results:
                    if ok and len(acc) < need[kind]:
                        acc.append(int(el))
                    elif not ok:
                        out["rejected"].append(dict(kind=kind_, element=int(el), feas=feas,
                                                    status=status))
                print(f"[{c['name']}] {kind}: screened {pos}/{len(cands)}, accepted {len(acc)}"
                      f" ({time.time() - t0:.0f}s)", flush=True)
    return out


def main(argv):
    idxs = [int(a) for a in argv] or [0, 1, 2, 4]
    workers = int(os.environ.get("SCREEN_WORKERS", os.cpu_count() or 1))
    os.makedirs(synthgrid._SCREEN_DIR, exist_ok=True)
    for idx in idxs:
        out = screen_config(idx, workers)
        path = synthgrid.screening_file(idx)
        with open(path, "w") as fh:
            json.dump(out, fh, indent=1)
        print(f"wrote {path}: {len(out['accepted_lines'])} lines, "
              f"{len(out['accepted_gens'])} gens, {len(out['rejected'])} rejected", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
