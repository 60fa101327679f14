#!/usr/bin/env python3
"""Benchmark: Newton steps/s of the NCL / interior-point method on the
synthetic 500-bus x 256-contingency AC-SCOPF, and time to solution.

One "step" is one Newton step of the inner interior-point loop at a fixed
mid-solve iterate: model evaluation and KKT assembly (eq. newtonsystem),
pivot-free block LDL^T with inertia correction, Schur complement and border
factor, solves with FP64 iterative refinement, recovery of the eliminated
directions, fraction-to-boundary and one trial evaluation.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload newton|screen]

Prints one JSON line.  --workload screen times batched contingency
screening (Section V-B) of the same network's candidate outages instead.  With --impl reference the CPU oracle is timed on a
bounded sample of the same workload (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The CPU baseline times the oracle on one core: numpy's BLAS pool reads this
# before it starts, so it is set ahead of every numpy import.
os.environ["OPENBLAS_NUM_THREADS"] = "1"

WORKLOADS = {
    2: ("syn500_k256: 500-bus, 90-generator synthetic grid (mean degree 2.8), 256 contingencies "
        "(220 line, 36 generator), random PV/PQ switch sets; seeded, screened"),
    4: ("syn2000_k128: 2000-bus, 360-generator synthetic grid (mean degree 2.7), 128 "
        "contingencies (100 line, 28 generator), random PV/PQ switch sets (blocks ~2x uneven); "
        "seeded, screened"),
}
SCALE_IDX = 4
METRIC = ("Newton steps/s and SCOPF time-to-solution at 500-bus×256-ctg (1e-6), "
          "vs plain FP64 GPU")
CONFIG_IDX = 2
# FP32 FMA peak from unit counts and clock: 148 SMs x 128 lanes x 2 flops x 2.032 GHz
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# FP64 peak of B300 from its nominal figure (1.25 TFLOP/s dense)
FP64_PEAK_TFLOPS = 1.25


# DRAM bytes (read + write) of one solve's forward and backward sweeps,
# from the ncu capture summarized in profiles/solve_sweeps_syn500_k256.md,
# valid only for the sweep kernels' source it was taken with: the digest
# covers the solve kernels' section of the source and the solve's launch
# function
SWEEP_TRAFFIC = {"source": "paper_2510_13333_b300/csrc/kernels_factor.cu",
                 "sha1": "a908fa075ea548fa73c0b54caca8a944e6f1a6ae",
                 # k_solve_fwd + k_border_gather + k_border_apply + k_solve_bwd (FP32)
                 "bytes_per_solve": 261414912 + 212736 + 296704 + 321260544}


def sweep_source_digest(text: str):
    """sha1 of the sweep kernels' source: from the solves section marker to
    the first kernel after it that is not a solve kernel, plus the
    launch_solve function."""
    import hashlib
    try:
        a = text.index("// ---------------------------------------------------------------- solves")
        b = text.index("k_ruiz_entries(", a)
        b = text.rindex("\n", a, b)
        c = text.index("void launch_solve(")
        d = text.index("#define INST(T)", c)
    except ValueError:
        return None
    return hashlib.sha1((text[a:b] + text[c:d]).encode()).hexdigest()


def sweep_traffic():
    try:
        with open(os.path.join(ROOT, SWEEP_TRAFFIC["source"])) as fh:
            if sweep_source_digest(fh.read()) != SWEEP_TRAFFIC["sha1"]:
                return None
    except OSError:
        return None
    return SWEEP_TRAFFIC["bytes_per_solve"]


def max_over_ranks(ms, dist, device):
    """The largest per-rank time: a job's step time is its slowest replica's."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units every replica processed over the slowest
    replica's time (ms)."""
    return world * units_per_rank / (ms / 1e3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class Clocks:
    """nvidia-smi sampling around the timed region: one nvidia-smi process
    in loop mode (-lms 50).  Samples read between mark() (or start()) and
    stop() count; if none landed there, the first one read after the mark
    is kept."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.samples = []   # (host time read, fields)
        self._p = None
        self._t = None
        self.t0 = None

    def start(self):
        self.t0 = time.perf_counter()
        try:
            self._p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-i",
                 str(int(os.environ.get("LOCAL_RANK", "0"))), "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._p = None
            return

        def run():
            for line in self._p.stdout:
                line = line.strip()
                if line:
                    self.samples.append((time.perf_counter(), [x.strip() for x in line.split(",")]))
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()

    def mark(self):
        """The timed region starts now."""
        self.t0 = time.perf_counter()

    def stop(self):
        t1 = time.perf_counter()
        time.sleep(0.06)   # the sample taken at the end of the region
        if self._p is not None:
            self._p.terminate()
            try:
                self._p.wait(timeout=5)
            except Exception:
                self._p.kill()
        if self._t:
            self._t.join(timeout=5)
        inside = [f for t, f in self.samples if self.t0 <= t <= t1 + 0.06]
        if not inside:
            inside = [f for t, f in self.samples if t >= self.t0][:1]
        sm = [float(f[0]) for f in inside if f[0].replace(".", "").isdigit()]
        mx = [float(f[1]) for f in inside if len(f) > 1 and f[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for f in inside for i in range(4)
                          if len(f) > 3 + i and f[3 + i].lower().startswith("active")})
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


# ------------------------------------------------------------- reference arm
def one_blas_thread():
    """BLAS limited to one thread around an oracle timing: threadpoolctl
    where it is installed, else the OPENBLAS_NUM_THREADS setting above."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:
        import contextlib
        return contextlib.nullcontext()
    return threadpool_limits(limits=1)


ORACLE_SAMPLE_CTG = 8      # contingencies in the oracle's bounded sample
ORACLE_SAMPLE_ITERATE = 30  # IPM iterations before the timed steps (as the GPU arm)


class OracleSample:
    """The CPU oracle on a bounded sample of the benchmark workload: the
    500-bus network with the first ORACLE_SAMPLE_CTG of its 256 contingencies.
    Like the GPU arm, the timed Newton steps are taken at the iterate the
    oracle itself reaches after ORACLE_SAMPLE_ITERATE interior-point
    iterations, from the delta_w it ended with."""

    def __init__(self, n_ctg=ORACLE_SAMPLE_CTG, iterate_at=ORACLE_SAMPLE_ITERATE, idx=CONFIG_IDX):
        import numpy as np
        import synthgrid
        from dataclasses import replace
        from oracle.linsolve import SparseLDLSolver
        from oracle.ncl import NCLSolver, Options
        from oracle.scopf_model import SCOPFModel
        from oracle import symbolic
        inst = synthgrid.config_instance(idx)
        self.net_name = f"{inst.net.n_bus}-bus"
        self.full_blocks = inst.K + 1
        inst.ctgs = inst.ctgs[:n_ctg]
        self.blocks = n_ctg + 1
        with one_blas_thread():   # BLAS on one thread; the C LDL^T is single-threaded
            t0 = time.perf_counter()
            M = SCOPFModel(inst)
            perm, _ = symbolic.kkt_permutation(M)
            S = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm),
                          replace(Options(), max_inner=iterate_at))
            r = S.solve()
            self.setup_s = time.perf_counter() - t0
        self.M, self.S, self.np = M, S, np
        self.st, self.prm, self.mu = r.state, r.params, r.mu
        self.dw_last = next((h["delta_w"] for h in reversed(r.history) if h["delta_w"] > 0), 0.0)
        self.iterate = (f"oracle iterate after {r.inner_iters} IPM iterations (mu {r.mu:.1e}, "
                        f"rho {r.params.rho:.0e})")
        self.tries = []

    def step(self):
        """One oracle Newton step (model, KKT, LDL^T with inertia correction,
        solve, recovery, fraction to boundary, one trial evaluation);
        returns its wall time."""
        S, st, prm, mu = self.S, self.st, self.prm, self.mu
        with one_blas_thread():
            t0 = time.perf_counter()
            res = S.residuals(st, prm)
            H = self.M.hessian(st.w, st.lam)
            sol, delta, tries, _, _ = S.newton_direction(st, prm, res, mu, H, self.dw_last)
            d = S.recover(st, prm, res, mu, sol)
            ap, az = S.frac_to_boundary(st, d, max(0.99, 1 - mu))
            trial = S.step(st, d, ap, az)
            S.theta(trial, self.M.constraints(trial.w))
            dt = time.perf_counter() - t0
        self.tries.append(tries)
        return dt

    def describe(self, n_steps, sec):
        return (f"oracle Newton step (numpy/scipy + C LDL^T, 1 thread) on the {self.net_name} "
                f"network with {self.blocks - 1} of {self.full_blocks - 1} contingencies ({self.blocks} of "
                f"{self.full_blocks} blocks), {self.iterate}; {n_steps} steps timed, "
                f"{sec / n_steps:.3f} s each, {np_mean(self.tries):.1f} factorizations per "
                f"step; full-size rate extrapolated linearly in blocks "
                f"(x {self.full_blocks / self.blocks:.1f})")


def np_mean(v):
    return sum(v) / len(v) if v else 0.0


def oracle_tts_118():
    """The oracle's own time to solution on the 118-bus x 32 workload (the
    smallest block-arrow case; one host core): seconds, IPM iterations and
    seconds per iteration of a full NCL solve at tol 1e-6."""
    import synthgrid
    from oracle.linsolve import SparseLDLSolver
    from oracle.ncl import NCLSolver
    from oracle.scopf_model import SCOPFModel
    from oracle import symbolic
    inst = synthgrid.config_instance(1)
    with one_blas_thread():
        t0 = time.perf_counter()
        M = SCOPFModel(inst)
        perm, _ = symbolic.kkt_permutation(M)
        t1 = time.perf_counter()
        r = NCLSolver(M, SparseLDLSolver(perm_fn=lambda K: perm)).solve()
        t2 = time.perf_counter()
    return {"seconds": t2 - t1, "setup_s": t1 - t0, "status": r.status,
            "inner_iters": r.inner_iters, "s_per_iter": (t2 - t1) / max(1, r.inner_iters),
            "objective": r.objective, "cores": 1}


def gpu_tts_118(P, torch, precision, ipm_graph=1):
    """The library's time to solution on the same 118-bus x 32 workload
    (latency-bound: 48k KKT rows), with the device-resident iteration
    (ipm_graph=1) or the host loop."""
    import synthgrid
    lib = P.SCOPF(synthgrid.config_instance(1), precision=precision, ipm_graph=ipm_graph)
    lib.ncl_solve()   # warm-up (graphs, caches)
    torch.cuda.synchronize()
    n0 = P.scopf_launch_count()
    t0 = time.perf_counter()
    r = lib.ncl_solve()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    launches = P.scopf_launch_count() - n0
    return {"seconds": dt, "status": r["call_status"], "inner_iters": r["inner_iters"],
            "ms_per_iter": 1e3 * dt / max(1, r["inner_iters"]), "objective": r["objective"],
            "factorizations": r["factorizations"],
            "host_round_trips_per_iter": r["host_round_trips"] / max(1, r["inner_iters"]),
            "launches_per_iter": launches / max(1, r["inner_iters"]),
            "graph_iters": r["graph_iters"]}


def host_cpu():
    """The host's CPU model and logical core count (the oracle's machine)."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": model, "nproc": os.cpu_count()}


def oracle_step_sample(n_steps: int = 3, idx: int = CONFIG_IDX):
    """The cpu_baseline leg: n_steps oracle Newton steps of the bounded
    sample; returns (seconds per full-size step extrapolated in blocks,
    description, cores)."""
    o = OracleSample(idx=idx)
    t = sum(o.step() for _ in range(n_steps))
    return t / n_steps * o.full_blocks / o.blocks, o.describe(n_steps, t), 1


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, times --steps Newton
    steps (after --warmup untimed ones) of its bounded sample.  ms_per_step
    is the measured time of one sampled step; value is the full-size rate,
    extrapolated linearly in contingency blocks (the step's work is per
    block)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    o = OracleSample()
    for _ in range(args.warmup):
        o.step()
    o.tries.clear()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step()
    sec = time.perf_counter() - t0
    ms_sample = 1e3 * sec / args.steps
    value = 1e3 / (ms_sample * o.full_blocks / o.blocks)
    line = {"metric": METRIC, "value": value, "unit": "Newton steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_sample,
            "value_basis": (f"ms_per_step is one step of the {o.blocks}-block sample as timed; "
                            f"value = 1000 / (ms_per_step x {o.full_blocks}/{o.blocks}), the "
                            f"full-size rate extrapolated linearly in blocks"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "syn500_k256: 500-bus, 90-generator synthetic grid, 256 "
                                   "contingencies (220 line, 36 generator)",
                       "sample_blocks": o.blocks, "full_blocks": o.full_blocks,
                       "setup_s": o.setup_s, "flush_l2": False},
            "cpu_baseline": {"value": value, "unit": "Newton steps/s", "cores": 1,
                             "kind": "oracle", "sample": o.describe(args.steps, sec),
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "Newton steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PHASE_KEYS = ("factor", "solve", "assemble", "residual", "schur", "front_init", "ipm")


def iteration_stats(names, hist, prec_fp32, prec_fp64, skip=10):
    """The metric's per-iteration rate from the iteration log of one solve:
    IPM iterations (each one Newton step with its inertia corrections,
    refinement and line search) per second over iterations skip..end, from
    the log's wall times; mean and median.  An iteration's time is set mostly
    by its number of factorizations (one, or more with inertia corrections),
    so the log is also split by that count and by the precision of the
    factors that made the step.  The median falls in one of the modes (one
    factorization or two, whichever holds just over half of the iterations)."""
    import numpy as np
    names = list(names)
    h = hist[skip:] if hist.shape[0] > skip else hist
    if not h.shape[0]:
        return {}
    it_ms = h[:, names.index("ms")]
    nf = h[:, names.index("factorizations")].astype(int)
    pr = h[:, names.index("precision")].astype(int)
    rs = h[:, names.index("refine_steps")]
    return {
        "iteration_ms_mean_10_end": float(it_ms.mean()),
        "iterations_per_s_mean_10_end": 1e3 / float(it_ms.mean()),
        "iteration_ms_median_10_end": float(np.median(it_ms)),
        "iterations_per_s_median_10_end": 1e3 / float(np.median(it_ms)),
        "iteration_ms_median_by_factorizations": {
            str(k): {"iterations": int((nf == k).sum()),
                     "ms_median": float(np.median(it_ms[nf == k]))}
            for k in sorted(set(nf.tolist()))},
        "iteration_ms_mean_by_precision": {
            lab: {"iterations": int((pr == v).sum()), "ms_mean": float(it_ms[pr == v].mean()),
                  "refine_steps_mean": float(rs[pr == v].mean())}
            for lab, v in (("fp32", prec_fp32), ("fp64", prec_fp64)) if (pr == v).any()},
    }


def dominant_phase(phases, solves):
    """The phase with the largest total time.  The phase timers see only the
    first block solve of each kkt solve (the refinement's solves run inside
    the device-resident loop's graph), so the solve phase is counted as its
    per-solve time times the number of block solves."""
    tot = {k: phases[k][0] for k in PHASE_KEYS}
    ms, calls = phases["solve"]
    if calls:
        tot["solve"] = ms / calls * max(solves, calls)
    return max(PHASE_KEYS, key=lambda k: tot[k])


def live_peaks():
    """FP32 FMA, FP64 FMA and FP64 tensor-MMA throughput measured now with
    the library's own probe kernels (TFLOP/s, best of 5 launches)."""
    import paper_2510_13333_b300 as P
    return {name: P.scopf_peak_probe(k) for k, name in P.PEAK_KINDS.items()}


def phase_work(sz, prec_bytes):
    """Algorithmic work of one call of each timed phase: (amount, unit, what).
    Bytes are the data the method must move once per call; flops count an
    FMA as 2."""
    N, nnz, nnzL = sz.n_kkt, sz.nnz_kkt, sz.nnz_L
    nc, nblk = sz.n_border, sz.n_blocks
    b = prec_bytes
    return {
        "assemble": (8 * sz.n_elem_values + 24 * sz.n_contrib + 16 * nnz + 48 * N, "B",
                     "element values written, (slot, coefficient, value) per contribution, "
                     "pointer + value per stored entry, iterate and right-hand-side vectors"),
        # power-of-two Ruiz scaling: one sweep for FP32 factors, none for FP64
        # (exact either way; FP64 has the range without it)
        "front_init": ((20 if b == 4 else 0) * nnz + 24 * nnz, "B",
                       ("one Ruiz sweep over (value, column, row, column scale) per stored "
                        "entry, then" if b == 4 else "unit scales, then") +
                       " each front original's value, offset, scales and write"),
        "factor": (sz.factor_flops, "flop", "sum over pivots of (f-c-1)(f-c) on the fronts"),
        "schur": (nblk * nc * nc * b + 8 * nc * nc, "B",
                  "every block's border front read once, S written (the n_c^3/3 dense factor "
                  "is negligible)"),
        "solve": (2 * b * nnzL + 16 * N, "B", "factor entries read by both sweeps, plus the "
                  "right-hand side in and the solution out"),
        "residual": (16 * nnz + 24 * N, "B", "value + column per stored entry, x, b, r"),
    }


def phase_rooflines(sz, phases, solves, prec_bytes, peaks_live):
    """Achieved fraction of each phase's roof.  Per call: the phase's CUDA-
    event time over its calls; the solve phase's timers see only the first
    block solve of each kkt solve, so its per-call time is the timed solves'
    mean."""
    peaks, kind = measured_peaks()
    hbm = peaks["hbm_gbs"]
    work = phase_work(sz, prec_bytes)
    out = {}
    for k, (amount, unit, what) in work.items():
        ms, calls = phases.get(k, (0.0, 0))
        if not calls or ms <= 0:
            continue
        per_call_s = ms / calls / 1e3
        if unit == "flop":
            key = "fp32_fma" if prec_bytes == 4 else "fp64_fma"
            derived = FP32_PEAK_TFLOPS if prec_bytes == 4 else FP64_PEAK_TFLOPS
            ach = amount / per_call_s / 1e12
            out[k] = {"bound": "alu", "achieved": ach, "unit": "TFLOP/s", "peak": derived,
                      "frac": ach / derived, "peak_probe": peaks_live.get(key),
                      "frac_of_probe": ach / peaks_live[key] if peaks_live.get(key) else None,
                      "per_call": amount, "ms_per_call": per_call_s * 1e3, "calls": calls,
                      "work": what}
            if k == "factor":
                # the second roof, that of the small fronts' memory traffic:
                # b nnz(L) written + 8 nnz(K) read
                hb = prec_bytes * sz.nnz_L + 8 * sz.nnz_kkt
                out[k]["hbm"] = {"bytes_per_call": hb, "achieved_gbs": hb / per_call_s / 1e9,
                                 "peak_gbs": hbm, "frac": hb / per_call_s / 1e9 / hbm}
        else:
            ach = amount / per_call_s / 1e9
            out[k] = {"bound": "hbm", "achieved": ach, "unit": "GB/s", "peak": hbm,
                      "peak_kind": kind, "frac": ach / hbm, "per_call": amount,
                      "ms_per_call": per_call_s * 1e3, "calls": calls, "work": what}
    return out


def roofline(sz, phases, dom, prec_bytes=4, peaks_live=None):
    """Roofline object of the dominant phase (factor: ALU; else HBM)."""
    ph = phase_rooflines(sz, phases, 0, prec_bytes, peaks_live or {})
    r = dict(ph[dom])
    r["phase"] = dom
    if dom == "solve":
        r["kernel"] = "k_solve_fwd + k_border_solve + k_solve_bwd (one solve)"
        r["traffic"] = sweep_traffic()
        r["algorithmic_bytes"] = r["per_call"]
    elif dom == "factor":
        r["kernel"] = "k_factor + k_factor_med + k_factor_big (block LDL^T, all blocks)"
        r["traffic"] = None
    else:
        r["traffic"] = None
    return r


# -------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    import synthgrid
    import paper_2510_13333_b300 as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    idx = SCALE_IDX if args.workload == "scale" else CONFIG_IDX
    inst = synthgrid.config_instance(idx)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    t0 = time.perf_counter()
    loop = {"device_loop": 0, "ipm_graph": 0} if args.host_loop else {}
    if args.workload == "condensed":
        loop["dual_first"] = 1
    tune = None
    if not args.no_autotune:
        # supernode tile shapes for this instance (scopf_autotune: Newton
        # steps of each candidate from a common iterate, CUDA events)
        t0 = time.perf_counter()
        tuned, cands = P.autotune(inst, precision=P.PREC_MIXED, **loop)
        loop["cluster_max_tasks"] = tuned.cluster_max_tasks
        loop["relax_max_nodes"] = tuned.relax_max_nodes
        tune = {"seconds": time.perf_counter() - t0,
                "chosen": {"cluster_max_tasks": tuned.cluster_max_tasks,
                           "relax_max_nodes": tuned.relax_max_nodes},
                "candidates": cands}
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        t0 = time.perf_counter()
    lib = P.SCOPF(inst, precision=P.PREC_MIXED, **loop)
    t_create = time.perf_counter() - t0
    torch.cuda.synchronize()
    handle_bytes = free0 - torch.cuda.mem_get_info()[0]
    sz = lib.sizes
    # ---- time to solution (full NCL solve from the flat start)
    tts = {}
    for name, prec in (("mixed", P.PREC_MIXED), ("fp64", P.PREC_FP64)):
        if args.tts == "none" or (name == "fp64" and args.tts != "both"):
            continue
        lib.set_precision(prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = lib.ncl_solve()
        torch.cuda.synchronize()
        tts[name] = {"seconds": time.perf_counter() - t0, "status": r["call_status"],
                     "objective": r["objective"], "inner_iters": r["inner_iters"],
                     "outer_iters": r["outer_iters"], "factorizations": r["factorizations"],
                     "fp64_fallbacks": r["fp64_fallbacks"], "max_violation": r["max_violation"],
                     "kkt_error": r["kkt_error"], "feas_rt": r["feas_rt"],
                     "host_round_trips_per_iter": r["host_round_trips"] / max(1, r["inner_iters"]),
                     "graph_iters": r["graph_iters"]}
        names, hist = lib.history(0)
        tts[name].update(iteration_stats(names, hist, P.PREC_MIXED, P.PREC_FP64))
    if idx == CONFIG_IDX and args.tts != "none":
        tts["118bus_k32"] = {"mixed": gpu_tts_118(P, torch, P.PREC_MIXED),
                             "fp64": gpu_tts_118(P, torch, P.PREC_FP64),
                             "mixed_host_loop": gpu_tts_118(P, torch, P.PREC_MIXED, 0),
                             "fp64_host_loop": gpu_tts_118(P, torch, P.PREC_FP64, 0)}
    # ---- a mid-solve iterate: the state after a fixed number of IPM iterations
    lib.set_precision(P.PREC_MIXED)
    lib2 = P.SCOPF(inst, precision=P.PREC_MIXED, max_inner=args.iterate_at,
                   **{k: v for k, v in loop.items() if k != "device_loop"})
    r = lib2.ncl_solve()
    st = lib2.get_state()
    lam_n, nu0_n, rho = lib2.ncl_params_tensors()
    mu = r["mu"]
    dw_last = r["delta_w_last"]
    del lib2
    direction = lib.new_state()

    apps = [0.0]   # preconditioner applications (block solves) of the last step

    def step(l):
        out, tries = l.scopf_newton_step(st, lam_n, nu0_n, rho, mu, dw_last, direction)
        apps[0] = out[5]
        return out, tries

    launches = [0]

    def timed(l, k, on_start=None):
        for _ in range(args.warmup):
            step(l)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l.scopf_timing(True)
        n0 = P.scopf_launch_count()
        torch.cuda.nvtx.range_push("timed")
        if on_start:
            on_start()
        e0.record(s)
        for _ in range(k):
            step(l)
        e1.record(s)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        launches[0] = P.scopf_launch_count() - n0
        phases = l.scopf_timing(False)
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        return ms, phases

    peaks_live = live_peaks()
    clocks = Clocks()
    clocks.start()
    ms_mixed, ph_mixed = timed(lib, args.steps, clocks.mark)
    launches_mixed = launches[0]
    apps_mixed = apps[0]
    clk = clocks.stop()
    lib.set_precision(P.PREC_FP64)
    ms_fp64, ph_fp64 = timed(lib, max(2, args.steps // 4))
    fp64_steps = max(2, args.steps // 4)
    lib.set_precision(P.PREC_MIXED)
    # ---- end to end through host buffers (pinned): every step copies its inputs
    # host->device and its direction device->host.  The copies run on their own
    # stream, overlapped with the neighbouring steps' compute: inputs and
    # directions are double-buffered on the device, and step i's inputs are
    # uploaded (and step i-2's direction read back) while step i-1 computes.
    host = {k: v.cpu().pin_memory() for k, v in st.items()}
    host_l, host_n = lam_n.cpu().pin_memory(), nu0_n.cpu().pin_memory()
    outs = [{"w": torch.empty(sz.n, dtype=torch.float64).pin_memory(),
             "lam": torch.empty(sz.m, dtype=torch.float64).pin_memory(),
             "yc": torch.empty(sz.p, dtype=torch.float64).pin_memory()} for _ in range(2)]
    h2d = sum(v.numel() * 8 for v in host.values()) + 8 * (host_l.numel() + host_n.numel())
    d2h = 8 * (sz.n + sz.m + sz.p)
    dev_in = [{k: torch.empty_like(v) for k, v in st.items()} for _ in range(2)]
    dls = [torch.empty_like(lam_n) for _ in range(2)]
    dns = [torch.empty_like(nu0_n) for _ in range(2)]
    dirs = [direction, lib.new_state()]
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()

    def upload(b):
        for k in st:
            dev_in[b][k].copy_(host[k], non_blocking=True)
        dls[b].copy_(host_l, non_blocking=True)
        dns[b].copy_(host_n, non_blocking=True)

    def download(b):
        for k in ("w", "lam", "yc"):
            outs[b][k].copy_(dirs[b][k], non_blocking=True)

    def e2e_run(nsteps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        done = [None, None]
        with torch.cuda.stream(copy):
            e0.record(copy)
            upload(0)
        ready = [copy.record_event(), None]
        for i in range(nsteps):
            b = i % 2
            with torch.cuda.stream(copy):
                if done[1 - b] is not None:       # step i-1 used buffer 1-b
                    copy.wait_event(done[1 - b])
                    download(1 - b)
                if i + 1 < nsteps:
                    upload(1 - b)
                ready[1 - b] = copy.record_event()
            comp.wait_event(ready[b])
            lib.scopf_newton_step(dev_in[b], dls[b], dns[b], rho, mu, dw_last, dirs[b])
            done[b] = comp.record_event()
        with torch.cuda.stream(copy):
            last = (nsteps - 1) % 2
            copy.wait_event(done[last])
            download(last)
            e1.record(copy)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    e2e_run(args.warmup)
    if dist:
        dist.barrier()
    ms_e2e = max_over_ranks(e2e_run(args.steps), dist, "cuda")

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    K = args.steps
    value = job_rate(K, world, ms_mixed)
    fp64_value = job_rate(fp64_steps, world, ms_fp64)
    # roofline of the dominant phase (from CUDA events on the handle's stream)
    dom = dominant_phase(ph_mixed, apps_mixed * K)
    roof = roofline(sz, ph_mixed, dom, 4, peaks_live)
    try:
        cpu_s, cpu_desc, cores = oracle_step_sample(idx=idx)
        cpu = {"value": 1.0 / cpu_s, "unit": "Newton steps/s", "cores": cores, "kind": "oracle",
               "sample": cpu_desc, "host": host_cpu()}
        if idx == CONFIG_IDX:
            cpu["tts_118bus_k32"] = oracle_tts_118()
        if "fp64" in tts:
            # the oracle's time to solution at this size, extrapolated (not run):
            # its sampled seconds per Newton step times the IPM iterations of the
            # GPU's FP64 solve (each iteration one Newton step and its trials)
            cpu["tts_extrapolated"] = {
                "seconds": cpu_s * tts["fp64"]["inner_iters"],
                "basis": "oracle s per Newton step (sampled, extrapolated in blocks) x the "
                         "GPU FP64 solve's IPM iterations; not a measured solve"}
    except Exception as exc:  # keep the GPU number even if the CPU sample fails
        cpu = {"value": None, "unit": "Newton steps/s", "cores": 1, "kind": "oracle",
               "sample": f"failed: {exc}"}
    line = {
        "metric": (METRIC if idx == CONFIG_IDX else
                   "Newton steps/s and SCOPF time-to-solution at 2000-bus×128-ctg (1e-6), vs "
                   "plain FP64 GPU") + (", condensed primal variant (dual rows eliminated first)"
                                        if args.workload == "condensed" else ""),
        "value": value, "unit": "Newton steps/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms_mixed / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 block factors + f64 (model, Schur, refinement)", "data": "synthetic",
        "config": {"workload": WORKLOADS[idx] + ("; condensed primal variant (dual-first "
                                                 "order: -C eliminated first, then a pivot-free "
                                                 "Cholesky of A + B' C^-1 B)"
                                                 if args.workload == "condensed" else ""),
                   "n_kkt": sz.n_kkt, "nnz_kkt": sz.nnz_kkt, "nnz_L": sz.nnz_L,
                   "blocks": sz.n_blocks, "border": sz.n_border,
                   "iterate": f"state after {args.iterate_at} IPM iterations (mu {mu:.1e}, "
                              f"rho {rho:.0e}, last delta_w {dw_last:.1e})",
                   "flush_l2": False, "inputs_exceed_l2": True,
                   "parallelism": "replicas only" if world > 1 else "1 GPU"},
        "fp64_newton_steps_per_s": fp64_value,
        "speedup_mixed_vs_fp64": value / fp64_value,
        "time_to_solution": tts,
        "create_s": t_create,
        "autotune": tune,
        "memory": {"device_bytes_handle": handle_bytes, "front_bytes": sz.front_bytes,
                   "bytes_per_block": handle_bytes / sz.n_blocks,
                   "note": "device memory the handle holds (free-memory difference around "
                           "scopf_create: model, KKT pattern and values, fronts, work vectors)"},
        "phases_ms_per_step": {k: v[0] / K for k, v in ph_mixed.items()},
        "block_solves_per_step": apps_mixed,
        "phases_ms_per_step_fp64": {k: v[0] / fp64_steps for k, v in ph_fp64.items()},
        "roofline": roof,
        "roofline_phases": phase_rooflines(sz, ph_mixed, 0, 4, peaks_live),
        "roofline_phases_fp64": phase_rooflines(sz, ph_fp64, 0, 8, peaks_live),
        "peaks_probe_tflops": peaks_live,
        "cpu_baseline": cpu,
        "e2e": {"value": job_rate(K, world, ms_e2e), "unit": "Newton steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clk,
        "gpu_launches": launches_mixed,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------- screening workload
SCREEN_EPS = 1e-6      # first stage held within 1e-6 of u0 (scenarios decouple)
SCREEN_RHO_CAP = 1e6
SCREEN_TOL = 1e-4


def oracle_screen_sample(n_sample: int = 8):
    """The CPU oracle screening candidates one by one (screen_candidate, a
    two-scenario NCL solve each) on the first n_sample candidates of the
    500-bus screening batch; returns (seconds per contingency, description)."""
    import synthgrid
    from oracle.screening import screen_candidate
    inst, u0, _, _ = synthgrid.screening_batch(CONFIG_IDX)
    with one_blas_thread():
        t0 = time.perf_counter()
        for cand in inst.ctgs[:n_sample]:
            screen_candidate(inst, cand, u0, eps=SCREEN_EPS, rho_cap=SCREEN_RHO_CAP,
                             accept_tol=SCREEN_TOL)
        t = time.perf_counter() - t0
    desc = (f"oracle screen_candidate (numpy/scipy + C LDL^T, 1 thread), one two-scenario NCL "
            f"solve per candidate, first {n_sample} of {len(inst.ctgs)} candidates of the "
            f"500-bus screening batch ({t:.1f} s)")
    return t / n_sample, desc


def run_screen(args):
    """Batched screening of the 500-bus workload's candidate outages at the
    stored base-case control u0 (Section V-B, Table 1's task): one step is
    one scopf_screen call over all candidates."""
    import numpy as np
    import torch
    import synthgrid
    import paper_2510_13333_b300 as P

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:        # replicas only: one screening batch per process
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    inst, u0, _, stored = synthgrid.screening_batch(CONFIG_IDX)
    n_ctg = len(inst.ctgs)
    lib = P.SCOPF(inst, precision=P.PREC_MIXED)
    sz = lib.sizes
    steps = max(1, min(args.steps, 10))

    def screen():
        return lib.scopf_screen(u0, eps=SCREEN_EPS, rho_cap=SCREEN_RHO_CAP,
                                accept_tol=SCREEN_TOL)

    for _ in range(args.warmup):
        acc, viol, res = screen()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks()
    clocks.start()
    lib.scopf_timing(True)
    n0 = P.scopf_launch_count()
    t0 = time.perf_counter()
    e0.record(s)
    for _ in range(steps):
        acc, viol, res = screen()
    e1.record(s)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = P.scopf_launch_count() - n0
    phases = lib.scopf_timing(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    value = n_ctg * steps / (ms / 1e3)
    dom = dominant_phase(phases, phases["solve"][1] + res["refine_steps"] * steps)
    try:
        cpu_s, cpu_desc = oracle_screen_sample()
        cpu = {"value": 1.0 / cpu_s, "unit": "contingencies/s", "cores": 1, "kind": "oracle",
               "sample": cpu_desc}
    except Exception as exc:
        cpu = {"value": None, "unit": "contingencies/s", "cores": 1, "kind": "oracle",
               "sample": f"failed: {exc}"}
    stored = np.array(stored)
    line = {
        "metric": "contingencies screened/s at a fixed base-case control (500-bus, all "
                  "candidates in one batch)",
        "value": value, "unit": "contingencies/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 block factors + f64 (model, Schur, refinement)", "data": "synthetic",
        "config": {"workload": f"syn500 screening batch: 500-bus grid, base case + {n_ctg} "
                               f"candidate outages examined by the oracle's screening, u0 "
                               f"+- {SCREEN_EPS:g}, rho cap {SCREEN_RHO_CAP:g}, accept "
                               f"|(r_k,t_k)|_inf <= {SCREEN_TOL:g}",
                   "n_kkt": sz.n_kkt, "blocks": sz.n_blocks, "flush_l2": False,
                   "inputs_exceed_l2": True},
        "s_per_contingency": ms / 1e3 / steps / n_ctg,
        "screen": {"status": res["status"], "outer_iters": res["outer_iters"],
                   "inner_iters": res["inner_iters"], "fp64_fallbacks": res["fp64_fallbacks"],
                   "accepted": int(acc[1:].sum()), "rejected": int((~acc[1:]).sum()),
                   "base_accepted": bool(acc[0]),
                   "agree_with_stored_u0pm1e-3_verdicts": int(np.sum(acc[1:] == stored))},
        "phases_ms_per_step": {k: v[0] / steps for k, v in phases.items()},
        "roofline": roofline(sz, phases, dom, 4, live_peaks()),
        "cpu_baseline": cpu,
        "e2e": {"value": n_ctg * steps / wall, "unit": "contingencies/s",
                "h2d_bytes_per_step": 8 * sz.n_border,
                "d2h_bytes_per_step": 12 * sz.n_blocks,
                "note": "scopf_screen takes u0 and returns verdicts in host memory; host clock"},
        "clocks": clk,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------ ill-conditioning study (q_min -> q_max)
ILLCOND_DELTAS = (1.0, 0.3, 0.1, 0.03, 0.01, 0.003)


def run_illcond(args):
    """Full NCL solves with the generators' reactive bands narrowed around
    the base-case reactive output q* of the unstressed solution:
    [max(q_min, q* - delta w), min(q_max, q* + delta w)], w = (q_max -
    q_min) / 2.  q_min close to q_max is the regime Section V-C names as the
    source of ill-conditioning (the eq. pvpq complementarity).  Per delta and
    precision: status, IPM iterations, factorizations per iteration (the
    inertia corrections), refinement steps per iteration, FP64 fallbacks and
    time to solution."""
    import numpy as np
    import torch
    import synthgrid
    import paper_2510_13333_b300 as P

    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rows = []
    for idx in (1, CONFIG_IDX):
        base = synthgrid.config_instance(idx)
        nb, ng = base.net.n_bus, base.net.n_gen
        lib = P.SCOPF(base, precision=P.PREC_FP64)
        r = lib.ncl_solve()
        # base-case q_g^0 in the natural variable order: theta (nb - 1), v at the
        # nb - ng buses without a generator, then q_g^0 per generator
        q0 = lib.get_state()["w"][(nb - 1) + (nb - ng):(nb - 1) + (nb - ng) + ng].cpu().numpy()
        del lib
        half = 0.5 * (base.net.qmax - base.net.qmin)
        for delta in ILLCOND_DELTAS:
            inst = synthgrid.config_instance(idx)
            net = inst.net
            net.qmin = np.maximum(base.net.qmin, q0 - delta * half)
            net.qmax = np.minimum(base.net.qmax, q0 + delta * half)
            lib = P.SCOPF(inst, precision=P.PREC_MIXED)
            for name, prec in (("mixed", P.PREC_MIXED), ("fp64", P.PREC_FP64)):
                lib.set_precision(prec)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = lib.ncl_solve()
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                rows.append({"network": inst.name, "K": len(inst.ctgs), "delta": delta,
                             "band_pu": float(np.median(net.qmax - net.qmin)),
                             "precision": name, "status": r["call_status"],
                             "inner_iters": r["inner_iters"], "outer_iters": r["outer_iters"],
                             "factorizations_per_iter": r["factorizations"] / max(1, r["inner_iters"]),
                             "refine_steps_per_iter": r["refine_steps"] / max(1, r["inner_iters"]),
                             "fp64_fallbacks": r["fp64_fallbacks"], "seconds": dt,
                             "objective": r["objective"], "max_violation": r["max_violation"]})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            del lib
    print(json.dumps({"metric": "ill-conditioning study: NCL solves with q_min -> q_max",
                      "unit": "see rows", "data": "synthetic", "rows": rows}), flush=True)


# tile shapes (cluster_max_tasks, relax_max_nodes) of the time-to-solution
# spread.  The work-item size changes no arithmetic (children are summed in
# a fixed order); the amalgamation limit changes the supernodes, and with
# them the factors' rounding, a rounding-level perturbation of the path
SPREAD_SHAPES = ((16, 8), (16, 1), (16, 2), (16, 3), (16, 4), (16, 6))


def run_tts_spread(args):
    """Time to solution in both precisions under the tile shapes of
    SPREAD_SHAPES, at 500-bus x 256 (or with --scale the 2000-bus x 128 case,
    first four shapes).  The shapes change no arithmetic of the
    method, only the factors' rounding, which moves the interior-point path:
    the spread over shapes is the path noise a single time-to-solution
    comparison sits in."""
    import numpy as np
    import torch
    import synthgrid
    import paper_2510_13333_b300 as P

    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    idx = SCALE_IDX if args.scale else CONFIG_IDX
    inst = synthgrid.config_instance(idx)
    rows = []
    for cl, rx in SPREAD_SHAPES[:4] if args.scale else SPREAD_SHAPES:
        lib = P.SCOPF(inst, precision=P.PREC_MIXED, cluster_max_tasks=cl, relax_max_nodes=rx)
        for name, prec in (("mixed", P.PREC_MIXED), ("fp64", P.PREC_FP64)):
            lib.set_precision(prec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = lib.ncl_solve()
            torch.cuda.synchronize()
            rows.append({"cluster_max_tasks": cl, "relax_max_nodes": rx, "precision": name,
                         "seconds": time.perf_counter() - t0, "status": r["call_status"],
                         "inner_iters": r["inner_iters"], "objective": r["objective"],
                         "fp64_fallbacks": r["fp64_fallbacks"],
                         "max_violation": r["max_violation"]})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del lib
    summary = {}
    for name in ("mixed", "fp64"):
        sec = np.array([r["seconds"] for r in rows if r["precision"] == name])
        it = np.array([r["inner_iters"] for r in rows if r["precision"] == name])
        summary[name] = {"seconds_median": float(np.median(sec)), "seconds_min": float(sec.min()),
                         "seconds_max": float(sec.max()), "iters_median": float(np.median(it)),
                         "iters_min": int(it.min()), "iters_max": int(it.max())}
    ratio = [a["seconds"] / b["seconds"] for a, b in zip(rows[1::2], rows[0::2])]
    summary["fp64_over_mixed_seconds_per_shape"] = ratio
    summary["fp64_over_mixed_median_seconds"] = (summary["fp64"]["seconds_median"] /
                                                 summary["mixed"]["seconds_median"])
    print(json.dumps({"metric": "time to solution at " + ("2000-bus x 128" if args.scale else
                                                          "500-bus x 256") +
                                " over tile shapes (rounding-level path perturbations)",
                      "unit": "s", "data": "synthetic", "rows": rows, "summary": summary}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iterate-at", type=int, default=30)
    ap.add_argument("--tts", default="both", choices=["none", "mixed", "both"],
                    help="which full NCL solves to time (time to solution)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip scopf_autotune and use the default tile shapes")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-driven refinement loop (every kernel launched from the host, "
                         "for profilers that attribute launches to NVTX ranges)")
    ap.add_argument("--scale", action="store_true",
                    help="tts_spread on the 2000-bus x 128 case")
    ap.add_argument("--workload", default="newton",
                    choices=["newton", "scale", "condensed", "screen", "illcond", "peaks",
                             "tts_spread"],
                    help="newton: the Newton step (default); scale: the same on the 2000-bus "
                         "x 128 scale-up workload, with its memory footprint; condensed: the "
                         "newton workload on the condensed primal variant; screen: batched "
                         "screening; illcond: NCL solves with narrowed reactive bands; peaks: "
                         "the arithmetic probes; tts_spread: time to solution under six "
                         "amalgamation limits (the path's rounding noise)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "peaks":
        if args.impl != "reference" and int(os.environ.get("RANK", "0")) == 0:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            print(json.dumps({"metric": "arithmetic throughput of the library's probe kernels",
                              "unit": "TFLOP/s", "peaks": live_peaks(),
                              "derived": {"fp32_fma": FP32_PEAK_TFLOPS,
                                          "fp64_nominal": FP64_PEAK_TFLOPS}}), flush=True)
        return
    if args.workload == "illcond":
        if args.impl != "reference":
            run_illcond(args)
        return
    if args.workload == "tts_spread":
        if args.impl != "reference":
            run_tts_spread(args)
        return
    if args.workload == "screen":
        if args.impl == "reference":
            if int(os.environ.get("RANK", "0")) == 0:
                cpu_s, desc = oracle_screen_sample()
                v = 1.0 / cpu_s
                print(json.dumps({"metric": "contingencies screened/s", "value": v,
                                  "unit": "contingencies/s", "impl": "reference",
                                  "higher_is_better": True, "data": "synthetic",
                                  "cpu_baseline": {"value": v, "unit": "contingencies/s",
                                                   "cores": 1, "kind": "oracle", "sample": desc},
                                  "e2e": {"value": v, "unit": "contingencies/s",
                                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
                      flush=True)
        else:
            run_screen(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)   # newton (500-bus x 256) or scale (2000-bus x 128)


if __name__ == "__main__":
    main()
