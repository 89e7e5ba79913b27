"""Benchmark of the GB300 C0IP biharmonic multigrid (arXiv 2412.05082).

One step = one pass of the whole hot path over the workload: the six
problems of the 2D sweep (Q2-Q4 on 512^2 cells, Q5-Q7 on 256^2 cells), each
solved by FP64 MG-GMRES to a true relative residual ||b - A x|| / ||b|| of
1e-8 (colored MVS, one pre- and one post-smoothing step, fast-diagonalization
local solvers, right preconditioning in the flexible form, restart 50; Sec.
5.1), which runs apply_A, the residual, the patch gather / solve / scatter,
the transfers, the V-cycle and GMRES.  The six solves run as one batch
(bh_batch_solve: each level operation one launch over all problems, the patch
work of a color one launch per degree as parallel graph branches, the
lockstep V-cycle replayed as a CUDA graph, tiles tuned on the batch itself);
every problem takes the iterations and arithmetic of its own solve.

Right-hand side: b = A x* with x* i.i.d. uniform[-1, 1] (seed k), so that the
FP64 rounding floor of the true residual, eps ||A|| ||x|| / ||b||, is O(eps)
and a 1e-8 true residual is reachable at every degree; for b itself i.i.d.
uniform that floor is 1e-8 .. 3e-7 at these sizes (reported per degree in the
breakdown).

value = sum of the paper's DoF counts (kN+1)^2 solved / device time (CUDA
events), the solve inputs resident in HBM; L2 is flushed (256 MiB write)
before every timed step.  e2e = the same through bh_batch_solve_host with
pinned host buffers (copies inside the timed region).  The FP32 V-cycle
(the mixed form, Sec. 5.2) with compensated FP32 defects (key `mixed`) and
with FP64 defects (key `mixed_r64`) is timed on the same problems and
reported beside it.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run one process per GPU (torchrun); the solves are independent
replicas (weak scaling, no collective on the data path).
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workload  # noqa: E402

METRIC = "DoF/s: C0IP apply, patch smoother, MG-GMRES solve to 1e-8; serve p50/p99 latency"
UNIT = "DoF/s"
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12   # 2 DFMA / clk / SM at 2070 MHz


def _measured_hbm_gbs():
    """The measured HBM copy bandwidth of this machine's GPUs (driver-written
    peaks file), else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


HBM_GBS = _measured_hbm_gbs()
# The paper's solver throughput for the same six problems (2D, GMRES with one
# MVS pre- and post-step, inexact local solvers, to 1e-8; one A100, FP64): the
# data behind its solver-throughput figure (Fig. 3), DoF/s per degree.
PAPER_SOLVE_2D_MVS = {2: 8.47e6, 3: 1.60e7, 4: 1.77e7, 5: 2.41e7, 6: 2.29e7, 7: 2.19e7}


def paper_rate(problems):
    """The paper's rate for the whole workload: all DoFs over the sum of its
    per-problem solve times."""
    dofs = [workload.paper_dofs(*p) for p in problems]
    return sum(dofs) / sum(n / PAPER_SOLVE_2D_MVS[k] for n, (_, k, _) in zip(dofs, problems))
FP32_PEAK_TFLOPS = 152 * 256 * 2.070e9 / 1e12  # 128 FFMA / clk / SM


def config_for(problems, precision="fp64"):
    return {
        "workload": "2D C0IP biharmonic sweep (paper sizes): Q2-Q4 on 512^2 and Q5-Q7 on 256^2 "
                    "cells; MG-GMRES to a true relative residual of 1e-8 (colored MVS 1+1, FDM "
                    "local solver, right preconditioning (flexible), restart 50), %s; the six "
                    "solves run as one batch" % precision,
        "problems": [{"d": d, "k": k, "cells": N, "dofs": workload.paper_dofs(d, k, N)}
                     for d, k, N in problems],
        "dof_count": "(kN+1)^d including boundary nodes (the paper's convention)",
        "rhs": "b = A x*, x* i.i.d. uniform[-1,1] (PCG64, seed k): FP64 rounding floor of the "
               "true residual O(eps); for b itself i.i.d. uniform the floor is 1e-8..3e-7 at "
               "these sizes (breakdown: uniform_rhs_floor)",
        "stop": "true residual ||b - A x||_2 / ||b||_2 <= 1e-8 (right preconditioning)",
        "l2": "flushed before every timed step (256 MiB write)",
    }


def flop_per_unknown_apply(d, k):
    """FP64 flops of one apply_A / residual per unknown: the band nonzeros of
    the sum-factorized sweeps (2 flops per FMA).  Per output cell of k rows the
    M and L bands hold k^2 + 2k entries and B 3k^2 + 2k (5k + 6 per row for the
    three together); 2D: one x-split (M, L, B) and one y-combination (B, L, M):
    2 (5k + 6) FMAs per unknown; 3D: x-split 5k+6, y-mix 8k+12, z 5k+6."""
    fma = 2 * (5 * k + 6) if d == 2 else (5 * k + 6) + (8 * k + 12) + (5 * k + 6)
    return 2 * fma


def mvs2_fma_per_patch(k):
    """FP64 FMAs of the fused 2D colored-MVS kernel per patch (m = 2k-1,
    window 4k+1): x-split T_M on the window rows and T_L, T_B on the 2k+1
    middle rows, y-combination on the m^2 patch nodes, four FDM contractions
    and the eigenvalue scaling.  Band sums over the m patch positions: M and L
    hold (2k+1) + (2k-2)(k+1) entries, B (4k+1) + (2k-2)(3k+1)."""
    m, w, wm = 2 * k - 1, 4 * k + 1, 2 * k + 1
    sm = (2 * k + 1) + (2 * k - 2) * (k + 1)
    sb = (4 * k + 1) + (2 * k - 2) * (3 * k + 1)
    return w * sm + wm * sm + wm * sb + m * (sb + 2 * sm) + 4 * m ** 3 + m * m


def mvs2_fp64_ops_interior(k):
    """FP64 operations the fused 2D MVS kernel executes on a patch away from
    the boundary: the same band contractions, with the four FDM contractions
    in the folded form (per line 2k^2 + k - 2 forward, 2k^2 - 1 backward)."""
    m = 2 * k - 1
    return mvs2_fma_per_patch(k) - 4 * m ** 3 + 2 * m * (4 * k * k + k - 3)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.fh = None
        # BH_CLOCKS_CSV keeps the raw samples where the caller wants them.
        self.keep = bool(os.environ.get("BH_CLOCKS_CSV"))
        self.path = os.environ.get("BH_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "bh_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
            if self.fh is not None:
                self.fh.close()
                if not self.keep and os.path.exists(self.path):
                    os.unlink(self.path)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not self.keep:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---- the CPU oracle timed on the host cores (spawned worker processes, each
# single-threaded in Python with its share of the host's BLAS threads) --------
_ORACLE = {}


def _oracle_problem(k, L):
    """Oracle hierarchy and right-hand side b = A x* of the 2D problem (k, L)."""
    from oracle import mg
    key = (k, L)
    if key not in _ORACLE:
        H = mg.Hierarchy(2, k, L)
        A = H.A[L]
        _ORACLE[key] = (H, A @ workload.vector_uniform(A.shape[0], k))
    return _ORACLE[key]


def _oracle_setup(problems):
    for k, L in problems:
        _oracle_problem(k, L)


def _oracle_solve(key):
    """One oracle MG-GMRES solve (right, true residual 1e-8); (seconds, iters, relres)."""
    from oracle import krylov
    H, b = _oracle_problem(*key)
    t0 = time.perf_counter()
    _, it, _, rr = krylov.gmres(H.A[H.L], b, H.preconditioner, 1e-8)
    return time.perf_counter() - t0, it, rr


def _oracle_best(k, L, reps):
    """Best of `reps` oracle solves of (k, L) (hierarchy setup not timed)."""
    _oracle_problem(k, L)
    runs = [_oracle_solve((k, L)) for _ in range(reps)]
    return min(r[0] for r in runs), runs[0][1], runs[0][2]


class _Pool:
    """A spawn-started process pool whose workers get `threads` BLAS threads."""

    VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

    def __init__(self, workers, threads, initializer=None, initargs=()):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.saved = {v: os.environ.get(v) for v in self.VARS}
        for v in self.VARS:
            os.environ[v] = str(threads)
        self.ex = cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"),
                                         initializer=initializer, initargs=initargs)

    def __enter__(self):
        return self.ex

    def __exit__(self, *exc):
        self.ex.shutdown()
        for v, val in self.saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val


def cpu_baseline(budget_s=40.0, reps=3):
    """The CPU oracle (as it stands) on the workload's family: the six
    problems (2D, k = 2..7, same smoother, local solver, GMRES protocol and
    right-hand side kind) solved concurrently, one spawned process per problem
    with cpu_count / 6 BLAS threads each, on meshes of N = 8, 16, 32, ... cells
    while the time budget lasts (best of `reps` per size); the largest common
    size reached is reported, the benchmark's own sizes (512^2 / 256^2) as not
    run when they do not fit."""
    ncpu = os.cpu_count() or 1
    threads = max(1, ncpu // 6)
    ks = list(range(2, 8))
    sizes, t_start = [], time.perf_counter()
    with _Pool(6, threads) as ex:
        L = 3
        while True:
            t0 = time.perf_counter()
            res = list(ex.map(_oracle_best, ks, [L] * 6, [reps] * 6))
            wall = time.perf_counter() - t0
            N = 2 ** L
            dofs = sum(workload.paper_dofs(2, k, N) for k in ks)
            tmax = max(r[0] for r in res)
            sizes.append({"cells": N, "dofs": dofs, "solve_s_max": tmax, "wall_s": wall,
                          "value": dofs / tmax, "iters": [r[1] for r in res],
                          "true_relres_max": max(r[2] for r in res)})
            # the next level costs about 4.5x (4x the unknowns, the same iterations)
            if time.perf_counter() - t_start + 4.5 * wall > budget_s or L >= 8:
                break
            L += 1
    top = sizes[-1]
    return {"value": top["value"], "unit": UNIT, "cores": 6 * threads, "kind": "oracle",
            "sample": "oracle MG-GMRES solves (MVS 1+1, separable local matrices by dense LU, "
                      "right preconditioning, true residual 1e-8, b = A x*) of the 2D sweep "
                      "family k = 2..7 on %d^2 cells, the six run concurrently in six spawned "
                      "processes with %d BLAS thread(s) each; value = their paper DoF count / "
                      "the slowest solve, best of %d" % (top["cells"], threads, reps),
            "sizes": sizes, "largest_cells": top["cells"],
            "not_run": "512^2 (k = 2..4) and 256^2 (k = 5..7) cells: beyond the %.0f s budget "
                       "(the oracle's time grows about 4.5x per level)" % budget_s,
            "host_cpus": ncpu}


def rough_rhs(bh, torch, params, seed, stream):
    """b = A_L x* on the device for x* ~ U[-1, 1] (seed), by the library's apply
    on a context of the problem's shape; returns (b, x*)."""
    with bh.Context(params, stream) as c:
        n = c.num_unknowns()
        xs = torch.tensor(workload.vector_uniform(n, seed), dtype=torch.float64, device="cuda")
        b = torch.empty_like(xs)
        c.apply_A(params.level, xs, b)
        torch.cuda.synchronize()
    return b, xs


def measure_batched(bh, torch, stream):
    """The batched form on 64 independent 2D problems (k ~ U{2..7}, levels
    with 1e4-1e6 DoFs, seed 1234; b = A x*): one right-preconditioned solve of
    all of them in lockstep with autotuned tiles, against the same problems
    solved one after another."""
    from paper_2412_05082_gb300 import autotune
    probs = workload.batch_problems(64, 1234)
    params = [bh.default_params(d, k, L) for d, k, L in probs]
    bs = [rough_rhs(bh, torch, p, i, stream)[0] for i, p in enumerate(params)]
    xs = [torch.empty_like(b) for b in bs]
    dofs = sum(workload.paper_dofs(d, k, 2 ** L) for d, k, L in probs)
    with bh.Batch(params, stream) as batch:
        tiles = autotune.tune_batch(batch, probs)
        batch.solve(bs, xs, 1e-8, 200)
        torch.cuda.synchronize()
        l0 = batch.launches()
        t0 = time.perf_counter()
        its, rr = batch.solve(bs, xs, 1e-8, 200)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        launches = batch.launches() - l0
        # the persistent form of the same V-cycle (one cooperative launch each)
        batch.set_persistent(True)
        batch.solve(bs, xs, 1e-8, 200)
        torch.cuda.synchronize()
        l0 = batch.launches()
        t0 = time.perf_counter()
        its_p, rr_p = batch.solve(bs, xs, 1e-8, 200)
        torch.cuda.synchronize()
        tp = time.perf_counter() - t0
        launches_p = batch.launches() - l0
        batch.set_persistent(False)
    ctxs = [bh.Context(p, stream) for p in params]
    for c, b, x in zip(ctxs, bs, xs):
        c.solve(b, x, 1e-8, 200)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its1 = [c.solve(b, x, 1e-8, 200)[0] for c, b, x in zip(ctxs, bs, xs)]
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    return {"workload": "64 independent 2D problems, k ~ U{2..7}, levels with 1e4-1e6 DoFs "
                        "(seed 1234), b = A x* with x* uniform[-1,1], FP64 MG-GMRES (MVS, right, "
                        "true residual) to 1e-8",
            "dofs": dofs, "value": dofs / tb, "unit": UNIT, "seconds": tb,
            "launches_per_solve": launches, "tiles_patches_per_block": tiles,
            "sequential_value": dofs / ts, "speedup_vs_sequential": ts / tb,
            "iterations_equal_to_sequential": sum(a == b for a, b in zip(its, its1)),
            "max_iters": max(its), "max_true_relres": max(rr),
            "persistent": {"value": dofs / tp, "seconds": tp, "launches_per_solve": launches_p,
                           "vs_graph": tb / tp, "iterations_equal_to_graph": its_p == its,
                           "max_true_relres": max(rr_p)}}


def measure_serving(bh, torch, stream, nreq):
    """The serving form on the first nreq requests of the Poisson stream
    (rate 200/s, seed 2024; 2D and 3D, k = 2..7, 1e4-2e7 DoFs; b = A x* with
    x* uniform[-1, 1], computed on the device before the replay), replayed at
    their arrival times: p50/p99 latency and throughput with 8 slots in the
    mixed form (FP32 V-cycle with compensated FP32 defects) and with 8 slots in FP64."""
    import numpy as np
    reqs = workload.serving_requests(1000, 200.0, 2024)[:nreq]
    rhs = [None] * len(reqs)
    shapes = {}
    for i, (_, d, k, L, s) in enumerate(reqs):
        shapes.setdefault((d, k, L), []).append(i)
    for (d, k, L), idx in shapes.items():
        with bh.Context(bh.default_params(d, k, L), stream) as c:
            n = c.num_unknowns()
            y = torch.empty(n, dtype=torch.float64, device="cuda")
            for i in idx:
                xs = torch.tensor(workload.vector_uniform(n, reqs[i][4]), dtype=torch.float64,
                                  device="cuda")
                c.apply_A(L, xs, y)
                rhs[i] = y.cpu().numpy()
            del y
        torch.cuda.empty_cache()
    dofs = sum(workload.paper_dofs(d, k, 2 ** L) for _, d, k, L, _ in reqs)
    out = {"workload": "first %d requests of the Poisson stream (200 req/s, seed 2024), 2D and "
                       "3D, k = 2..7, 1e4-2e7 DoFs, b = A x* with x* uniform[-1,1], right GMRES "
                       "to a true residual of 1e-8" % nreq, "dofs": dofs, "requests": nreq}
    for name, mixed in (("served_mixed", 7), ("served_fp64", 0)):
        xs = [np.zeros_like(b) for b in rhs]
        with bh.Server(slots=8, mixed_max_degree=mixed) as srv:
            start = time.perf_counter()
            tickets = []
            for (ta, d, k, L, _), b, x in zip(reqs, rhs, xs):
                while time.perf_counter() - start < ta:
                    time.sleep(0.0002)
                tickets.append(srv.submit(d, k, L, b, x))
            res = [srv.wait(t) for t in tickets]
            wall = time.perf_counter() - start
            st = srv.stats()
        lat = np.array([r["latency_s"] for r in res])
        svc = np.array([r["service_s"] for r in res])
        out[name] = {"slots": 8, "precision": "FP32 V-cycle with compensated FP32 defects" if mixed
                     else "FP64", "value": dofs / wall, "unit": UNIT, "wall_s": wall,
                     "p50_latency_s": float(np.percentile(lat, 50)),
                     "p99_latency_s": float(np.percentile(lat, 99)),
                     "p50_service_s": float(np.percentile(svc, 50)),
                     "p99_service_s": float(np.percentile(svc, 99)),
                     "failed": int(sum(r["status"] != 0 for r in res)),
                     "max_relres": float(max(r["relres"] for r in res)),
                     "hierarchies_created": st["created"], "evictions": st["evictions"]}
    return out


def breakdown_3d(bh, torch, dev, stream, time_op):
    """The 3D sweep (Q2, Q3 on 128^3, Q4-Q7 on 64^3 cells): apply, one colored
    MVS step (inexact, and exact local solvers), and right-preconditioned
    MG-GMRES to a true residual of 1e-8 on b = A x*: FP64, the FP32 V-cycle of
    Sec. 5.2 (k <= 4) and the FP32 V-cycle with FP64 or compensated FP32
    defects (every k), with the relative error of each solution against x*."""
    out = {}
    for d, k, N in workload.SWEEP_3D:
        L = workload.level_of(N)
        dofs = workload.paper_dofs(d, k, N)
        row = {"dofs": dofs}
        with bh.Context(bh.default_params(d, k, L), stream) as ctx:
            n = ctx.num_unknowns()
            xstar = torch.tensor(workload.vector_uniform(n, k), dtype=torch.float64, device=dev)
            b = torch.empty_like(xstar)
            ctx.apply_A(L, xstar, b)
            x = torch.zeros_like(b)
            row["apply"] = dofs / time_op(lambda: ctx.apply_A(L, xstar, x), 5)
            x.zero_()
            row["mvs_step"] = dofs / time_op(lambda: ctx.smooth(L, x, b, 1), 3)
            # one timed solve (the first on this context) to save time at 9e7 unknowns
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            itr = ctx.solve(b, x, 1e-8, 100, raise_on_noconv=False)
            e1.record(stream)
            torch.cuda.synchronize()
            row["solve_fp64_right"] = dofs / (e0.elapsed_time(e1) / 1e3)
            row["fp64_right_iters"], row["fp64_right_relres"] = itr[0], itr[1]
            row["fp64_right_err_vs_xstar"] = float((x - xstar).abs().max() / xstar.abs().max())
        with bh.Context(bh.default_params(d, k, L, local_solver=bh.EXACT), stream) as c2:
            row["mvs_exact_step"] = dofs / time_op(lambda: c2.smooth(L, x, b, 1), 2)
        for prec, name, kmax in ((bh.MIXED_FP32, "mixed_right", 4),
                                 (bh.MIXED_FP32_R64, "mixed_r64_right", 7),
                                 (bh.MIXED_FP32_RC, "mixed_rc_right", 7)):
            if k > kmax:
                continue
            with bh.Context(bh.default_params(d, k, L, precision=prec), stream) as c2:
                itm = c2.solve(b, x, 1e-8, 100, raise_on_noconv=False)
                row["solve_" + name] = dofs / time_op(
                    lambda: c2.solve(b, x, 1e-8, 100, raise_on_noconv=False), 1)
                row[name + "_iters"], row[name + "_relres"] = itm[0], itm[1]
                row[name + "_err_vs_xstar"] = float((x - xstar).abs().max() / xstar.abs().max())
        del b, x, xstar
        torch.cuda.empty_cache()
        out["k%d" % k] = row
    return out


def max_over_ranks(t, dist, device):
    """The slowest rank's time (every rank gets it); t itself without a
    process group.  The replicas share no data, so this reduction is the only
    collective of a multi-GPU run."""
    if dist is None:
        return t
    import torch
    v = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v)


# Tables 1-3 of Sec. 5.1: which smoother, steps and local solver each printed
# column uses, and whether it is run with CG (additive) or GMRES (multiplicative).
TABLE_COLUMNS = {
    "tab1_avs2_exact_2d": (2, "avs", 2, "exact"),
    "tab1_mvs_exact_2d": (2, "mvs", 1, "exact"),
    "tab2_avs2_inexact_2d": (2, "avs", 2, "fdm"),
    "tab2_mvs_inexact_2d": (2, "mvs", 1, "fdm"),
    "tab3_avs1_inexact_3d": (3, "avs", 1, "fdm"),
    "tab3_avs2_inexact_3d": (3, "avs", 2, "fdm"),
    "tab3_mvs1_inexact_3d": (3, "mvs", 1, "fdm"),
    "tab3_mvs2_inexact_3d": (3, "mvs", 2, "fdm"),
}


def table_entries(golden):
    """Every printed entry of the tables as (DoFs, column, row, col, d, k, L),
    smallest problem first."""
    entries = []
    for name, (d, _, _, _) in TABLE_COLUMNS.items():
        levels = golden["tab3_levels"] if d == 3 else golden["levels"]
        for i, L in enumerate(levels):
            for j, k in enumerate(golden["degrees"]):
                if golden[name][i][j] is not None:
                    entries.append(((k * 2 ** L + 1) ** d, name, i, j, d, k, L))
    return sorted(entries)


def run_tables(args):
    """Fractional iteration counts nu_frac = -8 n / log10(|r_n| / |r_0|) of the
    paper's Tables 1-3 (Sec. 5.1) on the GPU at the printed levels, with r the
    residual each Krylov method's stopping test measures (preconditioned for
    left GMRES, the convention of deal.II, the library of Sec. 5): the paper's
    sine right-hand side, CG with the additive smoother (atomic AVS) and left-
    preconditioned GMRES with the colored multiplicative one, the damping of
    Sec. 5.1, exact coarse solve, relative reduction 1e-8.  Entries are run in
    increasing size; 3D entries above --tables-max-dofs-3d and everything after
    the time budget are reported as null.  Prints one JSON line."""
    import torch
    import paper_2412_05082_gb300 as bh
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_tables_nu_frac.json")))
    entries = table_entries(golden)
    out = {}
    for name in TABLE_COLUMNS:
        rows, cols = len(golden[name]), len(golden["degrees"])
        out[name] = {"levels": golden["tab3_levels"] if name.startswith("tab3") else golden["levels"],
                     "degrees": golden["degrees"], "paper": golden[name],
                     "gpu": [[None] * cols for _ in range(rows)],
                     "iters": [[None] * cols for _ in range(rows)]}
    t0, skipped = time.perf_counter(), []
    for dofs, name, i, j, d, k, L in entries:
        _, smoother, steps, ls = TABLE_COLUMNS[name]
        if (d == 3 and dofs > args.tables_max_dofs_3d) or time.perf_counter() - t0 > args.tables_budget_s:
            skipped.append([name, k, L])
            continue
        p = bh.default_params(d, k, L, pre_steps=steps, post_steps=steps,
                              local_solver=bh.EXACT if ls == "exact" else bh.FDM,
                              gmres_side=bh.LEFT)
        if smoother == "avs":
            p.smoother, p.krylov = bh.AVS_ATOMIC, bh.CG
        with bh.Context(p, stream) as c:
            b = torch.empty(c.num_unknowns(), dtype=torch.float64, device="cuda")
            c.rhs(L, bh.RHS_PAPER_SINE, b)
            x = torch.zeros_like(b)
            it, _ = c.solve(b, x, 1e-8, 300, raise_on_noconv=False)
            # the ratio of the stopping test: preconditioned residual for
            # left GMRES, recursively updated residual for CG
            est = c.stats()["last_estimate"]
        nu = -8.0 * it / math.log10(est) if 0.0 < est < 1.0 else None
        out[name]["gpu"][i][j] = None if nu is None else round(nu, 2)
        out[name]["iters"][i][j] = it
        print("%s k=%d L=%d dofs=%d: nu_frac %s (paper %s)" % (name, k, L, dofs, nu, golden[name][i][j]),
              file=sys.stderr, flush=True)
    print(json.dumps({"tables": out, "skipped": skipped, "seconds": time.perf_counter() - t0,
                      "max_dofs_3d": args.tables_max_dofs_3d,
                      "protocol": "paper sine right-hand side; CG + atomic AVS, left GMRES(50) + "
                                  "colored MVS; default damping (2D AVS 1/4, MVS 1; 3D AVS 0.1, "
                                  "MVS 0.7); exact coarse solve; relative reduction 1e-8; "
                                  "nu_frac = -8 n / log10(|r_n| / |r_0|), r the residual of the stopping test "
                                  "(preconditioned for left GMRES)"}), flush=True)
    return 0


REFERENCE_CELLS = 16


def run_reference(args):
    """The reference arm: the CPU oracle timed as it stands on the host cores.
    Each step is a bounded sample of the workload: the six problems of the
    sweep family (2D, k = 2..7, b = A x*, right MG-GMRES to a true residual of
    1e-8) on 16^2 cells, solved concurrently by six spawned processes that
    hold the hierarchies (set up once, not timed)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    L = workload.level_of(REFERENCE_CELLS)
    keys = [(k, L) for k in range(2, 8)]
    ncpu = os.cpu_count() or 1
    threads = max(1, ncpu // 6)
    with _Pool(6, threads, _oracle_setup, (keys,)) as ex:
        list(ex.map(_oracle_solve, keys))  # every worker builds its hierarchies
        for _ in range(args.warmup):
            list(ex.map(_oracle_solve, keys))
        t0 = time.perf_counter()
        for _ in range(args.steps):
            res = list(ex.map(_oracle_solve, keys))
        dt = time.perf_counter() - t0
    problems = [(2, k, REFERENCE_CELLS) for k, _ in keys]
    dofs = sum(workload.paper_dofs(*p) for p in problems) * args.steps
    value = dofs / dt
    sample = ("oracle MG-GMRES solves (right, true residual 1e-8, b = A x*) of the 2D sweep "
              "family k = 2..7 on %d^2 cells per step, the six run concurrently in six spawned "
              "processes with %d BLAS thread(s) each; paper DoF count / wall time"
              % (REFERENCE_CELLS, threads))
    cfg = config_for(problems)
    cfg["workload"] = ("2D C0IP biharmonic sweep family at a size the CPU oracle finishes per "
                       "step: Q2-Q7 on %d^2 cells (the GPU arm runs Q2-Q4 on 512^2 and Q5-Q7 on "
                       "256^2); MG-GMRES to a true relative residual of 1e-8 (colored MVS 1+1, "
                       "separable local solver, right preconditioning, restart 50), FP64"
                       % REFERENCE_CELLS)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": cfg,
            "iterations": {str(k): it for (k, _), (_, it, _) in zip(keys, res)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 6 * threads, "kind": "oracle",
                             "sample": sample, "host_cpus": ncpu},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-breakdown", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched and serving measurements")
    ap.add_argument("--serve-requests", type=int, default=500,
                    help="requests of the Poisson stream replayed by the serving measurement")
    ap.add_argument("--cpu-budget-s", type=float, default=40.0,
                    help="time budget of the CPU oracle baseline")
    ap.add_argument("--tables", action="store_true",
                    help="reproduce the nu_frac of the paper's Tables 1-3 instead of the benchmark")
    ap.add_argument("--tables-max-dofs-3d", type=float, default=2e7)
    ap.add_argument("--tables-budget-s", type=float, default=240.0)
    args = ap.parse_args()
    if args.tables:
        return run_tables(args)
    if args.impl == "reference":
        # the oracle needs no GPU: this process never touches a device
        return run_reference(args)

    # the CPU baseline's worker processes are spawned before any CUDA call
    cpu = None
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_budget_s)

    import torch
    import paper_2412_05082_gb300 as bh
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()

    problems = workload.SWEEP_2D
    levels = [workload.level_of(N) for _, _, N in problems]
    from paper_2412_05082_gb300 import autotune
    # inputs: x* (seeded) and b = A x* by the library's apply, resident in HBM
    ctxs, rhs, xstar, xs, hostb, hostx = [], [], [], [], [], []
    for (d, k, N), L in zip(problems, levels):
        ctx = bh.Context(bh.default_params(d, k, L), stream)
        n = ctx.num_unknowns()
        xt = torch.tensor(workload.vector_uniform(n, k), dtype=torch.float64, device=dev)
        b = torch.empty_like(xt)
        ctx.apply_A(L, xt, b)
        ctxs.append(ctx)
        xstar.append(xt)
        rhs.append(b)
        xs.append(torch.empty(n, dtype=torch.float64, device=dev))
        hostb.append(b.cpu().pin_memory())
        hostx.append(torch.empty(n, dtype=torch.float64).pin_memory())
    torch.cuda.synchronize()
    plist = [(d, k, L) for (d, k, _), L in zip(problems, levels)]
    batch = bh.Batch([bh.default_params(d, k, L) for d, k, L in plist], stream)
    tiles = autotune.tune_batch(batch, plist)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    iters = {}

    def step():
        its, rrs = batch.solve(rhs, xs, 1e-8, 200)
        for (d, k, N), it, rr in zip(problems, its, rrs):
            iters[k] = (it, rr)

    def step_host():
        batch.solve_host(hostb, hostx, 1e-8, 200)

    def timed(fn, steps):
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return ts

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = bh.kernel_launches()
    with Clocks(local_rank) as clk:
        ts = timed(step, args.steps)
    launches = bh.kernel_launches() - launches0
    t_total = max_over_ranks(sum(ts), dist, dev)
    if dist:
        dist.barrier()
    dofs_step = sum(workload.paper_dofs(*p) for p in problems)
    value = dofs_step * args.steps * world / t_total
    err = {k: float((x - xt).abs().max() / xt.abs().max())
           for (_, k, _), x, xt in zip(problems, xs, xstar)}

    # end to end through the C ABI with host buffers (copies inside the region)
    step_host()
    te = timed(step_host, args.steps)
    t_e2e = max_over_ranks(sum(te), dist, dev)
    bytes_h2d = sum(8 * c.num_unknowns() for c in ctxs)

    # the mixed forms on the same problems, inside the same flexible FP64
    # GMRES with the same stop: the FP32 V-cycle with compensated FP32 defects
    # (BH_MIXED_FP32_RC, the `mixed` key) and with FP64 defects (R64)
    def mixed_leg(prec, label, steps):
        with bh.Batch([bh.default_params(d, k, L, precision=prec) for d, k, L in plist],
                      stream) as mb:
            mtiles = autotune.tune_batch(mb, plist)
            xm = [torch.empty_like(x) for x in xs]
            for _ in range(2):
                its_m, rr_m = mb.solve(rhs, xm, 1e-8, 200)
            tm = timed(lambda: mb.solve(rhs, xm, 1e-8, 200), steps)
            leg = {"value": dofs_step * len(tm) * world / max_over_ranks(sum(tm), dist, dev),
                   "unit": UNIT, "ms_per_step": statistics.mean(tm) * 1e3,
                   "precision": label,
                   "iterations": {str(k): {"iters": it, "true_relres": rr,
                                           "err_vs_xstar": float((x - xt).abs().max() /
                                                                 xt.abs().max())}
                                  for (_, k, _), it, rr, x, xt in zip(problems, its_m, rr_m, xm,
                                                                       xstar)},
                   "tiles_patches_per_block": mtiles}
            leg["speedup_vs_fp64"] = leg["value"] / value
            del xm
        return leg

    mixed = mixed_leg(bh.MIXED_FP32_RC, "FP32 V-cycle with compensated FP32 (double-float) "
                      "defects (BH_MIXED_FP32_RC) in flexible FP64 GMRES, same true-residual stop",
                      min(args.steps, 5))
    mixed_r64 = mixed_leg(bh.MIXED_FP32_R64, "FP32 V-cycle with FP64 defects (BH_MIXED_FP32_R64) "
                          "in flexible FP64 GMRES, same true-residual stop", min(args.steps, 3))
    # the persistent form of the headline batch's V-cycle (one cooperative launch
    # per V-cycle instead of the graph replay), on the same solves
    batch.set_persistent(True)
    batch.solve(rhs, xs, 1e-8, 200)
    tpers = timed(lambda: batch.solve(rhs, xs, 1e-8, 200), min(args.steps, 3))
    batch.set_persistent(False)
    persistent = {"value": dofs_step * len(tpers) * world / max_over_ranks(sum(tpers), dist, dev),
                  "unit": UNIT, "ms_per_step": statistics.mean(tpers) * 1e3}
    persistent["vs_graph"] = persistent["value"] / value

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / paper_rate(problems),
        "vs_baseline_basis": "against the paper's A100 solver throughput for the same six "
                             "problems (Fig. 3 data; all DoFs / sum of solve times = %.3g DoF/s; "
                             "the paper stops on its own Krylov residual); another machine: "
                             "context, not the target" % paper_rate(problems),
        "dtype": "f64",
        "data": "synthetic", "config": config_for(problems),
        "e2e": {"value": dofs_step * args.steps * world / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": bytes_h2d, "d2h_bytes_per_step": bytes_h2d},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "iterations": {str(k): {"iters": it, "true_relres": rr, "err_vs_xstar": err[k]}
                       for k, (it, rr) in iters.items()},
        "all_true_relres_le_1e-8": all(rr <= 1.0001e-8 for _, rr in iters.values()),
        "tiles_patches_per_block": tiles,
        "mixed": mixed,
        "mixed_r64": {key: mixed_r64[key] for key in ("value", "unit", "ms_per_step", "precision",
                                                       "speedup_vs_fp64")},
        "persistent_vcycle": persistent,
    }

    # dominant kernel: the fused colored-MVS kernel (8 launches per smoothing step)
    def time_op(fn, reps=10):
        fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return statistics.median(ts)

    roof_k = 4
    i4 = [p[1] for p in problems].index(roof_k)
    d, k, N = problems[i4]
    L = levels[i4]
    ctx = ctxs[i4]
    xr = torch.zeros_like(xs[i4])
    t_step = time_op(lambda: ctx.smooth(L, xr, rhs[i4], 1), 10)
    patches = (N - 1) ** 2
    flops_launch = 2 * mvs2_fma_per_patch(k) * patches / 8   # one launch = one color
    achieved = flops_launch / (t_step / 8) / 1e12
    probe = bh.fp64_fma_rate(stream)
    result["roofline"] = {
        "kernel": "mvs2_color_kernel (fused colored MVS: local residual + FDM + update), "
                  "2D Q4 512^2, one launch per color",
        "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": achieved / FP64_PEAK_TFLOPS,
        # dram__bytes_read.sum + dram__bytes_write.sum of one launch of this kernel in this
        # configuration, from one ncu capture of the unchanged kernel (62.96 MB + 0.75 MB)
        "traffic": 63.71e6, "traffic_unit": "bytes per launch",
        "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2070 MHz (derived from the unit counts "
                       "and clock; the measured-peaks file has no FP64 entry)",
        "measured_peak_tflops": probe,
        "measured_peak_source": "the library's FP64 FMA probe on this GPU (bh_fp64_fma_rate: "
                                "register-only FMA chains, 4 blocks x 128 threads per SM)",
        "frac_of_measured_peak": achieved / probe,
        "hbm_roofline": "not the bound: FP64 machine balance = derived FP64 peak / measured HBM "
                        "copy bandwidth = %.2f flop/B, while this kernel does about %.0f flop per "
                        "DRAM byte; an HBM fraction of 60 %% is unreachable in FP64, the FP64 pipe "
                        "saturates first" % (FP64_PEAK_TFLOPS * 1e12 / (HBM_GBS * 1e9),
                                             flops_launch / 63.71e6),
        "fma_per_patch": mvs2_fma_per_patch(k), "patches_per_launch": patches / 8,
        "launch_ms": t_step / 8 * 1e3,
    }
    # the rate of the FP64 operations the kernel executes (interior patches,
    # 99 % of them at this size, take the folded FDM) and the FP64 MMA probe
    executed = 2 * mvs2_fp64_ops_interior(k) * patches / 8 / (t_step / 8) / 1e12
    result["roofline"].update({
        "fp64_tensor_mma_probe_tflops": bh.fp64_mma_rate(stream),
        "executed_ops_per_interior_patch": mvs2_fp64_ops_interior(k),
        "executed_tflops": executed, "executed_frac_of_measured_peak": executed / probe})
    n4 = ctx.num_unknowns()
    r4 = torch.empty(n4, dtype=torch.float64, device=dev)
    t_res = time_op(lambda: ctx.residual(L, xs[i4], rhs[i4], r4), 20)
    result["roofline_residual_sweeps"] = {
        "kernel": "sweep_kernel x-split + y-combine (residual), 2D Q4 512^2", "bound": "alu",
        "achieved": flop_per_unknown_apply(d, k) * n4 / t_res / 1e12, "peak": FP64_PEAK_TFLOPS,
        "unit": "TFLOP/s",
        "frac": flop_per_unknown_apply(d, k) * n4 / t_res / 1e12 / FP64_PEAK_TFLOPS}

    if not args.no_breakdown:
        bd = {}
        for (d, k, N), L, ctx, b, x, xt in zip(problems, levels, ctxs, rhs, xs, xstar):
            dofs = workload.paper_dofs(d, k, N)
            n = ctx.num_unknowns()
            y = torch.empty(n, dtype=torch.float64, device=dev)
            row = {"dofs": dofs, "solve_iters": iters[k][0], "true_relres": iters[k][1]}
            row["apply"] = dofs / time_op(lambda: ctx.apply_A(L, b, y))
            for sm, name in ((bh.AVS_ATOMIC, "avs_atomic"), (bh.AVS_COLORED, "avs_colored"),
                             (bh.MVS_COLORED, "mvs")):
                with bh.Context(bh.default_params(d, k, L, smoother=sm), stream) as c2:
                    row[name + "_step"] = dofs / time_op(lambda: c2.smooth(L, y, b, 1), 5)
            # exact local solvers (dense inverse per boundary-type combination)
            for sm, name in ((bh.AVS_ATOMIC, "avs_exact"), (bh.MVS_COLORED, "mvs_exact")):
                with bh.Context(bh.default_params(d, k, L, smoother=sm,
                                                  local_solver=bh.EXACT), stream) as c2:
                    row[name + "_step"] = dofs / time_op(lambda: c2.smooth(L, y, b, 1), 5)
            # the headline protocol on one context (right, true residual, b = A x*)
            row["solve_fp64_single"] = dofs / time_op(lambda: ctx.solve(b, x, 1e-8, 200), 3)
            # the FP32 V-cycle (Sec. 5.2, Q2-Q4) and the FP32 V-cycle with FP64
            # defects (every degree), both in flexible GMRES, on one context
            for prec, name, kmax in ((bh.MIXED_FP32, "mixed_right", 4),
                                     (bh.MIXED_FP32_R64, "mixed_r64_right", 7),
                                     (bh.MIXED_FP32_RC, "mixed_rc_right", 7)):
                if k > kmax:
                    continue
                with bh.Context(bh.default_params(d, k, L, precision=prec), stream) as c2:
                    itm = c2.solve(b, y, 1e-8, 200, raise_on_noconv=False)
                    row[name + "_err_vs_xstar"] = float((y - xt).abs().max() / xt.abs().max())
                    row["solve_" + name] = dofs / time_op(
                        lambda: c2.solve(b, y, 1e-8, 200, raise_on_noconv=False), 3)
                    row[name + "_iters"], row[name + "_relres"] = itm[0], itm[1]
            # b itself i.i.d. uniform: the FP64 rounding floor of the true
            # residual (right GMRES stops on its Givens estimate), and the
            # paper's left protocol (preconditioned residual) on that b
            bu = torch.tensor(workload.rhs_uniform(n, k), dtype=torch.float64, device=dev)
            itu = ctx.solve(bu, y, 1e-8, 200, raise_on_noconv=False)
            row["uniform_rhs_floor"] = {"iters": itu[0], "true_relres": itu[1]}
            with bh.Context(bh.default_params(d, k, L, gmres_side=bh.LEFT), stream) as c2:
                itl = c2.solve(bu, y, 1e-8, 200, raise_on_noconv=False)
                row["solve_fp64_left_uniform"] = dofs / time_op(
                    lambda: c2.solve(bu, y, 1e-8, 200, raise_on_noconv=False), 2)
                row["left_uniform_iters"], row["left_uniform_true_relres"] = itl[0], itl[1]
            # the additive smoother's protocol: two pre- and post-steps, CG
            with bh.Context(bh.default_params(d, k, L, smoother=bh.AVS_ATOMIC, pre_steps=2,
                                              post_steps=2, krylov=bh.CG), stream) as c2:
                itc = c2.solve(b, y, 1e-8, 300, raise_on_noconv=False)
                row["solve_avs2_cg"] = dofs / time_op(
                    lambda: c2.solve(b, y, 1e-8, 300, raise_on_noconv=False), 2)
                row["avs2_cg_iters"] = itc[0]
            del y, bu
            bd["k%d" % k] = row
        result["breakdown_dofs_per_s"] = bd
        result["breakdown3d_dofs_per_s"] = breakdown_3d(bh, torch, dev, stream, time_op)
    if not args.no_forms:
        result["batched"] = measure_batched(bh, torch, stream)
        result["serving"] = measure_serving(bh, torch, stream, args.serve_requests)
    if cpu is not None:
        result["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(result), flush=True)
    for c in ctxs:
        c.close()
    batch.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
