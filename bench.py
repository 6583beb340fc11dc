"""Benchmark of the nested-VSIE operator apply on one B300 (and replicas under torchrun).

A step is one full matrix-free apply of the discretised VSIE operator (charge prescale,
far-field N-body sums over volume and interface source points, FP64 near-field/self
correction and mass) on the nested-sphere k0 = 10 workload: 80^3 voxel grid clipped to the
unit ball (1,608,576 tetrahedra, centroid far rule, four-point rule within two voxel
widths), two icospheres at subdivision 6 (163,840 triangles), 1,772,416 collocation
points x 2,100,096 far-field source points = 3.72e12 pair interactions per apply.

metric value: interactions/s of the mixed-precision (FP32 far field) apply, inputs
resident in HBM.  e2e: the same through vsie_apply_host (host buffers, copies timed).
--impl reference: the FP64 CPU oracle on a bounded sample of rows of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# the oracle timings report one core: hold numpy's BLAS/OpenMP pools to one thread (set
# before numpy loads them; nothing on the GPU path uses them)
for _var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "nested80_k10"
METRIC = "Helmholtz interactions/s & GMRES solve time, mixed vs FP64 on 1 B300 at rel err 1e-5"
UNIT = "interactions/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def make_workload(name):
    from paper_2607_06429_b300 import workloads as W
    return W.CONFIGS[name]()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


_ORACLE = {}


def oracle_of(w):
    """The FP64 oracle's discretisation of workload w, built once per run."""
    from oracle import vsie_oracle as O
    if id(w) not in _ORACLE:
        _ORACLE[id(w)] = O.Discretisation.from_workload(w)
    return _ORACLE[id(w)]


def one_thread():
    """Limit the BLAS/OpenMP pools to one thread while the oracle is timed, so that the
    reported core count (1) is the one used (threadpoolctl where it is installed; the
    environment variables set at start-up otherwise)."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:
        import contextlib
        return contextlib.nullcontext()
    return threadpool_limits(limits=1)


def oracle_rows_rate(w, rows_count, seed=0, time_budget=None):
    """FP64 CPU oracle applied to a seeded sample of rows; returns (interactions/s, sample
    description, seconds)."""
    with one_thread():
        return _oracle_rows_rate(w, rows_count, seed, time_budget)


def _oracle_rows_rate(w, rows_count, seed=0, time_budget=None):
    from paper_2607_06429_b300 import workloads as W
    D = oracle_of(w)
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(w.n, size=rows_count, replace=False))
    x = W.random_vector(w.n, 1)
    t0 = time.perf_counter()
    done = 0
    for r in rows:
        D.apply_rows(x, np.array([r]))
        done += 1
        if time_budget and time.perf_counter() - t0 > time_budget:
            break
    dt = time.perf_counter() - t0
    nsrc = w.n_far_sources()
    return done * nsrc / dt, f"{done} seeded rows x {nsrc} far-field source points (FP64 numpy, 1 thread)", dt


def _oracle_worker(name, tasks, results, idx):
    """One process of OraclePool: builds the oracle of workload ``name`` once, then serves
    row requests (BLAS pools held to one thread by the environment set at import)."""
    from paper_2607_06429_b300 import workloads as W
    try:
        w = make_workload(name)
        D = oracle_of(w)
    except Exception as e:  # noqa: BLE001 - reported to the parent
        results.put(("error", idx, f"{type(e).__name__}: {e}"))
        return
    xs = {}
    results.put(("ready", idx, None))
    while True:
        task = tasks.get()
        if task is None:
            break
        rows, seeds, budget = task
        key = tuple(seeds)
        if key not in xs:
            cols = [W.random_vector(w.n, s) for s in seeds]
            xs[key] = cols[0] if len(cols) == 1 else np.stack(cols, axis=1)
        x = xs[key]
        t0 = time.perf_counter()
        done, vals = [], []
        for r in rows:
            vals.append(D.apply_rows(x, np.array([r]))[0])
            done.append(int(r))
            if budget and time.perf_counter() - t0 > budget:
                break
        results.put(("rows", idx, (done, vals, time.perf_counter() - t0)))


class OraclePool:
    """The FP64 CPU oracle of one workload in ``cores`` spawned processes (rows of A x are
    independent), each holding its own copy of the discretisation.  Started with 'spawn'
    (safe after CUDA initialisation); ``start`` returns at once so that the processes build
    their discretisations while the GPU sections run."""

    def __init__(self, name, cores):
        import multiprocessing as mp
        self.ctx = mp.get_context("spawn")
        self.name = name
        self.cores = int(cores)
        self.tasks = [self.ctx.Queue() for _ in range(self.cores)]
        self.results = self.ctx.Queue()
        self.procs = [self.ctx.Process(target=_oracle_worker, args=(name, self.tasks[i], self.results, i),
                                       daemon=True) for i in range(self.cores)]
        for p in self.procs:
            p.start()
        self.ready = 0

    def wait_ready(self, timeout=900):
        while self.ready < self.cores:
            kind, _, msg = self.results.get(timeout=timeout)
            if kind == "error":
                raise RuntimeError(f"oracle process failed: {msg}")
            if kind == "ready":
                self.ready += 1

    def rows(self, rows, seeds, budget=None):
        """Oracle rows of A X (X the seeded columns ``seeds``) spread over the processes;
        each process stops after ``budget`` seconds.  Returns ({row: value(s)}, wall
        seconds of the parallel phase)."""
        self.wait_ready()
        rows = [int(r) for r in rows]
        parts = [rows[i::self.cores] for i in range(self.cores)]
        t0 = time.perf_counter()
        busy = 0
        for i, part in enumerate(parts):
            if part:
                self.tasks[i].put((part, list(seeds), budget))
                busy += 1
        out = {}
        for _ in range(busy):
            kind, _, payload = self.results.get(timeout=3600)
            done, vals, _ = payload
            out.update(zip(done, vals))
        return out, time.perf_counter() - t0

    def close(self):
        for q in self.tasks:
            q.put(None)
        for p in self.procs:
            p.join(timeout=30)


def host_cores():
    """Cores this process may run on, and the number the oracle pool uses (at most 16, so
    that the per-process copies of a large discretisation fit in host memory)."""
    try:
        avail = len(os.sched_getaffinity(0))
    except AttributeError:
        avail = os.cpu_count() or 1
    return avail, max(1, min(avail, 16))


def run_reference(args):
    """The oracle as it stands, on the host cores (one process per core, rows of the same
    workload spread over them): each step times a bounded sample of seeded rows."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    avail, cores = host_cores()
    pool = OraclePool(args.workload, cores)
    w = make_workload(args.workload)
    nsrc = w.n_far_sources()
    rng = np.random.default_rng(2024)
    per_step = 2 * cores
    try:
        for _ in range(args.warmup):
            pool.rows(rng.choice(w.n, size=min(w.n, cores), replace=False), [1])
        vals = []
        for _ in range(args.steps):
            got, wall = pool.rows(rng.choice(w.n, size=min(w.n, per_step), replace=False), [1])
            vals.append(len(got) * nsrc / wall)
    finally:
        pool.close()
    value = float(np.mean(vals))
    sample = (f"per step: {min(w.n, per_step)} seeded rows x {nsrc} far-field source points "
              f"(FP64 numpy, {cores} processes of one thread; {avail} cores available)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "nproc": avail},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def _info(info, seconds):
    return {"seconds": seconds, "iterations": info.iterations, "refinements": info.refinements,
            "rel_residual": info.rel_residual, "fp64_applies": info.fp64_applies,
            "fp32_applies": info.fp32_applies}


def row_sample_apply_seconds(torch, op, x, precision, rows):
    """Time of a full apply at ``precision`` from a contiguous block of rows
    (vsie_apply_rows): rows carry equal far-field work, so the full apply takes n/rows
    times as long (an extrapolation, used where the full FP64 apply takes minutes)."""
    r0 = min(op.n // 3, op.n - rows)
    op.apply_rows(x, r0, r0 + min(rows, 256), precision=precision)
    _, dt = _timed(torch, lambda: op.apply_rows(x, r0, r0 + rows, precision=precision))
    return dt * op.n / rows, {"rows": rows, "seconds": dt}


def sampled_residual(D, b, x, rows):
    """||b - A x|| / ||b|| over the given rows, with A from the oracle (rows independent)."""
    rows = np.asarray(rows)
    r = b[rows] - D.apply_rows(x, rows)
    return float(np.linalg.norm(r) / np.linalg.norm(b[rows]))


def solve_headline(torch, op, t32_s, tol=1e-5, D=None):
    """Time-to-solution on the benchmark mesh (Sec. 3.1 settings: x0 = 0, no restart, no
    preconditioner, plane wave along +x) at the paper's GMRES tolerance: the mixed solve
    measured (FP32-apply GMRES, its final residual formed with the double-float apply), the
    FP64 GMRES extrapolated: the mixed solve's time with every apply replaced by the FP64
    apply timed on a row sample, one FP64 apply per iteration plus the final residual."""
    b = op.plane_wave_rhs([[1.0, 0.0, 0.0]])[0].contiguous()
    t64, s64 = row_sample_apply_seconds(torch, op, b, 64, 4096)
    t48, s48 = row_sample_apply_seconds(torch, op, b, 48, 16384)
    (x, info), dt = _timed(torch, lambda: op.solve(b, mode=32, tol=tol, inner_tol=0.5 * tol, max_iters=2000,
                                                   max_refinements=4, raise_on_fail=False))
    mixed = _info(info, dt)
    mixed["status"] = info.status
    if D is not None:
        with one_thread():
            rows = np.sort(np.random.default_rng(11).choice(op.n, size=32, replace=False))
            mixed["rel_residual_oracle_rows"] = sampled_residual(D, b.cpu().numpy(), x.cpu().numpy(), rows)
            mixed["oracle_rows"] = 32
    overhead = max(0.0, dt - info.fp32_applies * t32_s - info.fp64_applies * t48)
    fp64 = overhead + (info.iterations + 1) * t64
    return {"workload": "nested80_k10", "n": op.n, "tol": tol, "mixed": mixed,
            "apply_seconds": {"fp32_measured": t32_s, "double_float_from_rows": t48, "fp64_from_rows": t64,
                              "row_samples": {"48": s48, "64": s64}},
            "fp64_extrapolated": {"seconds": fp64, "iterations": info.iterations, "basis":
                                  "the mixed solve's non-apply time + (iterations + 1) FP64 applies, "
                                  "the FP64 apply time taken from a 4,096-row sample"},
            "speedup_mixed_vs_fp64": fp64 / dt}


def solve_timing(torch, B, W, name="nested24_k10", tol=1e-8, fp64_tol8=True):
    """Time-to-solution of the FP64 GMRES solve and of the mixed solve (FP32-apply inner
    GMRES inside FP64 iterative refinement) on the same right-hand side (plane wave +x),
    both to the relative residual tol measured with the FP64 apply."""
    w = W.nested_k10(24, 4, 10.0)
    op = B.Operator.from_workload(w)
    op.autotune()
    b = op.plane_wave_rhs([[1.0, 0.0, 0.0]])[0].contiguous()
    out = {"workload": name, "n": op.n, "n_far_sources": op.n_far_sources, "tol": tol}
    x = torch.empty_like(b)
    y = torch.empty_like(b)
    for prec in (32, 48, 64):
        op.apply(b, y, precision=prec)
        _, dt = _timed(torch, lambda: op.apply(b, y, precision=prec))
        out[f"apply{prec}_interactions_per_s"] = op.n * op.n_far_sources / dt
    modes = [("mixed", dict(mode=32, inner_tol=1e-4, max_refinements=20))]
    if fp64_tol8:
        modes.append(("fp64", dict(mode=64)))
    for mode, kw in modes:
        (x, info), dt = _timed(torch, lambda: op.solve(b, tol=tol, max_iters=2000, **kw))
        out[mode] = _info(info, dt)
    if fp64_tol8:
        out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    # the same two solves to the paper's GMRES tolerance (Sec. 3.1), the metric's 1e-5
    paper_tol = 1e-5
    for mode, kw in (("mixed", dict(mode=32, inner_tol=1e-4, max_refinements=20)),
                     ("fp64", dict(mode=64))):
        (x, info), dt = _timed(torch, lambda: op.solve(b, tol=paper_tol, max_iters=2000, **kw))
        out[f"{mode}_tol1e-5"] = _info(info, dt)
    out["speedup_mixed_vs_fp64_tol1e-5"] = out["fp64_tol1e-5"]["seconds"] / out["mixed_tol1e-5"]["seconds"]
    # the batched mixed solve: 64 plane waves (Fibonacci directions) in one lockstep solve,
    # tensor-core FP32 inner applies, FP64 multi-RHS residuals; per right-hand side against
    # the single-column mixed and FP64 solves above (columns are independent systems)
    nb = 64
    B64 = op.plane_wave_rhs(W.fibonacci_dirs(nb)).contiguous()
    (X, infos), dt = _timed(torch, lambda: op.solve_batched(B64, mode=32, tol=tol, max_iters=1000, restart=400,
                                                            inner_tol=1e-4, max_refinements=20))
    r = B64 - op.apply_batched(X, precision=64)
    worst = float((torch.linalg.norm(r, dim=1) / torch.linalg.norm(B64, dim=1)).max())
    # the same residuals with the oracle's rows (4 columns x 64 seeded rows)
    from oracle import vsie_oracle as O
    D = O.Discretisation.from_workload(w)
    rows = np.sort(np.random.default_rng(24).choice(op.n, size=64, replace=False))
    Bh, Xh = B64.cpu().numpy(), X.cpu().numpy()
    with one_thread():
        worst_o = max(sampled_residual(D, Bh[c], Xh[c], rows) for c in (0, 21, 42, 63))
    its = [i.iterations for i in infos]
    out["batched_mixed"] = {
        "nrhs": nb, "seconds": dt, "seconds_per_rhs": dt / nb,
        "max_rel_residual_fp64": worst, "max_rel_residual_oracle_rows": worst_o,
        "iterations_mean": float(np.mean(its)), "iterations_max": max(its),
        "refinements_max": max(i.refinements for i in infos),
        "speedup_per_rhs_vs_mixed_single": out["mixed"]["seconds"] / (dt / nb)}
    if fp64_tol8:
        out["batched_mixed"]["speedup_per_rhs_vs_fp64_single"] = out["fp64"]["seconds"] / (dt / nb)
    op.close()
    return out


def tf32_peak(pk, sustained):
    """Dense TF32 tensor peak: the measured BF16 peak (burst, or sustained under the power
    cap for a kernel timed inside a long step) x the nominal TF32/BF16 ratio 1.1/2.25."""
    key = "bf16_tflops_sustained" if sustained and "bf16_tflops_sustained" in pk else "bf16_tflops"
    return pk[key] * 1.1 / 2.25, f"{key} {pk[key]} TFLOP/s x 1.1/2.25 (TF32 vs BF16 nominal)"


def batched_timing(torch, op, W, nrhs=64, steps=1, fp64=False, pool=None, oracle_budget=10.0):
    """Tensor-core multi-RHS apply (vsie_apply_batched) on the same operator: one block of
    nrhs right-hand sides per step; pair interactions counted per right-hand side.  Error
    against the oracle on seeded rows of two columns (the first and the last)."""
    seeds = [1000 + r for r in range(nrhs)]
    X = torch.from_numpy(np.stack([W.random_vector(op.n, sd) for sd in seeds])).cuda()
    Y = op.apply_batched(X)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        op.apply_batched(X, Y)
    b.record()
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / steps * 1e-3
    rate = op.n * op.n_far_sources * nrhs / t
    # tensor roofline: a block runs for seconds, so the sustained peak; algorithmic work 8
    # real FLOP per pair and right-hand side (one complex multiply-add), executed 24 (three
    # split TF32 products of it)
    pk, pk_kind = peaks()
    peak, basis = tf32_peak(pk, sustained=True)
    out = {"nrhs": nrhs, "seconds_per_block": t, "interactions_per_s": rate,
           "roofline": {"bound": "tensor", "achieved": rate * 8 / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": rate * 8 / 1e12 / peak, "executed_tflops": rate * 24 / 1e12,
                        "executed_frac": rate * 24 / 1e12 / peak, "peak_basis": f"{pk_kind} {basis}"}}
    if pool is not None:
        cols = [0, nrhs - 1]
        rows = np.random.default_rng(77).choice(op.n, size=16 * pool.cores, replace=False)
        got, _ = pool.rows(rows, [seeds[c] for c in cols], budget=oracle_budget)
        rr = np.array(sorted(got))
        ref = np.array([got[r] for r in rr])                   # (rows, 2)
        Yh = Y[cols].cpu().numpy()[:, rr].T
        errs = np.linalg.norm(Yh - ref, axis=0) / np.linalg.norm(ref, axis=0)
        out["rel_err_vs_oracle"] = {"max_over_columns": float(errs.max()), "columns": cols,
                                    "rows": int(len(rr))}
    if fp64:
        # the FP64 multi-RHS apply (the residual operator of the batched solve)
        op.apply_batched(X, Y, precision=64)
        torch.cuda.synchronize()
        a.record()
        op.apply_batched(X, Y, precision=64)
        b.record()
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b) * 1e-3
        out["fp64_seconds_per_block"] = t64
        out["fp64_interactions_per_s"] = op.n * op.n_far_sources * nrhs / t64
    return out


def multifreq_timing(torch, B, W, mesh="nested24_k10", nfreq=8, ndir=64, steps=2, oracle=True):
    """Multi-frequency batched apply: the same nested mesh at nfreq wavenumbers in [6, 12],
    ndir plane waves per wavenumber, all operators in one CUDA-graph plan whose tensor-core
    sums run as one persistent launch per source class; against the same work as separate
    per-operator batched applies.  Error per right-hand side against the oracle on seeded
    rows (first and last direction at the lowest and highest wavenumber)."""
    from oracle import vsie_oracle as O
    freqs = np.linspace(6.0, 12.0, nfreq)
    makers = {"nested24_k10": lambda k: W.nested_k10(24, 4, k), "nested80_k10": lambda k: W.nested_k10(80, 6, k)}
    wls = [makers[mesh](float(k)) for k in freqs]
    ops = [B.Operator.from_workload(w) for w in wls]
    dirs = W.fibonacci_dirs(ndir)
    xs = [op.plane_wave_rhs(dirs).contiguous() for op in ops]
    ys = [torch.empty_like(x) for x in xs]
    ops[0].autotune(far=False, batched=True)  # the launch uses the leading operator's shape
    g = B.BatchedGraph(ops, xs, ys)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(steps):
        g.launch()
    b.record()
    torch.cuda.synchronize()
    t_graph = a.elapsed_time(b) * 1e-3 / steps
    inter = float(ops[0].n) * float(ops[0].n_far_sources) * ndir * nfreq
    out = {"mesh": mesh, "wavenumbers": [float(k) for k in freqs], "rhs_per_wavenumber": ndir,
           "rhs_total": ndir * nfreq, "graph_nodes": g.nodes, "seconds_per_launch": t_graph,
           "interactions_per_s": inter / t_graph}
    if mesh == "nested24_k10":
        torch.cuda.synchronize()
        a.record()
        for _ in range(steps):
            for op, x, y in zip(ops, xs, ys):
                op.apply_batched(x, y)
        b.record()
        torch.cuda.synchronize()
        out["separate_applies_seconds"] = a.elapsed_time(b) * 1e-3 / steps
    if oracle:
        errs = []
        with one_thread():
            for p in (0, nfreq - 1):
                D = O.Discretisation.from_workload(wls[p])
                rows = np.random.default_rng(31 + p).choice(ops[p].n, size=8, replace=False)
                X = xs[p][[0, ndir - 1]].cpu().numpy().T          # (n, 2)
                ref = D.apply_rows(X, rows)                       # (8, 2)
                got = ys[p][[0, ndir - 1]].cpu().numpy()[:, rows].T
                errs.append(float((np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)).max()))
                del D
        out["rel_err_vs_oracle"] = {"max": max(errs), "per_wavenumber": dict(zip(["6", "12"], errs)),
                                    "sample": "8 seeded rows x directions 0 and 63 at k0 = 6 and 12"}
    g.close()
    for op in ops:
        op.close()
    return out


def cuboid_timing(torch, B, W, N=91, steps=2):
    """The paper's cuboid discretisation (Sec. 3 sphere benchmark grid, N^3 cells on
    [-3, 3]^3): FP32 apply interactions/s with the far-sum kernel's own time, and the cuboid
    oracle timed beside it on a few seeded rows (error of those rows stated)."""
    from oracle import cuboid_oracle as CO
    w = W.sphere_in_cube(N)
    op = B.Operator.from_cuboid(w)
    x = torch.from_numpy(W.random_vector(op.n, 4)).cuda()
    y = torch.empty_like(x)
    op.apply(x, y, precision=32)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        op.apply(x, y, precision=32)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    phase, _ = op.apply_timed(x, y, precision=32)
    inter = float(op.n) * float(op.n_far_sources)
    D = CO.CuboidDiscretisation.from_workload(w)
    xh = W.random_vector(op.n, 4)
    rows = np.random.default_rng(0).choice(op.n, size=4, replace=False)
    with one_thread():
        t0 = time.perf_counter()
        ref = np.array([D.apply_rows(xh, np.array([r]))[0] for r in rows])
        dt = time.perf_counter() - t0
    got = y.cpu().numpy()[rows]
    op.close()
    return {"workload": f"sphere_cube{N}", "n": op.n, "n_far_sources": op.n_far_sources,
            "ms_per_apply": ms, "interactions_per_s": inter / (ms * 1e-3),
            "far_volume_ms": phase["far_volume"],
            "far_volume_interactions_per_s": inter / (phase["far_volume"] * 1e-3),
            "rel_err_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "oracle_interactions_per_s": len(rows) * op.n_far_sources / dt,
            "oracle_sample": f"{len(rows)} seeded rows (FP64 numpy, 1 thread)"}


def bem_timing(torch, B, W, subdiv=(4, 3), k0=3.0, steps=3, vsie_grid=48, fp64_solve=True):
    """The nested PMCHWT boundary element solver (Sec. 2.4: the paper's comparison method for
    piecewise-constant media, P1 Galerkin) on icosphere interfaces r = 1, 0.5 with layers
    (rho, c) = (1.5, 0.8), (3.0, 0.6) at k0 = 3: FP32/FP64 apply rates, the apply against the
    N-body kernel's FP32-pipe bound, mixed and FP64 GMRES to the paper's 1e-5, the far field
    against the layered-sphere series, the FP64 oracle matrix on a small mesh of the same
    problem, and the same problem solved by the VSIE (tetrahedral layered ball) for the
    paper's VSIE-versus-BEM comparison (benchmark 2)."""
    from oracle import bem_oracle as BO
    from oracle import series
    radii, rho, c = [1.0, 0.5], [1.5, 3.0], [0.8, 0.6]
    dirs = W.fibonacci_dirs(64)
    ref = series.layered_sphere_far_field(dirs, [1, 0, 0], k0, radii, rho, c)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))  # noqa: E731
    out = {"workload": f"nested_spheres_ico{subdiv[0]}_ico{subdiv[1]}_k{k0:g}"}
    t0 = time.perf_counter()
    op = B.BemOperator.nested_spheres(subdiv, radii, k0, rho, c)
    torch.cuda.synchronize()
    out["create_s"] = time.perf_counter() - t0
    nt = [20 * 4 ** s for s in subdiv]
    q = op.n_points // sum(nt)
    np0, np1 = nt[0] * q, nt[1] * q
    pairs = float(np0) ** 2 + float(np0 + np1) ** 2 + float(np1) ** 2
    out.update(n_unknowns=op.n, n_points=op.n_points, n_near_pairs=op.n_near_pairs, pairs_per_apply=pairs)
    x = torch.from_numpy(W.random_vector(op.n, 11)).cuda()
    y = torch.empty_like(x)
    for prec in (32, 48, 64):
        op.apply(x, y, precision=prec)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_steps = steps if prec != 64 else 1
        a.record()
        for _ in range(n_steps):
            op.apply(x, y, precision=prec)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n_steps
        out[f"apply_ms_fp{prec}"] = ms
        out[f"pairs_per_s_fp{prec}"] = pairs / (ms * 1e-3)
    # bem_nbody_kernel<float>: 57 FP32-pipe operations and 3 MUFU operations per pair, so the
    # FP32 pipe binds (128 lanes per SM per clock)
    props = torch.cuda.get_device_properties(0)
    f_hz = 2032e6
    bound = props.multi_processor_count * 128 * f_hz / 57.0
    out["roofline_fp32"] = {"bound": "alu", "achieved": out["pairs_per_s_fp32"] / 1e9, "peak": bound / 1e9,
                            "unit": "Gpairs/s", "frac": out["pairs_per_s_fp32"] / bound,
                            "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes/clk at 2032 MHz "
                                          "/ 57 FP32-pipe operations per pair (whole apply timed)"}
    b = op.rhs([1.0, 0.0, 0.0])
    for mode in ((32, 64) if fp64_solve else (32,)):
        t = time.perf_counter()
        xs, info = op.solve(b, mode=mode, tol=1e-5, max_iters=3000, inner_tol=1e-3)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        out[f"solve_mode{mode}"] = {"seconds": dt, "iterations": info.iterations, "refinements": info.refinements,
                                    "rel_residual": info.rel_residual, "fp32_applies": info.fp32_applies,
                                    "fp64_applies": info.fp64_applies}
        if mode == 32:
            ff_bem = op.far_field(xs, dirs).cpu().numpy()
            out["far_field_rel_err_vs_series"] = rel(ff_bem, ref)
    if not fp64_solve:
        it = out["solve_mode32"]["iterations"]
        out["solve_mode64_extrapolated_s"] = (it + 1) * out["apply_ms_fp64"] * 1e-3
        out["solve_mode64_basis"] = "(mixed iterations + 1) FP64 applies at the measured FP64 apply time"
    op.close()
    # the oracle's dense matrix on the ico-1 / ico-1 mesh of the same problem
    small = B.BemOperator.nested_spheres((1, 1), radii, k0, rho, c)
    D = BO.BemDiscretisation.nested([W.icosphere(1, R) for R in radii], k0, rho, c)
    xh = W.random_vector(D.n, 12)
    with one_thread():
        t = time.perf_counter()
        yref = D.assemble() @ xh
        dt = time.perf_counter() - t
    xd = torch.from_numpy(xh).cuda()
    out["rel_err_vs_oracle"] = {"fp64": rel(small.apply(xd, precision=64).cpu().numpy(), yref),
                                "fp32": rel(small.apply(xd, precision=32).cpu().numpy(), yref),
                                "mesh": "ico1/ico1 (168 unknowns), full matrix", "oracle_seconds": dt}
    small.close()
    # the VSIE on the same layered ball (tetrahedra, centroid collocation)
    w = W.layered_ball(vsie_grid, 5, 4, k0, R2=0.5, rho1=rho[0], c1=c[0], rho2=rho[1], c2=c[1])
    vop = B.Operator.from_workload(w)
    t = time.perf_counter()
    p, vinfo = vop.solve(vop.plane_wave_rhs([1.0, 0.0, 0.0])[0].contiguous(), mode=32, tol=1e-5)
    torch.cuda.synchronize()
    vdt = time.perf_counter() - t
    ff_vsie = vop.far_field(p, dirs).cpu().numpy()
    vop.close()
    out["vsie_same_problem"] = {"workload": w.name, "n": int(w.n), "solve_s": vdt, "iterations": vinfo.iterations,
                                "far_field_rel_err_vs_series": rel(ff_vsie, ref),
                                "far_field_rel_diff_vs_bem": rel(ff_vsie, ff_bem)}
    # the paper's VSIE-versus-BEM density benchmark: nested cubes of 7 and 5 mm, rho2 = rho0/2,
    # c1 = c2 = c0/1.2, lambda0 = 3 mm; the cuboid VSIE against the BEM on cube surfaces
    cw = W.nested_cubes(0.125)
    cop = B.Operator.from_cuboid(cw)
    t = time.perf_counter()
    xc, cinfo = cop.solve(cop.plane_wave_rhs(np.array([1.0, 0.0, 0.0]))[0], mode=32, tol=1e-5)
    torch.cuda.synchronize()
    cdt = time.perf_counter() - t
    ff_cub = cop.far_field(xc, dirs).cpu().numpy()
    cn = cop.n
    cop.close()
    cbem = B.BemOperator([W.cube_surface(28, 3.5), W.cube_surface(20, 2.5)], 2.0 * np.pi / 3.0, [1.0, 0.5],
                         [1.0 / 1.2, 1.0 / 1.2])
    t = time.perf_counter()
    xcb, cbinfo = cbem.solve(cbem.rhs([1.0, 0.0, 0.0]), mode=32, tol=1e-5, max_iters=3000)
    torch.cuda.synchronize()
    cbdt = time.perf_counter() - t
    ff_cbem = cbem.far_field(xcb, dirs).cpu().numpy()
    out["papers_nested_cubes"] = {
        "vsie": {"discretisation": "cuboid, h = 0.125 mm", "n": int(cn), "solve_s": cdt,
                 "iterations": cinfo.iterations},
        "bem": {"discretisation": "P1 on cube surfaces, 0.25 mm", "n": cbem.n, "solve_s": cbdt,
                "iterations": cbinfo.iterations},
        "far_field_rel_diff": rel(ff_cub, ff_cbem)}
    cbem.close()
    return out


def bem_apply_only(args):
    """--steps applies (at --precision: 32, 48 or 64) of the nested-sphere boundary element
    operator (the bem section's problem) and one JSON line with their times: the command the
    profiles use."""
    import torch
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import workloads as W
    sub = tuple(int(v) for v in args.bem_apply_only.split(","))
    op = B.BemOperator.nested_spheres(sub, [1.0, 0.5], 3.0, [1.5, 3.0], [0.8, 0.6])
    x = torch.from_numpy(W.random_vector(op.n, 1)).cuda()
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    ms = []
    for _ in range(max(1, args.steps)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        op.apply(x, y, precision=args.precision)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    print(json.dumps({"bem_mesh": list(sub), "n_unknowns": op.n, "n_points": op.n_points,
                      "precision": args.precision, "ms_per_apply": ms}))
    op.close()


def large_timing(torch, B, W, nrhs=16):
    """The large workload (128^3 grid, k0 = 25, 7,250,176 unknowns, 8,560,896 far-field
    source points) with 16 plane waves: one timed tensor-core multi-RHS apply, the FP32
    single-column and double-float apply rates from row samples (rows carry equal work),
    and the cost of a refined solve per GMRES iteration that follows from them."""
    w = W.nested_k25(128, 7, 25.0)
    t0 = time.perf_counter()
    op = B.Operator.from_workload(w)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    X = op.plane_wave_rhs(W.fibonacci_dirs(nrhs)).contiguous()
    Y = torch.empty_like(X)
    (_, dt) = _timed(torch, lambda: op.apply_batched(X, Y))
    t32, s32 = row_sample_apply_seconds(torch, op, X[0].contiguous(), 32, 65536)
    t48, s48 = row_sample_apply_seconds(torch, op, X[0].contiguous(), 48, 4096)
    pairs = float(op.n) * float(op.n_far_sources)
    out = {"workload": "nested128_k25", "n": op.n, "n_far_sources": op.n_far_sources, "nrhs": nrhs,
           "create_s": create_s, "batched_seconds": dt, "batched_interactions_per_s": pairs * nrhs / dt,
           "fp32_apply_seconds_from_rows": t32, "double_float_apply_seconds_from_rows": t48,
           "row_samples": {"32": s32, "48": s48},
           "per_iteration_seconds": {"batched_16_rhs": dt, "16_single_column_fp32": 16 * t32},
           "refined_solve_seconds": "iterations x batched_seconds + refinements x 16 x double-float apply"}
    op.close()
    return out


def field_points(m, seed=5):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    return d * rng.uniform(1.05, 3.0, m)[:, None]


def field_timing(torch, op, W, D=None, m=65536):
    """Scattered field at m exterior points (shell 1.05 < |x| < 3 around the unit-ball
    scatterer) through vsie_scattered_field, FP32 far sums plus the near rows of the points
    within the near radii; the oracle on four of the points (error and rate)."""
    from oracle import vsie_oracle as O
    pts = field_points(m)
    xh = W.random_vector(op.n, 6)
    x = torch.from_numpy(xh).cuda()
    op.scattered_field(x, pts[:1024], precision=32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ps = op.scattered_field(x, pts, precision=32)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {"points": m, "n_far_sources": op.n_far_sources, "seconds": dt,
           "interactions_per_s": m * float(op.n_far_sources) / dt,
           "note": "wall time of the blocking call: point upload, far sums, near-row build and apply"}
    if D is not None:
        with one_thread():
            t0 = time.perf_counter()
            ref = O.scattered_field(D, xh, pts[:4])
            dto = time.perf_counter() - t0
        got = ps.cpu().numpy()[:4]
        out["rel_err_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        out["oracle_interactions_per_s"] = 4 * float(op.n_far_sources) / dto
        out["oracle_sample"] = "4 of the exterior points (FP64 numpy, 1 thread)"
    return out


def adjoint_timing(torch, op, W, D=None, steps=2):
    """The adjoint apply A^H lam (FP32 far sums with swapped roles, gather, correction
    transpose), the gradient channels of lam, and the plane-wave right-hand side and
    far-field pattern on 128 directions, on the benchmark operator; event-timed.  Errors
    against the oracle: entries of A^H lam from oracle columns, channels at source points of
    both classes, the far field on 16 directions, the plane wave."""
    from oracle import vsie_oracle as O
    lam_h = W.random_vector(op.n, 8)
    lam = torch.from_numpy(lam_h).cuda()
    x = torch.empty_like(lam)
    dirs = W.fibonacci_dirs(128)

    def timed(fn, reps):
        r = fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            r = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, r

    inter = float(op.n) * float(op.n_far_sources)
    adj_ms, _ = timed(lambda: op.adjoint_apply(lam, x, precision=32), steps)
    ch_ms, (phi, psi) = timed(lambda: op.gradient_channels(lam, precision=32), 1)
    ff_ms, ff = timed(lambda: op.far_field(lam, dirs), steps)
    pw_ms, pw = timed(lambda: op.plane_wave_rhs(dirs[:8]), steps)
    out = {"adjoint_ms": adj_ms, "adjoint_interactions_per_s": inter / (adj_ms * 1e-3),
           "gradient_channels_ms": ch_ms,
           "gradient_channels_interactions_per_s": inter / (ch_ms * 1e-3),
           "far_field_128_dirs_ms": ff_ms,
           "far_field_terms_per_s": 128.0 * op.n_far_sources / (ff_ms * 1e-3),
           "plane_wave_8_dirs_ms": pw_ms}
    if D is not None:
        with one_thread():
            cols = np.array([3, op.n // 2, D.n_tet + 5, op.n - 1])
            ref = D.matrix_columns(cols).conj().T @ lam_h
            got = x.cpu().numpy()[cols]
            out["adjoint_rel_err_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            xyz, own, cls = op.source_points()
            pick = np.concatenate([np.nonzero(cls == c)[0][:2] for c in (0, 1, 2)])
            rphi, rpsi = O.gradient_channels(D, lam_h, xyz[pick])
            gphi, gpsi = phi.cpu().numpy()[pick], psi.cpu().numpy()[pick]
            out["channels_rel_err_vs_oracle"] = float(max(np.linalg.norm(gphi - rphi) / np.linalg.norm(rphi),
                                                          np.linalg.norm(gpsi - rpsi) / np.linalg.norm(rpsi)))
            rff = D.far_field(lam_h, dirs[:16])
            out["far_field_rel_err_vs_oracle"] = float(np.linalg.norm(ff.cpu().numpy()[:16] - rff) /
                                                       np.linalg.norm(rff))
            rpw = np.stack([D.plane_wave(d) for d in dirs[:2]])
            out["plane_wave_rel_err_vs_oracle"] = float(np.linalg.norm(pw.cpu().numpy()[:2] - rpw) /
                                                        np.linalg.norm(rpw))
            out["oracle_sample"] = ("4 columns of A (adjoint entries), 2 source points per class "
                                    "(channels), 16 directions (far field), 2 plane waves")
    return out


def reduce_step_time(t_ms, world, dist, device="cuda"):
    """The step time of the whole job: the maximum over ranks of each rank's mean."""
    if world <= 1:
        return float(t_ms)
    import torch
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(interactions_per_step, world, t_ms):
    """Interactions of all ranks (one replica apply each) per second of the slowest rank."""
    return float(interactions_per_step) * world / (t_ms * 1e-3)


def rank_seed(rank):
    """Each replica applies the operator to its own seeded right-hand side."""
    return 1 + int(rank)


def flush_l2(torch, buf):
    buf.add_(1.0)


class Sections:
    """Optional sections of the JSON line, run in order of importance while the run's wall
    clock stays within its budget (skipped sections are listed, not silently dropped); a
    section that raises is reported with its error instead of ending the run."""

    def __init__(self, budget_s):
        self.t0 = time.perf_counter()
        self.budget = budget_s
        self.skipped = []
        self.failed = {}
        self.seconds = {}

    def elapsed(self):
        return time.perf_counter() - self.t0

    def run(self, name, fn, estimate_s=0.0):
        if self.elapsed() + estimate_s > self.budget:
            self.skipped.append(name)
            return None
        t = time.perf_counter()
        try:
            return fn()
        except Exception as e:  # noqa: BLE001 - reported in the line
            self.failed[name] = f"{type(e).__name__}: {e}"
            return None
        finally:
            self.seconds[name] = round(time.perf_counter() - t, 1)


# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the volume (G-class) far-sum
# kernel on the benchmark workload, from the ncu capture summarised in
# profiles/nbody_kernel_PolG2_nested80_k10.md; None once the kernel changes until recaptured.
G_KERNEL_DRAM_BYTES = 91616768


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--budget-s", type=float, default=1500.0,
                    help="wall-clock budget of the whole run; optional sections past it are skipped")
    ap.add_argument("--parallelism", default="replicas", choices=["replicas", "rows"],
                    help="N > 1: independent replica applies, or one apply sharded by rows")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in work shapes (profiling: no candidate launches)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the cuboid-grid apply, exterior-field and adjoint timings")
    ap.add_argument("--multifreq-mesh", default="auto", choices=["auto", "nested24_k10", "nested80_k10", "none"])
    ap.add_argument("--no-bem", action="store_true",
                    help="skip the nested PMCHWT boundary element section")
    ap.add_argument("--bem-apply-only", default=None, metavar="S1,S2",
                    help="profiling: only --steps applies (at --precision) of the boundary element "
                         "operator on icosphere interfaces of these subdivisions, then exit")
    ap.add_argument("--large", action="store_true",
                    help="also time the k0 = 25, 128^3 workload's 16-RHS apply (about 5 minutes)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.bem_apply_only:
        return bem_apply_only(args)

    sec = Sections(args.budget_s)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the oracle processes build their discretisations while the GPU sections run
    avail, cores = host_cores()
    pool = OraclePool(args.workload, cores) if (not args.no_cpu_baseline and world == 1) else None

    import torch
    import torch.distributed as dist
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import workloads as W

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    w = make_workload(args.workload)
    t0 = time.perf_counter()
    op = B.Operator.from_workload(w)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    # work shapes of the persistent kernels picked by timing candidates on this operator
    t0 = time.perf_counter()
    tuning = op.autotune(far=args.precision == 32, batched=args.precision == 32 and not args.no_batched) \
        if args.precision == 32 and not args.no_autotune else None
    autotune_s = time.perf_counter() - t0
    n, nsrc = op.n, op.n_far_sources
    inter = float(n) * float(nsrc)

    sharded = None
    if world > 1 and args.parallelism == "rows":
        from paper_2607_06429_b300 import sharded as SH
        sharded = SH.RowShardedApply.from_operator(op, precision=args.precision)
        seed = 1                                   # one system, every rank the same x
    else:
        seed = rank_seed(rank)
    xh = W.random_vector(n, seed)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty_like(x)
    l2buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step():
        if sharded is not None:
            return sharded(x)
        op.apply(x, y, precision=args.precision)
        return y

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phase_ms = []
    launches = 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush_l2(torch, l2buf)
            ev[s][0].record(stream)
            yt = step()
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        # per-kernel device times of the same apply (events between its phases)
        for s in range(min(args.steps, 3)):
            flush_l2(torch, l2buf)
            ms, launches = op.apply_timed(x, y, precision=args.precision)
            phase_ms.append(ms)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = float(np.mean(step_ms))
    t_ms = reduce_step_time(t_ms, world, dist)
    if world > 1:
        dist.barrier()
    clocks = clk.summary()
    y_result = yt.cpu().numpy()

    # end-to-end through the host-buffer entry point (pinned host memory)
    hx = torch.from_numpy(W.random_vector(n, 3)).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    op.apply_host_ptr(hx.data_ptr(), hy.data_ptr(), 1, args.precision)
    e2e_ms = []
    for _ in range(max(2, min(args.steps, 3))):
        t1 = time.perf_counter()
        op.apply_host_ptr(hx.data_ptr(), hy.data_ptr(), 1, args.precision)
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    e2e_t = float(np.mean(e2e_ms))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    if sharded is not None:
        value = inter / (t_ms * 1e-3)               # one apply of the whole system per step
        scaling = "strong"
    else:
        value = whole_job_value(inter, world, t_ms)
        scaling = "weak"
    # roofline of the dominant kernel: FP32 far-field sum over volume sources (G class)
    pk, pk_kind = peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    f_mhz = clocks["sm_mhz"] or pk.get("sm_max_mhz", 2032.0)
    g_ms = float(np.mean([p["far_volume"] for p in phase_ms]))
    n_g = nsrc - 3 * w.n_tri if w.grad_alpha is None else None
    probe = sec.run("pipe_probe", lambda: B.pipe_probe())
    rf = None
    if n_g:
        achieved = n * n_g / (g_ms * 1e-3)
        # ALU roofline: 3 MUFU ops (rsqrt, sin, cos) per pair at 16/clk/SM vs ~20 FP32-pipe
        # ops per pair at 128/clk/SM; the binding pipe is the MUFU one.
        xu = n_sm * 16 * f_mhz * 1e6 / 3.0
        fma = n_sm * 128 * f_mhz * 1e6 / 20.0
        peak = min(xu, fma)
        rf = {"bound": "alu", "kernel": "nbody_kernel<float,PolG2> (volume far field) + fixup",
              "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Ginteractions/s", "frac": achieved / peak,
              "peak_basis": f"min(MUFU {n_sm} SMs x 16/clk / 3 per pair, FP32 {n_sm} x 128/clk / 20 per pair) "
                            f"at {f_mhz:.0f} MHz (median SM clock sampled under load)",
              "traffic": G_KERNEL_DRAM_BYTES, "kernel_ms": g_ms,
              "algorithmic_bytes_per_launch": 20.0 * n_g + 16.0 * n + 16.0 * n,
              "measured_pipes_per_clk_per_sm": probe}
        # the timed apply's far sums as a whole (G and K concurrently when the autotuner chose
        # it): every class takes 3 MUFU operations per pair, so the same MUFU bound applies
        other_ms = float(np.mean([p["prescale"] + p["correction"] for p in phase_ms]))
        far_ms = max(t_ms - other_ms, 1e-9)
        rf["apply_far_sums"] = {"achieved": inter / (far_ms * 1e-3) / 1e9, "peak": xu / 1e9,
                                "unit": "Ginteractions/s", "frac": inter / (far_ms * 1e-3) / xu,
                                "far_ms": far_ms,
                                "concurrent_gk": (tuning or {}).get("concurrent_gk")}

    # error of the timed result against the oracle on seeded rows, and the oracle's rate on
    # all host cores (rows are independent): the CPU baseline
    cpu = None
    err = None
    if pool is not None and sharded is None:
        def oracle_rows():
            rows = np.random.default_rng(0).choice(n, size=min(n, 256 * cores), replace=False)
            got, wall = pool.rows(rows, [seed], budget=args.cpu_seconds)
            rr = np.array(sorted(got))
            ref = np.array([got[r] for r in rr])
            e = {"rel_l2": float(np.linalg.norm(y_result[rr] - ref) / np.linalg.norm(ref)),
                 "max_row_rel": float(np.max(np.abs(y_result[rr] - ref)) / np.max(np.abs(ref))),
                 "rows": int(len(rr)), "tolerance": 1e-5 if args.precision == 32 else 1e-12}
            c = {"value": len(rr) * nsrc / wall, "unit": UNIT, "cores": cores, "nproc": avail, "kind": "oracle",
                 "sample": f"{len(rr)} seeded rows x {nsrc} far-field source points (FP64 numpy, "
                           f"{cores} processes of one thread, {avail} cores available; rows independent)",
                 "seconds": round(wall, 2)}
            return e, c
        r = sec.run("oracle_rows", oracle_rows)
        if r:
            err, cpu = r

    solve80 = None
    if not args.no_solve and args.precision == 32 and args.workload == WORKLOAD:
        D80 = oracle_of(w) if (world == 1 and not args.no_cpu_baseline) else None
        solve80 = sec.run("solve_nested80", lambda: solve_headline(torch, op, t_ms * 1e-3, D=D80), estimate_s=450)

    batched = None
    if not args.no_batched and args.precision == 32:
        batched = sec.run("batched", lambda: batched_timing(torch, op, W, fp64=n * nsrc < 1e11, pool=pool),
                          estimate_s=60)

    extras = None
    if not args.no_extras and args.precision == 32:
        D = None
        if world == 1 and not args.no_cpu_baseline:
            D = sec.run("oracle_main", lambda: oracle_of(w), estimate_s=30)
        extras = {"adjoint": sec.run("adjoint", lambda: adjoint_timing(torch, op, W, D), estimate_s=60),
                  "field": sec.run("field", lambda: field_timing(torch, op, W, D), estimate_s=20),
                  "cuboid": sec.run("cuboid", lambda: cuboid_timing(torch, B, W), estimate_s=20)}

    if pool is not None:
        pool.close()

    solve24 = None
    if not args.no_solve:
        solve24 = sec.run("solve_nested24", lambda: solve_timing(torch, B, W, fp64_tol8=False), estimate_s=90)

    bem = None
    if not args.no_bem and args.precision == 32:
        bem = sec.run("bem", lambda: bem_timing(torch, B, W), estimate_s=90)

    multifreq = None
    if not args.no_batched and args.precision == 32 and args.multifreq_mesh != "none":
        mesh = args.multifreq_mesh
        if mesh == "auto":
            mesh = "nested80_k10" if sec.elapsed() + 400 < sec.budget else "nested24_k10"
        op.close()  # room for the eight operators of the multi-frequency plan
        multifreq = sec.run("multifreq", lambda: multifreq_timing(
            torch, B, W, mesh=mesh, steps=1 if mesh == "nested80_k10" else 2), estimate_s=30)

    large = None
    if args.large and args.precision == 32:
        large = sec.run("large", lambda: large_timing(torch, B, W), estimate_s=300)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True,
        "scaling": scaling, "vs_baseline": None, "dtype": "f32" if args.precision == 32 else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n_targets": n, "n_far_sources": nsrc,
                   "interactions_per_step": inter, "nnz_correction": op.nnz,
                   "precision": args.precision, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": (f"rows{world}" if sharded is not None else f"replicas{world}")
                   if world > 1 else "single"},
        "e2e": {"value": inter / (e2e_t * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 16 * n, "ms_per_step": e2e_t},
        "rel_err_vs_oracle": err,
        "gpu_launches": launches * args.steps,
        "phase_ms": {k: float(np.mean([p[k] for p in phase_ms])) for k in phase_ms[0]},
        "create_s": create_s,
        "autotune": tuning, "autotune_s": autotune_s,
        "roofline": rf, "peaks": pk_kind,
        "solve": {"nested80_k10": solve80, "nested24_k10": solve24},
        "batched": batched,
        "multifreq": multifreq,
        "large": large,
        "bem": bem,
        "extras": extras,
        "cpu_baseline": cpu,
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "sections": {"seconds": sec.seconds, "skipped": sec.skipped, "failed": sec.failed,
                     "budget_s": args.budget_s, "elapsed_s": round(sec.elapsed(), 1)},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
