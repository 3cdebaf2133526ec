#!/usr/bin/env python3
"""Benchmark: large dense single solves of graph-form ADMM on B300.

One step (per rank) is one full solve -- setup (Sinkhorn-Knopp equilibration, Gram,
Cholesky, inverse factor) plus ADMM iterations to eps_abs = 1e-4, eps_rel = 1e-3 -- of each of
  (a) tall Lasso, A 40000 x 10000 ~ N(0, 1/n)          (factor of I + A^T A),
  (b) fat l1-logistic regression, A 2000 x 40000 ~ N(0, 1/n)  (factor of I + A A^T),
i.e. two solves per step.  value = solves/s over all ranks (replicas: each rank solves its
own instances, no collective on the data path).  Inputs are resident in HBM when the timed
region starts; e2e repeats the measurement through the same C API from pinned host memory.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s & p50/p99 latency at eps_rel=1e-3, served vs plain; proj HBM GB/s"
WORKLOAD = ("large dense single solves: tall Lasso 40000x10000 (I+A^TA factor) + fat l1-logistic "
            "2000x40000 (I+AA^T factor), eps_abs=1e-4, eps_rel=1e-3, 2 solves per step")


# B300 HBM3e nominal bandwidth (context beside the measured copy bandwidth)
HBM_NOMINAL_GBS = 7700.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d["bf16_tflops_sustained"], src="measured")
    except Exception:
        return dict(hbm=6400.0, bf16=1800.0, bf16_sus=1400.0, src="fallback")


# FP64 and FP32 SIMT peaks from unit counts and clocks: 148 SMs x 2.032 GHz; FP32 128 lanes x 2
# flop; FP64 at the 1.25 TFLOP/s the part is rated for.
FP32_SIMT_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
FP64_TFLOPS = 1.25


def problem_seeds(rank: int):
    """Seeds of the two large solves a rank runs: rank 0 runs the named workload (seeds 10000,
    10001); every other rank runs its own independent replica of it."""
    return 10_000 + 100 * rank, 10_001 + 100 * rank


def problems(rank: int):
    import workloads as W
    sa, sb = problem_seeds(rank)
    a = W.lasso(40000, 10000, seed=sa, nnz_frac=0.1, noise_std=0.01, lam_frac=0.1)
    b = W.logistic(2000, 40000, seed=sb, nnz_frac=0.05, lam_frac=0.05)
    return [a, b]


class Clocks:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[5:9]) if v.lower() == "active"})
        out.update(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


def _dist():
    """(dist, rank, world size, local rank).  One process per GPU under torchrun: NCCL when a GPU
    is present, gloo otherwise (POGS_DIST_BACKEND overrides).  The replicas exchange only the
    barrier and the maximum of their timed intervals -- the path itself has no collective."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = os.environ.get("POGS_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")
        dist.init_process_group(backend)
        return dist, dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def _max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def job_rate(units_per_rank: int, world_size: int, t_ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world_size / (t_ms_max / 1000.0)


# ----------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on a bounded sample of the same workload.
# ----------------------------------------------------------------------------------------------
def _oracle_iters(prob):
    """The oracle's own iteration count on a large benchmark problem at the benchmark's stopping
    test, from the stored full oracle run (tests/golden/make_bench_refs.py), or None."""
    try:
        m, n = prob.A.shape
        with open(os.path.join(ROOT, "tests", "golden", f"bench_{prob.name}_{m}x{n}.json")) as f:
            rec = json.load(f)
        return dict(iters=int(rec["iters"]), obj=float(rec["obj"]), seconds=rec.get("seconds"))
    except Exception:
        return None


def oracle_full_size_timing(probs, iters, sample_iters):
    """The oracle as it stands, timed on the full-size problems on the host cores: its setup
    (Sinkhorn-Knopp equilibration and the FP64 Gram + Cholesky factorization) once, then
    `sample_iters[i]` ADMM iterations of problem i with that cached factor.  Every iteration does
    the same work (two passes of A, the triangular solves, the proxes), so a solve to the
    iteration count `iters[i]` takes t_setup + iters[i] * t_iter; nothing is scaled by size.
    Returns (solves/s, per-problem details)."""
    from oracle import admm as OA
    from oracle import equil as OE
    from oracle import project as OPJ
    total = 0.0
    parts = []
    for prob, it, k in zip(probs, iters, sample_iters):
        m, n = prob.A.shape
        A = prob.A.astype(np.float64)
        t0 = time.perf_counter()
        eq = OE.equilibrate(A, 10)
        t_eq = time.perf_counter() - t0
        t0 = time.perf_counter()
        factor = OPJ.Projector(eq.Ahat)
        t_fac = time.perf_counter() - t0
        prm = OA.Params(max_iter=k, abs_tol=0.0, rel_tol=0.0, gap_stop=False)
        t0 = time.perf_counter()
        OA.solve(A, prob.f, prob.g, prm, eq=eq, factor=factor)
        t_iter = (time.perf_counter() - t0) / k
        t_solve = t_eq + t_fac + it * t_iter
        total += t_solve
        rec = dict(shape=[m, n], t_equil_s=t_eq, t_factor_s=t_fac, t_iter_s=t_iter, iters_timed=k, iters=it,
                   solve_s=t_solve)
        ref = _oracle_iters(prob)
        if ref:
            rec["oracle_own_iters"] = ref["iters"]
        parts.append(rec)
        del A, eq, factor
    return len(probs) / total, parts


def oracle_sample_check(pool, served_obj, seconds=20.0, one_thread_seconds=0.0, one_thread_pool=None):
    """The oracle as it stands, solving the distinct problems of `pool` one after another until
    `seconds` have passed (a bounded sample; its sequential throughput is the workload's CPU
    baseline), and every GPU result for a sampled problem checked against the oracle's
    objective at the same stopping test.

    served_obj: {index into pool: [objective of every GPU result for that problem]}.
    one_thread_seconds > 0 also times the same problems in order with BLAS limited to one
    thread, for about that long (`value_1thread`); one_thread_pool is the Python expression that
    rebuilds `pool` in the child process that does it.
    Returns (cpu_baseline, check)."""
    from oracle import admm as OA
    t0 = time.perf_counter()
    ref = {}
    for k, pb in enumerate(pool):
        if ref and time.perf_counter() - t0 >= seconds:
            break
        r = OA.solve(pb.A, pb.f, pb.g, OA.Params())
        ref[k] = (float(r.obj), int(r.status))
    elapsed = time.perf_counter() - t0
    errs, checked = [], 0
    for k, (obj, status) in ref.items():
        if status != 0:
            continue
        for v in served_obj.get(k, []):
            errs.append(abs(v - obj) / max(1.0, abs(obj)))
            checked += 1
    cpu = dict(value=len(ref) / elapsed, unit="solves/s", cores=_threads(), cpu_count=os.cpu_count(),
               kind="oracle",
               sample=f"first {len(ref)} of {len(pool)} distinct problems, solved in sequence ({elapsed:.1f} s)")
    if one_thread_seconds > 0 and one_thread_pool:
        # the same problems in order, in a child process with one BLAS thread
        out = oracle_one_thread(
            "import json, time, workloads as W\n"
            "from oracle import admm as OA\n"
            f"probs = {one_thread_pool}\n"
            "t1 = time.perf_counter(); done = 0\n"
            "for pb in probs:\n"
            f"    if done and time.perf_counter() - t1 >= {one_thread_seconds}: break\n"
            "    OA.solve(pb.A, pb.f, pb.g, OA.Params()); done += 1\n"
            "print(json.dumps(dict(done=done, seconds=time.perf_counter() - t1)))\n")
        if out:
            cpu["value_1thread"] = out["done"] / out["seconds"]
            cpu["sample_1thread"] = (f"first {out['done']} of the same problems in a child process with one BLAS "
                                     "thread")
    check = dict(payloads=len(ref), oracle_converged=sum(1 for o in ref.values() if o[1] == 0),
                 requests_checked=checked, max_rel_obj_err=max(errs) if errs else None,
                 within_1e_3=sum(e <= 1e-3 for e in errs), within_1e_2=sum(e <= 1e-2 for e in errs))
    return cpu, check


def oracle_one_thread(script: str, timeout: float = 300.0):
    """Run `script` (Python source that prints one JSON line last) in a child process whose BLAS
    uses one thread: the thread counts are set in its environment before NumPy loads.  The child
    runs only the oracle (no CUDA).  Returns the parsed line, or None if the child failed."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", script], env=env, cwd=ROOT, capture_output=True, text=True,
                           timeout=timeout)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:  # noqa: BLE001
        return None


def _threads():
    try:
        from threadpoolctl import threadpool_info
        return max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, on the benchmark's own
    full-size problems.  Each problem's setup (equilibration, Gram + Cholesky) is timed once at
    full size; each step is then one full-size ADMM iteration of each problem with its cached
    factor (W untimed, K timed).  value = solves/s of a solve to the iteration counts the GPU
    path and the oracle both take on these problems (90 and 449): 2 / sum(setup + iters * t_iter)."""
    dist, rank, ws, _ = _dist()
    if rank != 0:
        return
    from oracle import admm as OA
    from oracle import equil as OE
    from oracle import project as OPJ
    probs = problems(0)
    iters = [90, 449]
    t_run = time.perf_counter()
    state = []
    for prob in probs:
        A = prob.A.astype(np.float64)
        t0 = time.perf_counter()
        eq = OE.equilibrate(A, 10)
        t_eq = time.perf_counter() - t0
        t0 = time.perf_counter()
        factor = OPJ.Projector(eq.Ahat)
        t_fac = time.perf_counter() - t0
        state.append((A, prob, eq, factor, t_eq, t_fac))
    one = OA.Params(max_iter=1, abs_tol=0.0, rel_tol=0.0, gap_stop=False)

    def step():
        out = []
        for A, prob, eq, factor, *_ in state:
            t0 = time.perf_counter()
            OA.solve(A, prob.f, prob.g, one, eq=eq, factor=factor)
            out.append(time.perf_counter() - t0)
        return out

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    per = [step() for _ in range(args.steps)]
    t_steps = time.perf_counter() - t0
    wall = time.perf_counter() - t_run
    t_iter = [float(np.mean([p[i] for p in per])) for i in range(len(probs))]
    details = []
    total = 0.0
    for (A, prob, eq, factor, t_eq, t_fac), ti, it in zip(state, t_iter, iters):
        solve_s = t_eq + t_fac + it * ti
        total += solve_s
        details.append(dict(shape=list(prob.A.shape), t_equil_s=t_eq, t_factor_s=t_fac, t_iter_s=ti, iters=it,
                            solve_s=solve_s))
    value = len(probs) / total
    sample = ("FP64 oracle on the full-size problems: setup (equilibration + Gram + Cholesky) timed once per "
              f"problem, then {args.steps} timed full-size iterations of each (after {args.warmup} untimed); "
              f"solve time = setup + {iters} iterations x the measured time per iteration")
    line = dict(impl="reference", metric=METRIC, value=value, unit="solves/s", n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000.0 * t_steps / max(1, args.steps), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD, l2="inputs larger than L2",
                            step="one full-size ADMM iteration of each of the two problems"),
                cpu_baseline=dict(value=value, unit="solves/s", cores=_threads(), cpu_count=os.cpu_count(),
                                  kind="oracle", sample=sample),
                e2e=dict(value=value, unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                wall_s=wall, details=details)
    print(json.dumps(line))


# ----------------------------------------------------------------------------------------------
def run_ours(args):
    import torch

    dist, rank, ws, local = _dist()
    torch.cuda.set_device(local)
    import paper_1503_08366_b300 as P

    stream = torch.cuda.current_stream()
    probs = problems(rank)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()

    def fn(p, conv):
        return type(p)(*(conv(getattr(p, k)) for k in "habcde"))

    D = [(dev(p.A), fn(p.f, dev), fn(p.g, dev)) for p in probs]
    H = [(pin(p.A), fn(p.f, pin), fn(p.g, pin)) for p in probs]
    outs_d = [tuple(torch.empty(k, dtype=torch.float32, device="cuda") for k in (p.n, p.m, p.n, p.m)) for p in probs]
    outs_h = [tuple(torch.empty(k, dtype=torch.float32).pin_memory() for k in (p.n, p.m, p.n, p.m)) for p in probs]
    prm = P.pogs_default_params(loop_mode=args.loop_mode)

    def one_solve(i, inputs, outs, ev=None):
        A, f, g = inputs[i]
        if ev is not None:
            ev[0].record(stream)
        h = P.pogs_setup(A, prm, stream=stream)
        info = P.pogs_solve(h, f, g, prm, *outs[i])
        P.pogs_free(h)
        if ev is not None:
            ev[1].record(stream)
        if info.status != 0:
            raise RuntimeError(f"solve {i} did not converge: {info.as_dict()}")
        return info

    for _ in range(args.warmup):
        for i in range(len(probs)):
            one_solve(i, D, outs_d)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    lat_events = []
    launches0 = P.pogs_kernel_launches()
    _barrier(dist)
    torch.cuda.synchronize()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    infos = []
    for _ in range(args.steps):
        for i in range(len(probs)):
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            infos.append(one_solve(i, D, outs_d, ev))
            lat_events.append(ev)
    e_end.record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    launches = P.pogs_kernel_launches() - launches0
    clk = clocks.stop()
    t_ms = _max_over_ranks(dist, e_start.elapsed_time(e_end))
    solves = len(probs) * args.steps * ws
    value = job_rate(len(probs) * args.steps, ws, t_ms)
    lats = sorted(a.elapsed_time(b) for a, b in lat_events)
    p50 = float(np.percentile(lats, 50))
    p99 = float(np.percentile(lats, 99))

    # ---- end to end through the same API, pinned host buffers -------------------------------
    torch.cuda.synchronize()
    _barrier(dist)
    e2 = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    e2[0].record(stream)
    for _ in range(args.steps):
        for i in range(len(probs)):
            one_solve(i, H, outs_h)
    e2[1].record(stream)
    torch.cuda.synchronize()
    t_e2e = _max_over_ranks(dist, e2[0].elapsed_time(e2[1]))
    e2e_value = solves / (t_e2e / 1000.0)
    h2d = sum(p.A.nbytes + sum(getattr(p.f, k).nbytes + getattr(p.g, k).nbytes for k in "habcde") for p in probs)
    d2h = sum(4 * 2 * (p.m + p.n) for p in probs) + 2 * 112

    # ---- per-kernel breakdown and the dominant kernel's roofline --------------------------------
    # Each iteration kernel is timed live with CUDA events on the launching stream (20 launches
    # back to back on the solved state, after the timed region); setup phases come from the
    # setup's own events.  Shares are of one step: per-launch time x launches per solve.
    peaks = _peaks()
    comp = {}        # (kernel, problem index) -> dict(total ms, per-launch ms, bytes per launch, launches)
    per_problem = []
    proj = []
    for i, p in enumerate(probs):
        A, f, g = D[i]
        h = P.pogs_setup(A, prm, stream=stream)
        info = P.pogs_solve(h, f, g, prm, *outs_d[i])
        rep = P.pogs_get_setup_report(h)
        kt = P.pogs_time_kernels(h, reps=20)
        P.pogs_free(h)
        it = info.iters
        tall = p.m >= p.n
        sym = kt["LinvT"][1] == 0.0   # the inverse applied as one symmetric product
        names = dict(prox="prox", A_pass1="colsum" if tall else "rowdot", Linv="symv" if sym else "trmv",
                     A_pass2="rowdot" if tall else "colsum", check="check")
        if not sym:
            names["LinvT"] = "trmv_t"
        for name, t in (("equil", rep.equil_ms), ("gram", rep.gram_ms), ("factor", rep.factor_ms),
                        ("inverse", rep.inverse_ms), ("ingest", rep.ingest_ms)):
            comp[(name, i)] = dict(total=t, ms=t, bytes=None, launches=1)
        for k, name in names.items():
            comp[(name, i)] = dict(total=kt[k][0] * it, ms=kt[k][0], bytes=kt[k][1], launches=it)
        proj_ms = sum(kt[k][0] for k in ("A_pass1", "Linv", "LinvT", "A_pass2"))
        proj_b = sum(kt[k][1] for k in ("A_pass1", "Linv", "LinvT", "A_pass2"))
        proj.append(dict(shape=[p.m, p.n], ms=proj_ms, bytes=proj_b, gbs=proj_b / proj_ms / 1e6,
                         frac=proj_b / proj_ms / 1e6 / peaks["hbm"],
                         frac_nominal=proj_b / proj_ms / 1e6 / HBM_NOMINAL_GBS))
        per_problem.append(dict(shape=[p.m, p.n], cls=p.name, iters=it, obj=info.obj, setup_ms=info.setup_ms,
                                solve_ms=info.solve_ms, setup=rep.as_dict(),
                                kernels={names[k]: dict(ms=v[0], bytes=v[1]) for k, v in kt.items() if k in names}))
    totals = {}
    for (name, i), r in comp.items():
        totals[name] = totals.get(name, 0.0) + r["total"]
    (dom, di) = max(comp, key=lambda key: comp[key]["total"])
    rec = comp[(dom, di)]
    pm, pn = probs[di].m, probs[di].n
    p_, q_ = max(pm, pn), min(pm, pn)
    shape = f"{pm}x{pn}"
    step_ms = t_ms / args.steps
    if rec["bytes"] is not None:
        achieved = rec["bytes"] / rec["ms"] / 1e6
        roof = dict(kernel=dom, shape=shape, bound="hbm", achieved=achieved, peak=peaks["hbm"], unit="GB/s",
                    frac=achieved / peaks["hbm"], bytes_per_launch=rec["bytes"], ms_per_launch=rec["ms"],
                    launches_per_step=rec["launches"], peak_src=peaks["src"] + " hbm_gbs (burst copy)")
    elif dom in ("factor", "inverse"):
        fl = q_ ** 3 / 3.0   # Cholesky: q^3/3 flop; triangular inverse: q^3/3 flop
        mixed = prm.chol_prec == P.CHOL["MIXED"]
        peak = FP32_SIMT_TFLOPS if (mixed or dom == "inverse") else FP64_TFLOPS
        roof = dict(kernel=dom, shape=shape, bound="alu", achieved=fl / rec["ms"] / 1e9, peak=peak,
                    unit="TFLOP/s", peak_src=("FP32 SIMT" if peak == FP32_SIMT_TFLOPS else "FP64")
                    + " from unit counts and clocks")
        roof["frac"] = roof["achieved"] / peak
    elif dom == "gram":
        fl = float(p_) * q_ * q_   # lower triangle of G: q(q+1)/2 dot products of length p
        used = per_problem[di]["setup"]["gram_prec_used"]
        if used == P.GRAM["FP32"]:
            roof = dict(kernel="gram", shape=shape, bound="alu", achieved=fl / rec["ms"] / 1e9,
                        peak=FP32_SIMT_TFLOPS, unit="TFLOP/s", peak_src="FP32 SIMT from unit counts and clocks")
        else:
            eff = fl * (3 if used == P.GRAM["BF16X3"] else 1)
            pk = peaks["bf16"] * (0.5 if used == P.GRAM["TF32"] else 1.0)
            roof = dict(kernel="gram", shape=shape, bound="tensor", achieved=eff / rec["ms"] / 1e9, peak=pk,
                        unit="TFLOP/s", peak_src=peaks["src"] + " bf16 burst"
                        + (" x 1/2 (tf32 nominal ratio)" if used == P.GRAM["TF32"] else ""))
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        by = 2 * 4.0 * pm * pn * (2 * 10 + 1) if dom == "equil" else 2 * 4.0 * pm * pn
        roof = dict(kernel=dom, shape=shape, bound="hbm", achieved=by / rec["ms"] / 1e6, peak=peaks["hbm"],
                    unit="GB/s", frac=by / rec["ms"] / 1e6 / peaks["hbm"], peak_src=peaks["src"] + " hbm_gbs")
    roof["traffic"] = _traffic(dom, shape)
    shares = {k: v / sum(totals.values()) for k, v in sorted(totals.items(), key=lambda kv: -kv[1])}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        its = [pp["iters"] for pp in per_problem]
        v, parts = oracle_full_size_timing(probs, its, sample_iters=[5, 20])
        cpu = dict(value=v, unit="solves/s", cores=_threads(), cpu_count=os.cpu_count(), kind="oracle",
                   sample=("FP64 oracle on the full-size problems: setup (equilibration + Gram + Cholesky) "
                           "timed once each, then 5 (tall) and 20 (fat) full-size iterations with the cached "
                           f"factor; solve time = setup + the GPU solves' iteration counts {its} x the measured "
                           "time per iteration"), parts=parts)

    extras = {}
    if rank == 0 and ws == 1 and not args.no_extras:
        extras["small_lasso"] = _extra("small_lasso", small_lasso_measure)
        extras["serve"] = _extra("serve", lambda: serve_measure(args))
        extras["batch"] = _extra("batch", lambda: batch_measure(args))

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="solves/s", n_gpus=ws, steps=args.steps, warmup=args.warmup,
                    ms_per_step=step_ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
                    data="synthetic (seeded N(0,1/n) matrices of the paper's Lasso/logistic classes)",
                    config=dict(workload=WORKLOAD, l2="inputs larger than L2 (1.6 GB and 320 MB matrices)",
                                parallelism="replicas" if ws > 1 else "single GPU",
                                gram_prec=prm.gram_prec, chol_prec=prm.chol_prec, refine_steps=prm.refine_steps),
                    latency_ms=dict(p50=p50, p99=p99, n=len(lats)),
                    e2e=dict(value=e2e_value, unit="solves/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
                    gpu_launches=launches, roofline=roof, proj_hbm=proj, time_shares=shares,
                    per_problem=per_problem, clocks=clk, cpu_baseline=cpu, **extras)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def small_lasso_measure(reps=50):
    """The 200 x 100 Lasso (A ~ N(0, 1/100), 10 nonzeros in x_true, lambda = 0.1 ||A^T b||_inf):
    one plain solve through the C ABI from host arrays (setup + iterations + copies), timed over
    `reps` solves after warm-up; the oracle as it stands on the same problem with all host cores
    and with BLAS limited to one thread; and the GPU objective against the oracle's at the same
    stopping test."""
    import torch
    import paper_1503_08366_b300 as P
    import workloads as W
    from oracle import admm as OA
    prob = W.lasso_small(0)
    prm = P.pogs_default_params(max_iter=2000)

    def gpu_once():
        with P.Solver(prob.A, prm) as s_:
            return s_.solve(prob.f, prob.g)[0]
    for _ in range(5):
        gpu_once()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        info = gpu_once()
        ts.append(time.perf_counter() - t0)
    oprm = OA.Params(max_iter=2000)

    def oracle_times(k):
        out, r = [], None
        for _ in range(k):
            t0 = time.perf_counter()
            r = OA.solve(prob.A, prob.f, prob.g, oprm)
            out.append(time.perf_counter() - t0)
        return out, r
    o_all, ref = oracle_times(5)
    one = oracle_one_thread(
        "import json, time, numpy as np, workloads as W\n"
        "from oracle import admm as OA\n"
        "prob = W.lasso_small(0); ts = []\n"
        "for _ in range(5):\n"
        "    t0 = time.perf_counter(); OA.solve(prob.A, prob.f, prob.g, OA.Params(max_iter=2000))\n"
        "    ts.append(time.perf_counter() - t0)\n"
        "print(json.dumps(dict(ts=ts)))\n")
    o_one = one["ts"] if one else [float("nan")]
    med = lambda v: float(np.median(v))
    return dict(workload="plain single Lasso solve 200x100, eps_abs=1e-4, eps_rel=1e-3, max_iter 2000",
                gpu=dict(ms_per_solve=1e3 * med(ts), solves_per_s=1.0 / med(ts), iters=info.iters,
                         status=info.status, obj=info.obj, reps=reps,
                         timing="wall clock per pogs_setup + pogs_solve + pogs_free call from host arrays"),
                oracle=dict(ms_per_solve=1e3 * med(o_all), solves_per_s=1.0 / med(o_all), iters=ref.iters,
                            obj=ref.obj, cores=_threads(), cpu_count=os.cpu_count()),
                oracle_1thread=dict(ms_per_solve=1e3 * med(o_one), solves_per_s=1.0 / med(o_one), cores=1,
                                    how="child process with one BLAS thread"),
                obj_rel_err=abs(info.obj - ref.obj) / max(1.0, abs(ref.obj)))


def _extra(name, fn):
    """Run one extra comparison of the default line; a failure is recorded, not raised."""
    try:
        t0 = time.perf_counter()
        out = fn()
        out["wall_s"] = time.perf_counter() - t0
        return out
    except Exception as e:  # noqa: BLE001
        return dict(error=f"{type(e).__name__}: {e}")


def _traffic(kernel, shape):
    """DRAM bytes (read + write) per launch of `kernel` on `shape` from the committed ncu summary,
    or None if the kernel's source changed since the counters were taken."""
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(f"{kernel}@{shape}")
        if not rec:
            return None
        src = open(os.path.join(ROOT, "paper_1503_08366_b300", "csrc", rec["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != rec["sha16"]:
            return None
        return rec["bytes_per_launch"]
    except Exception:
        return None


# ----------------------------------------------------------------------------------------------
# Extra workloads (not the default bench line): many small instances, and serving.
# ----------------------------------------------------------------------------------------------
def run_batch(args):
    print(json.dumps(batch_measure(args)))


def batch_measure(args):
    """2048 independent instances (Lasso / Huber / SVM / NNLS, m log-U[64, 2048], n log-U[32, 512])
    in one pogs_solve_batch call, vs the plain single-problem path one instance at a time."""
    import torch
    import paper_1503_08366_b300 as P
    import workloads as W
    probs = W.batch_mix(count=args.count)
    prm = P.pogs_default_params()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dprobs = [W.Problem(p.name, dev(p.A), W.FnParams(*(dev(getattr(p.f, k)) for k in "habcde")),
                        W.FnParams(*(dev(getattr(p.g, k)) for k in "habcde")), p.meta) for p in probs]
    P.pogs_solve_batch(dprobs, prm)                     # tunes the launch configuration once
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = P.pogs_solve_batch(dprobs, prm)
    torch.cuda.synchronize()
    t_dev = time.perf_counter() - t0
    t0 = time.perf_counter()
    P.pogs_solve_batch(probs, prm)
    t_host = time.perf_counter() - t0
    st = [r[0].status for r in res]
    # algorithmic bytes of every pass the method makes, per instance: setup (2 passes of A per
    # Sinkhorn-Knopp sweep, the rescale and the Gram read) and, per iteration, two passes of A,
    # two sweeps of the triangular factor and ~14 vectors of length m + n
    peaks = _peaks()
    algo = 0.0
    for pb, r in zip(probs, res):
        m, n = pb.A.shape
        q = min(m, n)
        algo += (2 * prm.sk_sweeps + 3) * 4.0 * m * n
        algo += r[0].iters * (8.0 * m * n + 4.0 * q * (q + 1) + 56.0 * (m + n))
    achieved = algo / t_dev / 1e9
    # the batch's time is set by its slowest instance: time the instances that converge within
    # max_iter as a batch of their own, to separate the engine's rate from that tail
    conv = [i for i, r in enumerate(res) if r[0].status == 0]
    bulk = None
    if 0 < len(conv) < len(probs):
        sub = [dprobs[i] for i in conv]
        P.pogs_solve_batch(sub, prm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.pogs_solve_batch(sub, prm)
        torch.cuda.synchronize()
        t_sub = time.perf_counter() - t0
        b_sub = 0.0
        for i in conv:
            m, n = probs[i].A.shape
            q = min(m, n)
            b_sub += (2 * prm.sk_sweeps + 3) * 4.0 * m * n
            b_sub += res[i][0].iters * (8.0 * m * n + 4.0 * q * (q + 1) + 56.0 * (m + n))
        bulk = dict(count=len(conv), value=len(conv) / t_sub, unit="solves/s", achieved=b_sub / t_sub / 1e9,
                    frac=b_sub / t_sub / 1e9 / peaks["hbm"], iters_max=max(res[i][0].iters for i in conv))
    cpu, check = (None, None) if args.no_cpu_baseline else \
        oracle_sample_check(probs, {i: [r[0].obj] for i, r in enumerate(res)}, one_thread_seconds=10.0,
                            one_thread_pool=f"W.batch_mix(count={args.count})")
    # plain: the single-problem path, one instance at a time (a bounded sample, extrapolated)
    k = min(args.plain_sample, len(probs))
    t0 = time.perf_counter()
    for pb in dprobs[:k]:
        with P.Solver(pb.A, prm) as sv:
            sv.solve(pb.f, pb.g, device_out=True)
    torch.cuda.synchronize()
    t_plain = (time.perf_counter() - t0) / k * len(probs)
    return (dict(workload="batch", metric="solves/s", value=len(probs) / t_dev, unit="solves/s",
                          e2e=dict(value=len(probs) / t_host, unit="solves/s"),
                          plain=dict(value=len(probs) / t_plain, unit="solves/s", sample=k),
                          statuses={str(s_): st.count(s_) for s_ in set(st)},
                          iters_mean=float(np.mean([r[0].iters for r in res])),
                          iters_max=int(max(r[0].iters for r in res)), cpu_baseline=cpu, oracle_check=check,
                          converged_only=bulk,
                          roofline=dict(bound="hbm", achieved=achieved, peak=peaks["hbm"], unit="GB/s",
                                        frac=achieved / peaks["hbm"], bytes=algo,
                                        peak_src=peaks["src"] + " hbm_gbs",
                                        note="algorithmic bytes of all passes (setup + per-iteration "
                                             "8mn + 4q(q+1) + 56(m+n)) over the whole batch time; "
                                             "instances staged in shared memory or resident in L2 "
                                             "read fewer bytes from DRAM"),
                          config=dict(count=len(probs), classes="lasso,huber,svm,nnls", m="log-U[64,2048]",
                                      n="log-U[32,512]")))


def _pool(trace, size):
    """Request payloads: `size` distinct problems drawn like the trace (class, m, n); request i
    carries payload i mod size."""
    return [trace[i].problem() for i in range(min(size, len(trace)))]


def run_serve(args):
    print(json.dumps(serve_measure(args)))


def censored_percentile(done_ms, unfinished_lower_ms, q):
    """Percentile q of a latency sample in which some requests had not finished when the run
    stopped: each of those counts at its lower bound (stop time - arrival), so the result is a
    lower bound on the true percentile (exact when nothing is unfinished)."""
    v = list(done_ms) + list(unfinished_lower_ms)
    return float(np.percentile(np.asarray(v), q)) if v else None


def serve_measure(args):
    """Poisson arrivals at 2000 req/s, mixed Lasso / logistic / Huber / SVM / NNLS with
    m log-U[100, 8000], n log-U[50, 4000], served with continuous batching under a 120 GB budget,
    vs the same trace served one request at a time by the single-problem path (run to the end
    of the trace unless --plain-limit is given; latencies of requests a limited run did not
    reach count at their lower bound)."""
    import torch
    import paper_1503_08366_b300 as P
    import workloads as W
    trace = W.serve_trace(count=args.requests)
    pool = _pool(trace, args.pool)
    prm = P.pogs_default_params()
    n_req = len(trace)

    big = [min(pool[i % len(pool)].A.shape) > 512 for i in range(n_req)]
    fin, steps = [], []
    served_obj = {}

    def served():
        lat, iters, st = [], [], []
        with P.Server(int(120e9), large_workers=args.workers, max_resident=args.max_resident, params=prm) as srv:
            t0 = time.monotonic()
            i = 0
            while len(lat) < n_req:
                now = time.monotonic() - t0
                while i < n_req and trace[i].arrival_s <= now:
                    srv.submit(pool[i % len(pool)], i)
                    i += 1
                if srv.pending() > 0:
                    ts = time.monotonic()
                    srv.step(args.step_iters)
                    steps.append(time.monotonic() - ts)
                else:
                    time.sleep(min(1e-4, max(0.0, trace[i].arrival_s - now)) if i < n_req else 0)
                for tag, info, _s, _a, done_s, *_ in srv.poll():
                    lat.append(done_s - (t0 + trace[tag].arrival_s))
                    fin.append((tag, done_s - t0))
                    served_obj.setdefault(tag % len(pool), []).append(info.obj)
                    iters.append(info.iters)
                    st.append(info.status)
            wall = time.monotonic() - t0
        return wall, lat, iters, st

    def plain(limit_s):
        lat, st = [], []
        t0 = time.monotonic()
        for i, req in enumerate(trace):
            now = time.monotonic() - t0
            if limit_s is not None and now > limit_s:
                break
            if req.arrival_s > now:
                time.sleep(req.arrival_s - now)
            pb = pool[i % len(pool)]
            with P.Solver(pb.A, prm) as sv:
                info, *_ = sv.solve(pb.f, pb.g)
            lat.append(time.monotonic() - (t0 + req.arrival_s))
            st.append(info.status)
        return time.monotonic() - t0, lat, st

    wall, lat, iters, st = served()
    pwall, plat, pst = plain(args.plain_limit)
    # requests the plain run did not reach: latency at least (end of the run - arrival)
    punf = [(pwall - trace[i].arrival_s) * 1e3 for i in range(len(plat), n_req)]
    cpu, check = (None, None) if args.no_cpu_baseline else oracle_sample_check(pool, served_obj)
    pct = lambda v, q: float(np.percentile(np.asarray(v) * 1e3, q)) if v else None

    def by_class(large):
        """Completions of one class (large: min(m, n) > 512, served by the worker threads):
        count, when the last one finished, and how many finished in each 10 s of the run."""
        t = sorted(d for tag, d in fin if big[tag] == large)
        if not t:
            return dict(count=0)
        return dict(count=len(t), last_s=t[-1], per_10s=np.bincount((np.asarray(t) // 10).astype(int)).tolist())
    return (dict(
        workload="serve", metric="solves/s & p50/p99 latency at eps_rel=1e-3, served vs plain",
        value=len(lat) / wall, unit="solves/s", latency_ms=dict(p50=pct(lat, 50), p99=pct(lat, 99)),
        statuses={str(s_): st.count(s_) for s_ in set(st)}, iters_mean=float(np.mean(iters)),
        small=by_class(False), large=by_class(True), cpu_baseline=cpu, oracle_check=check,
        step_calls=dict(count=len(steps), total_s=float(np.sum(steps)), p50_ms=pct(steps, 50),
                        max_ms=pct(steps, 100)),
        plain=dict(value=len(plat) / pwall, unit="solves/s", served=len(plat), of=n_req,
                   statuses={str(s_): pst.count(s_) for s_ in set(pst)},
                   latency_ms=dict(p50=censored_percentile([x * 1e3 for x in plat], punf, 50),
                                   p99=censored_percentile([x * 1e3 for x in plat], punf, 99),
                                   censored=len(punf)),
                   limit_s=args.plain_limit),
        served_p99_below_plain_p99=(pct(lat, 99) is not None and
                                    pct(lat, 99) < censored_percentile([x * 1e3 for x in plat], punf, 99)),
        config=dict(requests=n_req, rate_hz=2000, budget_gb=120, payload_pool=len(pool), step_iters=args.step_iters,
                    max_resident=args.max_resident,
                    large_workers=args.workers, m="log-U[100,8000]", n="log-U[50,4000]",
                    classes="lasso,logistic,huber,svm,nnls")))


def _precision_refs(name, m, n):
    """Oracle reference results for the precision study, written by tests/golden/make_precision_refs.py."""
    path = os.path.join(ROOT, "tests", "golden", f"precision_{name}_{m}x{n}.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return None


def run_precision(args):
    """Gram precision x refinement on dense NNLS and inequality-form LP, 30000 x 15000.

    Per (class, gram mode, refinement): the solve (setup and iteration times, iterations,
    status, objective, residuals), its objective error against the stored FP64 oracle results
    (the oracle stopped by the same test, and a much tighter oracle run standing in for p*),
    and the accuracy of one projection of seeded (c, d), measured as the FP64 residual of the
    normal equations the exact projection satisfies, (c + A^T d) - (I + A^T A) x and y - A x
    (tall case), relative to ||c + A^T d||."""
    import torch
    import workloads as W
    import paper_1503_08366_b300 as P

    torch.cuda.set_device(0)
    modes = [("BF16", 0), ("BF16", 1), ("TF32", 0), ("TF32", 1), ("BF16X3", 0)]
    out = []
    for gen in (W.nnls_precision_large, W.lp_precision_large):
        prob = gen()
        m, n = prob.A.shape
        refs = _precision_refs(prob.name, m, n) or {}
        Adev = torch.from_numpy(prob.A).cuda()
        rng = np.random.default_rng(77)
        c = rng.standard_normal(n).astype(np.float32)
        d = rng.standard_normal(m).astype(np.float32)
        for gram, refine in modes:
            prm = P.pogs_default_params(gram_prec=gram, refine_steps=refine, max_iter=5000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with P.Solver(Adev, prm) as s:
                torch.cuda.synchronize()
                setup_s = time.perf_counter() - t0
                rep = P.pogs_get_setup_report(s.handle)
                info, x, y, mu, nu = s.solve(prob.f, prob.g)
                xp, yp = s.project(c, d, prm)
                Ah = s.ahat().astype(np.float64)
            rhs = c.astype(np.float64) + Ah.T @ d.astype(np.float64)
            xp64, yp64 = xp.astype(np.float64), yp.astype(np.float64)
            kkt = rhs - (xp64 + Ah.T @ (Ah @ xp64))
            rec = dict(cls=prob.name, gram=gram, refine=refine, gram_used=rep.gram_prec_used, status=info.status,
                       iters=info.iters, obj=info.obj, r_pri=info.r_pri, r_dual=info.r_dual, eps_pri=info.eps_pri,
                       eps_dual=info.eps_dual, r_pri_unscaled=info.r_pri_unscaled,
                       r_dual_unscaled=info.r_dual_unscaled, setup_ms=info.setup_ms, solve_ms=info.solve_ms,
                       gram_ms=rep.gram_ms, factor_ms=rep.factor_ms,
                       proj_kkt_rel=float(np.linalg.norm(kkt) / np.linalg.norm(rhs)),
                       proj_graph_rel=float(np.linalg.norm(yp64 - Ah @ xp64) / max(np.linalg.norm(yp64), 1e-30)))
            for key in ("same_tol", "tight"):
                if key in refs:
                    po = refs[key]["obj"]
                    rec[f"obj_relerr_vs_oracle_{key}"] = abs(info.obj - po) / max(1.0, abs(po))
            out.append(rec)
            del Ah
        del Adev
    line = dict(workload="precision", metric="relative objective error vs FP64 oracle and projection accuracy",
                config=dict(shape=[30000, 15000], classes="nnls, lp (10% nonzeros stored dense)",
                            eps_abs=1e-4, eps_rel=1e-3, chol_prec="MIXED",
                            oracle="stored oracle results: tests/golden/precision_<class>_30000x15000.json"),
                results=out)
    print(json.dumps(line))


def run_next(args):
    """Rows beyond the single-solve path: (1) warm start and factor reuse -- a Lasso
    regularisation path of 10 weights on one handle (one setup), each solve started from the
    previous solution, against the same path started cold; (2) the wider prox library and
    classes -- basis pursuit, entropy maximization and portfolio optimization solves."""
    import torch
    import workloads as W
    import paper_1503_08366_b300 as P

    torch.cuda.set_device(0)
    out = {}
    # (1) regularisation path, 20000 x 8000 Lasso
    base = W.lasso(20000, 8000, seed=50_000)
    A = torch.from_numpy(base.A).cuda()
    lam_max = float(np.max(np.abs(base.A.astype(np.float64).T @ base.f.b.astype(np.float64))))
    fracs = [0.5, 0.35, 0.25, 0.18, 0.12, 0.09, 0.06, 0.045, 0.03, 0.02]
    prm = P.pogs_default_params(max_iter=20000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with P.Solver(A, prm) as s:
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        runs = {}
        for mode in ("cold", "warm"):
            x0 = nu0 = None
            iters, objs = [], []
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for frac in fracs:
                g = W.FnParams.make(base.n, W.H["ABS"], c=frac * lam_max)
                info, x, y, mu, nu = s.solve(base.f, g, x0=x0, nu0=nu0)
                if info.status != 0:
                    raise RuntimeError(f"path solve did not converge: {info.as_dict()}")
                iters.append(info.iters)
                objs.append(info.obj)
                if mode == "warm":
                    x0, nu0 = x, nu
            torch.cuda.synchronize()
            runs[mode] = dict(seconds=time.perf_counter() - t1, iters=iters, objs=objs)
    out["lasso_path"] = dict(shape=[20000, 8000], weights=len(fracs), setup_s=setup_s,
                             cold=dict(solves_per_s=len(fracs) / runs["cold"]["seconds"], iters=runs["cold"]["iters"]),
                             warm=dict(solves_per_s=len(fracs) / runs["warm"]["seconds"], iters=runs["warm"]["iters"]),
                             max_obj_rel_diff=float(max(abs(a - b) / max(1.0, abs(b)) for a, b in
                                                        zip(runs["warm"]["objs"], runs["cold"]["objs"]))))
    del A
    # (2) the remaining Appendix A classes
    cls = []
    for name, gen, shape in (("basis_pursuit", W.basis_pursuit, (2000, 8000)), ("entropy", W.entropy, (2000, 20000)),
                             ("portfolio", W.portfolio, (20000, 100))):
        prob = gen(*shape, seed=51_000)
        prm = P.pogs_default_params(max_iter=20000)
        Ad = torch.from_numpy(np.ascontiguousarray(prob.A)).cuda()
        reps = []
        for _ in range(3):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            with P.Solver(Ad, prm) as s:
                info, x, *_ = s.solve(prob.f, prob.g)
            torch.cuda.synchronize()
            reps.append(time.perf_counter() - t1)
        cls.append(dict(cls=name, shape=list(prob.A.shape), status=info.status, iters=info.iters, obj=info.obj,
                        r_pri=info.r_pri, eps_pri=info.eps_pri, r_dual=info.r_dual, eps_dual=info.eps_dual,
                        setup_ms=info.setup_ms, solve_ms=info.solve_ms, wall_s_median=float(np.median(reps))))
        del Ad
    out["classes"] = cls
    # (3) indirect projection (CGLS, no Gram and no factorization) against the direct one
    ind = []
    for name, gen, shape in (("lasso", W.lasso, (40000, 10000)), ("logistic", W.logistic, (10000, 40000))):
        prob = gen(*shape, seed=52_000)
        Ad = torch.from_numpy(np.ascontiguousarray(prob.A)).cuda()
        row = dict(cls=name, shape=list(prob.A.shape))
        for mode in ("DIRECT", "CGLS"):
            prm = P.pogs_default_params(max_iter=20000, proj_mode=mode)
            reps = []
            for _ in range(2):
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                with P.Solver(Ad, prm) as s:
                    info, x, *_ = s.solve(prob.f, prob.g)
                torch.cuda.synchronize()
                reps.append(time.perf_counter() - t1)
            row[mode.lower()] = dict(status=info.status, iters=info.iters, obj=info.obj, setup_ms=info.setup_ms,
                                     solve_ms=info.solve_ms, wall_s_median=float(np.median(reps)))
        row["obj_rel_diff"] = abs(row["cgls"]["obj"] - row["direct"]["obj"]) / max(1.0, abs(row["direct"]["obj"]))
        ind.append(row)
        del Ad
    out["indirect"] = ind
    # (4) sparse A (CSR passes): 200000 x 20000 Lasso, 100 nonzeros per row (0.5%), direct and CGLS
    prob = W.sparse_lasso(200000, 20000, seed=53_000, per_row=100)
    M = prob.A
    dev = tuple(torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (M.indptr.astype(np.int32), M.indices,
                                                                             M.data))
    sparse = dict(shape=list(M.shape), nnz=int(M.nnz), per_row=100)
    peaks = _peaks()
    for mode in ("DIRECT", "CGLS"):
        prm = P.pogs_default_params(max_iter=20000, proj_mode=mode)
        reps = []
        for _ in range(2):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            h = P.pogs_setup_csr(*dev, M.shape, prm)
            info = P.pogs_solve(h, prob.f, prob.g, prm)
            torch.cuda.synchronize()
            reps.append(time.perf_counter() - t1)
            if mode == "DIRECT" and len(reps) == 2:
                kt = P.pogs_time_kernels(h, reps=20)
                passes = {}
                for k in ("A_pass1", "A_pass2"):
                    ms, by = kt[k]
                    passes[k] = dict(us=ms * 1000.0, bytes=by, gbs=by / ms / 1e6, frac=by / ms / 1e6 / peaks["hbm"])
                sparse["csr_passes"] = passes
                sparse["iteration_us"] = kt["iteration"][0] * 1000.0
            P.pogs_free(h)
        sparse[mode.lower()] = dict(status=info.status, iters=info.iters, obj=info.obj, setup_ms=info.setup_ms,
                                    solve_ms=info.solve_ms, wall_s_median=float(np.median(reps)))
    out["sparse"] = sparse
    del dev
    # (5) sparse LDL^T of K on a banded A (where K factors with little fill): 200000 x 100000,
    # 17 nonzeros per row, against the indirect projection on the same handle type
    prob = W.banded_lasso(200000, 100000, seed=54_000, half_band=8)
    M = prob.A
    dev = tuple(torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (M.indptr.astype(np.int32), M.indices,
                                                                             M.data))
    st, _, _ = P.pogs_ldl_analyze(M.indptr, M.indices, M.shape)
    ldl = dict(shape=list(M.shape), nnz=int(M.nnz), half_band=8, symbolic=st)
    for mode in ("LDL", "CGLS"):
        prm = P.pogs_default_params(max_iter=20000, proj_mode=mode)
        reps = []
        for _ in range(2):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            h = P.pogs_setup_csr(*dev, M.shape, prm)
            info = P.pogs_solve(h, prob.f, prob.g, prm)
            torch.cuda.synchronize()
            reps.append(time.perf_counter() - t1)
            if mode == "LDL" and len(reps) == 2:
                kt = P.pogs_time_kernels(h, reps=10)
                ldl["solve_us"] = kt["Linv"][0] * 1000.0
                ldl["iteration_us"] = kt["iteration"][0] * 1000.0
            P.pogs_free(h)
        ldl[mode.lower()] = dict(status=info.status, iters=info.iters, obj=info.obj, setup_ms=info.setup_ms,
                                 solve_ms=info.solve_ms, wall_s_median=float(np.median(reps)))
    ldl["obj_rel_diff"] = abs(ldl["ldl"]["obj"] - ldl["cgls"]["obj"]) / max(1.0, abs(ldl["cgls"]["obj"]))
    out["sparse_ldl"] = ldl
    del dev
    print(json.dumps(dict(workload="next", metric="warm-start path solves/s and iterations; class solves; "
                          "indirect vs direct projection; sparse A", **out)))


def run_kernels(args):
    """One full-size problem of the default step (--shape tall: the 40000x10000 Lasso, fat: the
    2000x40000 logistic): setup, one solve, then each kernel of one ADMM iteration timed with CUDA
    events through pogs_time_kernels (launched back to back from the host; small kernels read the
    host's launch rate).  The launch sequence is fixed, so a profiler can select launches by
    index: the setup's Sinkhorn-Knopp passes come first, then the timed launches."""
    import torch
    import workloads as W
    import paper_1503_08366_b300 as P
    torch.cuda.set_device(0)
    prob = (W.lasso_tall_large if args.shape == "tall" else W.logistic_fat_large)()
    A = torch.from_numpy(prob.A).cuda()
    with P.Solver(A, P.pogs_default_params()) as s:
        info, *_ = s.solve(prob.f, prob.g)
        kt = P.pogs_time_kernels(s.handle, reps=args.reps)
    print(json.dumps(dict(workload="kernels", shape=list(prob.A.shape), iters=info.iters, obj=info.obj,
                          reps=args.reps, kernels={k: dict(ms=v[0], bytes=v[1]) for k, v in kt.items()})))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="large",
                    choices=["large", "batch", "serve", "precision", "next", "kernels"])
    ap.add_argument("--shape", default="fat", choices=["fat", "tall"], help="kernels workload: which problem")
    ap.add_argument("--reps", type=int, default=10, help="kernels workload: timed launches per kernel")
    ap.add_argument("--count", type=int, default=2048, help="batch workload: instances")
    ap.add_argument("--plain-sample", type=int, default=128, help="batch workload: plain-path sample")
    ap.add_argument("--requests", type=int, default=20000, help="serve workload: requests in the trace")
    ap.add_argument("--pool", type=int, default=256, help="serve workload: distinct payloads")
    ap.add_argument("--workers", type=int, default=8, help="serve workload: threads for large requests")
    ap.add_argument("--step-iters", type=int, default=25, help="serve workload: iterations per step")
    ap.add_argument("--max-resident", type=int, default=8192, help="serve workload: resident small requests")
    ap.add_argument("--plain-limit", type=float, default=None,
                    help="serve workload: stop the plain run after this many seconds (default: run the whole trace)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the small-Lasso, batch and serving comparisons")
    ap.add_argument("--loop-mode", type=int, default=0,
                    help="0: one graph per solve (conditional WHILE node); 1: host-checked loop over a "
                         "captured iteration (for profilers that skip conditional graphs)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "next":
        run_next(args)
    elif args.workload == "kernels":
        run_kernels(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
