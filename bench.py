#!/usr/bin/env python
"""Throughput benchmark of the QCP solution-map derivative (JVP + VJP).

Workload (default): the large sparse QCP (n = 100 000, m = 220 000; cone
{0}^20000 x R+^150000 x lognormal second-order-cone blocks on 50 000 rows;
A with 2.2 M entries in power-law columns, P banded plus 200 k random upper
entries), one forward and one adjoint direction, relative residual
tolerance 1e-6, FP64 data, synthetic seeded data with an optimum built by
construction.  One step = the JVP and the VJP in one
qcp_derivative_jvp_vjp_multi call (engine auto: the stream engine for a
problem this size).  --workload config2 runs the n = 2000 SOC problem with
16 + 16 directions at rtol 1e-10 (cluster engine), --workload example the
paper's example shape, cones a problem with every cone family (PSD,
exponential and power blocks: the pass engine), config4 / learned the
batched and learned forms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload config3|config2|example|cones|config1|config4|learned]

Prints one JSON line (rank 0).  `value` counts JVP+VJP solves per second
over all ranks with inputs resident in device memory; `e2e` measures the
same through the public API with the inputs copied from pinned host memory
and the outputs copied back inside the timed region.  With N > 1 (torchrun)
every rank solves its own instance (replicas, weak scaling); there is no
collective on the data path.  `--impl reference` times the CPU FP64 oracle
on the same workload: dense LU of the bordered derivative system where it
fits (configs 1, 2, example, cones), else a bounded sample of its matrix-free
LSMR iterations.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

L2_FLUSH_BYTES = 256 << 20
# mean LSQR iterations per solve of config 3 at rtol 1e-6 with 16
# equilibration sweeps (GB300 runs: 2727 JVP, 3093 VJP), for the CPU
# oracle's per-iteration sample when the GPU's own count is not at hand
CONFIG3_ITERS_PER_SOLVE = 2910.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# --------------------------------------------------------------------------- workloads
def workload(name, rank):
    import qcpgen as g
    if name == "config1":
        prob = g.config1(seed=rank)
        dirs = g.make_directions_batch(prob, 5 + 1000 * rank, 2)
        return prob, dirs, 1e-10, "tiny QP n=50 m=80 {0}^20 x R+^60, 2 JVP + 2 VJP directions"
    if name == "config2":
        prob = g.config2(seed=rank)
        dirs = g.make_directions_batch(prob, 5 + 1000 * rank, 16)
        return prob, dirs, 1e-10, ("single SOC QCP n=2000 m=5500 {0}^500 x R+^2000 x SOC(10)^300, "
                                   "16 JVP + 16 VJP directions")
    if name == "config3":
        prob = g.config3(seed=rank)
        dirs = g.make_directions_batch(prob, 5 + 1000 * rank, 1)
        return prob, dirs, 1e-6, ("large sparse QCP n=100000 m=220000 {0}^20000 x R+^150000 x lognormal SOC "
                                  "blocks on 50000 rows, 1 JVP + 1 VJP direction")
    if name == "example":
        prob = g.paper_example(seed=rank)
        dirs = g.make_directions_batch(prob, 5 + 1000 * rank, 16)
        # rtol 1e-9: at 1e-10 rounding stalls the true residual of a few
        # directions near 1.3e-10 (they then report QCP_NOT_CONVERGED)
        return prob, dirs, 1e-9, ("the paper's example shape (Sec. 4): x in R^1000, r in R^2000, "
                                   "[C D; E 0; f^T 0] with C 2000x1000 dense, {0}^2000 x R+^1000 x {0}, "
                                   "P diagonal on r; 16 JVP + 16 VJP directions")
    if name == "cones":
        prob = g.small_qcp(11 + rank, 1500, 100, 600, (5,) * 40, nnz_per_row=8, psd_orders=(8,) * 30,
                           exp_kinds=("ray", "sint", "yint") * 33 + ("ray",),
                           pow_blocks=(("ray", 0.3), ("sint", 0.6), ("yint", 0.45), ("ray", 0.7)) * 25)
        dirs = g.make_directions_batch(prob, 5 + 1000 * rank, 8)
        return prob, dirs, 1e-9, ("every cone family: QCP n=1500 m=2580 {0}^100 x R+^600 x SOC(5)^40 x "
                                  "PSD(8)^30 x EXP^100 x POW^100 (exponents 0.3-0.7), dense P, "
                                  "8 JVP + 8 VJP directions")
    raise SystemExit(f"unknown workload {name}")


def algorithmic_bytes_split(prob):
    """Bytes one product with F or F^T must move (FP64 values 8 B, indices
    4 B), as (matrix, vectors): half of B_iter = 2 [12 (2 nnz(A) + nnz_up(P))
    + 4 (m + 2n + 3)] + 8 (8n + 14m + 9N), the per-iteration traffic of one F
    and one F^T product (the matrix part) plus the LSQR vector updates (the
    vector part).  Two systems whose passes share a launch's read of the
    matrix (paired stream iterations) move the matrix part once."""
    n, m, N = prob.n, prob.m, prob.N
    mat = 12 * (2 * prob.A.nnz + prob.P.nnz) + 4 * (m + 2 * n + 3)
    vec = 8 * (8 * n + 14 * m + 9 * N) / 2.0
    return float(mat), vec


def algorithmic_bytes_per_pass(prob):
    mat, vec = algorithmic_bytes_split(prob)
    return mat + vec


# the dominant kernel of each engine and the sources it is built from
KERNELS = {
    "stream": ("k_stream", ("qcpd_stream.cuh", "qcpd_df64.cuh", "qcpd_kernels.cuh", "qcpd_common.cuh")),
    # the stream engine's paired launches (a JVP and a VJP system in step)
    "stream_pair": ("k_stream2", ("qcpd_stream.cuh", "qcpd_df64.cuh", "qcpd_kernels.cuh", "qcpd_common.cuh")),
    "passes": ("k_pass", ("qcpd_kernels.cuh", "qcpd_common.cuh")),
    "persistent": ("k_persist", ("qcpd_kernels.cuh", "qcpd_common.cuh")),
    "cluster": ("k_cluster_df", ("qcpd_cluster_df.cuh", "qcpd_cluster.cuh", "qcpd_df64.cuh", "qcpd_kernels.cuh",
                                 "qcpd_common.cuh")),
    "cluster_fp64": ("k_cluster", ("qcpd_cluster.cuh", "qcpd_kernels.cuh", "qcpd_common.cuh")),
}


def kernel_source_hash(engine):
    h = hashlib.sha256()
    for f in KERNELS[engine][1]:
        with open(os.path.join(ROOT, "paper_2508_17522_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(engine, workload_name):
    """dram read+write bytes per system pass (one product with F or F^T of
    one system) of the engine's dominant kernel from a committed ncu summary
    (profiles/*.json), if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"{KERNELS[engine][0]}_{workload_name}_dram.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha") != kernel_source_hash(engine):
        return None
    return rec.get("dram_bytes_per_system_pass")


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6), ("sw_thermal_slowdown", 7),
                              ("sw_power_cap", 8)):
                if f[col].lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- oracle (CPU)
def oracle_step(prob, dirs):
    """The CPU FP64 oracle on one step of the workload: dense LU of the
    bordered derivative system, then every JVP and VJP direction."""
    from oracle import derivative as D
    fac = D.DenseFactor(prob)
    for d in dirs:
        D.jvp_dense(prob, d, fac)
        D.vjp_dense(prob, d, fac)
    return 2 * len(dirs)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def dense_workload(name):
    """Workloads whose (N+1)^2 bordered system the dense-LU oracle factors."""
    return name in ("config1", "config2", "example", "cones")


def oracle_sample(prob, dirs, budget_s=30.0):
    """A bounded sample of the dense-LU oracle on this workload (rank 0 only)."""
    t0 = time.perf_counter()
    solves = oracle_step(prob, dirs[:16])
    dt = time.perf_counter() - t0
    return {"value": solves / dt, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": (f"one full step on the host: dense LU of the bordered (N+1)x(N+1) derivative "
                       f"system (N={prob.N}) plus {len(dirs[:16])} JVP and {len(dirs[:16])} VJP solves, "
                       f"{dt:.1f} s; numpy/scipy FP64 with the BLAS threads of all {os.cpu_count()} cores")}


def oracle_lsmr_sample(prob, dirs, iters_per_solve, target_s=15.0):
    """A bounded sample of the oracle's matrix-free LSMR on this workload (dense
    LU does not fit): the seconds per iteration of scipy's LSMR on the JVP
    system (F and F^T products through scipy sparse matrices, FP64, one
    core), scaled to a solve of `iters_per_solve` iterations."""
    from oracle import derivative as D
    op = D.FOperator(prob)
    t0 = time.perf_counter()
    D.jvp_lsmr(prob, dirs[0], rtol=1e-30, maxiter=5, op=op)
    per = (time.perf_counter() - t0) / 5
    k = int(max(10, min(2000, target_s / max(per, 1e-6))))
    t0 = time.perf_counter()
    D.jvp_lsmr(prob, dirs[0], rtol=1e-30, maxiter=k, op=op)
    dt = time.perf_counter() - t0
    s_iter = dt / k
    return {"value": 1.0 / (s_iter * iters_per_solve), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": (f"{k} iterations of the oracle's matrix-free LSMR on the JVP system (N={prob.N}; scipy "
                       f"sparse F and F^T products, FP64, single-threaded) in {dt:.1f} s = {1e3 * s_iter:.1f} ms "
                       f"per iteration, scaled to {iters_per_solve:.0f} iterations per solve (the mean the GPU's "
                       f"equilibrated LSQR took); {os.cpu_count()} cores on the host")}


# --------------------------------------------------------------------------- learned form
def learned_bench(args, rank, local):
    """The learned preconditioner's family (the parametric family with a fixed
    pattern, n = 5000, m = 8000 times --scale, 0.1 by default): train on the
    method's own solves of --train instances (untimed), then time, on --held
    held-out instances, the adjoint solve of ||x*||^2 to rtol 1e-6 by
      plain       zero start, no scaling (the method of Sec. 3.1);
      c_alpha     zero start, the column scaling c^alpha the training chose
                  (the network's preconditioner target without the network);
      learned     network features + forward + decode, warm start and
                  diagonal preconditioner;
      best_plain  the fastest plain GPU form: the 16-sweep equilibration,
    all on engine auto (the cluster engine up to the full size).  value = learned
    solves/s; every row's rate and mean iterations ride along."""
    import torch
    import qcpgen as g
    import paper_2508_17522_gb300 as q
    from paper_2508_17522_gb300 import learned as L
    from paper_2508_17522_gb300.buildlib import build
    build()
    dev = torch.device("cuda", local)
    fam = g.config5_family(2 + 1000 * rank, scale=args.scale)
    train = [fam.instance(j) for j in range(args.train)]
    held = [fam.instance(1000 + j) for j in range(args.held)]
    t0 = time.time()
    lp = L.LearnedPreconditioner(seed=3, device=dev).fit(train, steps=800, lr=1e-3)
    log(f"learned: trained on {len(train)} instances (n={fam.n}) in {time.time() - t0:.1f} s")
    plans = [q.qcp_plan_create(q.problem_tensors(pr, dev), torch.float64) for pr in held]
    dirs = [L.adjoint_direction(pr) for pr in held]
    calpha = [(L.plan_scalings(pl)[1] ** lp.alpha).contiguous() for pl in plans]
    kinds = {
        "plain": lambda i: q.options(rtol=1e-6, engine="auto"),
        "c_alpha": lambda i: q.options(rtol=1e-6, engine="auto", precond="diag", precond_d=calpha[i]),
        "best_plain": lambda i: q.options(rtol=1e-6, engine="auto", precond="equilibrate"),
    }

    def run(kind):
        its, stat, eng = [], set(), set()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record()
        for i, (pl, pr, (wx, wy, ws)) in enumerate(zip(plans, held, dirs)):
            if kind == "learned":
                *_, info = lp.vjp(pl, pr, rtol=1e-6)
            else:
                *_, info = q.qcp_derivative_vjp(pl, wx, wy, ws, kinds[kind](i))
            its.append(info[0]["iters"])
            stat.add(info[0]["status"])
            eng.add(pl.last_engine())
        ev1.record()
        torch.cuda.synchronize(dev)
        return ev0.elapsed_time(ev1), its, stat, eng

    names = ["plain", "c_alpha", "learned", "best_plain"]
    for _ in range(max(args.warmup, 1)):
        for k in names:
            t, its_k, _, _ = run(k)
            log(f"learned: warm-up {k}: {t:.1f} ms, mean iterations {np.mean(its_k):.0f}")
    tot = {k: [0.0, [], set(), set()] for k in names}
    for _ in range(args.steps):
        for k in names:
            t, i, s_, e = run(k)
            tot[k][0] += t
            tot[k][1] += i
            tot[k][2] |= s_
            tot[k][3] |= e
    n = len(held) * args.steps
    rate = {k: n / (v[0] / 1e3) for k, v in tot.items()}
    rows = {k: {"solves_per_s": rate[k], "mean_iters": float(np.mean(v[1])), "status": sorted(v[2]),
                "engines": sorted(v[3])} for k, v in tot.items()}
    if rank == 0:
        print(json.dumps({
            "metric": "VJP solves/sec at 1e-6 rel residual, learned vs plain", "value": rate["learned"],
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot["learned"][0] / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (f"learned-preconditioner family n={fam.n} m={fam.m} (scale {args.scale} of "
                                    "n=5000 m=8000: 1 zero row, R+ blocks, one SOC of 25% of the rows, dense "
                                    f"P = F^T F + diag); {args.train} training and {args.held} held-out instances; "
                                    "VJP of ||x*||^2 at rtol 1e-6"),
                       "alpha": lp.alpha, "rows": rows,
                       "learned_over_plain": rate["learned"] / rate["plain"],
                       "learned_over_c_alpha": rate["learned"] / rate["c_alpha"],
                       "learned_over_best_plain": rate["learned"] / rate["best_plain"],
                       "training": f"{args.train} instances, 800 Adam steps on the GPU (untimed)"},
            "gpu_launches": None, "e2e": None, "roofline": None, "cpu_baseline": None}), flush=True)
    for pl in plans:
        pl.close()


# --------------------------------------------------------------------------- batched form
def config4_bench(args, rank, local):
    """The batched QCP form against the plain per-problem form on the same
    problems: the first --problems problems of the uneven batch (n ~ U[50,
    3000], m ~ U[1.5, 3] n, R+ and SOC blocks, dense P = G^T G + 1e-3 I), one
    JVP and one VJP direction each, rtol 1e-6, equilibration.
    Batched: one batch plan (autotuned for the VJP, untimed), per step one
    batched JVP and one batched VJP (engine auto).  Plain: one plan per
    problem, each autotuned for the VJP (untimed), per step each problem's
    JVP and VJP in turn on its own fastest engine.
    value = batched solves/s; the plain rate, their ratio and both
    rooflines (algorithmic bytes of every pass of every problem over the
    device time of the iteration launches) ride along."""
    import torch
    import qcpgen as g
    import paper_2508_17522_gb300 as q
    from paper_2508_17522_gb300.buildlib import build
    build()
    dev = torch.device("cuda", local)
    probs = g.config4(seed=rank, n_problems=args.problems)
    dirs = [g.make_directions(pr, 3) for pr in probs]
    cat = lambda nm: torch.as_tensor(np.concatenate([getattr(d, nm) for d in dirs]), device=dev)
    ins = {nm: cat(nm) for nm in ("dP", "dA", "dq", "db", "wx", "wy", "ws")}
    plan = q.qcp_batch_plan_create([q.problem_tensors(pr, dev) for pr in probs], torch.float64)
    plan.set_equilibration(args.equil_sweeps)
    best, _ = plan.autotune("vjp", iters=16, opts=q.options(precond="equilibrate"))
    opts = q.options(rtol=1e-6, maxiter=args.maxiter, precond="equilibrate", engine="auto")
    plans = []
    for pr in probs:  # each problem on its own fastest engine (autotuned, untimed)
        pl = q.qcp_plan_create(q.problem_tensors(pr, dev), torch.float64)
        pl.set_equilibration(args.equil_sweeps)
        pl.autotune("vjp", iters=16, opts=q.options(precond="equilibrate"))
        plans.append(pl)
    pins = [{nm: torch.as_tensor(getattr(d, nm), device=dev) for nm in ("dP", "dA", "dq", "db", "wx", "wy", "ws")}
            for d in dirs]
    bpp = [algorithmic_bytes_per_pass(pr) for pr in probs]
    acct = {"batched": [0.0, 0.0, [], set(), set()], "plain": [0.0, 0.0, [], set(), set()]}

    def record(kind, pl, info, which):
        ms, _ = pl.last_timing()
        a = acct[kind]
        a[0] += ms
        a[1] += sum(2 * i["iters"] * bpp[p] for p, i in zip(which, info))
        a[2] += [i["iters"] for i in info]
        a[3] |= {i["status"] for i in info}
        a[4].add(pl.last_engine())

    def step_batched():
        *_, ji = q.qcp_derivative_jvp(plan, ins["dP"], ins["dA"], ins["dq"], ins["db"], opts)
        record("batched", plan, ji, range(len(probs)))
        *_, vi = q.qcp_derivative_vjp(plan, ins["wx"], ins["wy"], ins["ws"], opts)
        record("batched", plan, vi, range(len(probs)))

    def step_plain():
        for p, (pl, d) in enumerate(zip(plans, pins)):
            *_, ji = q.qcp_derivative_jvp(pl, d["dP"], d["dA"], d["dq"], d["db"], opts)
            record("plain", pl, ji, [p])
            *_, vi = q.qcp_derivative_vjp(pl, d["wx"], d["wy"], d["ws"], opts)
            record("plain", pl, vi, [p])

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record()
        for _ in range(args.steps):
            fn()
        ev1.record()
        torch.cuda.synchronize(dev)
        return ev0.elapsed_time(ev1)

    for _ in range(args.warmup):
        step_batched()
        step_plain()
    for a in acct.values():
        a[:] = [0.0, 0.0, [], set(), set()]
    ms_b = timed(step_batched)
    ms_p = timed(step_plain)
    peak = (json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs")
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None) or 6800.0

    def roof(kind):
        a = acct[kind]
        gbs = a[1] / (a[0] / 1e3) / 1e9 if a[0] > 0 else None
        return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                "frac": gbs / peak if gbs else None, "traffic": None,
                "engines": sorted(a[4]), "iters_median": float(np.median(a[2])), "iters_max": int(max(a[2])),
                "status": sorted(a[3])}
    n_solves = 2 * len(probs) * args.steps
    vb, vp = n_solves / (ms_b / 1e3), n_solves / (ms_p / 1e3)
    if rank == 0:
        print(json.dumps({
            "metric": "JVP+VJP solves/sec at 1e-6 rel residual, batched vs plain", "value": vb,
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"uneven batch, problems 0..{len(probs) - 1} of 512 (n ~ U[50, 3000], dense P)",
                       "sum_n": int(sum(p.n for p in probs)), "sum_m": int(sum(p.m for p in probs)),
                       "nnz_up_P": int(sum(p.P.nnz for p in probs)), "autotuned": best,
                       "equil_sweeps": args.equil_sweeps,
                       "plain_solves_per_s": vp, "batched_over_plain": vb / vp,
                       "plain_ms_per_step": ms_p / args.steps},
            "roofline": roof("batched"), "roofline_plain": roof("plain"),
            "gpu_launches": None, "e2e": None, "cpu_baseline": None}), flush=True)
    for pl in plans:
        pl.close()
    plan.close()


# --------------------------------------------------------------------------- ranks
def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings over all ranks (the job
    takes as long as its slowest rank); identity without a process group."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_rate(solves_per_rank_step, world, steps, max_ms):
    """Solves per second of the whole job: every rank's solves over the
    slowest rank's time (replicas: each rank solves its own directions)."""
    return solves_per_rank_step * world * steps / (max_ms / 1e3)


# --------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precond", default="equilibrate", choices=["equilibrate", "none"])
    ap.add_argument("--workload", default="config3",
                    choices=["config1", "config2", "config3", "example", "cones", "learned", "config4"])
    ap.add_argument("--scale", type=float, default=0.1,
                    help="learned: size of the family relative to n=5000, m=8000 (1.0: the full size)")
    ap.add_argument("--train", type=int, default=40, help="learned: training instances")
    ap.add_argument("--held", type=int, default=8, help="learned: held-out instances timed")
    ap.add_argument("--problems", type=int, default=32,
                    help="config4: how many of the batch's problems (drawn from their own streams, from 0)")
    ap.add_argument("--engine", default="auto", choices=["auto", "cluster", "cluster_fp64", "passes", "persistent"])
    ap.add_argument("--maxiter", type=int, default=400000,
                    help="Krylov iteration cap (lower it only for profiling runs: solves then stop early)")
    ap.add_argument("--solver", default="lsqr", choices=["lsqr", "lsmr"],
                    help="Krylov solver: LSQR (default) or the paper's LSMR")
    ap.add_argument("--call", default="pair", choices=["pair", "separate"],
                    help="pair: the JVPs and VJPs in one qcp_derivative_jvp_vjp_multi call (side by side on the "
                         "cluster engine); separate: one _multi call per kind")
    ap.add_argument("--equil-sweeps", type=int, default=16,
                    help="sweeps of the row/column equilibration (plan setting; 16 is the plan's default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    metric = "JVP+VJP solves/sec at <=1e-6 rel err"

    if args.impl == "reference":
        if rank != 0:
            return
        if args.workload not in ("config1", "config2", "config3", "example", "cones"):
            raise SystemExit("the oracle reference arm covers config1, config2, config3, example and cones")
        prob, dirs, rtol, desc = workload(args.workload, 0)
        if dense_workload(args.workload):
            for _ in range(args.warmup):
                oracle_step(prob, dirs)
            t0 = time.perf_counter()
            solves = 0
            for _ in range(args.steps):
                solves += oracle_step(prob, dirs)
            dt = time.perf_counter() - t0
            val = solves / dt
            cores = os.cpu_count()
            sample = f"{args.steps} full step{'' if args.steps == 1 else 's'} of the dense-LU oracle on the host"
        else:
            # each step: a bounded sample of the matrix-free oracle, scaled to
            # the iterations a solve of this workload takes with 16
            # equilibration sweeps (measured on the GPU: about 2900)
            rec = None
            for _ in range(args.warmup + args.steps):
                rec = oracle_lsmr_sample(prob, dirs, CONFIG3_ITERS_PER_SOLVE, target_s=10.0)
            val, cores, sample = rec["value"], rec["cores"], rec["sample"]
            dt = 2 * len(dirs) * args.steps / val
        print(json.dumps({
            "impl": "reference", "metric": metric, "value": val, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "rtol": rtol},
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch
    torch.cuda.set_device(local)
    if args.workload == "learned":
        return learned_bench(args, rank, local)
    if args.workload == "config4":
        return config4_bench(args, rank, local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import paper_2508_17522_gb300 as q
    from paper_2508_17522_gb300.buildlib import build
    build()

    prob, dirs, rtol, desc = workload(args.workload, rank)
    k = len(dirs)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and dense_workload(args.workload):
        log("timing the CPU oracle sample ...")
        cpu = oracle_sample(prob, dirs)

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    plan = q.qcp_plan_create(q.problem_tensors(prob, dev), torch.float64, max_rhs=2 * k, stream=stream)
    plan.set_equilibration(args.equil_sweeps)
    opts = q.options(rtol=rtol, maxiter=args.maxiter, precond=args.precond, engine=args.engine, solver=args.solver)
    cat = lambda nm: np.concatenate([getattr(d, nm) for d in dirs])
    host = {nm: torch.as_tensor(cat(nm)).pin_memory() for nm in ("dP", "dA", "dq", "db", "wx", "wy", "ws")}
    with torch.cuda.stream(stream):
        devin = {nm: t.to(dev, non_blocking=True) for nm, t in host.items()}
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream.synchronize()

    launches = [0]
    pass_ms = [0.0]
    passes = [0]
    sys_passes = [0]  # sum over systems of the passes each ran (2 per LSQR iteration)
    shared = [0]  # system passes that shared a launch's read of M with another system's
    infos = []

    def account(info):
        launches[0] += plan.last_launches()
        ms, n_ = plan.last_timing()
        pass_ms[0] += ms
        passes[0] += n_
        sys_passes[0] += sum(2 * i["iters"] for i in info)
        shared[0] += plan.last_shared_passes()

    def step(inputs):
        if args.call == "pair":
            jout, vout, info = q.qcp_derivative_jvp_vjp_multi(
                plan, k, inputs["dP"], inputs["dA"], inputs["dq"], inputs["db"], k, inputs["wx"], inputs["wy"],
                inputs["ws"], opts)
            account(info)
            infos.append((info[:k], info[k:]))
            return list(jout) + list(vout)
        jout = q.qcp_derivative_jvp_multi(plan, k, inputs["dP"], inputs["dA"], inputs["dq"], inputs["db"], opts)
        account(jout[-1])
        vout = q.qcp_derivative_vjp_multi(plan, k, inputs["wx"], inputs["wy"], inputs["ws"], opts)
        account(vout[-1])
        infos.append((jout[-1], vout[-1]))
        return list(jout[:-1]) + list(vout[:-1])

    for _ in range(args.warmup):
        step(devin)
    torch.cuda.synchronize(dev)

    # ---- device-resident timed region (L2 flushed before every step)
    launches[0], pass_ms[0], passes[0], sys_passes[0], shared[0] = 0, 0.0, 0, 0, 0
    infos.clear()
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    total_ms = 0.0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        step(devin)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    dev_launches = launches[0]
    dev_pass_ms, dev_passes, dev_sys_passes, dev_shared = pass_ms[0], passes[0], sys_passes[0], shared[0]
    statuses = sorted({i["status"] for pair in infos for grp in pair for i in grp})
    max_res = max(i["rel_residual"] for pair in infos for grp in pair for i in grp)

    # ---- end to end through the public API with host buffers
    e2e_ms = 0.0
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = 0
    outs_host = None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ins = {nm: t.to(dev, non_blocking=True) for nm, t in host.items()}
        outs = step(ins)
        with torch.cuda.stream(stream):
            if outs_host is None:
                outs_host = [torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in outs]
                d2h = sum(o.numel() * o.element_size() for o in outs)
            for hdst, o in zip(outs_host, outs):
                hdst.copy_(o, non_blocking=True)
            e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)

    # ---- max over ranks
    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_ms], dist, dev)
    value = whole_job_rate(2 * k, world, args.steps, total_ms)
    e2e = whole_job_rate(2 * k, world, args.steps, e2e_ms)

    mean_iters = float(np.mean([i["iters"] for pair in infos for grp in pair for i in grp]))
    if rank == 0 and not args.no_cpu_baseline and not dense_workload(args.workload):
        log("timing a sample of the matrix-free CPU oracle ...")
        cpu = oracle_lsmr_sample(prob, dirs, mean_iters)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_note = "measured" if peak else "fallback"
    peak = peak or 6800.0
    engine = plan.last_engine()
    kkey = "stream_pair" if engine == "stream" and dev_shared > 0 else engine
    kname = KERNELS[kkey][0]
    # algorithmic bytes of every pass every system ran, over the device time
    # of the iteration launches
    bmat, bvec = algorithmic_bytes_split(prob)
    bsys = bmat + bvec
    alg_bytes = bsys * dev_sys_passes - bmat * dev_shared
    achieved = alg_bytes / (dev_pass_ms / 1e3) / 1e9
    avg_pass_s = (dev_pass_ms / 1e3) / max(dev_passes, 1)
    traffic = recorded_traffic(kkey, args.workload)

    if rank == 0:
        line = {
            "metric": metric, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "df64" if engine in ("cluster", "stream") else "f64",
            "data": "synthetic",
            "config": {"workload": desc, "rtol": rtol, "precond": args.precond, "equil_sweeps": args.equil_sweeps,
                       "solver": args.solver.upper(), "engine": engine,
                       "arithmetic": ("vectors in double-float (binary32 pairs), Krylov scalars f64, data f64"
                                      if engine in ("cluster", "stream") else "f64"),
                       "call": (f"qcp_derivative_jvp_vjp_multi ({k} JVP + {k} VJP systems in one call)"
                                if args.call == "pair" else "qcp_derivative_jvp_multi then qcp_derivative_vjp_multi"),
                       "mean_iters_per_solve": mean_iters,
                       "parallelism": f"replicas x{world}", "l2": "flushed before every timed step "
                       f"({L2_FLUSH_BYTES >> 20} MiB write)", "status": statuses,
                       "max_true_rel_residual": max_res},
            "roofline": {"bound": "hbm" if args.workload in ("config3", "config4") else "l2",
                         "bound_note": ("M and the vectors (about 145 MB per iteration) exceed the 129 MB L2"
                                        if args.workload in ("config3", "config4") else
                                        "the matrix is L2- and shared-memory-resident: the fraction is of algorithmic "
                                        "bytes over time, not of DRAM traffic"),
                         "kernel": kname, "achieved": achieved, "peak": peak,
                         "peak_source": peak_note, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "traffic_per": "system pass (dram read + write bytes, ncu)",
                         "per": "algorithmic bytes of all passes of all systems (one pass = one product with F "
                                "or F^T of one system; a pass that shared its launch's read of M with another "
                                "system's counts the vector part only) over the device time of the iteration "
                                "launches; a cluster-engine launch runs every pass of its systems",
                         "bytes_per_system_pass": bsys, "matrix_bytes_per_pass": bmat,
                         "system_passes": dev_sys_passes, "shared_passes": dev_shared,
                         "avg_pass_us": avg_pass_s * 1e6, "passes": dev_passes},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": dev_launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
