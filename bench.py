#!/usr/bin/env python3
"""Benchmark of the GB300 SVM trainer.

Default workload (the benchmark line): the covtype-shaped problem,
n = 581,012 training rows, d = 54 (10 dense N(0,1) columns and one-hot blocks
of 4 and 40 columns, 12 stored entries per row), labels from a random tanh
MLP (49% positive), RBF gamma = 0.1, C = 4, tau = 1e-3, plus 10,000 held-out
rows, trained in FP64 (the paper's arithmetic). All inputs are seeded
synthetic data (paper_1406_5161_gb300.synth); the paper's own datasets are
not used.

One step = one full training to the KKT tolerance through the C ABI
(svm_train: ingest, fused SMO steps with adaptive shrinking, gradient
reconstruction, threshold b) followed by the decision function on the 10,000
held-out rows (svm_decision). The metric is SMO iterations per second over
the timed steps; time-to-KKT is reported beside it, and, for the default
workload, the same solve in the mixed-precision pattern and the a9a-shaped
one-hot workload as extra fields.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload covtype|onehot|batch|serve|recon] [--precision fp64|mixed]

With N > 1 (launched by torch.distributed.run) every rank trains its own
replica (the solve does not shard); the value is the sum of all ranks'
iterations divided by the slowest rank's time. `--impl reference` times the
FP64 CPU oracle (plain SMO, no shrinking) on a bounded prefix of the same
workload on the host cores; only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import atexit
import hashlib
import json
import os
import statistics
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SMO iter/s"
UNIT = "iter/s"
WORKLOADS = {
    "covtype": ("covtype-shaped: n=581012, d=54 (10 dense + one-hot 4 + one-hot 40, 12 entries/row), "
                "C=4, gamma=0.1, tau=1e-3; train to KKT + decision on 10000 held-out rows"),
    "onehot": ("onehot_sparse (a9a-shaped): n=32561, d=123, 14 ones/row, C=1, gamma=0.05, "
               "tau=1e-3; train to KKT + decision on 10000 held-out rows"),
}
# fastest measured Table-3 policy per workload and precision
DEFAULT_POLICY = {("covtype", "fp64"): "Multi500", ("covtype", "mixed"): "Multi500",
                  ("onehot", "fp64"): "Multi5pc", ("onehot", "mixed"): "Multi5pc"}
DTYPE = {"fp64": "f64", "mixed": "mixed (bf16 values, f32 dots/exp, f64 f/step/b)"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="covtype", choices=["covtype", "onehot", "batch", "serve", "recon"],
                    help="covtype: the benchmark line (581,012 rows); onehot: the a9a-shaped "
                         "workload; batch: the one-vs-one x C x gamma grid (405 jobs) batched vs "
                         "one job at a time; serve: the served Poisson stream; recon: the "
                         "tensor-core contraction")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="covtype / onehot: FP64 throughout, or the mixed-precision pattern")
    ap.add_argument("--policy", default=None,
                    help="shrinking policy (Table 3); default: the fastest measured for the "
                         "workload and precision")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="reference arm: about how long its warm-up and timed steps take together")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra fields (other precision, the a9a-shaped workload)")
    ap.add_argument("--serve-jobs", type=int, default=100)
    ap.add_argument("--serve-nmax", type=int, default=10000)
    ap.add_argument("--serve-cluster", type=int, default=0, help="CTAs per served job (0 = server default)")
    ap.add_argument("--serve-burst", action="store_true",
                    help="submit every job at time 0 (saturated server) instead of the Poisson times")
    ap.add_argument("--plain-sample", type=int, default=0,
                    help="batch workload: jobs trained one at a time for the comparison "
                         "(0 = all 405; a smaller sample covers all 9 (C, gamma) cells of "
                         "evenly spaced pairs)")
    ap.add_argument("--wss2", action="store_true",
                    help="covtype / onehot: choose i_low by the second-order gain "
                         "(SVM_FLAG_WSS2) instead of the first-order rule")
    ap.add_argument("--cache-mb", type=int, default=0,
                    help="covtype / onehot: kernel-row cache budget in MiB (0 automatic, -1 off; "
                         "profiling of small cases)")
    ap.add_argument("--max-iter", type=int, default=0,
                    help="cap SMO steps per solve (profiling of small cases; not a bench value)")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clk", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200", "-f", self.path]
        if shutil.which("timeout"):
            cmd = ["timeout", "900"] + cmd   # never outlives a crashed run by much
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        if self.proc is not None:
            atexit.register(self._kill)

    def _kill(self):
        if self.proc is not None and self.proc.poll() is None:
            self.proc.kill()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- helpers
def job_totals(dist, seconds: float, units: float, device) -> tuple[float, float]:
    """Whole-job figures over replicas (one per rank, no data-path collective):
    the slowest rank's time and the sum of the units all ranks processed."""
    if dist is None:
        return seconds, units
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def _code_tokens(text: str) -> str:
    """C/C++ source without its comments and whitespace (string and character
    literals kept whole), so that the hash below changes with the code only."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            if not c.isspace():
                out.append(c)
            i += 1
    return "".join(out)


def kernel_source_hash(root: str = ROOT) -> str:
    """Hash of the fused step kernel's code (its sources without comments or
    whitespace): the committed ncu records carry it, and a record whose hash
    differs was taken on other code."""
    h = hashlib.sha256()
    for name in ("smo_step.cuh", "svm_internal.cuh", "fp64_math.cuh", "expfx_table.inc"):
        with open(os.path.join(root, "paper_1406_5161_gb300", "csrc", name), encoding="utf-8") as fh:
            h.update(_code_tokens(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, precision: str):
    """DRAM bytes per launch of the fused step kernel from the committed ncu
    summary of this workload, or None when there is none or the kernel source
    changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"smo_step_{workload}_{precision}_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_hash") != kernel_source_hash():
        return None
    return rec


def measured_issue(workload: str, precision: str):
    """Warp-instructions per row visit of the fused step on this workload's
    full-set level, from the committed ncu summary, or None when there is
    none or the kernel source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"smo_step_{workload}_{precision}_issue.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_hash") != kernel_source_hash():
        return None
    return rec


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def workload(name: str):
    from paper_1406_5161_gb300 import synth
    return synth.covtype_like() if name == "covtype" else synth.onehot_sparse()


def row_bytes(p, precision: str, binary: bool) -> tuple[float, float]:
    """Algorithmic bytes of the fused step: per active row visited, and per
    step for the two target rows. Per row: the CSR entries (column index, plus
    the value unless every value is 1.0), the row pointer, f read and write,
    the index set, and for non-binary rows the norm (FP64: 8 B per entry + 29,
    125 B at 12 entries; mixed precision with BF16 values and, for d < 2^16,
    16-bit columns: 4 B per entry + 29, 77 B, else 6 B per entry; binary: 4 B
    per entry + 25, 81 B at 14 entries)."""
    nnz_row = p.X.nnz / p.X.n
    if binary:
        per_entry, fixed = 4.0, 8 + 16 + 1
    elif precision == "fp64":
        per_entry, fixed = 8.0, 29
    else:
        per_entry, fixed = (4.0 if p.X.d < 65536 else 6.0), 29
    return per_entry * nnz_row + fixed, 2 * per_entry * nnz_row


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return 0
    import oracle
    name = args.workload if args.workload in WORKLOADS else "covtype"
    p = workload(name)
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    # SMO steps per timed step: a bounded prefix of the solve, sized so that
    # warm-up and timed steps together take about two minutes
    t0 = time.perf_counter()
    oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=50)
    per = (time.perf_counter() - t0) / 50
    m = int(max(50, min(15000, args.ref_seconds / max(1, args.steps + args.warmup) / max(per, 1e-6))))
    for _ in range(args.warmup):
        oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=m)
    t0 = time.perf_counter()
    iters = 0
    for _ in range(args.steps):
        r = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=m)
        iters += r["iters"]
    dt = time.perf_counter() - t0
    value = iters / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[name], "policy": "Original (oracle has no shrinking)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {m} SMO steps of the workload per step (FP64 oracle, "
                                       "Algorithm 1, no shrinking)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(p):
    """The oracle as it stands on the host cores, on a bounded prefix."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=100)
    per = (time.perf_counter() - t0) / 100
    m = int(max(100, min(15000, 12.0 / max(per, 1e-6))))
    t0 = time.perf_counter()
    r = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=m)
    dt = time.perf_counter() - t0
    # the single-thread form of the same oracle (bit-identical results), on a
    # shorter prefix
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=10)
    per1 = (time.perf_counter() - t0) / 10
    m1 = int(max(10, min(m, 4.0 / max(per1, 1e-6))))
    t0 = time.perf_counter()
    r1 = oracle.smo(p.X, p.y, p.C, p.gamma, p.tau, max_iter=m1)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    return {"value": r["iters"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {r['iters']} SMO steps of the same workload (FP64 oracle, no shrinking), "
                      f"{dt:.1f} s",
            "single_thread": {"value": r1["iters"] / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"first {r1['iters']} SMO steps, {dt1:.1f} s"}}


# ---------------------------------------------------------------- GPU arm
def solve_once(pkg, p, precision: str, policy_name: str, steps: int, warmup: int, flush, stream,
               with_decision: bool = True):
    """Untimed-by-contract extra: `steps` solves (after `warmup`) of another
    precision or workload, timed with CUDA events like the main line."""
    import torch
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    Zd = pkg.to_device(p.Z)
    prec = pkg.SVM_FP64 if precision == "fp64" else pkg.SVM_MIXED_BF16
    policy = pkg.POLICIES[policy_name]
    for _ in range(warmup):
        pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, shrink=policy, precision=prec, stream=stream)
    torch.cuda.synchronize()
    ms, iters, objs = [], 0, []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = pkg.svm_train(Xd, yd, p.C, p.gamma, p.tau, shrink=policy, precision=prec, stream=stream)
        if with_decision:
            pkg.svm_decision(Xd, yd, r["alpha"], r["b"], p.gamma, Zd, precision=prec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        iters += r["iters"]
        objs.append(r["stats"]["objective"])
    return {"value": iters / (sum(ms) / 1e3), "unit": UNIT, "time_to_kkt_ms": statistics.mean(ms),
            "iters_per_solve": iters / steps, "objective": objs[-1], "policy": policy_name,
            "steps": steps, "dtype": DTYPE[precision]}


def run_gb300(args, rank, world, local):
    import numpy as np
    import torch
    import paper_1406_5161_gb300 as pkg

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.load()
    p = workload(args.workload)
    policy = pkg.POLICIES[args.policy]
    prec = pkg.SVM_FP64 if args.precision == "fp64" else pkg.SVM_MIXED_BF16
    flags = pkg.SVM_FLAG_WSS2 if args.wss2 else 0
    Xd = pkg.to_device(p.X)
    yd = torch.as_tensor(p.y, device="cuda")
    Zd = pkg.to_device(p.Z)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def train(X, y, **kw):
        return pkg.svm_train(X, y, p.C, p.gamma, p.tau, shrink=policy, precision=prec,
                             max_iter=args.max_iter, flags=flags, cache_mb=args.cache_mb, **kw)

    for _ in range(max(args.warmup, 3)):
        r = train(Xd, yd, stream=stream)
        pkg.svm_decision(Xd, yd, r["alpha"], r["b"], p.gamma, Zd, precision=prec, stream=stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = pkg.svm_kernel_launches()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e2 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    iters = row_visits = 0
    ms_smo = ms_recon = 0.0
    stats = None
    for k in range(args.steps):
        flush.zero_()                    # L2 flushed between timed steps
        e0[k].record(stream)
        r = train(Xd, yd, stream=stream)
        e1[k].record(stream)
        pkg.svm_decision(Xd, yd, r["alpha"], r["b"], p.gamma, Zd, precision=prec, stream=stream)
        e2[k].record(stream)
        stats = r["stats"]
        iters += r["iters"]
        row_visits += stats["row_visits"]
        ms_smo += stats["ms_smo"]
        ms_recon += stats["ms_recon"]
    torch.cuda.synchronize()
    launches = pkg.svm_kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, c in zip(e0, e2)]
    kkt_ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    t_total, iters_all = job_totals(dist, sum(step_ms) / 1e3, float(iters), "cuda")
    value = iters_all / t_total

    # ---- end to end through the public API with host buffers
    e2e = None
    if rank == 0 or world > 1:
        from paper_1406_5161_gb300 import synth

        def pinned(a):
            t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
            t.numpy()[...] = a
            return t.numpy()

        def pinned_csr(X):
            return synth.CSR(X.n, X.d, pinned(X.indptr), pinned(X.indices), pinned(X.values))

        Xh, Zh, yh = pinned_csr(p.X), pinned_csr(p.Z), pinned(p.y)
        alpha_h = pinned(np.zeros(p.X.n))
        out_h = pinned(np.zeros(p.Z.n))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_iters = 0
        n_e2e = 1 if args.workload == "covtype" else max(1, min(3, args.steps))
        for _ in range(n_e2e):
            r = train(Xh, yh, alpha_out=alpha_h)
            pkg.svm_decision(Xh, yh, alpha_h, r["b"], p.gamma, Zh, precision=prec, out=out_h)
            e2e_iters += r["iters"]
        dt, e2e_all = job_totals(dist, time.perf_counter() - t0, float(e2e_iters), "cuda")
        nbytes = lambda X: X.indptr.nbytes + X.indices.nbytes + X.values.nbytes  # noqa: E731
        h2d = (nbytes(p.X) + p.y.nbytes) * 2 + 8 * p.X.n + nbytes(p.Z)
        d2h = 8 * p.X.n + 8 * p.Z.n
        e2e = {"value": e2e_all / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * dt / n_e2e}

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ---- roofline of the fused step kernel (algorithmic bytes / kernel time)
    b_row, b_targets = row_bytes(p, args.precision, bool(stats["binary_input"]))
    alg_bytes = row_visits * b_row + iters * b_targets
    achieved = alg_bytes / (ms_smo / 1e3) / 1e9
    peak, peak_kind = peaks()
    trec = measured_traffic(args.workload, args.precision)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": trec["dram_bytes_per_launch"] if trec else None,
                "kernel": "smo_persistent_kernel",
                "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                "bytes_per_row_visit": b_row, "row_visits_per_step": row_visits / args.steps,
                "kernel_ms_per_step": ms_smo / args.steps}
    if trec:
        roofline["traffic_launch"] = trec.get("launch")
        roofline["traffic_alg_bytes"] = trec.get("alg_bytes_per_launch")
    issue = None
    irec = measured_issue(args.workload, args.precision)
    if irec:
        # the FP64 row pass runs its inner products and exponentials on the
        # integer pipes (exact 128-bit sums, fixed-point exp), which leaves the
        # fused step bound by instruction issue and latency, not by the FP64
        # pipe or memory: warp-instructions executed (ncu, per row visit of
        # the full-set level) over the fused-step time, against one
        # instruction per clock per scheduler
        wpr = float(irec["warp_instr_per_row_visit"])
        ach = row_visits * wpr / (ms_smo / 1e3)
        peak_issue = 152 * 4 * 2.07e9
        issue = {"bound": "issue", "achieved": ach, "peak": peak_issue, "unit": "warp-instr/s",
                 "frac": ach / peak_issue, "warp_instr_per_row_visit": wpr,
                 "peak_source": "152 SMs x 4 schedulers x 1 warp-instruction per clock x 2.07 GHz",
                 "source": irec.get("source")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "policy": args.policy,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "n": int(p.X.n), "d": int(p.X.d), "held_out": int(p.Z.n)},
            "time_to_kkt_ms": statistics.mean(kkt_ms),
            "iters_per_solve": iters / args.steps,
            "recon_ms_per_step": ms_recon / args.steps,
            "objective": stats["objective"],
            "gpu_launches": int(launches),
            "clocks": clk, "roofline": roofline, "e2e": e2e}
    if issue:
        line["roofline_issue"] = issue
    if args.max_iter:
        line["config"]["max_iter"] = args.max_iter
    if args.cache_mb:
        line["config"]["cache_mb"] = args.cache_mb
    if args.wss2:
        line["config"]["selection"] = "second-order i_low (SVM_FLAG_WSS2)"
    if world == 1 and not args.no_extras and args.workload == "covtype" and not args.max_iter:
        other = "mixed" if args.precision == "fp64" else "fp64"
        line["extra_" + other] = solve_once(pkg, p, other, DEFAULT_POLICY[("covtype", other)], 1, 1,
                                            flush, stream)
        line["extra_onehot"] = dict(solve_once(pkg, workload("onehot"), "fp64",
                                               DEFAULT_POLICY[("onehot", "fp64")], 5, 3, flush, stream),
                                    workload=WORKLOADS["onehot"])
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p)
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """405 trainings (45 one-vs-one pairs x 3 C x 3 gamma) over one 50,000 x 256
    matrix: batched in one persistent launch vs one svm_train at a time."""
    import numpy as np
    import torch
    import paper_1406_5161_gb300 as pkg
    from paper_1406_5161_gb300 import synth

    torch.cuda.set_device(0)
    mc = synth.multiclass()
    jobs = []
    for a, b in mc.ovo_pairs():
        rows, y = mc.subproblem(a, b)
        for C in mc.Cs:
            for g in mc.gammas:
                jobs.append({"rows": rows.astype(np.int32), "y": y, "C": C, "gamma": g, "tau": mc.tau})
    Xd = pkg.to_device(mc.X)
    djobs = [dict(j, rows=torch.as_tensor(j["rows"], device="cuda"), y=torch.as_tensor(j["y"], device="cuda"))
             for j in jobs]
    prec = pkg.SVM_MIXED_BF16
    t0 = time.perf_counter()
    shape = pkg.svm_batch_autotune(Xd, djobs, precision=prec)
    tune_s = time.perf_counter() - t0
    # warm-up on a slice, then the timed full batch
    pkg.svm_train_batch(Xd, djobs[:20], precision=prec, **shape)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = pkg.svm_train_batch(Xd, djobs, precision=prec, **shape)
    torch.cuda.synchronize()
    batch_s = time.perf_counter() - t0
    # one job at a time on a sample: all 9 (C, gamma) cells of evenly spaced pairs
    npairs = len(mc.ovo_pairs())
    cells = len(mc.Cs) * len(mc.gammas)
    if args.plain_sample <= 0 or args.plain_sample >= len(jobs):
        idx = list(range(len(jobs)))
    else:
        take = max(1, args.plain_sample // cells)
        pairs = [round(k * (npairs - 1) / max(1, take - 1)) for k in range(take)] if take > 1 else [0]
        idx = [pp * cells + c for pp in pairs for c in range(cells)]
    subs = [(pkg.to_device(mc.X.take(jobs[i]["rows"])), torch.as_tensor(jobs[i]["y"], device="cuda")) for i in idx]
    pkg.svm_train(subs[0][0], subs[0][1], jobs[idx[0]]["C"], jobs[idx[0]]["gamma"], mc.tau, precision=prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = []
    for (Xs, ys), i in zip(subs, idx):
        plain.append(pkg.svm_train(Xs, ys, jobs[i]["C"], jobs[i]["gamma"], mc.tau, precision=prec))
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    rel = [abs(out["results"][i]["objective"] - r["stats"]["objective"]) / abs(r["stats"]["objective"])
           for i, r in zip(idx, plain)]
    batch_tps = len(jobs) / batch_s
    plain_tps = len(idx) / plain_s
    line = {"metric": "batched trains/s", "value": batch_tps, "unit": "trains/s",
            "workload": "multiclass 50000x256, 45 one-vs-one pairs x C{0.1,1,10} x gamma{0.002,0.01,0.05} = 405 jobs",
            "precision": "mixed (BF16 values, FP32 dots/exp, FP64 f/step/b)",
            "batched": {"trains_per_s": batch_tps, "seconds": batch_s, "iters_total": out["iters_total"],
                        "job_iters_per_s": out["iters_total"] / batch_s, "cluster_size": out["cluster_size"],
                        "lanes_per_row": out["lanes_per_row"], "clusters_in_flight": out["clusters"],
                        "autotune_s": tune_s, "not_converged": sum(r["status"] != 0 for r in out["results"])},
            "one_at_a_time": {"trains_per_s": plain_tps, "jobs": len(idx), "seconds": plain_s,
                              "batched_trains_per_s_same_jobs": len(idx) / (batch_s * sum(out["results"][i]["iters"] for i in idx) / max(1, out["iters_total"])),
                              "iters": int(sum(r["iters"] for r in plain)),
                              "job_iters_per_s": sum(r["iters"] for r in plain) / plain_s},
            "speedup_trains_per_s": batch_tps / plain_tps,
            "objective_rel_diff_max": max(rel),
            "objective_rel_diff_jobs": len(rel),
            "objective_rel_diff_over_1e-5": int(sum(x > 1e-5 for x in rel)),
            "pair_rows_min_max": [int(min(len(jobs[i]["rows"]) for i in idx)),
                                  int(max(len(jobs[i]["rows"]) for i in idx))]}
    print(json.dumps(line), flush=True)
    return 0


def run_recon(args):
    """The reconstruction / decision contraction on the tensor cores at the
    covtype shape (d = 54, 12 stored entries per row): out[q] = sum_k
    alpha_k y_k K(x_k, z_q) - b over 100,000 support vectors and 100,000
    query rows, mixed precision (BF16 values, FP32 accumulation and exp, FP64
    sums across tiles). Every row is a support vector. The timed call is the
    public svm_decision (SV compaction and BF16 densification included)."""
    import numpy as np
    import torch
    import paper_1406_5161_gb300 as pkg
    from paper_1406_5161_gb300 import synth

    torch.cuda.set_device(0)
    nsv = nq = 100_000
    p = synth.covtype_like(n=nsv, n_test=nq, seed=3)
    rng = np.random.default_rng(7)
    alpha = rng.uniform(0.01, p.C, nsv)
    Xd, Zd = pkg.to_device(p.X), pkg.to_device(p.Z)
    yd = torch.as_tensor(p.y, device="cuda")
    ad = torch.as_tensor(alpha, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def call():
        return pkg.svm_decision(Xd, yd, ad, 0.25, p.gamma, Zd, precision=pkg.SVM_MIXED_BF16, stream=stream)

    for _ in range(max(args.warmup, 3)):
        call()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = pkg.svm_kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        out = call()
        e1.record(stream)
    torch.cuda.synchronize()
    launches = pkg.svm_kernel_launches() - launches0
    clk = clocks.stop()
    ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
    d = p.X.d
    flops = 2.0 * nsv * nq * d                      # algorithmic: the inner products
    tflops = flops / (ms / 1e3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured bf16_tflops (burst cuBLAS)"
    except (OSError, ValueError, KeyError):
        peak, kind = 1900.0, "fallback"
    # the epilogue evaluates one exp2 per pair on the SFU: nominally 16 per
    # clock per SM; the library's microbenchmark measures the rate
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clk.get("sm_mhz") or 2070.0
    exp_nominal = 16.0 * sms * mhz * 1e6
    exp_measured = pkg.svm_diag_sfu_rate(stream=stream)
    pairs_s = nsv * nq / (ms / 1e3)
    line = {"metric": "RBF contraction TFLOP/s", "value": tflops, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"covtype-shaped contraction: {nsv} support vectors x {nq} queries, d={d}",
                       "l2": "flushed between timed calls (256 MiB write)"},
            "pairs_per_s": pairs_s, "gpu_launches": int(launches), "clocks": clk,
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "traffic": None, "kernel": "tc_rbf_kernel",
                         "peak_source": kind,
                         "note": "one exp2 per pair bounds the epilogue"},
            "sfu": {"ex2_per_s_measured": exp_measured, "ex2_per_s_nominal": exp_nominal,
                    "pairs_per_s": pairs_s, "frac_of_measured": pairs_s / exp_measured},
            "checksum": float(out.double().sum().item())}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """A Poisson stream (20 jobs/s) of training jobs of different n and d:
    served with continuous batching vs one svm_train at a time (FIFO)."""
    import numpy as np
    import torch
    import paper_1406_5161_gb300 as pkg
    from paper_1406_5161_gb300 import synth

    torch.cuda.set_device(0)
    specs = synth.serving_stream(n_jobs=args.serve_jobs)
    jobs = [synth.serving_job(sp, n=min(sp.n, args.serve_nmax)) for sp in specs]
    arrivals = np.array([sp.arrival_s for sp in specs])
    arrivals -= arrivals[0]
    if args.serve_burst:
        arrivals[:] = 0.0
    prec = pkg.SVM_MIXED_BF16
    # warm-up (library load, engine and kernels)
    with pkg.Server(budget_bytes=150 << 30, max_slots=64, precision=prec,
                    cluster_size=args.serve_cluster) as srv:
        srv.wait(srv.submit(jobs[0].X, jobs[0].y, jobs[0].C, jobs[0].gamma))
        t0 = time.perf_counter()
        tickets = []
        for p, at in zip(jobs, arrivals):
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            tickets.append(srv.submit(p.X, p.y, p.C, p.gamma, p.tau))
        outs = [srv.wait(t) for t in tickets]
        served_span = time.perf_counter() - t0
        info = srv.stats()
    ttm = np.array([o["time_to_model_ms"] for o in outs])
    ok = sum(o["status"] == pkg.SVM_OK for o in outs)
    # one at a time: the same stream through one svm_train after another
    pkg.svm_train(jobs[0].X, jobs[0].y, jobs[0].C, jobs[0].gamma, jobs[0].tau, precision=prec)
    dur = []
    objs = []
    for p in jobs:
        t = time.perf_counter()
        r = pkg.svm_train(p.X, p.y, p.C, p.gamma, p.tau, precision=prec)
        dur.append(time.perf_counter() - t)
        objs.append(r["stats"]["objective"])
    finish, ttm_plain = 0.0, []
    for at, du in zip(arrivals, dur):
        finish = max(finish, at) + du
        ttm_plain.append(1e3 * (finish - at))
    plain_span = finish
    rel = max(abs(o["objective"] - w) / abs(w) for o, w in zip(outs, objs))
    line = {"metric": "served trains/s", "value": len(jobs) / served_span, "unit": "trains/s",
            "workload": ("all jobs at t=0, " if args.serve_burst else "Poisson 20 jobs/s, ") +
                        f"{len(jobs)} jobs, n log-uniform [1e3, 2e5] capped at "
                        f"{args.serve_nmax}, d log-uniform [20, 2000], half dense / half CSR 0.5%",
            "precision": "mixed (BF16 values, FP32 dots/exp, FP64 f/step/b)",
            "served": {"trains_per_s": len(jobs) / served_span, "p50_ms": float(np.percentile(ttm, 50)),
                       "p99_ms": float(np.percentile(ttm, 99)), "span_s": served_span, "ok": ok,
                       "clusters": info["clusters"], "cluster_size": info["cluster_size"],
                       "engine_launches": info["engine_launches"]},
            "one_at_a_time": {"trains_per_s": len(jobs) / plain_span,
                              "p50_ms": float(np.percentile(ttm_plain, 50)),
                              "p99_ms": float(np.percentile(ttm_plain, 99)), "span_s": plain_span,
                              "busy_s": float(sum(dur))},
            "objective_rel_diff_max": rel}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.policy is None:
        args.policy = DEFAULT_POLICY.get((args.workload, args.precision), "Multi5pc")
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "recon":
        return run_recon(args)
    return run_gb300(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
