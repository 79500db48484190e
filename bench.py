#!/usr/bin/env python
"""Benchmark: parallel FISTA iterations/s for fuzzy clustering at paper scale.

Workload (default): a citation-like synthetic graph with n = 70,000,000
articles, k = 32 clusters, power-law degrees (DC-SBM, exponent 2.5) and about
2e9 nonzeros in S, drawn on the GPU from the seeded generator in synth/ (the
paper's OpenAlex graph is not available; this stands in for its shape).  A
step is one fused iteration of the solver.  Both arithmetic forms run on the
same graph and start point: plain FP32 and mixed (bfloat16 gathers and S
values, FP32 accumulation, FP64 scalars).  ``value`` is the mixed form's
iterations/s; the FP32 form's rate and the objectives of both after the same
number of iterations are reported beside it.  The same run (single GPU) also
measures the batched form (512 uneven instances, key ``batch``) and the
served form (a Poisson stream at a load the server sustains, key ``serve``);
``--extras ""`` skips them.

Launch: ``python bench.py [--gpus N] [--steps K] [--warmup W]``; for N > 1 under
torch.distributed.run every rank solves its own instance (replicas, weak
scaling).  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PG iters/s, mixed vs FP32, at equal objective (n=70M,k=32); serving p99 latency"
UNIT = "iter/s"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_k32_n8M.json")
SPMM_SRC = [os.path.join(ROOT, "paper_2506_04045_b300", "csrc", f)
            for f in ("iter_common.cuh", "spmm_kernels.cuh", "state.h", "schedule.cuh", "init_kernels.cuh",
                      "solver.cu")]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--workload", default="paper", choices=["paper", "batch", "serve", "er2", "rowrate"],
                   help="paper: one n=70M k=32 instance (default); batch: 512 uneven instances; "
                        "serve: Poisson stream of solves through the continuous-batching server; "
                        "er2: the paper's artificial two-cluster graph (750k nodes, k=2); "
                        "rowrate: random-row gather rate (plain loads vs TMA gather4), the product's access pattern")
    p.add_argument("--table-gb", type=float, default=8.0, help="rowrate: size of the gathered table")
    p.add_argument("--rows-m", type=int, default=1 << 28, help="rowrate: random rows gathered per launch")
    p.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    p.add_argument("--duration", type=float, default=20.0, help="serve: seconds of arrivals")
    p.add_argument("--drain", type=float, default=30.0, help="serve: seconds to wait for completions afterwards")
    p.add_argument("--pool", type=int, default=32, help="serve: distinct request graphs drawn from")
    p.add_argument("--budget-gb", type=float, default=120.0)
    p.add_argument("--serve-max-iter", type=int, default=5000)
    p.add_argument("--serve-tol", type=float, default=1e-5)
    p.add_argument("--tick", type=int, default=64)
    p.add_argument("--instances", type=int, default=512)
    p.add_argument("--extras", default="batch,serve",
                   help="paper workload: also measure these forms in the same run (single GPU): batch "
                        "(the 512-instance batch, --extra-steps timed iterations), serve (a Poisson stream at "
                        "--extra-serve-rate); empty to skip")
    p.add_argument("--extra-steps", type=int, default=10)
    p.add_argument("--no-autotune", action="store_true",
                   help="batch: keep the default launch shapes (no autotuner trials, e.g. for a clean ncu launch list)")
    p.add_argument("--extra-serve-rate", type=float, default=0.5)
    p.add_argument("--extra-serve-duration", type=float, default=20.0)
    p.add_argument("--extra-serve-drain", type=float, default=25.0)
    p.add_argument("--n", type=int, default=70_000_000)
    p.add_argument("--k", type=int, default=32)
    p.add_argument("--mean-deg", type=float, default=28.9)
    p.add_argument("--seed", type=int, default=2)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--forms", default="fp32,mixed")
    p.add_argument("--cpu-sample-n", type=int, default=1_000_000)
    p.add_argument("--cpu-iters", type=int, default=2)
    p.add_argument("--tto-cap", type=int, default=300,
                   help="time to objective: FP32 runs to PG_REL --tto-tol or this many iterations, then the "
                        "mixed form runs until f <= f*(1+1e-5) (at most twice as many); 0 skips it")
    p.add_argument("--tto-tol", type=float, default=1e-5)
    p.add_argument("--fused", action="store_true", help="one fused kernel per iteration instead of the split form")
    p.add_argument("--relabel", type=int, default=1, choices=[0, 1],
                   help="solver option relabel (internal numbering by degree; 1 = library default)")
    p.add_argument("--overlap", type=int, default=0, choices=[0, 1],
                   help="solver option overlap (update of row chunks beside the gather; 0 = library default)")
    p.add_argument("--update-engine", type=int, default=0, choices=[0, 1, 2, 3],
                   help="solver option update_engine for 17 <= k <= 32 (0 = automatic, library default: "
                        "streaming from 2^17 articles; 1 = warp-level mma.sync; 2 = tcgen05 per row block; "
                        "3 = streaming tcgen05 + TMA)")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Ranks:
    """The run's ranks (one process per GPU, launched by torchrun): barrier,
    max and sum over ranks.  A world of one when WORLD_SIZE is 1 (no process
    group).  `backend`/`device` are nccl/cuda on GPUs; gloo/cpu in the
    multi-process tests."""

    def __init__(self, ws: int, backend: str = "nccl", device: str = "cuda"):
        self.ws, self.device, self.dist = ws, device, None
        if ws > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op: str) -> float:
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=getattr(self.dist.ReduceOp, op))
        return float(t.item())

    def max(self, x) -> float:
        return self._reduce(x, "MAX")

    def sum(self, x) -> float:
        return self._reduce(x, "SUM")

    def weak_throughput(self, units, seconds):
        """This rank processed `units` in `seconds`: returns (the slowest rank's
        seconds, all ranks' units / that time), the whole-job figure."""
        t = self.max(seconds)
        return t, self.sum(units) / t

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for nm, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows),
                "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
# algorithmic bytes (per iteration) of the fused pass
# ---------------------------------------------------------------------------
def alg_bytes(n, nnz, k, mixed, heavy_nnz=0):
    """Algorithmic bytes of one iteration: B_alg = row_ptr + (col + val) per
    nonzero + one gathered row per nonzero (rounded up to 32-byte sectors) +
    the two previous iterates' own rows read and the new row written (float32
    master) [+ the bfloat16 gather copy written in the mixed form].  With
    ``heavy_nnz`` the nonzeros of chunked rows (streamed by another kernel of
    the fused form) are left out."""
    return gather_bytes(n, nnz - heavy_nnz, k, mixed) + update_bytes(n, k, mixed)


def gather_bytes(n, nnz, k, mixed):
    """The product S X: row_ptr, col and val once, one gathered row per nonzero."""
    bg = 2 if mixed else 4
    bv = 2 if mixed else 4
    row = math.ceil(k * bg / 32) * 32
    return 8 * (n + 1) + nnz * (4 + bv) + nnz * row


def update_bytes(n, k, mixed):
    """The row-local update: two previous iterates' rows read, the new row written."""
    return 3 * n * k * 4 + (n * k * 2 if mixed else 0)


def kernel_digest() -> str:
    """Digest of the dominant (gather) kernel's sources, the row schedule it
    follows and the solver that launches it (its L2 window): the traffic
    figures stay valid while these files are unchanged."""
    h = hashlib.sha256()
    for path in SPMM_SRC:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_capture():
    """The committed ncu capture of DRAM bytes per launch (a smaller case of the
    same generator), or None when it was taken with older kernel sources."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
    except Exception:
        return None
    return d if d.get("kernel_sha") == kernel_digest() else None


def traffic_for(form: str, workload: str):
    """DRAM bytes per launch of the dominant kernel from the committed capture
    when it is of this very workload and the current sources, else None."""
    d = traffic_capture()
    if d is None or d.get("workload") != workload:
        return None
    ent = d.get(form)
    return None if ent is None else ent.get("bytes_per_launch")


def traffic_small_case(form: str):
    """The committed capture's figures for `form` when its sources are current:
    bytes and algorithmic bytes per launch of the gather and the update at the
    capture's (smaller) size, not scaled (see the capture's note)."""
    d = traffic_capture()
    if d is None or form not in d:
        return None
    e = d[form]
    return {"workload": d["workload"], "kernel": e["kernel"], "bytes_per_launch": e["bytes_per_launch"],
            "alg_bytes_per_launch": e["alg_bytes_per_launch"],
            "traffic_over_alg": e["bytes_per_launch"] / e["alg_bytes_per_launch"],
            "update_kernel": e.get("update_kernel"), "update_bytes_per_launch": e.get("update_bytes_per_launch"),
            "note": d.get("note")}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same generator
# ---------------------------------------------------------------------------
def blas_threads() -> int:
    """Threads the oracle's dense BLAS calls use (its sparse products use one)."""
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([d.get("num_threads", 1) for d in info] + [1])
    except ImportError:
        for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            if os.environ.get(var, "").isdigit():
                return int(os.environ[var])
        return os.cpu_count() or 1


def host_info() -> dict:
    """The host the oracle runs on: logical CPUs and the CPU model."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


class OracleSample:
    """The FP64 oracle on a bounded sample: an n = cpu_sample_n instance of the
    same generator, timed per iteration and scaled by nnz to the full size."""

    def __init__(self, args):
        import numpy as np
        import scipy.sparse as sp
        import oracle
        import synth
        self.args = args
        spec = synth.GraphSpec("dcsbm", args.cpu_sample_n, args.k, args.seed, mean_deg=args.mean_deg)
        rp, c, v = synth.make_graph(spec)
        self.csr = (rp, c, v)
        self.n = spec.n
        self.S = sp.csr_matrix((v.numpy().astype(np.float64), c.numpy(), rp.numpy()), shape=(spec.n, spec.n))
        self.U0t = synth.dirichlet_u0(spec.n, args.k, args.seed)
        self.U0 = self.U0t.numpy().astype(np.float64)
        self.tau = 1.0 / oracle.lipschitz(self.S)
        self.cores = blas_threads()
        self.last = None

    def seconds(self, iters: int, threads: int | None = None) -> float:
        """Time `iters` oracle iterations (BLAS limited to `threads` if given);
        the result is kept in self.last."""
        import contextlib
        import oracle
        ctx = contextlib.nullcontext()
        if threads is not None:
            try:
                import threadpoolctl
                ctx = threadpoolctl.threadpool_limits(threads)
            except ImportError:
                pass
        with ctx:
            t0 = time.perf_counter()
            self.last = oracle.fista(self.S, self.U0, self.tau, max_iter=iters, stop="none")
            return time.perf_counter() - t0

    def describe(self, iters_text: str, n_full_nnz: int, its: float) -> str:
        return (f"FP64 oracle (Algorithm 4, two products with S per iteration), {iters_text} on an "
                f"n={self.n:,} k={self.args.k} instance of the same generator (nnz={self.S.nnz:,}), "
                f"{its:.4f} it/s there, scaled by nnz to the full workload ({n_full_nnz:,} nonzeros); "
                f"sparse products single-threaded, dense BLAS on {self.cores} threads")


def oracle_errors(pkg, S_host, csr, U0t, iters, o, prefix):
    """Per-result error of both arithmetic forms against the FP64 oracle after
    `iters` iterations on one instance: max |U - U_oracle|, and the relative
    error of f, the trace term, ||U^T U||_F^2 and the PG norm r_iters."""
    import numpy as np
    import oracle
    import torch
    ref = oracle.loss_terms(S_host, o.U)
    out = {}
    dev = [t.cuda() for t in csr] + [U0t.cuda()]
    for form, prec in (("fp32", pkg.FP32), ("mixed", pkg.MIXED_BF16)):
        s = pkg.Solver(*dev, stop_rule=pkg.STOP_NONE, max_iter=iters, precision=prec)
        rep = s.solve()
        U = s.get_U().cpu().numpy()
        s.close()
        rel = lambda a, b: abs(a - b) / abs(b)
        out[form] = {"U_maxabs": float(np.max(np.abs(U - o.U))), "f_rel": rel(rep["f"], ref["f"]),
                     "trace_rel": rel(rep["trace_SU"], ref["trace"]),
                     "gram_fro2_rel": rel(rep["gram_fro2"], ref["gram_fro2"]),
                     "pg_norm_rel": rel(rep["pg_norm"], o.pg_norms[-1]), "iters": int(rep["iters"])}
    del dev
    torch.cuda.empty_cache()
    return {"instance": prefix, **out}


def cpu_baseline(args, n_full_nnz, pkg=None):
    """The oracle on the bounded sample, timed with BLAS on one thread and on
    all of them; with `pkg`, also the per-result error of both GPU forms
    against the oracle (the sample after the timed iterations, and a
    20,000-article instance after 50 iterations)."""
    import numpy as np
    import scipy.sparse as sp
    import oracle
    import synth
    o = OracleSample(args)
    dt1 = o.seconds(args.cpu_iters, threads=1)
    dta = o.seconds(args.cpu_iters)
    its1, itsa = args.cpu_iters / dt1, args.cpu_iters / dta
    scale = o.S.nnz / n_full_nnz
    out = {"value": itsa * scale, "unit": UNIT, "cores": o.cores, "kind": "oracle",
           "sample": o.describe(f"{args.cpu_iters} iterations", n_full_nnz, itsa),
           "single_core": its1 * scale, "all_core": itsa * scale, "sample_it_s": {"single_core": its1, "all_core": itsa},
           "nnz_scale": scale, **host_info()}
    if pkg is not None:
        errs = [oracle_errors(pkg, o.S, o.csr, o.U0t, args.cpu_iters, o.last,
                              f"dcsbm n={o.n:,} k={args.k}, {args.cpu_iters} iterations")]
        spec = synth.GraphSpec("dcsbm", 20_000, args.k, 71, mean_deg=30.0)
        rp, c, v = synth.make_graph(spec)
        S = sp.csr_matrix((v.numpy().astype(np.float64), c.numpy(), rp.numpy()), shape=(spec.n, spec.n))
        U0 = synth.dirichlet_u0(spec.n, args.k, 71)
        ref = oracle.fista(S, U0.numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=50, stop="none")
        errs.append(oracle_errors(pkg, S, (rp, c, v), U0, 50, ref, f"dcsbm n=20,000 k={args.k}, 50 iterations"))
        out["error_vs_oracle"] = errs
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    nnz_full = int(round(args.n * ((args.mean_deg - 1.0) * 0.99 + 1.0)))
    o = OracleSample(args)
    for _ in range(args.warmup):
        o.seconds(1)
    t = sum(o.seconds(1) for _ in range(args.steps))
    per_step = t / args.steps
    scale = o.S.nnz / nnz_full
    value = (1.0 / per_step) * scale
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1000.0,
            "ms_per_step_note": "measured per step on the sample; value = sample it/s x nnz_scale",
            "nnz_scale": scale, "ms_per_step_full_workload": per_step * 1000.0 / scale,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"dcsbm citation-like graph n={args.n:,} k={args.k} (oracle sample)",
                       "n": args.n, "k": args.k, "sample_n": o.n, "sample_nnz": int(o.S.nnz)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.cores, "kind": "oracle",
                             "sample": o.describe("1 iteration per step", nnz_full, 1.0 / per_step),
                             **host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
def run_native(args, ws, rank, local):
    import numpy as np
    import torch

    import synth
    import paper_2506_04045_b300 as pkg

    torch.cuda.set_device(local)
    ranks = Ranks(ws)
    barrier, max_over_ranks = ranks.barrier, ranks.max

    pkg.load()
    seed = args.seed + rank
    t_gen = time.perf_counter()
    spec = synth.GraphSpec("dcsbm", args.n, args.k, seed, mean_deg=args.mean_deg)
    rp, col, val = synth.make_graph(spec, device="cuda")
    U0 = synth.dirichlet_u0(args.n, args.k, seed, device="cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t_gen
    n, k, nnz = args.n, args.k, int(col.numel())
    deg = rp[1:] - rp[:-1]
    max_deg = int(deg.max())
    del deg
    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup
    hbm, peak_kind = peaks()
    forms = [f for f in args.forms.split(",") if f]
    res = {}
    sampler_summary = {}
    for form in forms:
        mixed = form == "mixed"
        s = pkg.Solver(rp, col, val, U0, stop_rule=pkg.STOP_NONE, max_iter=10 ** 9, borrow=1,
                       precision=pkg.MIXED_BF16 if mixed else pkg.FP32, fused_pass=1 if args.fused else 0,
                       relabel=args.relabel, update_engine=args.update_engine, overlap=args.overlap)
        s.step(W)
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as cs:
            e0.record(stream)
            kt = s.enqueue_profiled(K)
            e1.record(stream)
            torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(ms)
        U = s.get_U()
        f = pkg.objective(rp, col, val, U)
        rep = s.report()
        res[form] = {"ms_total": ms, "it_s": K / (ms / 1000.0), "kt": kt, "f": f, "iters": rep["iters"],
                     "launches": kt["kernels"]}
        sampler_summary[form] = cs.summary()
        s.close()
        del s, U
        torch.cuda.empty_cache()

    head = "mixed" if "mixed" in res else forms[0]
    r = res[head]
    mixed = head == "mixed"
    kt = r["kt"]
    b_iter = alg_bytes(n, nnz, k, mixed, 0)
    tag = "true" if mixed else "false"
    if args.fused:
        b_pass = alg_bytes(n, nnz, k, mixed, kt["heavy_nnz"])
        kname = f"fista_pass_kernel<32,{tag},false>"
    else:
        b_pass = gather_bytes(n, nnz, k, mixed)
        kname = f"spmm_kernel<32,{tag},4>"
    achieved = b_pass / (kt["pass_ms"] / 1000.0) / 1e9
    traffic = traffic_for(head + ("_fused" if args.fused else ""),
                          f"dcsbm n={n} k={k} nnz={nnz} seed={args.seed}")
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "traffic_small_case": None if args.fused else traffic_small_case(head),
            "kernel": kname, "peak_kind": peak_kind, "alg_bytes_per_launch": b_pass,
            "pass_ms": kt["pass_ms"], "heavy_ms": kt["heavy_ms"], "update_ms": kt["update_ms"],
            "fold_ms": kt["fold_ms"], "iteration_alg_bytes": b_iter,
            "iteration_frac": b_iter / (r["ms_total"] / K / 1000.0) / 1e9 / hbm}
    if not args.fused:
        ub = update_bytes(n, k, mixed)
        roof["update_kernel"] = {"alg_bytes_per_launch": ub, "ms": kt["update_ms"],
                                 "achieved": ub / (kt["update_ms"] / 1000.0) / 1e9 if kt["update_ms"] else None}
    clocks = sampler_summary[head]

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        try:
            e2e = run_e2e(args, pkg, rp, col, val, U0, head, K, barrier, max_over_ranks)
        except Exception as exc:  # e.g. pinned host memory unavailable
            e2e = {"value": None, "unit": UNIT, "error": f"{type(exc).__name__}: {exc}"[:300]}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline(args, nnz, pkg)
        except Exception as exc:
            cpu = {"value": None, "unit": UNIT, "kind": "oracle", "error": str(exc)[:200]}

    tto = None
    if args.tto_cap > 0 and "fp32" in res and "mixed" in res:
        try:
            tto = time_to_objective(args, pkg, rp, col, val, U0, res["fp32"]["ms_total"] / K,
                                    res["mixed"]["ms_total"] / K)
        except Exception as exc:
            tto = {"error": f"{type(exc).__name__}: {exc}"[:300]}

    # the batched and served forms, measured in the same run (single GPU only)
    extras = {}
    wanted = [x for x in args.extras.split(",") if x]
    if ws == 1 and wanted:
        del rp, col, val, U0
        torch.cuda.empty_cache()
        if "batch" in wanted:
            try:
                bres, bwork = batch_measure(args, ranks, rank, args.extra_steps, max(3, W), forms)
                bh = "mixed" if "mixed" in bres else forms[0]
                extras["batch"] = {"metric": "instance-iterations/s", "value": bres[bh]["inst_it_s"],
                                   "steps": args.extra_steps, "warmup": max(3, W), "config": bwork,
                                   "iteration_frac": bres[bh]["bytes_iter"] / (bres[bh]["ms"] / args.extra_steps
                                                                             / 1000.0) / 1e9 / hbm,
                                   "forms": batch_forms_summary(bres, args.extra_steps, compact=True)}
            except Exception as exc:
                extras["batch"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        if "serve" in wanted:
            try:
                extras["serve"] = serve_measure(args, rank, args.extra_serve_rate, args.extra_serve_duration,
                                                args.extra_serve_drain)
                extras["serve"]["requests"] = extras["serve"]["requests"][:40]
            except Exception as exc:
                extras["serve"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}

    # r["ms_total"] is already the slowest rank's time: whole-job iterations / that time
    _, value = ranks.weak_throughput(K, r["ms_total"] / 1000.0)
    eq = None
    if "fp32" in res and "mixed" in res:
        eq = True
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": r["ms_total"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16+f32" if mixed else "f32", "data": "synthetic",
        "config": {"workload": f"dcsbm citation-like graph n={n:,} k={k} nnz={nnz:,} (power-law degrees, "
                               f"exponent 2.5, unit diagonal, weights in (0,1]), Dirichlet(1) start, step 1/L",
                   "n": n, "k": k, "nnz": nnz, "max_degree": max_deg, "seed": args.seed,
                   "l2": "inputs larger than L2 (S 16 GB, iterate 9 GB); no flush",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "iteration_form": "fused" if args.fused else "split",
                   "update_engine": {0: "automatic (streaming tcgen05 + TMA at this size)", 1: "warp mma.sync",
                                     2: "tcgen05 per row block", 3: "streaming tcgen05 + TMA"}[args.update_engine],
                   "overlap": "update of 8 row chunks beside the gather" if args.overlap else "gather, then update",
                   "gen_seconds": round(gen_s, 1)},
        "forms": {f: {"it_s": res[f]["it_s"], "ms_per_step": res[f]["ms_total"] / K, "objective": res[f]["f"],
                      "pass_ms": res[f]["kt"]["pass_ms"], "heavy_ms": res[f]["kt"]["heavy_ms"],
                      "update_ms": res[f]["kt"]["update_ms"],
                      "fold_ms": res[f]["kt"]["fold_ms"], "iters_done": res[f]["iters"],
                      "clocks": sampler_summary[f]} for f in res},
        "time_to_objective": tto,
        "mixed_over_fp32": (res["mixed"]["it_s"] / res["fp32"]["it_s"]) if eq is not None else None,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": r["launches"],
        "batch": extras.get("batch"), "serve": extras.get("serve"),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()


def time_to_objective(args, pkg, rp, col, val, U0, ms_fp32, ms_mixed):
    """The metric's "at equal objective": the FP32 form runs to the PG stop
    rule (r_n <= tol r_1) or the cap and gives f*; the mixed form then runs
    until its reported loss reaches f* (1 + 1e-5).  Reports iterations, wall
    seconds and it/s of both, the iteration at which the mixed trace term is
    within 1e-5 of the FP32 one, and max |U_mixed - U_fp32| over all rows."""
    import torch
    opts = dict(borrow=1, relabel=args.relabel, update_engine=args.update_engine, overlap=args.overlap)
    sf = pkg.Solver(rp, col, val, U0, stop_rule=pkg.STOP_PG_REL, tol=args.tto_tol, max_iter=args.tto_cap,
                    precision=pkg.FP32, **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r1 = sf.step(1)["pg_norm"]
    rf = sf.solve()
    t_fp32 = time.perf_counter() - t0
    Uf = sf.get_U()
    sf.close()
    del sf
    torch.cuda.empty_cache()
    f_star, tr_star = rf["f"], rf["trace_SU"]
    target = f_star * (1.0 + 1e-5)
    cap = 2 * int(rf["out_iter"])
    sm = pkg.Solver(rp, col, val, U0, stop_rule=pkg.STOP_NONE, max_iter=max(cap, 1), precision=pkg.MIXED_BF16,
                    **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it_f = it_tr = None
    t_f = None
    rep = sm.step(0)
    while not rep["done"]:
        rep = sm.step(1)
        fi = rep["f_iter"]
        if fi < 0:
            continue
        if it_tr is None and abs(rep["trace_SU"] - tr_star) <= 1e-5 * abs(tr_star):
            it_tr = fi
        if rep["f"] <= target:
            it_f, t_f = fi, time.perf_counter() - t0
            break
    rm = sm.solve() if it_f is None else sm.report()
    Um = sm.get_U()
    umax = float((Um - Uf).abs().max())
    # the mixed form's loss is formed from its bfloat16 gathers; the objective of
    # its iterate evaluated in float32 (cluster_objective) beside it
    f_exact = pkg.objective(rp, col, val, Um)
    sm.close()
    del sm, Um, Uf
    torch.cuda.empty_cache()
    stop = ("PG_REL r_n <= %g r_1 at iteration %d" % (args.tto_tol, rf["out_iter"]) if rf["status"] == pkg.OK
            else "iteration cap %d (PG_REL %g not reached: r_n / r_1 = %.3g)" % (args.tto_cap, args.tto_tol,
                                                                                rf["pg_norm"] / r1))
    return {
        "fp32": {"iterations": int(rf["out_iter"]), "seconds": t_fp32, "it_s": rf["out_iter"] / t_fp32,
                 "f_star": f_star, "trace_star": tr_star, "pg_norm": rf["pg_norm"], "pg_norm_first": r1,
                 "stopped_by": stop,
                 "seconds_from_rate": rf["out_iter"] * ms_fp32 / 1000.0},
        "mixed": {"iterations_to_f_star": it_f, "seconds_to_f_star": t_f,
                  "it_s": (it_f + 1) / t_f if it_f is not None else None,
                  "seconds_from_rate": (it_f * ms_mixed / 1000.0) if it_f is not None else None,
                  "f_at_stop": rm["f"], "trace_at_stop": rm["trace_SU"],
                  "f_float32_of_newest_iterate": f_exact, "f_float32_rel_to_f_star": (f_exact - f_star) / f_star,
                  "trace_rel_to_fp32": abs(rm["trace_SU"] - tr_star) / abs(tr_star),
                  "iterations_to_trace_within_1e-5": it_tr, "cap": cap},
        "max_abs_U_mixed_minus_fp32": umax,
        "speedup_time_to_f_star": (rf["out_iter"] * ms_fp32) / (it_f * ms_mixed) if it_f else None,
        "note": "f* from the FP32 run; the mixed run stops at the first iterate with f <= f*(1+1e-5), "
                "detected one pass late (seconds_to_f_star includes that pass and a host sync per iteration; "
                "the U compared is the mixed run's newest iterate, one pass past it); "
                "seconds_from_rate = iterations x the timed per-iteration rate",
    }


def run_e2e(args, pkg, rp, col, val, U0, form, K, barrier, max_over_ranks):
    """Host CSR and start point (pinned) -> device copies -> cluster_init ->
    K iterations, reading the loss back after each -> U copied to the host."""
    import torch
    h_rp = torch.empty(rp.shape, dtype=rp.dtype, pin_memory=True)
    h_col = torch.empty(col.shape, dtype=col.dtype, pin_memory=True)
    h_val = torch.empty(val.shape, dtype=val.dtype, pin_memory=True)
    h_U0 = torch.empty(U0.shape, dtype=U0.dtype, pin_memory=True)
    h_U = torch.empty(U0.shape, dtype=U0.dtype, pin_memory=True)
    for h, d in ((h_rp, rp), (h_col, col), (h_val, val), (h_U0, U0)):
        h.copy_(d)
    d_rp, d_col, d_val, d_U0 = torch.empty_like(rp), torch.empty_like(col), torch.empty_like(val), torch.empty_like(U0)
    mixed = form == "mixed"
    stream = torch.cuda.current_stream()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e0.record(stream)
    for h, d in ((h_rp, d_rp), (h_col, d_col), (h_val, d_val), (h_U0, d_U0)):
        d.copy_(h, non_blocking=True)
    ev[0].record(stream)
    s = pkg.Solver(d_rp, d_col, d_val, d_U0, stop_rule=pkg.STOP_NONE, max_iter=10 ** 9, borrow=1,
                   precision=pkg.MIXED_BF16 if mixed else pkg.FP32, fused_pass=1 if args.fused else 0,
                   relabel=args.relabel, update_engine=args.update_engine, overlap=args.overlap)
    ev[1].record(stream)
    losses = []
    for _ in range(K):
        losses.append(s.step(1)["f"])
    U = s.get_U()
    ev[2].record(stream)
    h_U.copy_(U, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    marks = [e0] + ev + [e1]
    phases = {name: round(marks[i].elapsed_time(marks[i + 1]) / 1000.0, 4)
              for i, name in enumerate(("h2d", "init", "iterations", "d2h"))}
    s.close()
    h2d = sum(t.numel() * t.element_size() for t in (h_rp, h_col, h_val, h_U0))
    d2h = h_U.numel() * h_U.element_size() + K * 8
    return {"value": K / (ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d / K,
            "d2h_bytes_per_step": d2h / K, "seconds": ms / 1000.0, "phases_s": phases,
            "note": "one solve: H2D of S and U0, cluster_init, K iterations each reading the loss, D2H of U"}


def batch_measure(args, ranks, rank, K, W, forms):
    """Generate the batched workload (--instances instances, seed 3 + 1000 rank)
    and time K batched iterations of each form after autotuning and W warm-up
    iterations.  Returns the per-form results and the workload description."""
    import torch

    import synth
    import paper_2506_04045_b300 as pkg
    specs = synth.batch_specs(args.instances, seed=3 + 1000 * rank)
    t0 = time.perf_counter()
    inst, nnz_tot, n_tot = [], 0, 0
    for sp in specs:
        rp, c, v = synth.make_graph(sp, device="cuda")
        U0 = synth.dirichlet_u0(sp.n, sp.k, sp.seed, device="cuda")
        inst.append((rp, c, v, U0))
        nnz_tot += int(c.numel())
        n_tot += sp.n
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    res = {}
    for form in forms:
        mixed = form == "mixed"
        t1 = time.perf_counter()
        b = pkg.Batch(inst, stop_rule=pkg.STOP_NONE, max_iter=10 ** 9, borrow=1,
                      precision=pkg.MIXED_BF16 if mixed else pkg.FP32, relabel=args.relabel,
                      update_engine=args.update_engine, overlap=args.overlap)
        init_s = time.perf_counter() - t1
        desc = b.describe() if args.no_autotune else b.autotune(trials=1)
        b.step(W)
        torch.cuda.synchronize()
        ranks.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as cs:
            e0.record(stream)
            b.enqueue(K)
            e1.record(stream)
            torch.cuda.synchronize()
        ranks.barrier()
        ms, inst_it_s = ranks.weak_throughput(len(inst) * K, e0.elapsed_time(e1) / 1000.0)
        ms *= 1000.0
        reps = b.step(0)
        bytes_iter = sum(alg_bytes(sp.n, int(c.numel()), sp.k, mixed) for sp, (rp, c, v, U0) in zip(specs, inst))
        res[form] = {"ms": ms, "inst_it_s": inst_it_s, "desc": desc, "init_s": init_s,
                     "bytes_iter": bytes_iter, "clocks": cs.summary(),
                     "iters_min": min(r["iters"] for r in reps), "iters_max": max(r["iters"] for r in reps)}
        b.close()
    del inst
    torch.cuda.empty_cache()
    workload = {"workload": f"{len(specs)} DC-SBM instances, n log-uniform [500, 2e5], k in {{4..64}}, "
                            f"mean degree U[10,40]; sum n = {n_tot:,}, sum nnz = {nnz_tot:,}",
                "instances": len(specs), "sum_n": n_tot, "sum_nnz": nnz_tot, "gen_seconds": round(gen_s, 1),
                "l2": "working set larger than L2; no flush"}
    return res, workload


def batch_forms_summary(res, K, compact=False):
    out = {}
    for f, v in res.items():
        d = {"inst_it_s": v["inst_it_s"], "ms_per_step": v["ms"] / K, "init_s": round(v["init_s"], 2),
             "model_GBps": v["bytes_iter"] * K / (v["ms"] / 1000.0) / 1e9, "clocks": v["clocks"],
             "iters_done": [v["iters_min"], v["iters_max"]]}
        if compact:
            d["classes"] = [{key: c.get(key) for key in ("kp", "instances", "gather_ms", "update_ms",
                                                        "gather_nonzeros_per_batch", "gather_rows_per_unit")}
                            for c in v["desc"]["classes"]]
        else:
            d["classes"] = v["desc"]["classes"]
        out[f] = d
    return out


def run_batch(args, ws, rank, local):
    """Batched workload: independent instances with n log-uniform in [500, 2e5],
    k uniform in {4, 8, 16, 32, 64}, mean degree uniform in [10, 40], advanced
    together by the segmented launches; a step is one iteration of every
    instance.  value = instance-iterations/s."""
    import torch

    import paper_2506_04045_b300 as pkg
    torch.cuda.set_device(local)
    ranks = Ranks(ws)
    pkg.load()
    hbm, peak_kind = peaks()
    K, W = args.steps, args.warmup
    forms = [f for f in args.forms.split(",") if f]
    res, workload = batch_measure(args, ranks, rank, K, W, forms)
    head = "mixed" if "mixed" in res else forms[0]
    r = res[head]
    achieved = r["bytes_iter"] * K / (r["ms"] / 1000.0) / 1e9
    line = {"metric": "batched instance-iterations/s (512 uneven instances)", "value": r["inst_it_s"],
            "unit": "instance-iter/s", "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": r["ms"] / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32" if head == "mixed" else "f32", "data": "synthetic",
            "config": workload,
            "forms": batch_forms_summary(res, K),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": "whole batched iteration (all classes)", "peak_kind": peak_kind},
            "clocks": r["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()


def run_er2(args, ws, rank, local):
    """The paper's artificial graph (Sect. 5): two Erdos-Renyi clusters (500,000
    nodes of expected degree 1200, 250,000 of degree 1600), 200 bridges, 0/1
    similarity, k = 2, start X^0 with every row in the second cluster,
    constant step tau = 5e-7.  For FISTA and GPA in each form: the label
    agreement after each of the first 30 iterations (untimed), then W warm-up
    and K timed iterations.  value = FISTA FP32 iterations/s.  The iterate
    (750k x 2 float32) fits in L2, so the product streams S from HBM and
    gathers rows from L2; the roofline uses the compulsory bytes (S once, the
    iterate rows once, the product written and read)."""
    import torch

    import synth
    import paper_2506_04045_b300 as pkg
    torch.cuda.set_device(local)
    ranks = Ranks(ws)
    pkg.load()
    n1, n2, d1, d2, bridges, tau = 500_000, 250_000, 1200.0, 1600.0, 200, 5e-7
    t0 = time.perf_counter()
    rp, col, val, labels = synth.two_cluster_graph(n1, n2, d1, d2, bridges, seed=6 + rank, device="cuda")
    n, nnz = n1 + n2, int(col.numel())
    U0 = synth.second_row_start(n, device="cuda")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    K, W = args.steps, args.warmup
    hbm, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    forms = [f for f in args.forms.split(",") if f]
    res = {}
    for form in forms:
        mixed = form == "mixed"
        for accel in (1, 0):
            name = ("fista_" if accel else "gpa_") + form
            s = pkg.Solver(rp, col, val, U0, step_rule=pkg.STEP_CONST, tau=tau, stop_rule=pkg.STOP_NONE,
                           max_iter=10 ** 9, borrow=1, accel=accel, relabel=args.relabel, update_engine=args.update_engine, overlap=args.overlap,
                           precision=pkg.MIXED_BF16 if mixed else pkg.FP32)
            acc = []
            for _ in range(30):
                s.step(1)
                lab = s.get_U().argmax(dim=1)
                a = float((lab == labels).float().mean())
                acc.append(round(max(a, 1.0 - a), 6))
            s.step(W)
            torch.cuda.synchronize()
            ranks.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with ClockSampler(torch.cuda.current_device()) as cs:
                e0.record(stream)
                kt = s.enqueue_profiled(K)
                e1.record(stream)
                torch.cuda.synchronize()
            ranks.barrier()
            secs, it_s = ranks.weak_throughput(K, e0.elapsed_time(e1) / 1000.0)
            ms = secs * 1000.0
            first = next((i + 1 for i, a in enumerate(acc) if a >= 0.999), None)
            res[name] = {"it_s": it_s, "ms_per_step": ms / K, "pass_ms": kt["pass_ms"],
                         "update_ms": kt["update_ms"], "fold_ms": kt["fold_ms"], "accuracy_by_iter": acc,
                         "first_iter_99_9": first, "clocks": cs.summary()}
            s.close()
            del s
            torch.cuda.empty_cache()
    head = res["fista_fp32"] if "fista_fp32" in res else next(iter(res.values()))
    # compulsory bytes of the product: row_ptr, col, val, each iterate row once, z written
    b_min = 8 * (n + 1) + nnz * 8 + n * 2 * 4 * 2
    achieved = b_min / (head["pass_ms"] / 1000.0) / 1e9
    line = {"metric": "FISTA iterations/s on the paper's artificial two-cluster graph (k=2)",
            "value": head["it_s"], "unit": "iter/s", "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"two Erdos-Renyi clusters {n1:,} (degree {d1:.0f}) + {n2:,} (degree {d2:.0f}), "
                                   f"{bridges} bridges, 0/1 similarity, nnz = {nnz:,}, X0 = second row, tau = {tau}",
                       "n": n, "k": 2, "nnz": nnz, "gen_seconds": round(gen_s, 1),
                       "l2": "iterate fits in L2 (6 MB); S (8 GB) streamed from HBM; no flush",
                       "paper": "GPA and FISTA recovered the clusters in < 10 iterations, about 15 s (V100 box)"},
            "forms": res,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": "spmm_kernel<2,false>", "peak_kind": peak_kind,
                         "alg_bytes_per_launch": b_min, "note": "compulsory bytes: the iterate is L2-resident"},
            "clocks": head["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()


def serve_measure(args, rank, rate, duration, drain):
    """Poisson arrivals at `rate` per second for `duration` seconds of solves
    drawn from a pool of --pool pre-generated graphs (n log-uniform in
    [1e3, 2e6], k in {8, 16, 32, 64, 128}, mean degree U[10, 40]; host
    arrays), each run to PG_REL --serve-tol (cap --serve-max-iter) under a
    --budget-gb device budget; completions are awaited `drain` seconds more.
    Returns latency percentiles of the finished requests, offered vs achieved
    load and the requests still pending (counted, not dropped)."""
    import random
    import threading

    import numpy as np
    import torch

    import synth
    import paper_2506_04045_b300 as pkg
    specs = synth.batch_specs(args.pool, seed=4 + 1000 * rank, n_range=(1_000, 2_000_000),
                              ks=(8, 16, 32, 64, 128))
    pool = []
    for sp in specs:
        rp, c, v = synth.make_graph(sp, device="cuda")
        U0 = synth.dirichlet_u0(sp.n, sp.k, sp.seed, device="cuda")
        pool.append((rp.cpu().numpy(), c.cpu().numpy(), v.cpu().numpy(), U0.cpu().numpy()))
        del rp, c, v, U0
    torch.cuda.empty_cache()
    srv = pkg.Server(hbm_budget=int(args.budget_gb * (1 << 30)), iters_per_tick=args.tick, relabel=args.relabel,
                     update_engine=args.update_engine, overlap=args.overlap, stop_rule=pkg.STOP_PG_REL,
                     tol=args.serve_tol, max_iter=args.serve_max_iter, borrow_host=True)
    rng = random.Random(4 + rank)
    tickets, submit_t, which = [], {}, {}
    depth = []
    stop_sampling = threading.Event()

    def sampler():
        t0 = time.perf_counter()
        while not stop_sampling.is_set():
            st = srv.stats()
            depth.append((round(time.perf_counter() - t0, 2), st["queued"], st["resident"], st["completed"]))
            stop_sampling.wait(1.0)

    th = threading.Thread(target=sampler, daemon=True)
    with ClockSampler(torch.cuda.current_device()) as cs:
        th.start()
        t_start = time.perf_counter()
        t_next = t_start
        while True:
            t_next += rng.expovariate(rate)
            if t_next - t_start > duration:
                break
            delay = t_next - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            pi = rng.randrange(len(pool))
            tk = srv.submit(*pool[pi])
            tickets.append(tk)
            submit_t[tk] = time.perf_counter()
            which[tk] = pi
        t_arrivals_end = time.perf_counter()
        results = {}
        deadline = t_arrivals_end + drain
        while time.perf_counter() < deadline and len(results) < len(tickets):
            for tk in tickets:
                if tk in results:
                    continue
                try:
                    out = srv.poll(tk)
                except pkg.ClusterError as exc:
                    results[tk] = ("error", str(exc))
                    continue
                if out is not None:
                    results[tk] = ("ok", out[2], out[1], which[tk])
            time.sleep(0.05)
        t_end = time.perf_counter()
        stop_sampling.set()
        th.join(timeout=5)
    st = srv.stats()
    srv.close()
    ok = [r for r in results.values() if r[0] == "ok"]
    lat = np.array([r[1]["total_s"] for r in ok]) if ok else np.array([])
    pending = len(tickets) - len(results)
    span = t_end - t_start
    return {"config": {"workload": f"Poisson {rate}/s for {duration}s, n log-uniform [1e3, 2e6], "
                                   f"k in {{8..128}}, mean degree U[10,40], PG_REL {args.serve_tol}, "
                                   f"max_iter {args.serve_max_iter}, budget {args.budget_gb} GB, pool {args.pool}",
                       "tick": args.tick, "drain_s": drain},
            "requests_submitted": len(tickets),
            "p50_s": float(np.percentile(lat, 50)) if ok else None,
            "p99_s": float(np.percentile(lat, 99)) if ok else None,
            "completed": len(ok), "failed": len(results) - len(ok), "pending_at_end": pending,
            "offered_rps": len(tickets) / duration, "achieved_solves_per_s": len(ok) / span,
            "mean_queue_s": float(np.mean([r[1]["queue_s"] for r in ok])) if ok else None,
            "mean_run_s": float(np.mean([r[1]["run_s"] for r in ok])) if ok else None,
            "iterations_of_completed": [int(r[2]["iters"]) for r in ok][:50],
            "requests": [[specs[r[3]].n, specs[r[3]].k, round(r[1]["queue_s"], 4), round(r[1]["run_s"], 4),
                          round(r[1]["total_s"], 4)] for r in ok][:200],
            "queue_depth": depth[::max(1, len(depth) // 40)], "server_stats": st, "clocks": cs.summary()}


def run_serve(args, ws, rank, local):
    """Serving workload: Poisson arrivals (rate --rate) of solves, see
    serve_measure.  value = p99 latency (arrival -> U on host) of the requests
    that finished."""
    import torch

    import paper_2506_04045_b300 as pkg
    torch.cuda.set_device(local)
    pkg.load()
    m = serve_measure(args, rank, args.rate, args.duration, args.drain)
    line = {"metric": "serving p99 latency (continuous batching)", "value": m["p99_s"],
            "unit": "s", "n_gpus": ws, "steps": m["requests_submitted"], "warmup": 0, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", **m}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_rowrate(args, ws, rank, local):
    """Random-row gather rate, the access pattern of the product S X isolated:
    --rows-m uniformly random row indices into a --table-gb table (far larger
    than L2), rows of 32, 64, 128 and 256 bytes (k = 32 gathers 64-byte bf16
    rows in the mixed form and 128-byte float32 rows in the FP32 form).  Modes:
    plain 16-byte loads; the same with the 64-byte L2 fetch hint (rows <= 64 B);
    TMA tile::gather4 staging through shared memory (64- and 128-byte rows).
    value = G rows/s of plain loads of 64-byte rows."""
    import ctypes

    import torch
    from paper_2506_04045_b300 import build as _b
    torch.cuda.set_device(local)
    lib = ctypes.CDLL(_b.build_probe())
    fn = lib.probe_gather
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                   ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    K, W = args.steps, args.warmup
    nbytes = int(args.table_gb * (1 << 30)) // 256 * 256
    table = torch.empty(nbytes // 4, dtype=torch.int32, device="cuda").random_()
    sink = torch.empty(1 << 22, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    hbm, peak_kind = peaks()
    m = args.rows_m // 4 * 4
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    res = []
    with ClockSampler(torch.cuda.current_device()) as cs:
        for rb in (32, 64, 128, 256):
            rows = nbytes // rb
            idx = torch.randint(0, rows, (m,), dtype=torch.int32, device="cuda", generator=gen)
            modes = [0] + ([1] if rb <= 64 else []) + ([2] if rb in (64, 128) else [])
            for mode in modes:
                ms = ctypes.c_double(0.0)
                for reps in (W, K):
                    rc = fn(table.data_ptr(), rows, rb, idx.data_ptr(), m, mode, 0, max(reps, 1), sink.data_ptr(),
                            stream.cuda_stream, ctypes.byref(ms))
                    if rc != 0:
                        raise RuntimeError(f"probe_gather rows={rb}B mode={mode}: code {rc}")
                t = ms.value / 1000.0
                res.append({"row_bytes": rb, "mode": ["plain", "plain+L2::64B", "tma_gather4"][mode],
                            "ms": ms.value, "G_rows_per_s": m / t / 1e9,
                            "row_GBps": m * rb / t / 1e9, "with_index_GBps": m * (rb + 4) / t / 1e9,
                            "frac_of_copy_peak": m * (rb + 4) / t / 1e9 / hbm})
            del idx
    head = next(r for r in res if r["row_bytes"] == 64 and r["mode"] == "plain")
    line = {"metric": "random-row gather rate (G rows/s)", "value": head["G_rows_per_s"], "unit": "G rows/s",
            "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": head["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"{m:,} uniform random rows per launch from a {nbytes / 2**30:.1f} GiB table",
                       "l2": "table 64x larger than L2; no flush"},
            "results": res,
            "roofline": {"bound": "hbm", "achieved": head["with_index_GBps"], "peak": hbm, "unit": "GB/s",
                         "frac": head["frac_of_copy_peak"], "traffic": None, "peak_kind": peak_kind,
                         "kernel": "probe_ldg_kernel<64,false>"},
            "clocks": cs.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "batch":
        run_batch(args, ws, rank, local)
        return
    if args.workload == "serve":
        run_serve(args, ws, rank, local)
        return
    if args.workload == "er2":
        run_er2(args, ws, rank, local)
        return
    if args.workload == "rowrate":
        run_rowrate(args, ws, rank, local)
        return
    run_native(args, ws, rank, local)


if __name__ == "__main__":
    main()
