#!/usr/bin/env python3
"""POTRF effective TFLOP/s (n^3/3 per second) of the mixed-precision recursive Cholesky
against the FP64 tree, on one GB300 (or N independent replicas under torchrun).

Workload (one "step" = one pass of the hot path over one matrix):
  A: n = 8192, B iid N(0,1), A = (B + B^T)/2, A_ii = rho * sum_{j!=i} |A_ij|, rho cycling
     through {1.05, 2, 8}; tree [F16,F16,F16,F16,F32|F64@128] (FP16 off-diagonal GEMMs with
     FP32 accumulation at the four outer levels, FP32 below, FP64 diagonal leaves of 128);
  step = hrp_potrf_async (factor) + hrp_potrs (1 right-hand side) on the device.
Every step factors its own resident copy of A (512 MB each, larger than L2), so no
input is re-read from L2 across steps.

Output: one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
step-by-step emulator of Alg. 1-3) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 8192
RHOS = (1.05, 2.0, 8.0)
TREE = "[F16,F16,F16,F16,F32|F64@128]"
LEAF = 128
FP64_TREE, FP64_LEAF = "[F64]", 64
METRIC = "POTRF TFLOP/s (n^3/3 per s) mixed vs FP64 tree on GB300 at stated backward error"
# FMA rates of the GB300s from a throughput microbenchmark (8 independent FMA chains
# per thread, 4 x 152 CTAs of 256 threads, CUDA-event timed, SM clock 2.0 GHz): FP64 1.20 and
# FP32 75.2 TFLOP/s.  ALU-bound kernels report against them (NVIDIA's nominal FP64 figure is
# 1.25 TFLOP/s).
FP64_MEASURED_TFLOPS = 1.20
FP32_MEASURED_TFLOPS = 75.2
# DRAM bytes (read + write) per launch of the leaf POTRF kernel from one ncu capture, reported
# while the kernel's device code is the code captured: the source up to its launcher, hashed.
LEAF_TRAFFIC = {"bytes": 162176, "source": "paper_2601_08082_gb300/csrc/k_leaf_cluster.cu",
                "until": "cudaError_t launch_potrf_leaf_cluster(", "sha1": "c1833c238d6246960dce60c58aa7a6d40dfe023a"}
# The leaves of trees with a level below FP64 run in double-float arithmetic on the FP32 pipe:
# one double-float multiply-add (the Dot2 accumulation step of the tile updates) is 12 FP32
# instructions, so FP64-class work done that way peaks at the FP32 rate / 12.
DF_OPS_PER_FMA = 12


def device_code_sha1(path, until):
    """SHA-1 of a CUDA source up to (not including) the first line that starts with `until`:
    the kernels, without the host launcher below them."""
    import hashlib
    text = open(path, "rb").read().decode()
    cut = text.find("\n" + until)
    return hashlib.sha1(text[: cut if cut >= 0 else len(text)].encode()).hexdigest()


def leaf_traffic():
    if LEAF_TRAFFIC["bytes"] is None:
        return None
    try:
        ok = device_code_sha1(os.path.join(ROOT, LEAF_TRAFFIC["source"]), LEAF_TRAFFIC["until"]) == LEAF_TRAFFIC["sha1"]
    except OSError:
        ok = False
    return LEAF_TRAFFIC["bytes"] if ok else None


def host_lower_bytes(n, blk=128):
    """Bytes hrp_potrf_host transfers for an n x n matrix: rows [128 b, n) of every 128-column
    block b (the lower triangle and the 128 x 128 diagonal blocks)."""
    return sum((n - c0) * min(blk, n - c0) * 8 for c0 in range(0, n, blk))


def accuracy_steps(warmup, nsteps, nrho):
    """(step, matrix index) of the first timed step of each input matrix: step s factors
    matrix s % nrho, so entry i of the result names the matrix that step really factored."""
    out = []
    for s in range(warmup, min(nsteps, warmup + nrho)):
        out.append((s, s % nrho))
    return out


def lpt_partition(costs, world):
    """Longest processing time first: the items, by decreasing cost (ties by index), each go
    to the rank with the least load so far (ties by rank).  Returns each rank's item indices in
    increasing order.  Graham's bound: the largest load is at most 4/3 of the optimum."""
    import heapq
    loads = [(0.0, r) for r in range(world)]
    heapq.heapify(loads)
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda j: (-costs[j], j)):
        load, r = heapq.heappop(loads)
        parts[r].append(i)
        heapq.heappush(loads, (load + costs[i], r))
    return [sorted(p) for p in parts]


def forward_error_colmajor(Lm, L64):
    """||L_hat - L||_F / ||L||_F for two factors held column-major as (n, ld) tensors, storage
    row c = matrix column c: the factors' lower triangles are the storage's upper triangles
    (the strict lower part of the storage holds the untouched input)."""
    import torch
    ref = torch.triu(L64)
    return float(torch.linalg.norm(torch.triu(Lm) - ref) / torch.linalg.norm(ref))


class Replicas:
    """One process per GPU (torchrun): RANK, WORLD_SIZE and LOCAL_RANK come from the
    environment.  The replicas share no data; the process group (NCCL on the GPUs, gloo in the
    CPU tests) only brackets the timed region with barriers and combines the per-rank figures:
    the max of the times, the sum of the work."""

    def __init__(self, backend="nccl", device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": device} if device is not None else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, self.dist.ReduceOp.MAX if self.dist is not None else None)

    def sum(self, x):
        return self._reduce(x, self.dist.ReduceOp.SUM if self.dist is not None else None)

    def gather_objects(self, obj):
        """Every rank's picklable obj, in rank order (a one-element list on one rank)."""
        if self.dist is None:
            return [obj]
        out = [None] * self.world
        self.dist.all_gather_object(out, obj)
        return out

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def tuned_fp64_tree(h, hrp, n):
    """The plain FP64 tree with the recursion cut-offs hrp_autotune picks at order n (one timed
    run per candidate), so the comparison is with the fastest FP64 configuration, not a fixed one."""
    base = hrp.tree_parse(FP64_TREE, leaf=FP64_LEAF)
    t, ms = h.autotune(base, n, reps=1)
    return t, {"leaf": t.leaf, "trsm_leaf": t.trsm_leaf or t.leaf, "tuned_at_n": n, "tuner_ms": ms}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained", p["bf16_tflops"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


class Clocks:
    """nvidia-smi sampling during the timed region.  The sampler is started and its first
    sample awaited before the region opens (nvidia-smi takes a few hundred milliseconds to
    start), and one sample after the region closes is awaited before it stops, so that the
    samples inside the region and the two that bracket it are always on record.  All waits
    are bounded; without nvidia-smi the summary has no samples."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, period_ms: int = 200, cmd=None, start_timeout_s: float = 5.0):
        self.device = device
        self.period = period_ms / 1e3
        self.cmd = cmd or ["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                           "--format=csv,noheader,nounits", "-lms", str(period_ms)]
        self.start_timeout = start_timeout_s
        self.proc = None
        self.lines = []                  # (monotonic time of arrival, line)
        self.t0 = self.t1 = None

    def _wait_for(self, pred, timeout):
        end = time.monotonic() + timeout
        while not pred() and time.monotonic() < end:
            if self.proc is not None and self.proc.poll() is not None:
                break
            time.sleep(0.01)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            self._wait_for(lambda: len(self.lines) > 0, self.start_timeout)
        except Exception:
            self.proc = None
        self.t0 = time.monotonic()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def __exit__(self, *a):
        self.t1 = time.monotonic()
        if self.proc:
            self._wait_for(lambda: any(t > self.t1 for t, _ in self.lines), 4 * self.period + 1.0)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _parse(line):
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 8:
            return None
        try:
            return float(parts[0]), float(parts[1]), parts[4:8]
        except ValueError:
            return None

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = [(t, r) for t, ln in self.lines for r in [self._parse(ln)] if r is not None]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "in_region": 0}
        t0 = self.t0 if self.t0 is not None else rows[0][0]
        t1 = self.t1 if self.t1 is not None else rows[-1][0]
        inside = [r for t, r in rows if t0 <= t <= t1]
        before = [r for t, r in rows if t < t0][-1:]
        after = [r for t, r in rows if t > t1][:1]
        use = before + inside + after
        sm = [r[0] for r in use]
        reasons = {nm for r in use for nm, v in zip(names, r[2]) if v.lower().startswith("active")}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in use), "reasons": sorted(reasons),
                "samples": len(use), "in_region": len(inside)}


def cpu_oracle_sample(n_s: int = 3072, rho: float = 2.0, mats=None, budget_s: float = 10.0):
    """Time the oracle (emulator of Alg. 1-3) with the same tree: on `mats` (the workload's
    own matrices, one after another until `budget_s` seconds of emulation have run), or on one
    n_s matrix of the same generator."""
    from oracle import tree as otree
    from synth import dominant_spd, seed_for
    t = otree.parse(TREE, leaf=LEAF)
    if mats is None:
        mats = [dominant_spd(n_s, rho, seed_for(1, 900 + n_s))]
        what = f"one n={n_s} matrix of the same generator (rho={rho})"
    else:
        what = None
    done, secs, flops = 0, 0.0, 0.0
    for A in mats:
        t0 = time.perf_counter()
        _, info, _ = otree.emulate_potrf(A, t)
        secs += time.perf_counter() - t0
        assert info == 0
        done += 1
        flops += A.shape[0] ** 3 / 3.0
        if secs >= budget_s:
            break
    if what is None:
        what = f"{done} of the workload's n={mats[0].shape[0]} matrices (rho {list(RHOS)[:done]})"
    return {"value": flops / secs / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"emulator of Alg. 1-3 (float64 numpy, tree {TREE}, leaf {LEAF}) on {what}; {secs:.1f} s",
            "seconds": secs}


def cpu_dense_sample(mats, nrhs: int = 4, budget_s: float = 10.0, seed_base: int = 10000):
    """Time the oracle's plain FP64 Cholesky and solve (oracle.dense) on `mats` one after
    another until `budget_s` seconds have run: the CPU baseline of the batched workload."""
    from oracle import dense
    from synth import rhs, seed_for
    done, secs, flops = 0, 0.0, 0.0
    for i, A in enumerate(mats):
        B = rhs(A.shape[0], nrhs, seed_for(3, seed_base + i))
        t0 = time.perf_counter()
        L, info = dense.cholesky(A)
        assert info == 0
        dense.potrs(L, B)
        secs += time.perf_counter() - t0
        done += 1
        flops += A.shape[0] ** 3 / 3.0
        if secs >= budget_s:
            break
    return {"value": flops / secs / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"plain FP64 Cholesky + {nrhs}-RHS solve (oracle.dense, float64 numpy) on the first "
                      f"{done} of the batch's systems; {secs:.1f} s"}


def run_reference(args, rank):
    if rank != 0:
        return 0
    n_s = 2048
    for _ in range(args.warmup):
        cpu_oracle_sample(n_s)
    secs = []
    for _ in range(args.steps):
        secs.append(cpu_oracle_sample(n_s)["seconds"])
    tot = sum(secs)
    val = args.steps * n_s ** 3 / 3.0 / tot / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16/f32/f64 emulated in f64",
            "data": "synthetic", "config": {"workload": f"mixed tree {TREE}, n={N} generator, sample n={n_s}",
                                            "n": n_s, "tree": TREE, "leaf": LEAF, "rho": 2.0, "nrhs": 0},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"emulator of Alg. 1-3 on one n={n_s} matrix per step"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, rank, world):
    """512 RBF systems (n ~ U[64, 2048], x_i ~ U[0,1]^3, length 0.5, jitter 1e-2), 4 RHS each:
    one graph-captured batched factorization + solve with a mixed tree, against a
    per-matrix loop of the FP64 tree."""
    import numpy as np
    import torch

    import paper_2601_08082_gb300 as hrp
    from synth import rbf_spd, rhs, seed_for, uniforms

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reps = Replicas("nccl", device=torch.device("cuda", local))
    h = hrp.Handle(local)
    batch = args.batch
    # the job's batch * world systems, shared among the ranks by LPT on n^3 (each rank then
    # holds about `batch` systems and the same share of the work)
    u = uniforms(seed_for(3, 0), 7, np.arange(batch * world, dtype=np.uint64))
    all_sizes = [int(64 + np.floor(x * (2048 - 64 + 1))) for x in u]
    mine = lpt_partition([float(n) ** 3 for n in all_sizes], world)[rank]
    sizes = [all_sizes[g] for g in mine]
    mats = [rbf_spd(all_sizes[g], seed_for(3, 1 + g)) for g in mine]
    A0 = [hrp.colmajor(A).cuda() for A in mats]
    B0 = [hrp.colmajor(rhs(all_sizes[g], 4, seed_for(3, 10000 + g))).cuda() for g in mine]
    As = [A.clone() for A in A0]
    Bs = [B.clone() for B in B0]
    tree = hrp.tree_parse(args.batch_tree, leaf=128)
    d_info = torch.zeros(len(mine), dtype=torch.int32, device="cuda")
    flops = sum(n ** 3 / 3.0 for n in sizes)

    def graph_ms(persistent):
        """(1) the factor + solve graph alone (no refinement): one replay per step."""
        h.set_batched_mode(persistent)
        h.potrf_batched(tree, As, d_info)
        h.potrs_batched(As, Bs)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                h.potrf_batched(tree, As, d_info, stream=s)
                h.potrs_batched(As, Bs, stream=s)
        gt = []
        for rep in range(args.warmup + args.steps):
            for A, a0 in zip(As, A0):
                A.copy_(a0)
            for B, b0 in zip(Bs, B0):
                B.copy_(b0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            if rep >= args.warmup:
                gt.append(e0.elapsed_time(e1))
        return sum(gt) / len(gt)

    g_pool = graph_ms(False)
    g_pers = graph_ms(True)
    h.set_batched_mode(False)               # the handle's default (the stream pool) for the POSV
    failed = [i for i, v in enumerate(d_info.cpu().tolist()) if v != 0]
    # (2) the full batched solve: mixed tree, fallback where it fails, FP64 refinement to 1e-12
    Xs = [torch.zeros_like(B) for B in B0]
    times = []
    for rep in range(args.warmup):
        out = h.posv_batched(tree, A0, B0, Xs, max_iter=30, tol=1e-12)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for rep in range(args.steps):
            torch.cuda.synchronize()
            reps.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = h.posv_batched(tree, A0, B0, Xs, max_iter=30, tol=1e-12)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    # every rank solves its LPT share (weak scaling: batch systems per rank on average): the
    # job's work over the slowest rank
    ms = reps.max(sum(times) / len(times))
    flops_rank = flops
    flops = reps.sum(flops_rank)
    worst = max(out["resid"])
    # per-matrix loop of the FP64 tree (the comparison named by the workload)
    t64 = hrp.tree_parse("[F64]", leaf=64)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for A, a0, B, b0 in zip(As, A0, Bs, B0):
        A.copy_(a0)
        h.potrf_async(t64, A, d_info[0:1])
        h.potrs(A, B)
    e1.record()
    torch.cuda.synchronize()
    ms64 = reps.max(e0.elapsed_time(e1))
    line = {"metric": METRIC + " (batched)", "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16 (fp32 acc) / f32 / f64", "data": "synthetic",
            "config": {"workload": f"{batch * world} RBF systems n~U[64,2048] over {world} rank(s) by LPT on n^3, "
                                   f"4 RHS, tree {args.batch_tree}, batched posv "
                                   "with FP32/FP64 fallback and FP64 refinement",
                       "batch": batch * world, "systems_rank0": len(mine), "sum_n3_over_3": flops,
                       "tree": args.batch_tree},
            "fp64_loop": {"ms": ms64, "tflops": flops / (ms64 * 1e-3) / 1e12},
            "speedup_vs_fp64_loop": ms64 / ms, "status": out["status"],
            "systems_refactored_with_fallback": int(sum(out["used_fallback"])),
            "max_refinement_rounds": int(max(out["iters"])), "worst_solution_residual": worst,
            "graph_factor_solve_ms": {"persistent": g_pers, "stream_pool": g_pool},
            "graph_systems_failing_mixed_tree": len(failed), "clocks": clk.summary(),
            "roofline": None,
            "roofline_note": "no single dominant kernel: each system's launch chain runs on one stream "
                             "of a 32-stream pool, with refinement rounds and fallback refactorizations"}
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_dense_sample(mats)
    reps.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    return 0


BLAS3_TREES = ["[F64]", "[F32]", "[F16,F16,F32]", "[F16,F16,F16,F16,F32]", "[F16]"]


def blas3_baseline(spec):
    """The paper's normalization (Sec. 4.2): a mixed list against the pure tree of its innermost
    (diagonal) precision; Pure F16 against FP32."""
    inner = spec.strip("[]").split(",")[-1]
    return "[F32]" if spec == "[F16]" else f"[{inner}]"


def run_blas3(args, rank, world):
    """Standalone recursive SYRK (C -= A A^T, A n x n) and TRSM (X L^T = B, B n x n) of order
    --blas3-n with the precision lists of Sec. 4.2: TFLOP/s (n^3 for SYRK and TRSM) and the
    speed-up over the baseline the paper uses for each list."""
    import numpy as np
    import torch

    import paper_2601_08082_gb300 as hrp

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reps = Replicas("nccl", device=torch.device("cuda", local))
    n = args.blas3_n
    h = hrp.Handle(local)
    g = torch.Generator(device="cuda")
    g.manual_seed(2601008082 + 4000 + rank)
    A = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64)
    C0 = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64)
    B0 = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64)
    # a well-conditioned lower factor: unit-ish diagonal, small off-diagonal entries
    Lf = torch.tril(torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64) / n ** 0.5, -1)
    Lf.diagonal().copy_(1.0 + torch.rand(n, generator=g, device="cuda", dtype=torch.float64))
    Lt = Lf.T.contiguous()                        # column-major storage of L
    C = torch.empty_like(C0)
    Bx = torch.empty_like(B0)
    stream = torch.cuda.current_stream()
    hs = hrp.Handle(local)
    hs.set_fp32_split(True)
    out = {"syrk": {}, "trsm": {}, "syrk_tf32x3": {}}
    for spec in BLAS3_TREES:
        t = hrp.tree_parse(spec, leaf=128)
        # syrk_tf32x3: the same SYRK with the FP32 levels on tensor cores (TF32 split)
        for op in ("syrk", "trsm", "syrk_tf32x3"):
            if op == "syrk_tf32x3" and "F32" not in spec:
                continue
            hh = hs if op == "syrk_tf32x3" else h
            times = []
            for rep in range(args.warmup + args.steps):
                if op != "trsm":
                    C.copy_(C0)
                else:
                    Bx.copy_(B0)
                torch.cuda.synchronize()
                reps.barrier()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if op != "trsm":
                    hh.syrk(t, A, C, stream=stream)
                else:
                    hh.trsm(t, Lt, Bx, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                if rep >= args.warmup:
                    times.append(e0.elapsed_time(e1))
            assert hh.check() == 0
            ms = reps.max(statistics.median(times))
            out[op][spec] = {"ms": ms, "tflops": world * float(n) ** 3 / (ms * 1e-3) / 1e12}
    for op in ("syrk", "trsm"):
        for spec, v in out[op].items():
            base = blas3_baseline(spec)
            if base != spec and base in out[op]:
                v["speedup_vs_" + base] = out[op][base]["ms"] / v["ms"]
    for spec, v in out["syrk_tf32x3"].items():
        v["speedup_vs_simt_fp32"] = out["syrk"][spec]["ms"] / v["ms"]
    hs.close()
    line = {"metric": "recursive SYRK / TRSM TFLOP/s (n^3 per s) by precision list", "unit": "TFLOP/s",
            "value": out["syrk"]["[F16,F16,F16,F16,F32]"]["tflops"], "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 (fp32 acc) / f32 / f64", "data": "synthetic (device generator)",
            "config": {"workload": f"hrp_syrk and hrp_trsm, n={n}, leaf 128, precision lists {BLAS3_TREES}",
                       "n": n, "value_is": "SYRK [F16,F16,F16,F16,F32]",
                       "l2": "inputs larger than L2 (128 MB+ operands, fresh copy per step)"},
            "syrk": out["syrk"], "trsm": out["trsm"]}
    reps.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    return 0


def run_fp8posv(args, rank, world):
    """n = 32768, A = (B + B^T)/2 with B iid N(0,1) and A_ii = 2 sum_{j!=i} |A_ij|, tree
    [F8,F16,F16,F32|F64@128] (E4M3 outermost off-diagonal level with one power-of-two scale per
    128 x 128 tile, FP16 at the next two levels, FP32 diagonal regions, FP64 leaves of 128):
    factorization rate, then hrp_posv with 16 right-hand sides refined to 1e-12.  The input
    (8.6 GB) is drawn on the device from a seeded torch generator; the oracle is not run at
    this size."""
    import torch

    import paper_2601_08082_gb300 as hrp

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reps = Replicas("nccl", device=torch.device("cuda", local))
    n, nrhs, rho, spec = args.n3, 16, 2.0, "[F8,F16,F16,F32|F64@128]"
    g = torch.Generator(device="cuda")
    g.manual_seed(2601008082 + 2000 + rank)
    Bt = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64)
    A = Bt + Bt.T
    del Bt
    A.mul_(0.5)
    A.diagonal().zero_()
    A.diagonal().copy_(rho * A.abs().sum(dim=1))
    Bm = torch.randn((nrhs, n), generator=g, device="cuda", dtype=torch.float64)   # column-major n x nrhs
    X = torch.zeros_like(Bm)
    h = hrp.Handle(local)
    tree = hrp.tree_parse(spec, leaf=128)
    d_info = torch.zeros(1, dtype=torch.int32, device="cuda")
    Af = torch.empty_like(A)
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        reps.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    tf = []
    with Clocks(local) as clk:
        for rep in range(args.warmup + args.steps):
            Af.copy_(A)
            _, t = timed(lambda: h.potrf_async(tree, Af, d_info, stream=stream))
            if rep >= args.warmup:
                tf.append(t)
    info = int(d_info.item())
    be = h.backward_error(A, Af)
    tp = []
    out = None
    for rep in range(1 + max(1, args.steps // 2)):
        out, t = timed(lambda: h.posv(tree, A, Bm, X, max_iter=30, tol=1e-12))
        if rep >= 1:
            tp.append(t)
    # the same factorization with the FP32 diagonal regions on tensor cores (TF32 split)
    hs = hrp.Handle(local)
    hs.set_fp32_split(True)
    ts = []
    for rep in range(1 + max(1, args.steps // 2)):
        Af.copy_(A)
        _, t = timed(lambda: hs.potrf_async(tree, Af, d_info, stream=stream))
        if rep >= 1:
            ts.append(t)
    split = {"ms": statistics.median(ts), "tflops": n ** 3 / 3.0 / (statistics.median(ts) * 1e-3) / 1e12,
             "info": int(d_info.item()), "backward_error": hs.backward_error(A, Af)}
    assert hs.check() == 0
    hs.close()
    fp64 = None
    if args.fp64_steps > 0:
        # cut-offs tuned at n = 8192 (tuning at n = 32768 would take minutes: ~10 s per run)
        tree64, tune64 = tuned_fp64_tree(h, hrp, 8192)
        Af.copy_(A)
        _, t64 = timed(lambda: h.potrf_async(tree64, Af, d_info, stream=stream))
        fp64 = {"ms": t64, "tflops": n ** 3 / 3.0 / (t64 * 1e-3) / 1e12, "tree": FP64_TREE, **tune64}
    # every rank factors its own matrix (weak scaling): the job's work over the slowest rank
    ms = reps.max(statistics.median(tf))
    flops = n ** 3 / 3.0
    line = {"metric": METRIC + " (n=32768 FP8 posv)", "value": world * flops / (ms * 1e-3) / 1e12,
            "unit": "TFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "e4m3 (block-scaled MMA, fp32 acc) / f16 (fp32 acc) / f32 / f64", "data": "synthetic (device generator)",
            "config": {"workload": f"n={n} rho={rho} tree {spec}, factor; posv with {nrhs} RHS to 1e-12",
                       "n": n, "tree": spec, "leaf": 128, "nrhs": nrhs,
                       "l2": "inputs larger than L2 (8.6 GB matrix, fresh copy per step)"},
            "info": info, "backward_error": be,
            "posv": {"ms": statistics.median(tp), "status": out["status"], "iters": out["iters"],
                     "resid": out["resid"], "used_fallback": out["used_fallback"],
                     "tflops_incl_refinement": flops / (statistics.median(tp) * 1e-3) / 1e12},
            "fp32_tf32x3": split,
            "fp64_tree": fp64, "speedup_vs_fp64_tree": (fp64["ms"] / ms) if fp64 else None,
            "clocks": clk.summary()}
    reps.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    return 0


def run_fp64_1024(args, rank, world):
    """The plain FP64 recursive Cholesky + solve at n = 1024: A = (B + B^T)/2, B iid N(0,1),
    A_ii = sum_{j!=i} |A_ij| + 1, one N(0,1) right-hand side, tree [F64] with leaf 64 (FP64
    leaves, FP64 SIMT GEMMs).  A step is hrp_potrf_async + hrp_potrs on a fresh resident copy;
    the factor and the solution are checked against the CPU oracle (plain Cholesky, two
    triangular solves) on every matrix, and the oracle itself is timed on the host as the CPU
    baseline."""
    import numpy as np
    import torch

    import paper_2601_08082_gb300 as hrp
    from oracle import dense
    from synth import dominant_spd, rhs, seed_for

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reps = Replicas("nccl", device=torch.device("cuda", local))
    n = 1024
    mats = [dominant_spd(n, 1.0, seed_for(0, 10 * rank + i), shift=1.0) for i in range(3)]
    bs = [rhs(n, 1, seed_for(0, 100 + 10 * rank + i)) for i in range(3)]
    # oracle: factor + solve on the host, its results also the reference of the check
    t0 = time.perf_counter()
    ref = []
    for A, b in zip(mats, bs):
        L0, info0 = dense.cholesky(A)
        ref.append((L0, dense.potrs(L0, b)))
    cpu_s = (time.perf_counter() - t0) / len(mats)
    h = hrp.Handle(local)
    tree = hrp.tree_parse("[F64]", leaf=64)
    A0 = [hrp.colmajor(A).cuda() for A in mats]
    B0 = [hrp.colmajor(b).cuda() for b in bs]
    nsteps = args.warmup + args.steps
    copies = [A0[s % 3].clone() for s in range(nsteps)]
    Bc = [B0[s % 3].clone() for s in range(nsteps)]
    d_info = torch.zeros(nsteps, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for s in range(args.warmup):
        h.potrf_async(tree, copies[s], d_info[s:s + 1], stream=stream)
        h.potrs(copies[s], Bc[s], stream=stream)
    torch.cuda.synchronize()
    reps.barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for s in range(args.warmup, nsteps):
        h.potrf_async(tree, copies[s], d_info[s:s + 1], stream=stream)
        h.potrs(copies[s], Bc[s], stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = reps.max(a.elapsed_time(b))
    assert int(d_info.max().item()) == 0 and int(d_info.min().item()) == 0
    err_l, err_x = 0.0, 0.0
    for s in range(args.warmup, min(nsteps, args.warmup + 3)):
        L0, x0 = ref[s % 3]
        L = np.tril(hrp.from_colmajor(copies[s]))
        x = hrp.from_colmajor(Bc[s])
        err_l = max(err_l, float(np.max(np.abs(L - L0)) / np.max(np.abs(L0))))
        err_x = max(err_x, float(np.max(np.abs(x - x0)) / np.max(np.abs(x0))))
    flops = n ** 3 / 3.0
    work = reps.sum(args.steps * flops)
    if rank == 0:
        line = {"metric": "POTRF TFLOP/s (n^3/3 per s), plain FP64 recursive Cholesky + 1-RHS solve, n=1024",
                "value": work / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "plain FP64 tree [F64] leaf 64, n=1024, A_ii = sum |A_ij| + 1, 1 RHS",
                           "n": n, "tree": "[F64]", "leaf": 64,
                           "l2": "inputs fit in L2 (8 MB each); a fresh resident copy per step"},
                "max_rel_err_L_vs_oracle": err_l, "max_rel_err_x_vs_oracle": err_x,
                "cpu_baseline": {"value": flops / cpu_s / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
                                 "kind": "oracle", "sample": "oracle Cholesky + solve of the 3 workload matrices"}}
        print(json.dumps(line), flush=True)
    h.close()
    return 0


def paired_ratio_ci(t_a, t_b, reps=2000, seed=7):
    """Mean of t_a / mean of t_b and a 95% bootstrap interval (pairs resampled together)."""
    import numpy as np
    a, b = np.asarray(t_a, dtype=np.float64), np.asarray(t_b, dtype=np.float64)
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(a), size=(reps, len(a)))
    boot = a[idx].mean(axis=1) / b[idx].mean(axis=1)
    return float(a.mean() / b.mean()), float(np.quantile(boot, 0.025)), float(np.quantile(boot, 0.975))


def run_policy(args, rank, world):
    """The learned precision-tree policy on held-out matrices of its training distribution
    (another generator seed): for each matrix, hrp_posv with tree = NULL (the library runs the
    feature pass, the network and its order gate, then the solve) against hrp_posv with the
    fixed fallback tree.  Reports the time ratio with a bootstrap interval and the failure rate."""
    import json as _json

    import numpy as np
    import torch

    import paper_2601_08082_gb300 as hrp
    from paper_2601_08082_gb300 import train_policy as tp
    from synth import rhs, seed_for

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reps = Replicas("nccl", device=torch.device("cuda", local))
    h = hrp.Handle(local)
    weights = os.path.join(ROOT, "paper_2601_08082_gb300", "policy_weights.json")
    h.policy_load(weights)
    with open(weights) as f:
        gate = _json.load(f).get("min_n", [0])[0]
    fb = hrp.policy_tree(0)
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    k = 0
    rows = []
    for i in range(args.policy_matrices * world):
        if i % world != rank:
            continue
        A, meta = tp.make_matrix(i, 9999, torch)
        A = A.contiguous()
        n = meta["n"]
        B = hrp.colmajor(rhs(n, 1, seed_for(7, 100 + i))).cuda()
        res = {}
        for name, tree in (("policy", None), ("fallback", fb)):
            X = torch.zeros_like(B)
            out, t = timed(lambda: h.posv(tree, A, B, X, tol=1e-12))
            res[name] = (t, int(out["status"]), int(out.get("used_fallback", 0)))
            if tree is None:
                k = int(h.last_policy_choice())
        rows.append({"n": n, "kind": meta["kind"], "pick": k, "t_policy": res["policy"][0],
                     "t_fallback": res["fallback"][0], "ok_policy": res["policy"][1] == 0,
                     "ok_fallback": res["fallback"][1] == 0, "policy_refactored": res["policy"][2]})
        del A
    gathered = reps.gather_objects(rows)
    if rank == 0:
        allr = [r for part in gathered for r in part]
        t_pol = [r["t_policy"] for r in allr]
        t_fb = [r["t_fallback"] for r in allr]
        ratio, lo, hi = paired_ratio_ci(t_pol, t_fb)
        line = {"metric": "policy POSV time (features + solve) / fixed-fallback POSV time, held-out matrices",
                "value": ratio, "unit": "ratio", "n_gpus": world, "steps": len(allr), "warmup": 0,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f16 / f32 / f64 trees",
                "data": "synthetic (device generator, held-out seed)",
                "config": {"workload": "learned policy on the training distribution: Gram G G^T/k + alpha I and "
                                       "rho-dominant matrices, n in {1024, 2048, 4096, 8192}, 1 RHS, POSV to 1e-12",
                           "matrices": len(allr)},
                "ratio_ci95": [lo, hi],
                "speedup": 1.0 / ratio,
                "failures_policy": sum(not r["ok_policy"] for r in allr),
                "failures_fallback": sum(not r["ok_fallback"] for r in allr),
                "policy_refactored_with_fallback": sum(r["policy_refactored"] != 0 for r in allr),
                "order_gate": gate,
                "picks": {str(k): sum(r["pick"] == k for r in allr) for k in range(8)},
                "by_n": {str(nn): {"matrices": sum(r["n"] == nn for r in allr),
                                   "ratio": (float(np.mean([r["t_policy"] for r in allr if r["n"] == nn]) /
                                                   np.mean([r["t_fallback"] for r in allr if r["n"] == nn]))
                                             if any(r["n"] == nn for r in allr) else None)}
                         for nn in (1024, 2048, 4096, 8192)}}
        print(json.dumps(line), flush=True)
    h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hrp", choices=["hrp", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="mixed8192", choices=["mixed8192", "batched", "fp8posv32768", "blas3", "policy",
                                                                  "fp64_1024"])
    ap.add_argument("--policy-matrices", type=int, default=48, help="held-out matrices per rank of the policy workload")
    ap.add_argument("--blas3-n", type=int, default=8192, help="order of the blas3 workload")
    ap.add_argument("--n3", type=int, default=32768, help="order of the fp8posv32768 workload")
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--batch-tree", default="[F16,F32|F64@128]")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "batched":
        return run_batched(args, rank, world)
    if args.workload == "fp8posv32768":
        return run_fp8posv(args, rank, world)
    if args.workload == "blas3":
        return run_blas3(args, rank, world)
    if args.workload == "policy":
        return run_policy(args, rank, world)
    if args.workload == "fp64_1024":
        return run_fp64_1024(args, rank, world)

    import numpy as np
    import torch

    import paper_2601_08082_gb300 as hrp
    from synth import dominant_spd, rhs, seed_for

    torch.cuda.set_device(local)
    reps = Replicas("nccl", device=torch.device("cuda", local))

    def barrier():
        reps.barrier()
        torch.cuda.synchronize()

    # inputs: one matrix per rho, generated on the host (same bits as the oracle sees)
    mats = [dominant_spd(N, rho, seed_for(1, 10 * rank + i)) for i, rho in enumerate(RHOS)]

    # oracle baseline on the same matrices (rank 0 only, before the GPU work)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_oracle_sample(mats=mats)
        cpu.pop("seconds", None)

    h = hrp.Handle(local)
    tree = hrp.tree_parse(TREE, leaf=LEAF)
    tree64, tune64 = tuned_fp64_tree(h, hrp, N) if args.fp64_steps > 0 else (None, None)
    stream = torch.cuda.current_stream()

    bvec = rhs(N, 1, seed_for(1, 100 + rank))
    A0 = [hrp.colmajor(A).cuda() for A in mats]
    nsteps = args.warmup + args.steps
    copies = [A0[s % len(RHOS)].clone() for s in range(nsteps)]
    B = [hrp.colmajor(bvec).cuda() for _ in range(nsteps)]
    d_info = torch.zeros(nsteps, dtype=torch.int32, device="cuda")
    flops = N ** 3 / 3.0

    def step(s):
        h.potrf_async(tree, copies[s], d_info[s:s + 1], stream=stream)
        launches = h.launch_count()
        h.potrs(copies[s], B[s], stream=stream)
        return launches + h.launch_count()

    for s in range(args.warmup):
        step(s)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    # the timed region lasts ~0.2 s: sample every 50 ms so that some samples fall inside it
    with Clocks(local, period_ms=50) as clk:
        barrier()
        e0.record(stream)
        for s in range(args.warmup, nsteps):
            launches += step(s)
        e1.record(stream)
        barrier()
    ms = reps.max(e0.elapsed_time(e1))
    infos = d_info.cpu().tolist()
    assert all(i == 0 for i in infos), infos
    value = world * args.steps * flops / (ms * 1e-3) / 1e12

    # accuracy of the timed factorizations (device FP64 backward error) and of the solves
    acc = {}
    for s, k in accuracy_steps(args.warmup, nsteps, len(RHOS)):
        be = h.backward_error(A0[k], copies[s])
        x = hrp.from_colmajor(B[s])
        r = mats[k] @ x - bvec
        acc[str(RHOS[k])] = {"backward_error": be,
                             "solution_residual": float(np.linalg.norm(r) / np.linalg.norm(bvec))}

    # roofline: one factorization in timing mode (per-kernel-class event timing)
    hrp.load().hrp_set_timing(h._h, 1)
    tmp = A0[1].clone()
    h.potrf(tree, tmp)
    import ctypes
    buf = (ctypes.c_double * 15)()
    hrp.load().hrp_get_timing(h._h, buf, 15)
    hrp.load().hrp_set_timing(h._h, 0)
    names = ["leaf_potrf_fp64", "leaf_trsm", "gemm_f16_tcgen05", "gemm_simt", "other"]
    classes = {names[c]: {"ms": buf[3 * c], "launches": int(buf[3 * c + 1]), "flops": buf[3 * c + 2]}
               for c in range(5)}
    tot_cls = sum(v["ms"] for v in classes.values()) or 1.0
    for v in classes.values():
        v["share"] = v["ms"] / tot_cls
    pk = peaks()
    # the leaf POTRF: the largest class on the critical stream (a timeline of the factorization
    # shows 4.3 ms of leaves there); the per-launch event timing of the other classes also
    # counts their side-stream launches, which overlap the leaves
    dom = "leaf_potrf_fp64"

    def roof(name):
        c = classes[name]
        avg_ms = c["ms"] / max(1, c["launches"])
        per_launch = c["flops"] / max(1, c["launches"])
        achieved = per_launch / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else 0.0
        if name == "gemm_f16_tcgen05":
            peak, bound, src = pk["bf16_tflops"], "tensor", f"{pk['src']} bf16 dense burst (FP16 same rate)"
        elif name in ("leaf_potrf_fp64",) and TREE != FP64_TREE:
            peak, bound = FP32_MEASURED_TFLOPS / DF_OPS_PER_FMA, "alu"
            src = (f"double-float on the FP32 pipe: FP32 {FP32_MEASURED_TFLOPS} TFLOP/s (FFMA microbenchmark, this "
                   f"pool) / {DF_OPS_PER_FMA} FP32 instructions per double-float multiply-add")
        elif name in ("leaf_potrf_fp64",):
            peak, bound, src = FP64_MEASURED_TFLOPS, "alu", "FP64 1.20 TFLOP/s (DFMA microbenchmark, this pool)"
        else:
            peak, bound, src = FP32_MEASURED_TFLOPS, "alu", "FP32 75.2 TFLOP/s (FFMA microbenchmark, this pool)"
        return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": leaf_traffic() if name == "leaf_potrf_fp64" else None, "kernel": name,
                "avg_launch_ms": avg_ms, "peak_src": src}

    # FP64 tree on the same matrices (the comparison of the metric)
    fp64 = None
    if args.fp64_steps > 0:
        t64 = []
        for i in range(args.fp64_steps):
            tmp = A0[i % len(RHOS)].clone()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.potrf_async(tree64, tmp, d_info[0:1], stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            t64.append(a.elapsed_time(b))
        fp64 = {"ms": min(t64), "tflops": flops / (min(t64) * 1e-3) / 1e12, "tree": FP64_TREE, **tune64}
        # forward error of the mixed factor against the FP64 tree's on the same matrix, and the
        # solve alone (POTRS, 1 RHS); reported when they can be taken, never failing the line
        try:
            i = (args.fp64_steps - 1) % len(RHOS)          # tmp holds the FP64 factor of A0[i]
            fp64["forward_error_mixed"] = forward_error_colmajor(copies[i], tmp)
            fp64["forward_error_rho"] = RHOS[i]
            Bx = hrp.colmajor(bvec).cuda()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.potrs(copies[i], Bx, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            fp64["potrs_ms"] = a.elapsed_time(b)
        except Exception as exc:                           # pragma: no cover (GPU only)
            fp64["extra_error"] = repr(exc)

    # end to end through the C ABI with host buffers: hrp_potrf_host (the lower triangle of A
    # copied from pinned host memory in 128-column blocks, overlapped with the factorization),
    # H2D of b, potrs, D2H of x
    e2e = None
    if args.e2e_steps > 0:
        hostA = [A.cpu().pin_memory() for A in A0]
        hostB = hrp.colmajor(bvec).pin_memory()
        hostX = torch.empty_like(hostB).pin_memory()
        dA = torch.empty_like(A0[0])
        dB = torch.empty_like(B[0])
        # this box's pinned host-to-device rate, one whole-matrix copy (context for e2e)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dA.copy_(hostA[0], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = dA.numel() * 8 / (a.elapsed_time(b) * 1e-3) / 1e9
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for s in range(args.e2e_steps):
            h.potrf_host(tree, hostA[s % len(RHOS)], dA, d_info[0:1], stream=stream)
            dB.copy_(hostB, non_blocking=True)
            h.potrs(dA, dB, stream=stream)
            hostX.copy_(dB, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        ems = a.elapsed_time(b)
        e2e = {"value": world * args.e2e_steps * flops / (ems * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(host_lower_bytes(N) + dB.numel() * 8), "d2h_bytes_per_step": int(dB.numel() * 8),
               "ms_per_step": ems / args.e2e_steps, "h2d_gbs_box": h2d_gbs}

    barrier()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16 (fp32 acc) / f32 / f64", "data": "synthetic",
            "config": {"workload": f"mixed tree {TREE} n={N} rho cycling {list(RHOS)}, factor + 1-RHS solve",
                       "n": N, "tree": TREE, "leaf": LEAF, "rhos": list(RHOS), "nrhs": 1,
                       "l2": "inputs larger than L2 (one resident 512 MB copy per step)",
                       "parallelism": f"replicas x{world}"},
            "fp64_tree": fp64,
            "speedup_vs_fp64_tree": (value / world) / fp64["tflops"] if fp64 else None,
            "accuracy": acc,
            "roofline": roof(dom),
            "roofline_gemm": roof("gemm_f16_tcgen05"),
            "roofline_leaf_trsm": roof("leaf_trsm"),
            "kernel_classes": classes,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    reps.close()
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
