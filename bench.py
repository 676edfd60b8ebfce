"""Benchmark: selected-kernel GEMM TFLOP/s over held-out shapes of the tuning grid.

Workload: the 200 held-out sizes (80/20 seeded split) of the 1,000-shape
FP32 tuning grid (M, N, K log-uniform in [16, 4096], batch in {1,..,16},
transA/transB in {N, T}, uniform[-1, 1] data).  One step = for every held-out
size, the deployed decision tree picks one of the deployed kernels and the
library launches it (select_kernel + gemm through the C-ABI), with every
input resident in HBM.  The step's inputs total ~7 GB, far above the 129 MB
L2, so consecutive steps start from a cold L2.

Also reported: the same metric end to end from pinned host buffers
(gemm_host_pipeline: every shape's H2D copies, GEMM and D2H copy inside the
timed region, uploads and downloads on the library's copy streams overlapping
the GEMMs); the share of
the per-shape exhaustive optimum (each held-out size re-run with the best of
all configs in the GB300 sweep table -- the 576 base configs and the split-K
kind -- untimed passes, per-shape medians of 3 on both sides); the dominant
kernel's roofline; the FP32 kernels on one large product beside the vendor
library's FP32 GEMM (``fp32_large``, context); the FP64 CPU oracle timed on a
bounded sample on the host cores (``cpu_baseline``).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import functools
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2008_13145_gb300 import workloads as wl  # noqa: E402

DEPLOY = os.path.join(ROOT, "paper_2008_13145_gb300", "deploy")
METRIC = "selected-kernel GEMM TFLOP/s and % of per-shape exhaustive optimum, FP32 vs TC"
WORKLOAD = "held-out 20% (200 shapes) of the 1000-shape FP32 tuning grid (seed 1)"
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
REF_TOTAL_S = 120.0  # oracle seconds for a whole --impl reference run
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12  # 80.5


def test_shapes():
    g = wl.shape_grid(1000, 1)
    _, te = wl.train_test_split(1000, 1)
    return [g[i] for i in te], te


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's);
    identity without a process group.  A control-path reduction only: the
    GEMMs of different ranks are independent replicas."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size: int, flops_per_step: float, steps: int, ms_total: float) -> float:
    """Whole-job TFLOP/s: the work of every rank over the slowest rank's time."""
    return world_size * flops_per_step * steps / (ms_total * 1e-3) / 1e12


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and "Active" in r[3 + i]
                          and "Not" not in r[3 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------- reference arm: the CPU oracle
@functools.lru_cache(maxsize=64)
def _oracle_inputs(one):
    """Host inputs of one sampled product, drawn once and reused by every step."""
    A, B, _ = wl.gemm_inputs(one, seed=5)
    return A, B


def cpu_oracle_sample(shapes, budget_s: float, nthreads: int):
    """FP64 oracle throughput on a bounded sample: the full product of batch
    entry 0 of the held-out shapes, in order, until the time budget is spent.
    Returns (TFLOP/s, description, seconds measured)."""
    from oracle import gemm as og
    og.build()
    flops, t_used, n_shapes = 0, 0.0, 0
    for sh in shapes:
        one = wl.Shape(sh.M, sh.N, sh.K, 1, sh.transA, sh.transB)
        A, B = _oracle_inputs(one)
        t0 = time.perf_counter()
        og.gemm(sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, A, B, nthreads=nthreads)
        t_used += time.perf_counter() - t0
        flops += one.flops
        n_shapes += 1
        if t_used >= budget_s:
            break
    return flops / t_used / 1e12, (f"full FP64 product of batch entry 0 of the first {n_shapes} held-out shapes "
                                   f"({flops / 1e9:.1f} GFLOP in {t_used:.1f} s, {nthreads} threads)"), t_used


def cpu_details(nthreads: int) -> dict:
    """The FP64 oracle on the small fixed case (256^3 NN, one thread and all
    threads) and on every VGG16 GEMM at batch 1 (all threads): GFLOP/s."""
    from oracle import gemm as og
    og.build()
    out = {}
    sh = wl.Shape(256, 256, 256, 1, "N", "N")
    A, B, _ = wl.gemm_inputs(sh, seed=0)
    for name, nt in (("single_gemm_256_1_thread", 1), (f"single_gemm_256_{nthreads}_threads", nthreads)):
        t0 = time.perf_counter()
        og.gemm("N", "N", 256, 256, 256, 1.0, A, B, nthreads=nt)
        out[name] = sh.flops / (time.perf_counter() - t0) / 1e9
    layers, total_f, total_t = {}, 0, 0.0
    for n, (name, sh) in enumerate(wl.vgg16_layers(1)):
        A, B, _ = wl.gemm_inputs(sh, seed=10 + n)
        t0 = time.perf_counter()
        og.gemm(sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, A, B, nthreads=nthreads)
        dt = time.perf_counter() - t0
        layers[name] = sh.flops / dt / 1e9
        total_f, total_t = total_f + sh.flops, total_t + dt
    out["vgg16_batch1_layers"] = layers
    out["vgg16_batch1_total"] = {"gflops": total_f / total_t / 1e9, "seconds": total_t, "threads": nthreads}
    out["unit"] = "GFLOP/s"
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    shapes, _ = test_shapes()
    steps, secs = [], []
    from oracle import gemm as og
    og.build()
    nthreads = og.max_threads()
    # Each step is a bounded sample: the whole run stays within about
    # REF_TOTAL_S of oracle work (the per-step budget shrinks as K + W grows).
    budget = min(args.ref_budget, max(0.3, REF_TOTAL_S / (args.warmup + args.steps)))
    for s in range(args.warmup + args.steps):
        v, desc, t = cpu_oracle_sample(shapes, budget, nthreads)
        if s >= args.warmup:
            steps.append(v)
            secs.append(t)
    val = statistics.median(steps)
    # Each step is a bounded sample of the workload; ms_per_step is the time a
    # timed step took, and the whole step's time is what the sampled rate implies.
    full_flops = sum(sh.flops for sh in shapes)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(secs) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "kind": "fp64 triple-loop CPU oracle",
                       "step": f"a bounded sample of the workload (about {budget:.1f} s of oracle work)",
                       "ms_per_step": "measured time of one sampled step (median over the timed steps)",
                       "ms_per_full_step_implied": full_flops / (val * 1e12) * 1e3},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": nthreads, "kind": "oracle", "sample": desc},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import torch
    from paper_2008_13145_gb300 import kselect as ks
    from paper_2008_13145_gb300 import tune

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    dep_path = os.path.join(DEPLOY, "f32.json")
    dep = json.load(open(dep_path))
    handle = ks.Handle(dep)
    table_shapes, perf, table_ids, _ = tune.load_table(os.path.join(DEPLOY, "table_f32.npz"))
    shapes, te = test_shapes()
    assert [table_shapes[i] for i in te] == shapes, "sweep table does not match the workload grid"
    best_cfg = [table_ids[int(np.argmax(perf[i]))] for i in te]

    bufs = [tune.alloc_inputs(sh, ks.PREC_F32, 1000 + 7 * rank + i) for i, sh in enumerate(shapes)]
    flops = sum(sh.flops for sh in shapes)
    chosen = [ks.select_kernel(handle, sh.M, sh.N, sh.K, sh.batch) for sh in shapes]
    # kernels per step: a split-K launch adds its reduction kernel
    launches_per_step = sum(1 + (ks.split_factor(c, sh.M, sh.N, sh.K, sh.batch)[0] > 1)
                            for c, sh in zip(chosen, shapes))

    def step(events=None, cfgs=None):
        for i, (sh, (A, B, C, lda, ldb, ldc)) in enumerate(zip(shapes, bufs)):
            if events is not None:
                events[i][0].record(stream)
            if cfgs is None:
                ks.gemm(handle, sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, A, lda, B, ldb, 0.0, C, ldc, sh.batch,
                        stream)
            else:
                ks.gemm_with_config(cfgs[i], sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, A, lda, B, ldb, 0.0, C,
                                    ldc, sh.batch, stream)
            if events is not None:
                events[i][1].record(stream)

    def per_launch_ms(cfgs=None):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in shapes]
        step(ev, cfgs)
        torch.cuda.synchronize(dev)
        return np.array([a.elapsed_time(b) for a, b in ev])

    def per_launch_median(cfgs=None, passes=3):
        return np.median([per_launch_ms(cfgs) for _ in range(passes)], axis=0)

    # Warm-up steps (selected kernels); the last ones also time every launch, after
    # the first has loaded every module.
    for _ in range(args.warmup - 1):
        step()
    sel_ms = per_launch_median()
    # Untimed reference passes: every shape with its exhaustive-best config (the
    # first loads the kernels the deployment does not use, the next ones are timed).
    per_launch_ms(best_cfg)
    exh_ms = per_launch_median(best_cfg)
    ratio = np.minimum(exh_ms / sel_ms, 1.0)
    live = {"geomean": float(np.exp(np.mean(np.log(ratio)))), "mean": float(np.mean(ratio)),
            "source": "per-shape launch times this run, median of 3 passes each: exhaustive-best config vs "
                      "selected config"}
    # Dominant kernel: the deployed config with the largest share of step time.
    by_cfg = {}
    for c, t, sh in zip(chosen, sel_ms, shapes):
        a = by_cfg.setdefault(c, [0.0, 0, 0])
        a[0] += t
        a[1] += sh.flops
        a[2] += 1
    dom = max(by_cfg, key=lambda c: by_cfg[c][0])
    dom_idx = [i for i, c in enumerate(chosen) if c == dom]

    # Timed region: K steps, dominant-kernel launches bracketed by events.
    dom_ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in dom_idx]
              for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly the timed steps
        e0.record(stream)
        for k in range(args.steps):
            evs = {i: ev for i, ev in zip(dom_idx, dom_ev[k])}
            for i, (sh, (A, B, C, lda, ldb, ldc)) in enumerate(zip(shapes, bufs)):
                if i in evs:
                    evs[i][0].record(stream)
                ks.gemm(handle, sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, A, lda, B, ldb, 0.0, C, ldc, sh.batch,
                        stream)
                if i in evs:
                    evs[i][1].record(stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
    ms_total = max_over_ranks(e0.elapsed_time(e1))
    ms_step = ms_total / args.steps
    value = job_throughput(ws, flops, args.steps, ms_total)
    dom_total = sum(a.elapsed_time(b) for evs in dom_ev for a, b in evs)
    dom_ms = dom_total / (len(dom_idx) * args.steps)
    dom_share = dom_total / e0.elapsed_time(e1)
    dom_flops = by_cfg[dom][1] / by_cfg[dom][2]
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12

    # The same deployed kernels chosen by the other selectors (untimed choice,
    # timed steps): the random forest of deploy/f32_forest.json and the MLP
    # performance model served by the batched selection kernel.
    selectors = {"decision_tree_b": {"value": value, "live_geomean": live["geomean"]}}
    alt = {}
    forest_path = os.path.join(DEPLOY, "f32_forest.json")
    if os.path.exists(forest_path):
        fdep = json.load(open(forest_path))
        if fdep["config_ids"] == dep["config_ids"]:
            hf = ks.Handle(fdep)
            alt["random_forest"] = [ks.select_kernel(hf, sh.M, sh.N, sh.K, sh.batch) for sh in shapes]
    if dep.get("mlp_params"):
        alt["mlp"] = [int(c) for c in tune.mlp_choose(np.asarray(dep["mlp_params"], np.float32), shapes,
                                                      dep["config_ids"])]
    for name, cfgs in alt.items():
        per_launch_ms(cfgs)
        r = np.minimum(exh_ms / per_launch_median(cfgs), 1.0)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(10):
            step(None, cfgs)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        selectors[name] = {"value": job_throughput(ws, flops, 10, max_over_ranks(e0.elapsed_time(e1))),
                           "live_geomean": float(np.exp(np.mean(np.log(r))))}

    # End to end from pinned host buffers through gemm_host_pipeline.
    hosts = []
    h2d = d2h = 0
    for sh, (A, B, C, lda, ldb, ldc) in zip(shapes, bufs):
        hA, hB = A.cpu().pin_memory(), B.cpu().pin_memory()
        hC = torch.empty(C.numel(), dtype=torch.float32).pin_memory()
        hosts.append((hA, hB, hC))
        h2d += hA.numel() * hA.element_size() + hB.numel() * hB.element_size()
        d2h += hC.numel() * 4
    # One pipelined call per step: the library uploads on its copy stream, runs
    # each selected GEMM on `stream` and downloads on a second copy stream, so
    # the host link carries uploads and downloads while the GPU computes.
    probs = ks.host_problems([dict(transA=sh.transA, transB=sh.transB, M=sh.M, N=sh.N, K=sh.K, batch=sh.batch,
                                   alpha=1.0, beta=0.0, A_host=hA, lda=lda, B_host=hB, ldb=ldb, C_host=hC, ldc=ldc,
                                   A_dev=A, B_dev=B, C_dev=C)
                              for sh, (A, B, C, lda, ldb, ldc), (hA, hB, hC) in zip(shapes, bufs, hosts)])
    ks.gemm_host_pipeline(handle, probs, stream)  # warm-up
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.steps):
        ks.gemm_host_pipeline(handle, probs, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_e2e = max_over_ranks(e0.elapsed_time(e1))
    e2e = job_throughput(ws, flops, args.steps, ms_e2e)

    tc = tc_families(args, ks, tune, shapes, te, bufs, stream, dev) if not args.no_tc else None
    tc_large = tc_large_shapes(ks) if not args.no_tc else None
    fp32_large = fp32_large_shape(ks) if not args.no_tc else None
    grouped = grouped_launch(ks, tune) if not args.no_tc else None
    vgg16 = vgg16_inference(ks) if not args.no_tc else None
    c0 = single_gemm_256(ks, tune)
    serving = mlp_serving(ks, tune, dep)

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu:
        from oracle import gemm as og
        v, desc, _ = cpu_oracle_sample(shapes, args.ref_budget, og.max_threads())
        cpu = {"value": v, "unit": "TFLOP/s", "cores": og.max_threads(), "kind": "oracle", "sample": desc,
               "details": cpu_details(og.max_threads())}
    clocks = clk.summary()
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        t = json.load(open(tp)).get(str(dom))
        traffic = t.get("bytes_per_launch") if t else None
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "family": "FP32 SIMT", "deployed_kernels": len(dep["config_ids"]),
                   "selector": f"decision tree {dep['meta']['tree']}", "shapes_per_step": len(shapes),
                   "gflop_per_step": flops / 1e9, "l2": "inputs 7 GB per step, larger than L2",
                   "deployment": os.path.relpath(dep_path, ROOT)},
        "pct_of_exhaustive_optimum": {"live": live, "sweep_table_test_split": dep["meta"]["scores"]["tree"]},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic, "kernel_config": dom,
                     "kernel_params": ks.config_params(dom), "share_of_step": dom_share},
        "e2e": {"value": e2e, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "selectors": selectors,
        "tc": tc,
        "tc_large": tc_large,
        "fp32_large": fp32_large,
        "grouped": grouped,
        "vgg16": vgg16,
        "single_gemm_256": c0,
        "mlp_serving": serving,
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def tc_families(args, ks, tune, shapes, te, bufs, stream, dev):
    """The same held-out shapes with each tensor-core family's deployed tree
    (and the FP32-input class whose deployment mixes SIMT and split-BF16x3
    kernels, "f32mix"):
    selected-kernel TFLOP/s (untimed warm-up, then timed steps) and the live
    share of the family's per-shape exhaustive optimum."""
    import torch
    out = {}
    for name, fam in (("tf32", ks.PREC_TF32), ("f32x3", ks.PREC_F32X3), ("bf16", ks.PREC_BF16),
                      ("f32mix", ks.PREC_F32)):
        dpath = os.path.join(DEPLOY, f"{name}.json")
        if not os.path.exists(dpath):
            continue
        dep = json.load(open(dpath))
        h = ks.Handle(dep)
        _, perf, ids, _ = tune.load_table(os.path.join(DEPLOY, f"table_{name}.npz"))
        best = [ids[int(np.argmax(perf[i]))] for i in te]
        fb = bufs if fam != ks.PREC_BF16 else [tune.alloc_inputs(sh, fam, 3000 + i) for i, sh in enumerate(shapes)]

        def run(cfgs=None, events=None, st=stream):
            for i, (sh, (A, B, C, lda, ldb, ldc)) in enumerate(zip(shapes, fb)):
                if events is not None:
                    events[i][0].record(st)
                if cfgs is None:
                    ks.gemm(h, sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, A, lda, B, ldb, 0.0, C, ldc, sh.batch, st)
                else:
                    ks.gemm_with_config(cfgs[i], sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, A, lda, B, ldb, 0.0, C,
                                        ldc, sh.batch, st)
                if events is not None:
                    events[i][1].record(st)

        def per_launch(cfgs=None):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in shapes]
            run(cfgs, ev)
            torch.cuda.synchronize(dev)
            return np.array([a.elapsed_time(b) for a, b in ev])

        for _ in range(args.warmup):
            run()
        sel = np.median([per_launch() for _ in range(3)], axis=0)
        run(best)  # loads the kernels the deployment does not use
        exh = np.median([per_launch(best) for _ in range(3)], axis=0)
        ratio = np.minimum(exh / sel, 1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_push(f"timed_{name}")  # lets a profiler select this family's timed steps
        e0.record(stream)
        for _ in range(args.steps):
            run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
        ms = e0.elapsed_time(e1) / args.steps
        flops = sum(sh.flops for sh in shapes)
        # The same step captured once in a CUDA graph (kernels selected at capture) and replayed.
        side = torch.cuda.Stream(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            run(st=side)
        with torch.cuda.stream(side):
            g.replay()
            torch.cuda.synchronize(dev)
            e0.record(side)
            for _ in range(args.steps):
                g.replay()
            e1.record(side)
        torch.cuda.synchronize(dev)
        ms_graph = e0.elapsed_time(e1) / args.steps
        out[name] = {"value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
                     "graph_value": flops / (ms_graph * 1e-3) / 1e12,
                     "pct_of_exhaustive_optimum": {"live_geomean": float(np.exp(np.mean(np.log(ratio)))),
                                                   "sweep_table_test_split": dep["meta"]["scores"]["tree"]["geomean"]},
                     "deployed_kernels": len(dep["config_ids"]),
                     "inputs": "bf16" if fam == ks.PREC_BF16 else "f32",
                     "accuracy": {"tf32": "<= 5e-3", "f32x3": "<= 1e-5 on this data (worst case 3*2^-16)",
                                  "bf16": "<= 2e-2 (bf16 inputs)",
                                  "f32mix": "FP32 SIMT or split-BF16x3, <= 1e-5 on this data"}[name]}
        if name == "f32mix":
            out[name]["families_deployed"] = sorted({ks.family_of(c) for c in dep["config_ids"]})
        if fb is not bufs:
            del fb
    return out


def measured_peaks() -> tuple[float, str]:
    """Dense BF16 tensor peak (TFLOP/s) for a kernel timed in isolation: the
    burst cuBLAS figure measured on the GB300s when the file is
    present, else the recorded fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    return 1900.0, "fallback (1.9 PFLOP/s bf16 burst)"


def tc_large_shapes(ks, n: int = 8192, reps: int = 10, warmup: int = 3):
    """The tensor-core families on large shapes: n^3 NN and NT through gemm()
    with each family's deployed handle (its decision tree picks the kernel),
    CUDA-event timed over `reps` back-to-back launches after `warmup`; every
    operand is 256 MB (FP32) or 128 MB (BF16), so the inputs exceed L2.  Each
    line also gives the fastest of the family's configs on the same product
    and the roofline fraction: BF16 against the measured dense BF16 peak, TF32
    against that peak times the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s),
    split-BF16 x3 as delivered FP32-accurate flops against the BF16 peak / 3
    (three BF16 products per product)."""
    import torch
    bf16_peak, src = measured_peaks()
    peaks = {"bf16": bf16_peak, "tf32": bf16_peak * 1.1 / 2.25, "f32x3": bf16_peak / 3}
    flops = 2.0 * n ** 3
    A32 = torch.empty(n * n, device="cuda")
    B32 = torch.empty(n * n, device="cuda")
    ks.fill_uniform(A32, n, n, n, 1, 71)
    ks.fill_uniform(B32, n, n, n, 1, 72)
    C = torch.empty(n * n, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(run):
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"shape": f"{n}^3", "peak_source": src, "timing": f"{warmup} warm-up + {reps} timed back-to-back launches"}
    for name, fam in (("bf16", ks.PREC_BF16), ("tf32", ks.PREC_TF32), ("f32x3", ks.PREC_F32X3)):
        dpath = os.path.join(DEPLOY, f"{name}.json")
        if not os.path.exists(dpath):
            continue
        h = ks.Handle(json.load(open(dpath)))
        A, B = (A32.to(torch.bfloat16), B32.to(torch.bfloat16)) if fam == ks.PREC_BF16 else (A32, B32)
        for tb in ("N", "T"):
            ms = timed(lambda: ks.gemm(h, "N", tb, n, n, n, 1.0, A, n, B, n, 0.0, C, n, 1))
            best_ms, best_id = min((timed(lambda c=c: ks.gemm_with_config(c, "N", tb, n, n, n, 1.0, A, n, B, n, 0.0,
                                                                             C, n, 1)), c)
                                   for c in ks.config_ids(fam))
            tf = flops / (ms * 1e9)
            out[f"{name}_N{tb}"] = {"value": tf, "unit": "TFLOP/s", "ms": ms,
                                    "config": ks.select_kernel(h, n, n, n, 1),
                                    "roofline": {"bound": "tensor", "achieved": tf, "peak": peaks[name],
                                                 "unit": "TFLOP/s", "frac": tf / peaks[name]},
                                    "best_config": best_id, "best_value": flops / (best_ms * 1e9)}
        del A, B
    return out


def fp32_large_shape(ks, n: int = 4096, reps: int = 10, warmup: int = 3):
    """The FP32 SIMT family on one large product: n^3 NN through gemm() with the
    FP32 deployment (its decision tree picks the kernel) and with each deployed
    kernel directly, CUDA-event timed like tc_large_shapes (A, B and C together
    exceed L2), against the FP32 FMA peak.  Beside it, as context only, the
    vendor library's FP32 GEMM on the same operands (torch.mm with TF32 off, i.e.
    cuBLAS computing in FP32 with FMA instructions), with the largest difference
    between its product and ours."""
    import torch
    dpath = os.path.join(DEPLOY, "f32.json")
    if not os.path.exists(dpath):
        return None
    dep = json.load(open(dpath))
    h = ks.Handle(dep)
    flops = 2.0 * n ** 3
    A = torch.empty(n * n, device="cuda")
    B = torch.empty(n * n, device="cuda")
    ks.fill_uniform(A, n, n, n, 1, 81)
    ks.fill_uniform(B, n, n, n, 1, 82)
    C = torch.empty(n * n, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(run):
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed(lambda: ks.gemm(h, "N", "N", n, n, n, 1.0, A, n, B, n, 0.0, C, n, 1))
    tf = flops / (ms * 1e9)
    per_cfg = {c: flops / (timed(lambda c=c: ks.gemm_with_config(c, "N", "N", n, n, n, 1.0, A, n, B, n, 0.0, C, n, 1))
                           * 1e9) for c in dep["config_ids"]}
    ks.gemm(h, "N", "N", n, n, n, 1.0, A, n, B, n, 0.0, C, n, 1)
    A2, B2 = A.view(n, n), B.view(n, n)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        lib_ms = timed(lambda: torch.mm(A2, B2))
        diff = (torch.mm(A2, B2) - C.view(n, n)).abs().max().item()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    best = max(per_cfg, key=per_cfg.get)
    return {"shape": f"{n}^3 NN", "timing": f"{warmup} warm-up + {reps} timed back-to-back launches",
            "value": tf, "unit": "TFLOP/s", "ms": ms, "config": ks.select_kernel(h, n, n, n, 1),
            "roofline": {"bound": "alu", "achieved": tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tf / FP32_PEAK_TFLOPS},
            "deployed_configs": {str(c): v for c, v in per_cfg.items()}, "best_config": best,
            "best_value": per_cfg[best],
            "vendor_fp32_gemm_context": {"what": "torch.mm, TF32 off (cuBLAS FP32 GEMM)", "value": flops / (lib_ms * 1e9),
                                         "unit": "TFLOP/s", "max_abs_diff_vs_ours": diff}}


def grouped_launch(ks, tune):
    """The 256-problem uneven group in one persistent launch per family, with
    the tile configuration the group classifier picks for it (gemm_grouped_select
    on the family's deployed selector; the autotuner's fastest config for this
    group when no selector is deployed), replayed from a CUDA graph."""
    gpath = os.path.join(DEPLOY, "grouped.json")
    if not os.path.exists(gpath):
        return None
    g = json.load(open(gpath))
    out = {}
    for name, r in g.items():
        fam = ks.PRECISIONS[name]
        probs, keep, flops = tune.grouped_workload(fam)
        cid = ks.grouped_select(ks.Handle(r["selector"]), probs) if r.get("selector") else r["config"]
        plan = ks.GroupedPlan(cid, probs)
        ms = tune.time_grouped_graph(plan, reps=20, warmup=3)
        out[name] = {"value": flops / (ms * 1e9), "unit": "TFLOP/s", "ms_per_launch": ms, "config": cid,
                     "problems": len(probs), "gflop": flops / 1e9,
                     "selector": "group tree" if r.get("selector") else "fastest on this group"}
        if r.get("selector_scores"):
            out[name]["selector_held_out_geomean"] = r["selector_scores"]["tree"]["geomean"]
        plan.close()
        if r.get("selector"):
            # The library call of the boundary, gemm_grouped(handle, problems,
            # precision, stream): selection inside the call, descriptors written
            # into the handle's workspace by the captured upload kernels on every
            # replay; captured once after a call that sizes the workspace.
            h = ks.Handle(r["selector"])
            ms_h = time_handle_call_graph(ks, h, probs, fam)
            out[name]["handle_call"] = {"value": flops / (ms_h * 1e9), "ms_per_launch": ms_h,
                                        "config": ks.grouped_select(h, probs),
                                        "note": "gemm_grouped(handle, ...) captured in a CUDA graph and replayed"}
        del keep
    return out


def time_handle_call_graph(ks, h, probs, precision, reps: int = 20, warmup: int = 3) -> float:
    """Mean ms of one replay of a CUDA graph holding one gemm_grouped(handle, ...) call."""
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ks.gemm_grouped(h, probs, precision, s)  # sizes the handle's workspace (outside the capture)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ks.gemm_grouped(h, probs, precision, s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        for _ in range(warmup):
            g.replay()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(reps):
            g.replay()
        e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def mlp_serving(ks, tune, dep, n: int = 4096, reps: int = 100):
    """The learned selector's batched inference kernel over n queued shapes
    (seeded grid shapes): microseconds per batch."""
    import torch
    if not dep.get("mlp_params"):
        return None
    h = ks.Handle({k: v for k, v in dep.items() if k != "known"})
    shapes = torch.from_numpy(tune.shape_rows(wl.shape_grid(n, 12))).cuda()
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(5):
        ks.select_kernels_batched(h, shapes, ids)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        ks.select_kernels_batched(h, shapes, ids)
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / reps
    return {"queued_shapes": n, "us_per_batch": us, "shapes_per_s": n / (us * 1e-6)}


def single_gemm_256(ks, tune, reps: int = 200):
    """The small fixed case: 256^3 NN FP32, alpha 1, beta 0, uniform[-1, 1) inputs,
    one fixed config (16x16 threads, 4x4 per thread, K-step 16, staged).  Its
    786 KB of operands and result stay in L2 across back-to-back launches, so
    it measures latency and launch overhead, reported as time, TFLOP/s and
    algorithmic GB/s."""
    import torch
    from paper_2008_13145_gb300 import workloads as wl
    sh = wl.Shape(256, 256, 256, 1, "N", "N")
    A, B, C, lda, ldb, ldc = tune.alloc_inputs(sh, ks.PREC_F32, 0)
    cid = next(c for c in ks.config_ids(ks.PREC_F32) if ks.config_params(c)[1:7] == [4, 4, 16, 16, 16, 1])
    for _ in range(10):
        ks.gemm_with_config(cid, "N", "N", 256, 256, 256, 1.0, A, lda, B, ldb, 0.0, C, ldc, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        ks.gemm_with_config(cid, "N", "N", 256, 256, 256, 1.0, A, lda, B, ldb, 0.0, C, ldc, 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    out = {"config": cid, "us_per_launch": ms * 1e3, "tflops": sh.flops / (ms * 1e9),
           "algorithmic_gbs": 3 * 256 * 256 * 4 / (ms * 1e6), "note": "back-to-back launches, L2-resident"}
    # the same product with the kernel the FP32 deployment selects
    h = ks.Handle(json.load(open(os.path.join(DEPLOY, "f32.json"))))
    for _ in range(10):
        ks.gemm(h, "N", "N", 256, 256, 256, 1.0, A, lda, B, ldb, 0.0, C, ldc, 1)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        ks.gemm(h, "N", "N", 256, 256, 256, 1.0, A, lda, B, ldb, 0.0, C, ldc, 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    out["selected"] = {"config": ks.select_kernel(h, 256, 256, 256, 1), "us_per_launch": ms * 1e3,
                       "tflops": sh.flops / (ms * 1e9)}
    return out


def vgg16_inference(ks, reps: int = 10):
    """VGG16 forward passes (im2col + selected GEMM + bias/ReLU + pooling, synthetic
    He-normal weights) with the FP32 and mixed FP32-input deployments, and in the
    paper's GEMM-batched layout (per image Cout x HW, weights shared)."""
    import torch
    from paper_2008_13145_gb300 import vgg
    out = {}
    for name, layout in (("f32", "nhwc"), ("f32mix", "nhwc"), ("f32", "batched")):
        h = ks.Handle(json.load(open(os.path.join(DEPLOY, f"{name}.json"))))
        for batch in (1, 16):
            net = vgg.VGG16(h, batch, layout=layout)
            x = torch.rand((batch, 224, 224, 3) if layout == "nhwc" else (batch, 3, 224, 224), device="cuda")
            for _ in range(3):
                net.forward(x)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                net.forward(x)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out[f"{name}{'' if layout == 'nhwc' else '_gemm_batched'}_batch{batch}"] = {"ms_per_inference": ms, "images_per_s": batch * 1e3 / ms,
                                           "tflops": net.flops / (ms * 1e9)}
            del net
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-budget", type=float, default=12.0, help="seconds of CPU oracle work per sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core, grouped and VGG16 lines")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
