"""Run one kernel configuration on one GEMM size a few times (an ncu target).

    python -m paper_2008_13145_gb300.profile_case --config 531 --shape 4096 4096 4096 1 N N --reps 3
    python -m paper_2008_13145_gb300.profile_case --grouped 1216 --reps 2

Inputs are filled on the device by the library; nothing is checked here
(parity lives in tests/).  Prints the CUDA-event time of the last launch.
"""
from __future__ import annotations

import argparse

from . import tune
from . import workloads as wl


def main(argv=None):
    import torch
    from . import kselect as ks
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int)
    ap.add_argument("--shape", nargs=6, metavar=("M", "N", "K", "BATCH", "TA", "TB"))
    ap.add_argument("--grouped", type=int, help="config id: run the 256-problem grouped workload")
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.grouped is not None:
        fam = ks.family_of(a.grouped)
        probs, keep = [], []
        for i, sh in enumerate(wl.grouped_problems(256, 3)):
            A, B, C, lda, ldb, ldc = tune.alloc_inputs(sh, fam, 500 + i)
            keep.append((A, B, C))
            probs.append(dict(M=sh.M, N=sh.N, K=sh.K, transA="N", transB="T", A=A, lda=lda, B=B, ldb=ldb, C=C,
                              ldc=ldc))
        plan = ks.GroupedPlan(a.grouped, probs)
        flops = sum(2 * q["M"] * q["N"] * q["K"] for q in probs)
        for _ in range(a.reps):
            e0.record()
            plan.run()
            e1.record()
    else:
        M, N, K, b = (int(x) for x in a.shape[:4])
        sh = wl.Shape(M, N, K, b, a.shape[4], a.shape[5])
        A, B, C, lda, ldb, ldc = tune.alloc_inputs(sh, ks.family_of(a.config), 1)
        flops = sh.flops
        for _ in range(a.reps):
            e0.record()
            ks.gemm_with_config(a.config, sh.transA, sh.transB, M, N, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, b)
            e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print(f"{ms:.4f} ms  {flops / (ms * 1e9):.1f} TFLOP/s")


if __name__ == "__main__":
    main()
