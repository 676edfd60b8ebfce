"""Run one kernel configuration on one GEMM size a few times (an ncu target).

    python -m paper_2008_13145_gb300.profile_case --config 531 --shape 4096 4096 4096 1 N N --reps 3
    python -m paper_2008_13145_gb300.profile_case --grouped 1216 --reps 2
    python -m paper_2008_13145_gb300.profile_case --vendor-fp32 --shape 4096 4096 4096 1 N N --reps 2

--vendor-fp32 runs the vendor library's FP32 GEMM instead (torch.mm with TF32
off, a batch-1 NN product only): a reference point for profiling, not part of
the library.

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
    ap.add_argument("--vendor-fp32", action="store_true", help="time torch.mm (cuBLAS FP32, TF32 off) instead")
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
    elif a.vendor_fp32:
        M, N, K, b = (int(x) for x in a.shape[:4])
        if b != 1 or a.shape[4] != "N" or a.shape[5] != "N":
            raise SystemExit("--vendor-fp32 takes batch-1 NN shapes only")
        A = torch.empty(M * K, device="cuda")
        B = torch.empty(K * N, device="cuda")
        ks.fill_uniform(A, M, K, K, 1, 1)
        ks.fill_uniform(B, K, N, N, 1, 2)
        A2, B2 = A.view(M, K), B.view(K, N)
        torch.backends.cuda.matmul.allow_tf32 = False
        flops = 2.0 * M * N * K
        for _ in range(a.reps):
            e0.record()
            torch.mm(A2, B2)
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
