"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The 200 held-out shapes of the 1,000-shape grid (M, N, K up to 4096, batch up to
16, every transpose), each GEMM selected by the committed deployment through the
handle exactly as the bench's timed step does (plain FP32 kernels and the split-K
kind included).  Inputs are drawn on the host (seeded) and uploaded; the oracle
evaluates sampled outputs one by one: per batch entry one seeded row in every
band of 64 rows x all columns plus one seeded column in every band of 64
columns x all rows, so every output tile of 64 x 64 or more is met."""
import json
import os

import numpy as np
import pytest

from oracle import gemm as og
from paper_2008_13145_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEPLOY = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2008_13145_gb300", "deploy")
CASES = [("f32.json", 1e-5, False), ("f32mix.json", 1e-5, False), ("f32x3.json", 1e-5, False), ("tf32.json", 5e-3, False),
         ("bf16.json", 2e-2, True)]
# (deployment, tolerance of its precision class, BF16 inputs)


def test_bench_workload_sampled(lib):
    import torch
    ks = lib
    handles = [(name, tol, bf16, ks.Handle(json.load(open(os.path.join(DEPLOY, name))))) for name, tol, bf16 in CASES]
    g = wl.shape_grid(1000, 1)
    _, te = wl.train_test_split(1000, 1)
    worst = {name: 0.0 for name, _, _ in CASES}
    nthreads = og.max_threads()
    for n, i in enumerate(te):
        sh = g[i]
        A, B, _ = wl.gemm_inputs(sh, seed=5000 + n, ld_multiple=8)
        pos = wl.band_positions(sh, 64, 64, seed=n)
        ldc = wl.round_up(sh.N, 4)
        refs = {}  # the oracle's entries, once per input type
        for name, tol, bf16, h in handles:
            tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            Ah, Bh = A, B
            if bf16:
                tA, tB = tA.to(torch.bfloat16), tB.to(torch.bfloat16)
                Ah = tA.float().cpu().numpy().reshape(A.shape)
                Bh = tB.float().cpu().numpy().reshape(B.shape)
            C = torch.full((sh.batch, sh.M, ldc), float("nan"), device="cuda")
            ks.gemm(h, sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, tA, A.shape[2], tB, B.shape[2], 0.0, C, ldc,
                    sh.batch)
            got = C.cpu().numpy()[pos[:, 0], pos[:, 1], pos[:, 2]]
            if bf16 not in refs:
                refs[bf16] = og.gemm_entries(sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, Ah, Bh, 0.0, None, pos,
                                             nthreads=nthreads)
            ref, den = refs[bf16]
            err = og.error_ratio(got, ref, den)
            assert err <= tol, (name, sh, ks.select_kernel(h, sh.M, sh.N, sh.K, sh.batch), err)
            worst[name] = max(worst[name], err)
            del tA, tB, C
    assert ks.device_status() == 0
    print("worst sampled error ratio over the 200 shapes:", worst)
