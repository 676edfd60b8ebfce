"""Explicit batch strides (gemm_strided_batched) against the FP64 oracle, entry by entry.

One A shared by every batch entry (stride 0), B entries separated by NaN-filled
gaps (one gap a multiple of 16 bytes, one not, so the unvectorised loads run
too) and C entries separated by sentinel gaps that must survive.  Every kernel
family: FP32 SIMT (staged and direct), the split-K kind, TF32, BF16 and
split-BF16 x3 in two tile shapes (whose kernels pack non-contiguous batches in
their pre-pass).
Tolerances as in the per-family parity tests."""
import numpy as np
import pytest

from oracle import gemm as og
from paper_2008_13145_gb300 import workloads as wl
from tests.gpu_helpers import SENTINEL

pytestmark = pytest.mark.gpu
CASES = [("f32 staged", 369, 1e-5), ("f32 direct", 368, 1e-5), ("split-K", 2533, 1e-5),
         ("tf32", 1008, 5e-3), ("bf16", 1108, 2e-2), ("f32x3", 1208, 1e-5), ("f32x3 BN 256", 1216, 1e-5)]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.mark.parametrize("name,cid,tol", CASES)
@pytest.mark.parametrize("ta,tb,gap_b", [("N", "T", 40), ("T", "N", 37), ("N", "N", 37), ("T", "T", 40)])
def test_strided_batched(lib, torch, name, cid, tol, ta, tb, gap_b):
    ks = lib
    M, N, K, batch = 70, 90, 300, 3
    shape = wl.Shape(M, N, K, batch, ta, tb)
    if name == "split-K":
        assert ks.split_factor(cid, M, N, K, batch)[0] > 1
    A3, B3, C3 = wl.gemm_inputs(shape, seed=40, beta_nonzero=True, ld_multiple=8)
    A = A3[:1]  # one matrix for every entry
    lda, ldb, ldc = A3.shape[2], B3.shape[2], C3.shape[2]
    sB = B3.shape[1] * ldb + gap_b
    sC = M * ldc + 24
    Bf = np.full(sB * batch, np.nan, np.float32)
    Cf = np.full(sC * batch + 64, SENTINEL, np.float32)
    for b in range(batch):
        Bf[b * sB:b * sB + B3.shape[1] * ldb] = B3[b].ravel()
        c = C3[b].copy()
        c[:, N:] = SENTINEL
        Cf[b * sC:b * sC + M * ldc] = c.ravel()
    bf16 = name == "bf16"
    tA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    tB = torch.from_numpy(Bf).cuda()
    if bf16:
        tA, tB = tA.to(torch.bfloat16), tB.to(torch.bfloat16)
    tC = torch.from_numpy(Cf).cuda()
    ks.gemm_strided_batched_with_config(cid, ta, tb, M, N, K, 0.75, tA, lda, 0, tB, ldb, sB, -0.5, tC, ldc, sC, batch)
    torch.cuda.synchronize()
    got = tC.cpu().numpy()
    Ah = tA.float().cpu().numpy().reshape(A.shape)
    Bh = tB.float().cpu().numpy()
    for b in range(batch):
        Cb = got[b * sC:b * sC + M * ldc].reshape(M, ldc)
        assert np.all(Cb[:, N:] == SENTINEL), "write into ldc padding"
        assert np.all(got[b * sC + M * ldc:(b + 1) * sC] == SENTINEL), "write into the gap after an entry"
        Bb = Bh[b * sB:b * sB + B3.shape[1] * ldb].reshape(1, B3.shape[1], ldb)
        ref, den = og.gemm(ta, tb, M, N, K, 0.75, Ah, Bb, -0.5, C3[b:b + 1])
        err = og.error_ratio(Cb[None, :, :N], ref, den)
        assert err <= tol, (name, b, err)
    assert np.all(got[sC * batch:] == SENTINEL)
    assert ks.device_status() == 0


def test_strided_through_handle(lib, torch):
    """gemm_strided_batched selects with the deployment, like gemm()."""
    import json
    import os
    ks = lib
    dep = json.load(open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                      "paper_2008_13145_gb300", "deploy", "f32.json")))
    h = ks.Handle(dep)
    M, N, K, batch = 64, 50, 200, 4
    rng = np.random.default_rng(41)
    A = rng.uniform(-1, 1, (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (batch, K, N)).astype(np.float32)
    C = torch.full((batch, M, N), float("nan"), device="cuda")
    ks.gemm_strided_batched(h, "N", "N", M, N, K, 1.0, torch.from_numpy(A).cuda(), K, 0,
                            torch.from_numpy(B).cuda(), N, K * N, 0.0, C, N, M * N, batch)
    got = C.cpu().numpy()
    for b in range(batch):
        ref, den = og.gemm("N", "N", M, N, K, 1.0, A[None], B[b:b + 1])
        assert og.error_ratio(got[b:b + 1], ref, den) <= 1e-5
