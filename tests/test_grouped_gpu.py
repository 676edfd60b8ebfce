"""GPU parity of the persistent grouped tensor-core launch (one launch for an
uneven group of GEMMs) against the FP64 oracle, eager and replayed from a
CUDA graph.  Tolerances as for the single-GEMM families."""
import json
import os

import numpy as np
import pytest

from oracle import gemm as og
from paper_2008_13145_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
FAMILIES = {"tf32": (1, 5e-3), "bf16": (2, 2e-2), "f32x3": (3, 1e-5)}
DEPLOY = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2008_13145_gb300", "deploy")


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def build_group(torch, shapes, fam, seed, ld_multiple=8):
    bf16 = fam == "bf16"
    probs, host = [], []
    for i, sh in enumerate(shapes):
        A, B, C0 = wl.gemm_inputs(sh, seed=seed + i, ld_multiple=ld_multiple, beta_nonzero=(i % 3 == 0))
        tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        if bf16:
            tA, tB = tA.to(torch.bfloat16), tB.to(torch.bfloat16)
        C = torch.from_numpy(np.where(np.isnan(C0), 0, C0).astype(np.float32)).cuda()
        beta = 0.5 if i % 3 == 0 else 0.0
        probs.append(dict(M=sh.M, N=sh.N, K=sh.K, transA=sh.transA, transB=sh.transB, alpha=1.0 - 0.1 * (i % 4),
                          beta=beta, A=tA, lda=A.shape[2], B=tB, ldb=B.shape[2], C=C, ldc=C0.shape[2]))
        host.append((tA.float().cpu().numpy().reshape(A.shape), tB.float().cpu().numpy().reshape(B.shape), C0))
    return probs, host


def check_group(probs, host, shapes, tol, full=True):
    worst = 0.0
    for q, (A, B, C0), sh in zip(probs, host, shapes):
        C = q["C"].cpu().numpy().reshape(sh.M, -1)[:, :sh.N]
        if full:
            ref, den = og.gemm(sh.transA, sh.transB, sh.M, sh.N, sh.K, q["alpha"], A, B, q["beta"], C0)
            err = og.error_ratio(C[None], ref, den)
        else:
            pos = wl.band_positions(sh, 64, 64, seed=1)  # meets every output tile
            ref, den = og.gemm_entries(sh.transA, sh.transB, sh.M, sh.N, sh.K, q["alpha"], A, B, q["beta"], C0, pos,
                                       nthreads=og.max_threads())
            err = og.error_ratio(C[pos[:, 1], pos[:, 2]], ref, den)
        worst = max(worst, err)
    assert worst <= tol, worst
    return worst


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_small_uneven_group_all_layouts(lib, torch, fam):
    rng = np.random.default_rng(1)
    shapes = [wl.Shape(int(rng.integers(1, 300)), int(rng.integers(1, 300)), int(rng.integers(16, 300)), 1,
                       "NT"[i % 2], "NT"[(i // 2) % 2]) for i in range(24)]
    probs, host = build_group(torch, shapes, fam, 100, ld_multiple=1 if fam == "tf32" else 8)
    cid = lib.config_ids(FAMILIES[fam][0])[3]  # BN 128, 2 stages
    lib.gemm_grouped_with_config(cid, probs)
    check_group(probs, host, shapes, FAMILIES[fam][1])
    assert lib.device_status() == 0


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_group_of_256_in_a_cuda_graph(lib, torch, fam):
    """The uneven 256-problem workload (M, N, K log-uniform in [32, 4096]): a
    plan captured in a CUDA graph and replayed gives the eager result."""
    shapes = wl.grouped_problems(256, 3)
    probs, host = build_group(torch, shapes, fam, 1000)
    cid = lib.config_ids(FAMILIES[fam][0])[8]  # BN 256, 4 stages
    plan = lib.GroupedPlan(cid, probs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.run(s)
    torch.cuda.synchronize()
    eager = [q["C"].clone() for q in probs]
    for q, (_, _, C0) in zip(probs, host):  # reset C (beta != 0 problems read it)
        q["C"].copy_(torch.from_numpy(np.where(np.isnan(C0), 0, C0).astype(np.float32)).cuda())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(s)
    g.replay()
    torch.cuda.synchronize()
    for q, e in zip(probs, eager):
        assert torch.equal(q["C"], e)
    check_group(probs, host, shapes, FAMILIES[fam][1], full=False)
    assert lib.device_status() == 0


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_handle_call_selects_and_is_captured_in_a_cuda_graph(lib, torch, fam):
    """gemm_grouped(handle, problems, precision, stream): the family's deployed
    group selector picks the tile config inside the call.  After one eager
    call (which sizes the handle's workspace) the call is captured in a CUDA
    graph; another group then runs through the same handle and overwrites the
    workspace, and the replay still equals the eager result bit for bit,
    because the graph carries its own descriptors.  Both match the oracle."""
    ks = lib
    sel = json.load(open(os.path.join(DEPLOY, "grouped.json")))[fam]["selector"]
    h = ks.Handle(sel)
    prec = FAMILIES[fam][0]
    rng = np.random.default_rng(7)
    shapes = [wl.Shape(int(rng.integers(1, 400)), int(rng.integers(1, 400)), int(rng.integers(1, 300)), 1,
                       "NT"[i % 2], "NT"[(i // 2) % 2]) for i in range(40)]
    probs, host = build_group(torch, shapes, fam, 2000, ld_multiple=1 if fam == "tf32" else 8)
    assert ks.family_of(ks.grouped_select(h, probs)) == prec
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ks.gemm_grouped(h, probs, prec, s)
    torch.cuda.synchronize()
    eager = [q["C"].clone() for q in probs]
    check_group(probs, host, shapes, FAMILIES[fam][1])

    def reset(ps, hs):
        for q, (_, _, C0) in zip(ps, hs):  # beta != 0 problems read C
            q["C"].copy_(torch.from_numpy(np.where(np.isnan(C0), 0, C0).astype(np.float32)).cuda())

    reset(probs, host)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ks.gemm_grouped(h, probs, prec, s)
    # a smaller group through the same handle between capture and replay
    others = [wl.Shape(int(rng.integers(1, 200)), int(rng.integers(1, 200)), int(rng.integers(1, 200)), 1, "N", "T")
              for _ in range(8)]
    oprobs, ohost = build_group(torch, others, fam, 3000)
    with torch.cuda.stream(s):
        ks.gemm_grouped(h, oprobs, prec, s)
    torch.cuda.synchronize()
    check_group(oprobs, ohost, others, FAMILIES[fam][1])
    with torch.cuda.stream(s):
        g.replay()
    torch.cuda.synchronize()
    for q, e in zip(probs, eager):
        assert torch.equal(q["C"], e)
    assert ks.device_status() == 0


def test_handle_call_under_capture_never_allocates(lib, torch):
    """A handle whose workspace is too small for the group refuses the call
    under capture (GEMM_ERR_UNSUPPORTED, nothing enqueued) instead of
    allocating; after gemm_grouped_reserve the same capture succeeds."""
    ks = lib
    sel = json.load(open(os.path.join(DEPLOY, "grouped.json")))["bf16"]["selector"]
    h = ks.Handle(sel)  # a fresh handle: no workspace yet
    shapes = [wl.Shape(150 + 10 * i, 130, 64 + 8 * i, 1, "N", "N") for i in range(6)]
    probs, host = build_group(torch, shapes, "bf16", 4000)
    ks.gemm_with_config(1100, "N", "T", 1, 1, 1, 1.0, probs[0]["A"], 1, probs[0]["B"], 1, 0.0,
                        torch.empty(1, device="cuda"), 1, 1)  # the device's status word exists
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g = torch.cuda.CUDAGraph()
        g.capture_begin()
        try:
            st = ks._lib.gemm_grouped(h.value, len(probs), ks._problems(probs), ks.PREC_BF16, ks.stream_handle(s))
        finally:
            g.capture_end()
    assert st == -2
    ks.gemm_grouped_reserve(h, probs, ks.PREC_BF16)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s):
        ks.gemm_grouped(h, probs, ks.PREC_BF16, s)
    with torch.cuda.stream(s):
        g2.replay()
    torch.cuda.synchronize()
    check_group(probs, host, shapes, FAMILIES["bf16"][1])


def test_plan_rejects_bad_problems(lib, torch):
    A = torch.zeros(64, device="cuda")
    good = dict(M=4, N=4, K=4, A=A, lda=4, B=A, ldb=4, C=A, ldc=4)
    with pytest.raises(lib.KSelectError):
        lib.GroupedPlan(1000, [dict(good, K=0)])
    with pytest.raises(lib.KSelectError):
        lib.GroupedPlan(1000, [dict(good, lda=3)])
    with pytest.raises(lib.KSelectError):
        lib.GroupedPlan(7, [good])  # a SIMT config cannot run a grouped launch
