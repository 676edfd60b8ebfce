"""GPU parity of the FP32 SIMT family against the FP64 oracle, through the C-ABI.

Tolerance: max |C - C_ref| / (|alpha||A||B| + |beta||C0|) <= 1e-5 for FP32.
Every output buffer is surrounded by sentinel guard regions (before, after and
in the ldc padding) that must survive each launch; beta = 0 launches start
from NaN-filled C, so reading C when beta == 0 shows up as NaN."""
import numpy as np
import pytest

from oracle import gemm as og
from paper_2008_13145_gb300 import workloads as wl
from tests.gpu_helpers import GUARD, SENTINEL, Out

pytestmark = pytest.mark.gpu
TOL_F32 = 1e-5
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


def pad_c(C0, ldc_extra=3):
    b, M, ldc = C0.shape
    out = np.full((b, M, ldc + ldc_extra), SENTINEL, np.float32)
    out[:, :, :ldc] = C0
    out[:, :, C0.shape[2]:] = SENTINEL
    return out


def run_case(ks, torch, cid, shape, alpha, beta, A, B, C0, N_valid=None):
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C0p = C0.copy()
    C0p[:, :, shape.N:] = SENTINEL
    out = Out(torch, C0p, beta, shape.N)
    ks.gemm_with_config(cid, shape.transA, shape.transB, shape.M, shape.N, shape.K, alpha, tA, A.shape[2], tB,
                        B.shape[2], beta, out.ptr, C0p.shape[2], shape.batch)
    torch.cuda.synchronize()
    return out.result(shape.N)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def find_cfg(ks, tm, tn, wx, wy, bk, staged):
    return next(c for c in ks.config_ids(ks.PREC_F32) if ks.config_params(c)[1:7] == [tm, tn, wx, wy, bk, staged])


def test_single_gemm_256(lib, torch):
    """256^3 NN, alpha 1, beta 0, uniform[-1,1] seed 0; 16x16 threads, 4x4 per thread, K-step 16, staged."""
    ks = lib
    shape = wl.Shape(256, 256, 256, 1, "N", "N")
    A, B, C0 = wl.gemm_inputs(shape, seed=0)
    cid = find_cfg(ks, 4, 4, 16, 16, 16, 1)
    C = run_case(ks, torch, cid, shape, 1.0, 0.0, A, B, C0)
    ref, den = og.gemm("N", "N", 256, 256, 256, 1.0, A, B)
    err = og.error_ratio(C, ref, den)
    assert err <= TOL_F32, err
    tC = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    gerr = ks.error_check(tC, torch.from_numpy(ref).cuda(), torch.from_numpy(den).cuda(), rows=256, cols=256,
                          batch=1, ldc=256, strideC=256 * 256)
    assert gerr == pytest.approx(err, rel=1e-12, abs=0)


@pytest.mark.parametrize("ta,tb", TRANS)
def test_every_config_ragged(lib, torch, ta, tb):
    """All 576 configs on a ragged batched shape, alpha -0.5, beta 0.25, NaN padding in A and B."""
    ks = lib
    shape = wl.Shape(37, 45, 29, 2, ta, tb)
    A, B, C0 = wl.gemm_inputs(shape, seed=11, beta_nonzero=True, ld_multiple=8)
    ref, den = og.gemm(ta, tb, shape.M, shape.N, shape.K, -0.5, A, B, 0.25, C0)
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C0p = C0.copy()
    C0p[:, :, shape.N:] = SENTINEL
    bad = []
    for cid in ks.config_ids(ks.PREC_F32):
        out = Out(torch, C0p, 0.25, shape.N)
        ks.gemm_with_config(cid, ta, tb, shape.M, shape.N, shape.K, -0.5, tA, A.shape[2], tB, B.shape[2], 0.25,
                            out.ptr, C0p.shape[2], shape.batch)
        err = og.error_ratio(out.result(shape.N), ref, den)
        if not err <= TOL_F32:
            bad.append((cid, ks.config_params(cid), err))
    assert not bad, bad[:10]


def test_beta_zero_does_not_read_c(lib, torch):
    ks = lib
    shape = wl.Shape(50, 33, 40, 3, "T", "N")
    A, B, C0 = wl.gemm_inputs(shape, seed=12)
    ref, den = og.gemm("T", "N", shape.M, shape.N, shape.K, 2.0, A, B)
    for cid in range(0, 576, 5):
        C = run_case(ks, torch, cid, shape, 2.0, 0.0, A, B, C0)
        assert og.error_ratio(C, ref, den) <= TOL_F32, cid


@pytest.mark.parametrize("ta,tb", TRANS)
def test_integer_inputs_exact(lib, torch, ta, tb):
    """|a|,|b| <= 8 with K <= 4096 keeps every partial sum an integer below 2^24: exact in FP32."""
    ks = lib
    shape = wl.Shape(70, 66, 300, 2, ta, tb)
    A, B, C0 = wl.gemm_inputs(shape, seed=13, kind="integer", bound=8, beta_nonzero=True)
    ref, _ = og.gemm(ta, tb, shape.M, shape.N, shape.K, 1.0, A, B, 1.0, C0)
    for cid in range(3, 576, 11):
        C = run_case(ks, torch, cid, shape, 1.0, 1.0, A, B, C0)
        assert np.array_equal(C.astype(np.float64), ref), cid


def test_several_tiles_with_tails(lib, torch):
    ks = lib
    shape = wl.Shape(300, 290, 77, 1, "N", "N")
    A, B, C0 = wl.gemm_inputs(shape, seed=14, beta_nonzero=True)
    ref, den = og.gemm("N", "N", shape.M, shape.N, shape.K, 1.0, A, B, -1.0, C0)
    big = [c for c in ks.config_ids(ks.PREC_F32) if ks.config_params(c)[1] * ks.config_params(c)[4] >= 64]
    for cid in big[::3]:
        C = run_case(ks, torch, cid, shape, 1.0, -1.0, A, B, C0)
        assert og.error_ratio(C, ref, den) <= TOL_F32, cid


def test_degenerate_sizes(lib, torch):
    ks = lib
    for (M, N, K) in [(1, 1, 1), (1, 300, 5), (300, 1, 5), (2, 3, 1), (5, 7, 4099)]:
        shape = wl.Shape(M, N, K, 2, "N", "T")
        A, B, C0 = wl.gemm_inputs(shape, seed=15, beta_nonzero=True)
        ref, den = og.gemm("N", "T", M, N, K, 1.0, A, B, 0.5, C0)
        for cid in (0, 101, 287, 431, 575):
            C = run_case(ks, torch, cid, shape, 1.0, 0.5, A, B, C0)
            assert og.error_ratio(C, ref, den) <= TOL_F32, (M, N, K, cid)
    # K == 0: C = beta * C
    shape = wl.Shape(9, 10, 0, 1, "N", "N")
    C0 = wl.uniform_matrix(9, 12, 12, 1, 3, 3)
    out = Out(torch, pad_c(C0[:, :, :12], 0), 0.5, 10)
    ks.gemm_with_config(7, "N", "N", 9, 10, 0, 1.0, 0, 1, 0, 1, 0.5, out.ptr, 12, 1)
    torch.cuda.synchronize()
    f = out.flat.cpu().numpy()[GUARD:GUARD + 9 * 12].reshape(9, 12)
    assert np.array_equal(f[:, :10], np.float32(0.5) * C0[0, :, :10])


def test_unaligned_operands_use_scalar_path(lib, torch):
    """Pointers 4 bytes past a 16-byte boundary and odd leading dimensions."""
    ks = lib
    M, N, K = 45, 39, 51
    rng = np.random.default_rng(16)
    A = rng.uniform(-1, 1, (M, K + 1)).astype(np.float32)
    B = rng.uniform(-1, 1, (K, N + 2)).astype(np.float32)
    ref, den = og.gemm("N", "N", M, N, K, 1.0, A[None], B[None])
    fa = torch.from_numpy(np.concatenate([[0.0], A.ravel()]).astype(np.float32)).cuda()
    fb = torch.from_numpy(np.concatenate([[0.0], B.ravel()]).astype(np.float32)).cuda()
    for cid in (1, 143, 289, 575):
        C = torch.full((M * (N + 1) + 1,), float("nan"), device="cuda")
        ks.gemm_with_config(cid, "N", "N", M, N, K, 1.0, fa.data_ptr() + 4, K + 1, fb.data_ptr() + 4, N + 2, 0.0,
                            C.data_ptr() + 4, N + 1, 1)
        torch.cuda.synchronize()
        got = C.cpu().numpy().ravel()[1:1 + M * (N + 1)].reshape(M, N + 1)[:, :N]
        assert og.error_ratio(got[None], ref, den) <= TOL_F32, cid


def test_full_size_sampled(lib, torch):
    """Largest grid-size shape in the staged 8x8-per-thread config, checked on sampled entries by the GPU reduction."""
    ks = lib
    shape = wl.Shape(4096, 3000, 4096, 2, "T", "N")
    A, B, _ = wl.gemm_inputs(shape, seed=17)
    cid = find_cfg(ks, 8, 8, 16, 16, 8, 1)
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.empty((2, 4096, 3000), device="cuda")
    ks.gemm_with_config(cid, "T", "N", 4096, 3000, 4096, 1.0, tA, A.shape[2], tB, B.shape[2], 0.0, C, 3000, 2)
    pos = wl.sample_positions(shape, 8, 8, seed=3)
    ref, den = og.gemm_entries("T", "N", 4096, 3000, 4096, 1.0, A, B, 0.0, None, pos, nthreads=og.max_threads())
    gerr = ks.error_check(C, torch.from_numpy(ref).cuda(), torch.from_numpy(den).cuda(), pos=torch.from_numpy(pos).cuda(),
                          ldc=3000, strideC=4096 * 3000)
    host = og.error_ratio(C.cpu().numpy()[pos[:, 0], pos[:, 1], pos[:, 2]], ref, den)
    assert gerr <= TOL_F32 and gerr == pytest.approx(host, rel=1e-12)


def test_error_check_kernel_semantics(lib, torch):
    ks = lib
    rng = np.random.default_rng(18)
    C = rng.standard_normal((3, 20, 24)).astype(np.float32)
    ref = C.astype(np.float64)[:, :, :21] + rng.standard_normal((3, 20, 21)) * 1e-6
    den = np.abs(rng.standard_normal((3, 20, 21))) + 0.1
    tC = torch.from_numpy(C).cuda()
    e = ks.error_check(tC, torch.from_numpy(ref).cuda(), torch.from_numpy(den).cuda(), rows=20, cols=21, batch=3,
                       ldc=24, strideC=480)
    assert e == pytest.approx(og.error_ratio(C[:, :, :21], ref, den), rel=1e-14)
    den[1, 2, 3] = 0.0
    ref[1, 2, 3] = C[1, 2, 3]
    e = ks.error_check(tC, torch.from_numpy(ref).cuda(), torch.from_numpy(den).cuda(), rows=20, cols=21, batch=3,
                       ldc=24, strideC=480)
    assert np.isfinite(e)
    ref[1, 2, 3] += 1e-3
    e = ks.error_check(tC, torch.from_numpy(ref).cuda(), torch.from_numpy(den).cuda(), rows=20, cols=21, batch=3,
                       ldc=24, strideC=480)
    assert e == float("inf")


def test_gemm_host_round_trip(lib, torch):
    """gemm_host: pinned host inputs copied to device staging, selected kernel, C copied back."""
    ks = lib
    h = ks.Handle({"precision": 0, "config_ids": [531, 173], "nodes": [
        {"feature": 0, "threshold": 100.5, "left": 1, "right": 2, "label": 0},
        {"feature": -1, "threshold": 0, "left": -1, "right": -1, "label": 1},
        {"feature": -1, "threshold": 0, "left": -1, "right": -1, "label": 0}]})
    for shape, beta in ((wl.Shape(77, 130, 45, 3, "T", "N"), 0.5), (wl.Shape(300, 64, 200, 1, "N", "T"), 0.0)):
        A, B, C0 = wl.gemm_inputs(shape, seed=21, beta_nonzero=beta != 0)
        hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
        hC = torch.from_numpy(np.where(np.isnan(C0), 0, C0).astype(np.float32)).pin_memory()
        dA, dB, dC = torch.empty_like(hA, device="cuda"), torch.empty_like(hB, device="cuda"), \
            torch.empty_like(hC, device="cuda")
        ks.gemm_host(h, shape.transA, shape.transB, shape.M, shape.N, shape.K, 1.0, hA, A.shape[2], hB, B.shape[2],
                     beta, hC, C0.shape[2], shape.batch, dA, dB, dC)
        torch.cuda.synchronize()
        ref, den = og.gemm(shape.transA, shape.transB, shape.M, shape.N, shape.K, 1.0, A, B, beta,
                           np.where(np.isnan(C0), 0, C0))
        assert og.error_ratio(hC.numpy()[:, :, :shape.N], ref, den) <= TOL_F32


# ---------------------------------------------------------------- split-K kind
def split_ids(ks):
    return [c for c in ks.config_ids(ks.PREC_F32) if c >= 2000]


@pytest.mark.parametrize("ta,tb", TRANS)
def test_split_kind_every_config(lib, torch, ta, tb):
    """Every split-K config on a shape it does split (two batch entries of a single
    tile, K = 1999 so the last split is ragged), alpha -0.5, beta 0.25, NaN padding
    in A and B, and an odd ldc so the reduction takes its scalar stores."""
    ks = lib
    shape = wl.Shape(37, 45, 1999, 2, ta, tb)
    A, B, C0 = wl.gemm_inputs(shape, seed=21, beta_nonzero=True, ld_multiple=8)
    C0 = pad_c(C0, ldc_extra=3)[:, :, :51]  # ldc 51
    ref, den = og.gemm(ta, tb, shape.M, shape.N, shape.K, -0.5, A, B, 0.25, C0[:, :, :shape.N])
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    bad = []
    for cid in split_ids(ks):
        S, kc = ks.split_factor(cid, shape.M, shape.N, shape.K, shape.batch)
        assert S > 1 and (S - 1) * kc < shape.K <= S * kc, (cid, S, kc)
        out = Out(torch, C0, 0.25, shape.N)
        ks.gemm_with_config(cid, ta, tb, shape.M, shape.N, shape.K, -0.5, tA, A.shape[2], tB, B.shape[2], 0.25,
                            out.ptr, C0.shape[2], shape.batch)
        err = og.error_ratio(out.result(shape.N), ref, den)
        if not err <= TOL_F32:
            bad.append((cid, ks.config_params(cid), S, err))
    assert not bad, bad[:10]


def test_split_kind_integer_exact(lib, torch):
    """Small integers: every partial sum and the split reduction are exact."""
    ks = lib
    shape = wl.Shape(70, 66, 1500, 3, "T", "N")
    A, B, C0 = wl.gemm_inputs(shape, seed=22, kind="integer", bound=8, beta_nonzero=True)
    ref, _ = og.gemm("T", "N", shape.M, shape.N, shape.K, 1.0, A, B, 1.0, C0)
    for cid in split_ids(ks)[::7]:
        assert ks.split_factor(cid, shape.M, shape.N, shape.K, shape.batch)[0] > 1
        C = run_case(ks, torch, cid, shape, 1.0, 1.0, A, B, C0)
        assert np.array_equal(C.astype(np.float64), ref), cid


def test_split_kind_deterministic_and_graph_capturable(lib, torch):
    """Two eager calls and a CUDA-graph replay give identical bits (the partials are
    summed in split order); beta = 0 over NaN-filled C."""
    ks = lib
    cid = 2000 + find_cfg(ks, 8, 4, 16, 8, 32, 1)
    shape = wl.Shape(300, 200, 3945, 8, "N", "T")
    S, _ = ks.split_factor(cid, shape.M, shape.N, shape.K, shape.batch)
    assert S > 1
    A, B, C0 = wl.gemm_inputs(shape, seed=23)
    ref, den = og.gemm("N", "T", shape.M, shape.N, shape.K, 1.5, A, B)
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    outs = []
    for _ in range(2):
        out = Out(torch, C0, 0.0, shape.N)
        ks.gemm_with_config(cid, "N", "T", shape.M, shape.N, shape.K, 1.5, tA, A.shape[2], tB, B.shape[2], 0.0,
                            out.ptr, C0.shape[2], shape.batch)
        outs.append(out.result(shape.N))
    assert og.error_ratio(outs[0], ref, den) <= TOL_F32
    assert np.array_equal(outs[0], outs[1])
    out = Out(torch, C0, 0.0, shape.N)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            ks.gemm_with_config(cid, "N", "T", shape.M, shape.N, shape.K, 1.5, tA, A.shape[2], tB, B.shape[2],
                                0.0, out.ptr, C0.shape[2], shape.batch, side)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.result(shape.N), outs[0])


def test_split_kind_unsplit_equals_base(lib, torch):
    """Where the cost model keeps S = 1 the split-K id runs its base kernel unchanged."""
    ks = lib
    base = find_cfg(ks, 8, 4, 16, 8, 32, 1)
    shape = wl.Shape(2048, 2048, 256, 1, "N", "N")
    assert ks.split_factor(2000 + base, shape.M, shape.N, shape.K, shape.batch)[0] == 1
    A, B, C0 = wl.gemm_inputs(shape, seed=24, beta_nonzero=True)
    a = run_case(ks, torch, base, shape, 0.75, -0.5, A, B, C0)
    b = run_case(ks, torch, 2000 + base, shape, 0.75, -0.5, A, B, C0)
    assert np.array_equal(a, b)
    assert ks.split_factor(base, 37, 45, 1999, 2) == (1, 1999)  # not of the split kind


def test_host_pipeline(lib, torch):
    """gemm_host_pipeline: uploads, selected GEMMs and downloads of 14 problems on
    three streams; every C lands in pinned host memory as the oracle has it
    (beta != 0 problems upload C first; K = 0 scales C; an empty problem is skipped)."""
    import json
    import os
    ks = lib
    dep = json.load(open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                      "paper_2008_13145_gb300", "deploy", "f32.json")))
    h = ks.Handle(dep)
    rng = np.random.default_rng(31)
    cases, keep = [], []
    for n in range(14):
        M, N, K = (int(x) for x in rng.integers(1, 700, 3))
        if n == 5:
            K = 0
        if n == 9:
            M = 0
        sh = wl.Shape(M, N, K, int(rng.choice([1, 2, 4])), "NT"[n % 2], "NT"[(n // 2) % 2])
        beta = 0.0 if n % 3 == 0 else 0.5
        A, B, C0 = wl.gemm_inputs(sh, seed=300 + n, beta_nonzero=beta != 0)
        hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
        hC = torch.from_numpy(C0.copy() if beta != 0 else np.zeros_like(C0)).pin_memory()
        dA, dB = torch.empty(max(A.size, 1), device="cuda"), torch.empty(max(B.size, 1), device="cuda")
        dC = torch.empty(max(C0.size, 1), device="cuda")
        keep.append((hA, hB, hC, dA, dB, dC))
        cases.append((sh, beta, A, B, C0, hC, dict(transA=sh.transA, transB=sh.transB, M=sh.M, N=sh.N, K=sh.K,
                                                   batch=sh.batch, alpha=1.25, beta=beta, A_host=hA.data_ptr(),
                                                   lda=A.shape[2], B_host=hB.data_ptr(), ldb=B.shape[2],
                                                   C_host=hC.data_ptr(), ldc=C0.shape[2], A_dev=dA, B_dev=dB,
                                                   C_dev=dC)))
    s = torch.cuda.Stream()
    ks.gemm_host_pipeline(h, [c[-1] for c in cases], s)
    s.synchronize()
    for sh, beta, A, B, C0, hC, _ in cases:
        got = hC.numpy()[:, :, :sh.N]
        if sh.M == 0:
            continue
        ref, den = og.gemm(sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.25, A, B, beta, C0 if beta != 0 else None)
        assert og.error_ratio(got, ref, den) <= TOL_F32, sh


def test_staged_configs_equal_their_direct_twins_bit_for_bit(lib, torch):
    """A staged config (shared-memory slices, warp lane map, interior-tile loop)
    and its unstaged twin (same TM, TN, work group and K-step, operands read
    straight from global memory) accumulate every element's K terms in the same
    order with the same packed FMAs, so on real-valued data their products must
    agree to the bit: whatever the staged path does to feed its FMAs, it may
    not change a result.  Interior and edge tiles (ragged M, N, K), every
    transpose pair, alpha and beta both non-trivial."""
    ks = lib
    for n_case, (M, N, K, b) in enumerate([(131, 97, 75, 2), (192, 256, 160, 1)]):
        for tA, tB in TRANS:
            shape = wl.Shape(M, N, K, b, tA, tB)
            A, B, C0 = wl.gemm_inputs(shape, seed=40 + n_case, beta_nonzero=True)
            gA, gB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            gC0 = torch.from_numpy(np.ascontiguousarray(C0)).cuda()
            ldc = C0.shape[2]
            for direct in range(0, 576, 2):
                outs = []
                for cid in (direct, direct + 1):
                    C = gC0.clone()
                    ks.gemm_with_config(cid, tA, tB, M, N, K, 0.75, gA, A.shape[2], gB, B.shape[2], -0.5, C, ldc, b)
                    outs.append(C)
                torch.cuda.synchronize()
                # bit patterns: the results, signed zeros, and the untouched NaN padding of C
                assert torch.equal(outs[0].view(torch.int32), outs[1].view(torch.int32)), (direct, shape)
