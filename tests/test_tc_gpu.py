"""GPU parity of the tensor-core families (tcgen05 + TMA + TMEM) against the FP64 oracle.

Tolerances on max |C - C_ref| / (|alpha||A||B| + |beta||C0|):
  TF32  5e-3 (inputs truncated to 10-bit mantissas: <= 2^-9 per product),
  BF16  2e-2 (BF16 inputs: products exact in FP32, only accumulation rounds),
  F32X3 1e-5 at every K: from K = 64 on, hi*hi + hi*lo + lo*hi misses lo*lo and
        the split residuals (<= 3 * 2^-16 per product in the worst case, averaged
        well below 1e-5 over K terms of uniform data); below K = 64 three BF16
        parts and six products leave terms below about 4 * 2^-24 per product."""
import numpy as np
import pytest

from oracle import gemm as og
from paper_2008_13145_gb300 import workloads as wl
from tests.gpu_helpers import Out

pytestmark = pytest.mark.gpu
FAMILIES = {"tf32": (1, 5e-3), "bf16": (2, 2e-2), "f32x3": (3, 1e-5)}
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def to_dev(torch, x, bf16):
    t = torch.from_numpy(x).cuda()
    return t.to(torch.bfloat16) if bf16 else t


def host_values(t):
    """What the kernel actually reads (BF16 values widened exactly), for the oracle."""
    return t.float().cpu().numpy()


def tc_ids(ks, fam):
    return ks.config_ids(FAMILIES[fam][0])


def run(ks, torch, cid, fam, shape, alpha, beta, seed, ld_multiple=8, kind="uniform", bound=8):
    bf16 = fam == "bf16"
    A, B, C0 = wl.gemm_inputs(shape, seed=seed, beta_nonzero=beta != 0, ld_multiple=ld_multiple, kind=kind,
                              bound=bound)
    tA, tB = to_dev(torch, A, bf16), to_dev(torch, B, bf16)
    out = Out(torch, C0, beta, shape.N)
    ks.gemm_with_config(cid, shape.transA, shape.transB, shape.M, shape.N, shape.K, alpha, tA, A.shape[2], tB,
                        B.shape[2], beta, out.ptr, C0.shape[2], shape.batch)
    torch.cuda.synchronize()
    C = out.result(shape.N)
    ref, den = og.gemm(shape.transA, shape.transB, shape.M, shape.N, shape.K, alpha, host_values(tA).reshape(A.shape),
                       host_values(tB).reshape(B.shape), beta, C0)
    return C, ref, den


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_tn_single_tile_family(lib, torch, fam):
    """One 128 x 128 tile, both operands K-contiguous (no pre-pass)."""
    ks = lib
    cid = tc_ids(ks, fam)[4]  # BN 128, 3 stages
    assert ks.config_params(cid)[2] == 128
    C, ref, den = run(ks, torch, cid, fam, wl.Shape(128, 128, 128, 1, "N", "T"), 1.0, 0.0, seed=1)
    assert og.error_ratio(C, ref, den) <= FAMILIES[fam][1]
    assert ks.device_status() == 0


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_every_config_ragged(lib, torch, fam):
    """All 9 configs: several tiles in M and N with ragged tails, K not a multiple of the slice."""
    ks = lib
    bad = []
    for cid in tc_ids(ks, fam):
        C, ref, den = run(ks, torch, cid, fam, wl.Shape(300, 333, 136, 2, "N", "T"), -0.5, 0.25, seed=2)
        err = og.error_ratio(C, ref, den)
        if not err <= FAMILIES[fam][1]:
            bad.append((cid, ks.config_params(cid), err))
    assert not bad, bad
    assert ks.device_status() == 0


@pytest.mark.parametrize("fam", ["tf32", "bf16"])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("T", "T")])
def test_mn_major_every_config(lib, torch, fam, ta, tb):
    """TF32 and BF16 operands stored MN-contiguous (A as K x M, B as K x N)
    with 16-byte aligned rows are read in place as MN-major tiles (TF32: boxes
    of 32 elements, 128-byte swizzle of 32-byte pieces): all 9 configs, two
    tiles plus a ragged tail in M and N, K not a multiple of the slice, two
    batch entries, alpha and beta."""
    ks = lib
    bad = []
    for cid in tc_ids(ks, fam):
        C, ref, den = run(ks, torch, cid, fam, wl.Shape(300, 333, 136, 2, ta, tb), -0.5, 0.25, seed=12)
        err = og.error_ratio(C, ref, den)
        if not err <= FAMILIES[fam][1]:
            bad.append((cid, ks.config_params(cid), err))
    assert not bad, bad
    assert ks.device_status() == 0


@pytest.mark.parametrize("fam,bound", [("tf32", 64), ("bf16", 16), ("f32x3", 128)])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("T", "T")])
def test_mn_major_integer_exact(lib, torch, fam, bound, ta, tb):
    """Small integers are exact in the operand format and their sums in FP32,
    so reading an MN-major operand transposed must give the FP64 product bit
    for bit, in every config (x3: its pre-pass splits an aligned MN-contiguous
    operand without transposing it, and the kernel reads the parts MN-major)."""
    ks = lib
    for cid in tc_ids(ks, fam):
        C, ref, _ = run(ks, torch, cid, fam, wl.Shape(200, 260, 320, 2, ta, tb), 1.0, 1.0, seed=13,
                        kind="integer", bound=bound)
        assert np.array_equal(C.astype(np.float64), ref), cid


@pytest.mark.parametrize("ta,tb", TRANS)
def test_x3_every_config_any_layout_odd_ld(lib, torch, ta, tb):
    """Split-BF16 x3 in all 9 configs with odd leading dimensions (so the
    pre-pass takes its unpaired loads), K not a multiple of the 64-wide slice,
    ragged M and N tails and two batch entries."""
    ks = lib
    bad = []
    for cid in tc_ids(ks, "f32x3"):
        C, ref, den = run(ks, torch, cid, "f32x3", wl.Shape(300, 333, 137, 2, ta, tb), 0.75, -0.5, seed=14,
                          ld_multiple=1)
        err = og.error_ratio(C, ref, den)
        if not err <= FAMILIES["f32x3"][1]:
            bad.append((cid, ks.config_params(cid), err))
    assert not bad, bad
    assert ks.device_status() == 0


@pytest.mark.parametrize("fam", list(FAMILIES))
@pytest.mark.parametrize("ta,tb", TRANS)
def test_layouts_and_unaligned_ld(lib, torch, fam, ta, tb):
    """Every transpose combination, with 16-byte aligned and unaligned leading dimensions."""
    ks = lib
    ids = tc_ids(ks, fam)
    for cid, ldm in ((ids[1], 8), (ids[8], 1)):
        C, ref, den = run(ks, torch, cid, fam, wl.Shape(190, 77, 99, 3, ta, tb), 1.5, -1.0, seed=3, ld_multiple=ldm)
        assert og.error_ratio(C, ref, den) <= FAMILIES[fam][1], (cid, ldm)


@pytest.mark.parametrize("fam,bound", [("tf32", 64), ("bf16", 16), ("f32x3", 128)])
def test_integer_inputs_exact(lib, torch, fam, bound):
    """Integers small enough to be exact in the operand format, with exact FP32 sums."""
    ks = lib
    cid = tc_ids(ks, fam)[2]
    C, ref, _ = run(ks, torch, cid, fam, wl.Shape(160, 200, 256, 2, "T", "N"), 1.0, 1.0, seed=4, kind="integer",
                    bound=bound)
    assert np.array_equal(C.astype(np.float64), ref)


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_degenerate_sizes(lib, torch, fam):
    ks = lib
    cid = tc_ids(ks, fam)[0]
    for M, N, K in [(1, 1, 1), (1, 300, 20), (300, 1, 20), (5, 7, 4099)]:
        C, ref, den = run(ks, torch, cid, fam, wl.Shape(M, N, K, 2, "N", "N"), 1.0, 0.5, seed=5)
        assert og.error_ratio(C, ref, den) <= FAMILIES[fam][1], (M, N, K)


@pytest.mark.parametrize("K", [1, 2, 3, 7, 15, 16, 63, 64, 65])
def test_x3_small_k_fp32_level(lib, torch, K):
    """The split-BF16 family at the FP32 tolerance for small K, where averaging
    over K terms no longer hides the two-part split's per-product error: K < 64
    runs three parts and six products, K >= 64 the three products.  Every
    config, 4 x 4 tiles of 128 x 128 outputs (enough elements for the error's
    tail to show), each layout of the operands in turn."""
    ks = lib
    bad = []
    for i, cid in enumerate(tc_ids(ks, "f32x3")):
        ta, tb = TRANS[i % 4]
        C, ref, den = run(ks, torch, cid, "f32x3", wl.Shape(512, 520, K, 2, ta, tb), 1.0, 0.0, seed=40 + K)
        err = og.error_ratio(C, ref, den)
        if not err <= FAMILIES["f32x3"][1]:
            bad.append((cid, ta, tb, err))
    assert not bad, bad


@pytest.mark.parametrize("fam", list(FAMILIES))
def test_full_size_sampled(lib, torch, fam):
    """4096^3 in the largest tile config, checked on sampled entries by the GPU FP64 reduction."""
    ks = lib
    bf16 = fam == "bf16"
    cid = tc_ids(ks, fam)[8]  # BN 256, 4 stages
    shape = wl.Shape(4096, 4096, 4096, 1, "N", "N")
    A, B, _ = wl.gemm_inputs(shape, seed=6, ld_multiple=8)
    tA, tB = to_dev(torch, A, bf16), to_dev(torch, B, bf16)
    C = torch.empty((4096, 4096), device="cuda")
    ks.gemm_with_config(cid, "N", "N", 4096, 4096, 4096, 1.0, tA, A.shape[2], tB, B.shape[2], 0.0, C, 4096, 1)
    pos = wl.sample_positions(shape, 4, 4, seed=7)
    ref, den = og.gemm_entries("N", "N", 4096, 4096, 4096, 1.0, host_values(tA).reshape(A.shape),
                               host_values(tB).reshape(B.shape), 0.0, None, pos, nthreads=og.max_threads())
    err = ks.error_check(C, torch.from_numpy(ref).cuda(), torch.from_numpy(den).cuda(), pos=torch.from_numpy(pos).cuda(),
                         ldc=4096, strideC=4096 * 4096)
    assert err <= FAMILIES[fam][1], err
    assert ks.device_status() == 0


def test_misaligned_direct_operand_is_rewritten(lib, torch):
    """A pointer 4 bytes off a 16-byte boundary takes the pre-pass instead of failing TMA alignment."""
    ks = lib
    M, N, K = 130, 64, 96
    rng = np.random.default_rng(8)
    A = rng.uniform(-1, 1, (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (N, K)).astype(np.float32)
    fa = torch.from_numpy(np.concatenate([[0.0], A.ravel()]).astype(np.float32)).cuda()
    tB = torch.from_numpy(B).cuda()
    C = torch.empty((M, N), device="cuda")
    ks.gemm_with_config(tc_ids(ks, "tf32")[0], "N", "T", M, N, K, 1.0, fa.data_ptr() + 4, K, tB, K, 0.0, C, N, 1)
    ref, den = og.gemm("N", "T", M, N, K, 1.0, A[None], B[None])
    assert og.error_ratio(C.cpu().numpy()[None], ref, den) <= 5e-3


def test_mixed_family_deployment_through_gemm(lib, torch):
    """The FP32-input deployment mixing SIMT and split-BF16x3 kernels: sizes that
    select either family give FP32-level results through gemm()."""
    import json
    import os
    ks = lib
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2008_13145_gb300",
                        "deploy", "f32mix.json")
    dep = json.load(open(path))
    h = ks.Handle(dep)
    fams = set()
    for i, sh in enumerate(wl.shape_grid(60, 99)[:60]):
        if sh.flops > 4e9:
            continue
        fams.add(ks.family_of(ks.select_kernel(h, sh.M, sh.N, sh.K, sh.batch)))
        A, B, C0 = wl.gemm_inputs(sh, seed=300 + i)
        tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        out = Out(torch, C0, 0.0, sh.N)
        ks.gemm(h, sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, tA, A.shape[2], tB, B.shape[2], 0.0, out.ptr,
                C0.shape[2], sh.batch)
        torch.cuda.synchronize()
        ref, den = og.gemm(sh.transA, sh.transB, sh.M, sh.N, sh.K, 1.0, A, B, nthreads=og.max_threads())
        assert og.error_ratio(out.result(sh.N), ref, den) <= 1e-5, (sh, ks.select_kernel(h, sh.M, sh.N, sh.K, sh.batch))
    assert fams == {0, 3}, fams


@pytest.mark.parametrize("K", [1, 2, 3, 7, 15])
def test_fp32_class_small_k_through_gemm(lib, torch, K):
    """gemm() with the FP32-input deployment (SIMT and split-BF16 kernels) at
    small K meets the FP32 tolerance whichever family the tree picks; a handle
    holding only the deployment's split-BF16 kernels makes gemm() run that
    family on every size."""
    import json
    import os
    ks = lib
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2008_13145_gb300",
                        "deploy", "f32mix.json")
    dep = json.load(open(path))
    x3_ids = [c for c in dep["config_ids"] if ks.family_of(c) == ks.PREC_F32X3]
    assert x3_ids, "the FP32-input deployment should hold split-BF16 kernels"
    handles = [ks.Handle(dep), ks.Handle({"precision": 0, "config_ids": x3_ids, "nodes": []})]
    for j, (M, N, batch, ta, tb) in enumerate([(700, 900, 1, "N", "N"), (257, 1030, 4, "T", "N"),
                                               (1500, 130, 2, "N", "T"), (64, 64, 16, "T", "T")]):
        sh = wl.Shape(M, N, K, batch, ta, tb)
        A, B, C0 = wl.gemm_inputs(sh, seed=600 + 10 * K + j)
        tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        ref, den = og.gemm(ta, tb, M, N, K, 1.0, A, B, nthreads=og.max_threads())
        for h in handles:
            out = Out(torch, C0, 0.0, N)
            ks.gemm(h, ta, tb, M, N, K, 1.0, tA, A.shape[2], tB, B.shape[2], 0.0, out.ptr, C0.shape[2], batch)
            torch.cuda.synchronize()
            err = og.error_ratio(out.result(N), ref, den)
            assert err <= 1e-5, (sh, ks.select_kernel(h, M, N, K, batch), err)
    assert ks.device_status() == 0


def test_bounded_wait_gives_up_and_context_survives(lib, torch):
    """The failure path: a bounded mbarrier wait on a barrier that nothing arrives
    at gives up after its limit (1 ms here), records code 1 in the status word,
    the host reads it as GEMM_ERR_TIMEOUT and clears it, and tensor-core GEMMs
    on the same context are correct afterwards."""
    import time
    ks = lib
    assert ks.device_status() == 0
    t0 = time.perf_counter()
    assert ks.wait_selftest(1_000_000) == 0
    assert time.perf_counter() - t0 < 5.0
    st = ks.i32()
    assert ks._lib.gemm_device_status(ks.ctypes.byref(st), 0) == -5 and st.value == 1  # GEMM_ERR_TIMEOUT, kept
    assert ks.device_status(clear=True) == 1
    assert ks.device_status() == 0
    C, ref, den = run(ks, torch, tc_ids(ks, "bf16")[4], "bf16", wl.Shape(128, 128, 128, 1, "N", "T"), 1.0, 0.0, seed=1)
    assert og.error_ratio(C, ref, den) <= FAMILIES["bf16"][1]
    assert ks.device_status() == 0


@pytest.mark.parametrize("cid", [7, 2533, 1000, 1116, 1216])
def test_empty_sizes_and_k_zero_every_family(lib, torch, cid):
    """The degenerate cases of C = alpha op(A) op(B) + beta C, in every family
    (SIMT, split-K, TF32, BF16, x3): K = 0 leaves C = beta C (beta = 0 writes
    exact zeros over a NaN-filled C); M, N or batch = 0 touches nothing.  Guard
    bands around C and its ldc padding must survive."""
    ks = lib
    bf16 = ks.family_of(cid) == ks.PREC_BF16
    dummy = torch.zeros(64, device="cuda", dtype=torch.bfloat16 if bf16 else torch.float32)
    for beta in (0.5, 0.0):
        C0 = wl.uniform_matrix(9, 10, 12, 2, 3, 3)
        out = Out(torch, C0, beta, 10)
        ks.gemm_with_config(cid, "N", "T", 9, 10, 0, 1.0, dummy, 1, dummy, 1, beta, out.ptr, 12, 2)
        torch.cuda.synchronize()
        want = np.float32(beta) * C0[:, :, :10] if beta != 0 else np.zeros((2, 9, 10), np.float32)
        assert np.array_equal(out.result(10), want), (cid, beta)
    for M, N, batch in ((0, 10, 2), (9, 0, 2), (9, 10, 0)):
        C0 = wl.uniform_matrix(9, 10, 12, 2, 4, 3)
        out = Out(torch, C0, 0.5, 10)
        ks.gemm_with_config(cid, "N", "T", M, N, 16, 1.0, dummy, 16, dummy, 16, 0.5, out.ptr, 12, batch)
        torch.cuda.synchronize()
        assert np.array_equal(out.result(10), C0[:, :, :10]), (cid, M, N, batch)
    assert ks.device_status() == 0


@pytest.mark.parametrize("cid", [7, 533, 2533, 1000, 1116, 1216])
def test_maximum_batch_every_family(lib, torch, cid):
    """batch = 65535, the largest the library accepts (the SIMT grid's z
    dimension; the tensor-core kernels walk 65535 tiles persistently): 4 x 5 x 6
    products against the oracle, and 65536 is refused before any launch."""
    ks = lib
    fam = ks.family_of(cid)
    bf16 = fam == ks.PREC_BF16
    shape = wl.Shape(4, 5, 6, 65535, "N", "T")
    A, B, C0 = wl.gemm_inputs(shape, seed=77, ld_multiple=8, beta_nonzero=True)
    tA, tB = to_dev(torch, A, bf16), to_dev(torch, B, bf16)
    C = torch.from_numpy(C0).cuda()
    ks.gemm_with_config(cid, "N", "T", 4, 5, 6, 1.0, tA, A.shape[2], tB, B.shape[2], -0.5, C, C0.shape[2], 65535)
    torch.cuda.synchronize()
    ref, den = og.gemm("N", "T", 4, 5, 6, 1.0, host_values(tA).reshape(A.shape), host_values(tB).reshape(B.shape),
                       -0.5, C0)
    tol = {ks.PREC_F32: 1e-5, ks.PREC_TF32: 5e-3, ks.PREC_BF16: 2e-2, ks.PREC_F32X3: 1e-5}[fam]
    assert og.error_ratio(C.cpu().numpy()[:, :, :5], ref, den) <= tol
    with pytest.raises(ks.KSelectError) as e:
        ks.gemm_with_config(cid, "N", "T", 4, 5, 6, 1.0, tA, A.shape[2], tB, B.shape[2], 0.0, C, C0.shape[2], 65536)
    assert e.value.status == -2
    assert ks.device_status() == 0
