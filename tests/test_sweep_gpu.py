"""The benchmark harness of Section 3.1 (data collection) on the GPU.

gemm_benchmark / gemm_benchmark_configs produce every throughput the pruning,
the tree and the MLP are trained on, so their contract is checked directly:
configs that cannot run report a status and no time; pass 2 re-times exactly
the configs whose probe is within refine_ratio of the fastest; the repetition
count R stays inside [min_reps, max_reps]; the reported time per launch agrees
with an independent CUDA-event timing of the same launches; and a sweep that
was killed while writing resumes without re-running finished shapes."""
import json

import numpy as np
import pytest

from paper_2008_13145_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def inputs(sh, seed=1):
    from paper_2008_13145_gb300 import tune
    return tune.alloc_inputs(sh, 0, seed)


def bench(ks, ids, sh, bufs, **kw):
    A, B, C, lda, ldb, ldc = bufs
    return ks.benchmark_configs(ids, sh.transA, sh.transB, sh.M, sh.N, sh.K, A, lda, B, ldb, C, ldc, sh.batch,
                                details=True, **kw)


def test_configs_that_cannot_run_report_status_and_no_time(lib, torch):
    ks = lib
    sh = wl.Shape(300, 200, 100, 2, "N", "N")
    ids = [369, 1001, 99999, 533, 1203]  # 1001 and 1203: reserved tensor-core slots; 99999: no such id
    ms, st, probe, reps = bench(ks, ids, sh, inputs(sh))
    bad = [1, 2, 4]
    assert list(st[bad]) == [-6, -6, -6]
    assert np.all(ms[bad] == 0) and np.all(probe[bad] == 0) and np.all(reps[bad] == 0)
    assert st[0] == 0 and st[3] == 0 and np.all(ms[[0, 3]] > 0) and np.all(reps[[0, 3]] >= 1)


def test_refine_pass_retimes_exactly_the_near_best(lib, torch):
    ks = lib
    sh = wl.Shape(512, 512, 512, 1, "N", "N")
    ids = ks.config_ids(ks.PREC_F32)[:576:13]  # 45 base configs of very different speeds
    ratio = 1.5
    ms, st, probe, reps = bench(ks, ids, sh, inputs(sh), refine_ratio=ratio, min_reps=2, max_reps=50,
                                min_total_ms=1.0)
    ok = st == 0
    assert ok.all()
    near = probe <= ratio * probe.min()
    assert near.sum() >= 1 and (~near).sum() >= 10, "both passes should be exercised"
    assert np.all(reps[near] >= 2), (reps[near], probe[near])
    assert np.all(reps[~near] == 1)
    assert np.array_equal(ms[~near], probe[~near])  # pass-1 time kept
    assert np.all(ms > 0)


def test_repetitions_stay_within_their_bounds(lib, torch):
    ks = lib
    sh = wl.Shape(256, 384, 128, 2, "T", "N")
    bufs = inputs(sh)
    A, B, C, lda, ldb, ldc = bufs
    ids = [533, 369, 2533]
    # a long target clamps R at max_reps, a tiny one at min_reps (every config refined)
    _, st, _, reps = bench(ks, ids, sh, bufs, min_reps=3, max_reps=5, min_total_ms=1e4, refine_ratio=1e9)
    assert np.all(st == 0) and np.all(reps == 5), reps
    _, st, _, reps = bench(ks, ids, sh, bufs, min_reps=4, max_reps=50, min_total_ms=1e-6, refine_ratio=1e9)
    assert np.all(st == 0) and np.all(reps == 4), reps
    for min_total, want in ((1e4, 5), (1e-6, 3)):
        st, ms, r = ks.gemm_benchmark(533, sh.transA, sh.transB, sh.M, sh.N, sh.K, A, lda, B, ldb, C, ldc, sh.batch,
                                      warmup=1, min_reps=3, max_reps=5, min_total_ms=min_total, with_reps=True)
        assert st == 0 and ms > 0 and r == want


def test_time_per_launch_agrees_with_event_timing(lib, torch):
    """The harness's mean time per launch against CUDA events around 30
    back-to-back launches of the same kernel on the same inputs (10 %)."""
    ks = lib
    sh = wl.Shape(2048, 2048, 2048, 1, "N", "N")
    A, B, C, lda, ldb, ldc = inputs(sh)
    cid = 533
    for _ in range(3):
        ks.gemm_with_config(cid, "N", "N", 2048, 2048, 2048, 1.0, A, lda, B, ldb, 0.0, C, ldc, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(30):
        ks.gemm_with_config(cid, "N", "N", 2048, 2048, 2048, 1.0, A, lda, B, ldb, 0.0, C, ldc, 1)
    e1.record()
    torch.cuda.synchronize()
    t_events = e0.elapsed_time(e1) / 30
    st, ms = ks.gemm_benchmark(cid, "N", "N", 2048, 2048, 2048, A, lda, B, ldb, C, ldc, 1, min_total_ms=10.0)
    assert st == 0 and abs(ms - t_events) <= 0.1 * t_events, (ms, t_events)
    msc, stc, _, reps = bench(ks, [cid], sh, (A, B, C, lda, ldb, ldc), min_total_ms=10.0)
    assert stc[0] == 0 and reps[0] > 1 and abs(msc[0] - t_events) <= 0.1 * t_events, (msc[0], t_events)


def test_sweep_resumes_after_a_kill(lib, torch, tmp_path, monkeypatch):
    """A sweep killed while writing its second record leaves one whole line and
    a partial one: the rerun keeps the first shape's record, drops the partial
    line and benchmarks exactly the two unfinished shapes."""
    from paper_2008_13145_gb300 import tune
    ks = lib
    shapes = [wl.Shape(64, 96, 32, 1, "N", "T"), wl.Shape(100, 50, 70, 2, "T", "N"), wl.Shape(33, 65, 17, 1, "N", "N")]
    ids = [369, 533, 71]
    out = tmp_path / "sweep.jsonl"
    full = tune.sweep(shapes, 0, str(out), config_ids=ids, log=None)
    lines = out.read_text().splitlines()
    assert len(lines) == 3 and full.shape == (3, 3) and np.all(full > 0)
    out.write_text(lines[0] + "\n" + lines[1][: len(lines[1]) // 2])
    calls = []
    orig = ks.benchmark_configs

    def counting(*a, **k):
        calls.append(a[3])  # M of the shape being benchmarked
        return orig(*a, **k)

    monkeypatch.setattr(ks, "benchmark_configs", counting)
    again = tune.sweep(shapes, 0, str(out), config_ids=ids, log=None)
    assert calls == [100, 33]
    recs = [json.loads(x) for x in out.read_text().splitlines()]
    assert [r["i"] for r in recs] == [0, 1, 2]
    assert recs[0] == json.loads(lines[0])
    assert np.array_equal(again[0], full[0]) and np.all(again > 0)
    # a finished sweep is not re-run at all
    calls.clear()
    tune.sweep(shapes, 0, str(out), config_ids=ids, log=None)
    assert calls == []
