"""Host-side pipeline functions of the library (no GPU needed) against the oracle.

CART, representatives and Top-N are exact integer/index work: the library must
reproduce the oracle's trees node for node and its column choices exactly."""
import numpy as np
import pytest

from oracle import select as osel


@pytest.fixture(scope="module")
def ks():
    from paper_2008_13145_gb300 import build
    build.build_library()
    from paper_2008_13145_gb300 import kselect
    return kselect


def same_tree(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert (x["feature"], x["left"], x["right"], x["label"]) == (y["feature"], y["left"], y["right"], y["label"])
        if x["feature"] >= 0:
            assert x["threshold"] == y["threshold"]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("tree", ["A", "B", "C"])
def test_tree_matches_oracle_with_many_ties(ks, seed, tree):
    rng = np.random.default_rng(seed)
    n = 150
    F = rng.integers(1, 7, (n, 5)).astype(np.float64)  # few distinct values: many tied splits
    y = rng.integers(0, 5, n)
    depth, leaf = osel.TREES[tree]
    same_tree(ks.tree_train(F, y, 5, depth, leaf), osel.tree_train(F, y, 5, depth, leaf))


@pytest.mark.parametrize("tree", ["A", "B", "C"])
def test_tree_matches_oracle_on_grid_sizes(ks, tree):
    from paper_2008_13145_gb300 import workloads as wl
    g = wl.shape_grid(400, 21)
    F = osel.selector_features([[s.M, s.N, s.K, s.batch] for s in g])
    y = ((F[:, 0] * F[:, 1] > 1e5).astype(int) + (F[:, 2] > 700).astype(int) * 2
         + (np.random.default_rng(2).random(400) < 0.15))
    depth, leaf = osel.TREES[tree]
    same_tree(ks.tree_train(F, y, 5, depth, leaf), osel.tree_train(F, y, 5, depth, leaf))


def test_selector_features_and_labels_match_oracle(ks):
    """The feature rows and the best-deployed-kernel labels the tuner trains on
    are the library's, bit for bit the oracle's (ties included)."""
    from paper_2008_13145_gb300 import workloads as wl
    sizes = [[s.M, s.N, s.K, s.batch] for s in wl.shape_grid(500, 3)] + [[0, 7, 1, 1], [4096, 4096, 4096, 65535]]
    assert np.array_equal(ks.selector_features(sizes), osel.selector_features(sizes))
    rng = np.random.default_rng(4)
    perf = rng.integers(0, 6, (300, 40)).astype(np.float64)  # many ties
    for cols in ([0], [5, 3, 9, 1], list(range(40)), [39, 0, 17, 17]):
        assert list(ks.best_labels(perf, cols)) == list(osel.best_labels(perf, cols))
    with pytest.raises(ks.KSelectError):
        ks.best_labels(perf, [40])
    with pytest.raises(ks.KSelectError):
        ks.selector_features([[1, -2, 3, 4]])


def test_tree_pure_and_single_sample(ks):
    F = np.array([[1.0, 2, 3, 4, 5]])
    assert ks.tree_train(F, np.array([2]), 3) == [{"feature": -1, "threshold": 0.0, "left": -1, "right": -1,
                                                    "label": 2}]
    F = np.tile(np.array([[5.0, 5, 5, 5, 5]]), (6, 1))
    nodes = ks.tree_train(F, np.array([0, 1, 1, 0, 1, 0]), 2)
    assert len(nodes) == 1 and nodes[0]["label"] == 0  # identical features: no split, tie -> lowest class


def test_tree_rejects_bad_input(ks):
    with pytest.raises(ks.KSelectError):
        ks.tree_train(np.ones((3, 5)), np.array([0, 5, 1]), 2)
    with pytest.raises(ks.KSelectError):
        ks.tree_train(np.full((3, 5), np.nan), np.array([0, 1, 1]), 2)
    with pytest.raises(ks.KSelectError) as e:  # too many nodes for the output buffer
        ks.tree_train(np.arange(500, dtype=float).reshape(100, 5), np.arange(100) % 2, 2, max_nodes=5)
    assert e.value.status == -2


@pytest.mark.parametrize("seed", range(5))
def test_representatives_match_oracle(ks, seed):
    rng = np.random.default_rng(seed)
    k, d, n = 6, 40, 90
    centres = rng.random((k, d)).astype(np.float32)
    centres[:, 3] += 0.8  # a shared favourite forces duplicates
    labels = rng.integers(0, k, n)
    for dedupe in (True, False):
        got = ks.representatives(centres, labels, dedupe)
        want = osel.representatives(centres.astype(np.float64), labels, dedupe)
        assert list(got) == list(want)


@pytest.mark.parametrize("seed", range(5))
def test_top_n_matches_oracle(ks, seed):
    rng = np.random.default_rng(seed)
    perf = rng.random((60, 30)).astype(np.float32) ** 3
    perf[:, 7] *= 3.0
    for n in (1, 4, 8, 15, 30):
        assert list(ks.top_n(perf, n)) == list(osel.top_n(perf.astype(np.float64), n))


# ---------------------------------------------------------------- regression-tree pruning (Section 4.1)
def same_partition(a, b):
    return len(set(zip(a.tolist(), b.tolist()))) == len(set(a.tolist())) == len(set(b.tolist()))


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("k", [1, 2, 4, 8, 15])
def test_tree_regress_matches_oracle(ks, seed, k):
    """Tie-free sizes, float32 performance vectors: the same leaves in the same
    order (exact labels) and leaf means within float rounding."""
    rng = np.random.default_rng(100 + seed)
    F = rng.permutation(4096)[:5 * 90].reshape(90, 5).astype(np.float64) + 16
    Y = (rng.random((90, 12)) ** 3).astype(np.float32)
    labels, centres = ks.tree_regress(F, Y, k)
    ref_labels, ref_centres = osel.tree_regression_partition(F, Y.astype(np.float64), k)
    assert np.array_equal(labels, ref_labels)
    assert np.allclose(centres, ref_centres, rtol=0, atol=1e-6)


def test_tree_regress_on_grid_sizes_with_ties(ks):
    """Grid-like sizes (repeated values, batch in 5 levels) and normalised rows:
    same partition as the oracle."""
    from paper_2008_13145_gb300 import workloads as wl
    shapes = wl.shape_grid(300, 9)
    F = osel.selector_features([[s.M, s.N, s.K, s.batch] for s in shapes])
    rng = np.random.default_rng(9)
    perf = rng.random((300, 20)) * np.log(F[:, :1]) * np.sqrt(F[:, 3:4])
    Y = osel.normalise(perf, "standard").astype(np.float32)
    for k in (4, 8, 15):
        labels, _ = ks.tree_regress(F, Y, k)
        ref, _ = osel.tree_regression_partition(F, Y.astype(np.float64), k)
        assert same_partition(labels, ref), k


def test_tree_regress_constant_leaves_stop(ks):
    F = osel.selector_features([[16, 16, 16, 1], [32, 16, 16, 1], [64, 16, 16, 1], [128, 16, 16, 1]])
    Y = np.array([[1, 0], [1, 0], [0, 1], [0, 1]], np.float32)
    labels, centres = ks.tree_regress(F, Y, 4)
    assert labels.tolist() == [0, 0, 1, 1] and np.array_equal(centres, [[1, 0], [0, 1]])
    with pytest.raises(ks.KSelectError):
        ks.tree_regress(F, np.full((4, 2), np.nan, np.float32), 2)
    with pytest.raises(ks.KSelectError):
        ks.tree_regress(F, Y, 0)


# ---------------------------------------------------------------- random-forest trees (Section 5.1 classifiers)
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_random_forest_tree_matches_oracle(ks, seed, m):
    """Node for node, with bootstrap-like repeated rows and the same per-node draws."""
    from paper_2008_13145_gb300 import workloads as wl
    rng = np.random.default_rng(200 + seed)
    shapes = wl.shape_grid(400, 10 + seed)
    F = osel.selector_features([[s.M, s.N, s.K, s.batch] for s in shapes])
    y = (np.log(F[:, 0]) + np.log(F[:, 1]) > 12).astype(np.int32) + (F[:, 3] > 4).astype(np.int32)
    boot = rng.integers(0, 400, 400)
    draws = rng.integers(0, 2 ** 32, (8192, 5), dtype=np.uint64).astype(np.uint32)
    for depth, leaf in ((None, 1), (6, 3)):
        got = ks.tree_train_rf(F[boot], y[boot], 3, m, draws, depth, leaf)
        want = osel.tree_train(F[boot], y[boot], 3, depth, leaf, max_features=m, draws=draws)
        same_tree(got, want)
        if m == 5:
            same_tree(got, ks.tree_train(F[boot], y[boot], 3, depth, leaf))


def test_forest_selector_votes_like_the_oracle(ks):
    """A deployment with a forest: select_kernel is the majority vote of the trees
    (lowest label on ties), each tree walked as the oracle walks it."""
    from paper_2008_13145_gb300 import workloads as wl
    rng = np.random.default_rng(77)
    shapes = wl.shape_grid(300, 21)
    F = osel.selector_features([[s.M, s.N, s.K, s.batch] for s in shapes])
    y = ((np.log(F[:, 0]) > 6).astype(np.int32) + (np.log(F[:, 2]) > 6.5) * 2 + (F[:, 3] > 4)) % 4
    y = y.astype(np.int32)
    trees = []
    for b in range(9):
        boot = rng.integers(0, 300, 300)
        draws = rng.integers(0, 2 ** 32, (8192, 5), dtype=np.uint64).astype(np.uint32)
        trees.append(ks.tree_train_rf(F[boot], y[boot], 4, 2, draws))
    ids = [11, 22, 33, 44]
    h = ks.Handle({"precision": 0, "config_ids": ids, "nodes": [], "forest": trees})
    Q = osel.selector_features([[s.M, s.N, s.K, s.batch] for s in wl.shape_grid(500, 22)])
    votes = np.zeros((len(Q), 4), np.int64)
    for t in trees:
        votes[np.arange(len(Q)), osel.tree_predict(t, Q)] += 1
    want = [ids[int(np.argmax(v))] for v in votes]  # argmax: lowest label among the tied maxima
    got = [ks.select_kernel(h, *map(int, q[:4])) for q in Q]
    assert got == want


def test_forest_deployment_validation(ks):
    leaf = lambda c: {"feature": -1, "threshold": 0.0, "left": -1, "right": -1, "label": c}
    split = {"feature": 0, "threshold": 100.0, "left": 1, "right": 2, "label": 0}
    ok = {"precision": 0, "config_ids": [5, 7]}
    h = ks.Handle({**ok, "forest": [[split, leaf(0), leaf(1)], [leaf(1)], [leaf(1)]]})
    assert ks.select_kernel(h, 50, 1, 1, 1) == 7 and ks.select_kernel(h, 500, 1, 1, 1) == 7
    h = ks.Handle({**ok, "forest": [[split, leaf(0), leaf(1)], [leaf(0)]]})
    assert ks.select_kernel(h, 50, 1, 1, 1) == 5  # 2 votes for label 0
    assert ks.select_kernel(h, 500, 1, 1, 1) == 5  # a 1-1 tie goes to the lower label
    with pytest.raises(ks.KSelectError):  # a leaf label outside the deployed set
        ks.Handle({**ok, "forest": [[leaf(0)], [leaf(2)]]})
    # raw ABI: two trees sharing a node, and a root out of range
    nodes = (ks.TreeNode * 3)(ks.TreeNode(0, 1, 2, 0, 100.0), ks.TreeNode(-1, -1, -1, 0, 0.0),
                              ks.TreeNode(-1, -1, -1, 1, 0.0))
    ids = (ks.i32 * 2)(5, 7)
    for roots in ([0, 1], [0, 3], [0, -1]):
        r = (ks.i32 * 2)(*roots)
        d = ks.Deployment(0, 2, ids, 3, nodes, None, 0, None, None, 2, r)
        hv = ks.vp()
        assert ks._lib.gemm_library_create(ks.ctypes.byref(d), ks.ctypes.byref(hv)) == -1, roots
    r = (ks.i32 * 300)(*([0] * 300))
    d = ks.Deployment(0, 2, ids, 3, nodes, None, 0, None, None, 300, r)
    hv = ks.vp()
    assert ks._lib.gemm_library_create(ks.ctypes.byref(d), ks.ctypes.byref(hv)) == -1


def test_grouped_select_reads_group_medians(ks):
    """gemm_grouped_select: the deployment's tree walked on (lower median M, N, K, count)."""
    from paper_2008_13145_gb300 import tune
    leaf = lambda c: {"feature": -1, "threshold": 0.0, "left": -1, "right": -1, "label": c}
    nodes = [{"feature": 2, "threshold": 500.0, "left": 1, "right": 2, "label": 0}, leaf(0),
             {"feature": 3, "threshold": 40.0, "left": 3, "right": 4, "label": 0}, leaf(1), leaf(2)]
    h = ks.Handle({"precision": 2, "config_ids": [1100, 1116, 1104], "nodes": nodes})
    rng = np.random.default_rng(5)
    for count in (1, 2, 7, 33, 64):
        for _ in range(5):
            probs = [dict(M=int(rng.integers(1, 3000)), N=int(rng.integers(1, 3000)), K=int(rng.integers(1, 3000)),
                          A=0, lda=1, B=0, ldb=1, C=0, ldc=1) for _ in range(count)]
            f = tune.group_features(probs)
            assert f[3] == count and f[2] == sorted(q["K"] for q in probs)[(count - 1) // 2]
            assert ks.grouped_select(h, probs) == ks.select_kernel(h, *f)
    with pytest.raises(ks.KSelectError):
        ks.grouped_select(h, [dict(M=-1, N=1, K=1, A=0, lda=1, B=0, ldb=1, C=0, ldc=1)])
