"""Pins for the pruning/selection oracle: closed forms, brute force, invariants,
and (where scikit-learn is present) library cross-checks."""
import itertools
import math

import numpy as np
import pytest

from oracle import select as osel


# ---------------------------------------------------------------- normalisation (Section 3.4)
def test_sigmoid_closed_form():
    perf = np.array([[0.85, 0.80, 1.0, 0.5]])
    x = osel.normalise(perf, "sigmoid")[0]
    assert x[0] == pytest.approx(0.5, abs=1e-15)
    assert x[1] == pytest.approx(1.0 / (1.0 + math.exp(2.5)), rel=1e-14)
    assert x[1] < 0.1
    assert x[2] == pytest.approx(1.0 / (1.0 + math.exp(-7.5)), rel=1e-14)


def test_standard_and_cutoffs():
    perf = np.array([[10.0, 9.5, 8.0, 0.0], [0.0, 0.0, 0.0, 0.0], [2.0, 1.0, 4.0, 3.8]])
    s = osel.normalise(perf, "standard")
    assert np.array_equal(s[0], [1.0, 0.95, 0.8, 0.0])
    assert np.array_equal(s[1], [0, 0, 0, 0])
    assert s[2].max() == 1.0
    r = osel.normalise(perf, "raw_cutoff")
    assert np.array_equal(r[0], [1.0, 0.95, 0.0, 0.0])
    sc = osel.normalise(perf, "standard_cutoff")
    assert sc[0][0] == 1.0 and sc[0][1] == pytest.approx(0.5) and sc[0][2] == 0.0
    assert sc[2][3] == pytest.approx(0.5)


# ---------------------------------------------------------------- k-means (Section 4.1)
def blobs(n_per, centres, spread, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([c + spread * rng.standard_normal((n_per, len(c))) for c in centres])


@pytest.mark.parametrize("k", [2, 3])
def test_kmeans_reaches_brute_force_optimum(k):
    X = blobs(3, [np.array([0.0, 0.0, 1.0]), np.array([1.0, 1.0, 0.0]), np.array([0.0, 1.0, 0.0])][:k],
              0.05, seed=k)
    if k == 2:
        X = X[:7]
    opt, _ = osel.brute_force_partition(X, k)
    u = np.random.default_rng(1).random((10, k))
    _, labels, inertia, _ = osel.kmeans(X, k, u)
    assert inertia == pytest.approx(opt, rel=1e-12)


def test_brute_force_small_case_by_hand():
    # 1-D points {0, 1, 10, 11}, k = 2: optimum {0,1} | {10,11}, cost 0.5 + 0.5.
    cost, labels = osel.brute_force_partition(np.array([[0.0], [1.0], [10.0], [11.0]]), 2)
    assert cost == pytest.approx(1.0)
    assert labels[0] == labels[1] != labels[2] == labels[3]


def test_lloyd_inertia_non_increasing():
    X = np.random.default_rng(4).random((60, 5))
    C0 = X[[0, 1, 2, 3]]
    prev = math.inf
    for it in range(1, 12):
        _, _, inertia, _ = osel.lloyd(X, C0, max_iter=it, tol=0.0)
        assert inertia <= prev + 1e-12
        prev = inertia


def test_kmeanspp_first_centre_and_far_point():
    X = np.array([[0.0], [0.1], [10.0]])
    C = osel.kmeanspp_init(X, 2, np.array([0.0, 0.5]))
    assert C[0, 0] == 0.0
    # D^2 = [0, 0.01, 100]: half the total lies past point 1, so point 2 is picked.
    assert C[1, 0] == 10.0


def test_kmeans_matches_sklearn_inertia():
    sk = pytest.importorskip("sklearn.cluster")
    X = blobs(20, [np.zeros(6), np.ones(6), np.r_[np.ones(3), np.zeros(3)]], 0.1, seed=9)
    u = np.random.default_rng(2).random((10, 3))
    _, labels, inertia, _ = osel.kmeans(X, 3, u)
    ref = sk.KMeans(3, n_init=10, random_state=0).fit(X)
    assert inertia == pytest.approx(ref.inertia_, rel=1e-9)


# ---------------------------------------------------------------- representatives / Top-N (Section 4.2)
def test_representatives_argmax_and_dedupe():
    centres = np.array([[0.1, 0.9, 0.8, 0.0],
                        [0.2, 0.95, 0.1, 0.3],
                        [1.0, 0.0, 0.0, 0.0]])
    labels = np.array([0, 0, 0, 1, 1, 2])
    assert list(osel.representatives(centres, labels, dedupe=True)) == [1, 3, 0]
    # without dedupe the smaller cluster with the same best config is dropped
    assert list(osel.representatives(centres, labels, dedupe=False)) == [1, 0]


def test_cluster_geomean_representative():
    X = np.array([[1.0, 0.5], [0.25, 1.0], [0.9, 0.8]])
    # geometric means: col0 (1*0.25)^(1/2)=0.5, col1 (0.5*1)^(1/2)=0.707 -> 1 for cluster {0,1}
    reps = osel.cluster_geomean_representatives(X, np.array([0, 0, 1]), 2)
    assert list(reps) == [1, 0]


def test_top_n_counts():
    perf = np.array([[1, 2, 3], [3, 2, 1], [0, 5, 1], [1, 1, 9], [2, 1, 8.0]])
    assert list(osel.top_n(perf, 2)) == [2, 0]
    assert list(osel.top_n(perf, 3)) == [2, 0, 1]


def test_top_n_fill():
    perf = np.array([[1.0, 0.5, 0.9], [1.0, 0.2, 0.95]])
    assert list(osel.top_n(perf, 3)) == [0, 2, 1]


# ---------------------------------------------------------------- score (Section 4.3)
def test_score_closed_form():
    perf = np.array([[4.0, 2.0, 1.0], [1.0, 1.0, 2.0]])
    s = osel.score(perf, deployed=np.array([1]))
    assert s["geomean"] == pytest.approx(math.sqrt(0.5 * 0.5))
    s = osel.score(perf, chosen=np.array([2, 0]))
    assert s["geomean"] == pytest.approx(math.sqrt(0.25 * 0.5))
    assert s["mean"] == pytest.approx(0.375)
    assert osel.score(perf)["geomean"] == 1.0
    assert osel.score(perf, deployed=np.arange(3))["geomean"] == 1.0


def test_top_n_all_is_optimal():
    perf = np.random.default_rng(0).random((30, 7))
    assert osel.score(perf, deployed=osel.top_n(perf, 7))["geomean"] == pytest.approx(1.0)


# ---------------------------------------------------------------- decision tree (Section 5.1)
def brute_best_split(F, y, n_classes, min_leaf):
    best = None
    n = len(y)
    for f in range(F.shape[1]):
        for t in sorted(set(F[:, f])):
            left = F[:, f] <= t
            nl = left.sum()
            if nl < min_leaf or n - nl < min_leaf:
                continue
            w = 0.0
            for side in (left, ~left):
                cnt = np.bincount(y[side], minlength=n_classes)
                w += side.sum() * (1 - np.sum((cnt / side.sum()) ** 2))
            if best is None or w / n < best - 1e-15:
                best = w / n
    return best


@pytest.mark.parametrize("seed", range(5))
def test_best_split_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    F = rng.integers(0, 6, (12, 3)).astype(float)
    y = rng.integers(0, 3, 12)
    s = osel.best_split(F, y, 3, 1)
    assert s[2] == pytest.approx(brute_best_split(F, y, 3, 1), abs=1e-14)


def test_tree_separable_is_perfect_and_limits_hold():
    rng = np.random.default_rng(1)
    F = rng.integers(16, 4096, (200, 4)).astype(float)
    y = (F[:, 0] > 500).astype(int) + 2 * (F[:, 2] > 1000).astype(int)
    nodes = osel.tree_train(F, y, 4)
    assert np.array_equal(osel.tree_predict(nodes, F), y)
    nodes_c = osel.tree_train(F, y, 4, max_depth=1, min_leaf=4)

    def depth(j):
        n = nodes_c[j]
        return 0 if n["feature"] < 0 else 1 + max(depth(n["left"]), depth(n["right"]))
    assert depth(0) <= 1
    assert all(n["n"] >= 4 for n in nodes_c)


def test_tree_matches_sklearn_on_tie_free_data():
    sk = pytest.importorskip("sklearn.tree")
    rng = np.random.default_rng(7)
    F = rng.permutation(1000)[:300].reshape(100, 3).astype(float)
    y = ((F[:, 0] > 400) ^ (F[:, 1] > 600)).astype(int) + (F[:, 2] > 800).astype(int)
    for name, (depth, leaf) in osel.TREES.items():
        nodes = osel.tree_train(F, y, 3, depth, leaf)
        ref = sk.DecisionTreeClassifier(max_depth=depth, min_samples_leaf=leaf, random_state=0).fit(F, y)
        Ft = rng.integers(0, 1000, (500, 3)).astype(float) + 0.25
        assert np.array_equal(osel.tree_predict(nodes, Ft), ref.predict(Ft)), name


# ---------------------------------------------------------------- PCA (Section 3.3)
def test_pca_matches_svd():
    X = np.random.default_rng(3).random((50, 8)) @ np.diag([5, 3, 1, 1, 0.5, 0.1, 0.1, 0.01])
    ev = osel.pca_explained_variance(X)
    s = np.linalg.svd(X - X.mean(0), compute_uv=False)
    assert np.allclose(ev, s ** 2 / np.sum(s ** 2), rtol=1e-10, atol=1e-14)
    assert osel.components_for(np.array([0.5, 0.3, 0.15, 0.05]), 0.8) == 2
    assert osel.components_for(np.array([0.5, 0.3, 0.15, 0.05]), 0.95) == 3


def test_pca_top_eigenpairs():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((80, 6)) @ np.diag([4, 3, 2, 1, 0.5, 0.1])
    mean, w, v, tot = osel.pca_top(X, 3)
    cov = np.cov(X.T)
    assert np.allclose(cov @ v, v * w, atol=1e-10)
    assert np.allclose(v.T @ v, np.eye(3), atol=1e-12)
    assert tot == pytest.approx(np.trace(cov)) and np.all(np.diff(w) <= 0)


def test_knn_by_hand():
    train = np.array([[0.0], [1.0], [2.0], [10.0], [11.0]])
    labels = np.array([0, 1, 1, 2, 2])
    assert list(osel.knn_predict(train, labels, np.array([[0.2], [10.4], [1.6]]), 1)) == [0, 2, 1]
    # 3-NN of 1.0: points 1.0, 0.0 and 2.0 (0.0 before 2.0 on the distance tie) -> labels {1, 0, 1} -> 1
    assert list(osel.knn_predict(train, labels, np.array([[1.0]]), 3)) == [1]
    # 2-NN of 0.5: labels 0 and 1 tie -> the nearer (index 0 first on the distance tie) wins
    assert list(osel.knn_predict(train, labels, np.array([[0.5]]), 2)) == [0]


# ---------------------------------------------------------------- regression-tree pruning (Section 4.1)
def planted_regions(seed, n=60, d=7):
    """Sizes whose performance vector depends only on which of three M ranges they fall in."""
    rng = np.random.default_rng(seed)
    F = np.column_stack([rng.permutation(n) * 10.0 + 16, rng.integers(16, 4096, n), rng.integers(16, 4096, n),
                         rng.choice([1, 2, 4, 8, 16], n)]).astype(np.float64)
    region = np.digitize(F[:, 0], [200.0, 450.0])
    proto = rng.random((3, d))
    return F, proto[region], region


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tree_regression_recovers_planted_regions(seed):
    F, Y, region = planted_regions(seed)
    labels, centres = osel.tree_regression_partition(F, Y, 3)
    # same partition (leaf numbering is the tree's own)
    pairs = set(zip(labels.tolist(), region.tolist()))
    assert len(pairs) == 3 and len({a for a, _ in pairs}) == 3 and len({b for _, b in pairs}) == 3
    for j in range(3):
        assert np.allclose(centres[j], Y[labels == j].mean(axis=0), rtol=0, atol=1e-15)
    # no gain left once the planted regions are separated: growth stops at 3 leaves
    labels5, _ = osel.tree_regression_partition(F, Y, 5)
    assert labels5.max() == 2


def test_tree_regression_limits_and_monotone_error():
    rng = np.random.default_rng(4)
    F = rng.random((40, 4)) * 1000
    Y = rng.random((40, 5))
    l1, c1 = osel.tree_regression_partition(F, Y, 1)
    assert np.all(l1 == 0) and np.allclose(c1[0], Y.mean(axis=0))
    sse = []
    for k in range(1, 12):
        labels, centres = osel.tree_regression_partition(F, Y, k)
        assert labels.max() == k - 1 and sorted(set(labels.tolist())) == list(range(k))
        sse.append(sum(osel.leaf_sse(Y[labels == j]) for j in range(k)))
    assert all(b <= a + 1e-12 for a, b in zip(sse, sse[1:]))
    labels, _ = osel.tree_regression_partition(F, Y, 40)  # every sample alone
    assert len(set(labels.tolist())) == 40


@pytest.mark.parametrize("k", [2, 3, 5, 8])
def test_tree_regression_matches_sklearn(k):
    """scikit-learn's best-first regression tree (max_leaf_nodes) gives the same
    partition on tie-free continuous data."""
    tree = pytest.importorskip("sklearn.tree")
    rng = np.random.default_rng(10 + k)
    F = rng.random((80, 4)) * 4096
    Y = rng.random((80, 6)) ** 3
    labels, _ = osel.tree_regression_partition(F, Y, k)
    sk = tree.DecisionTreeRegressor(max_leaf_nodes=k, random_state=0).fit(F, Y)
    leaf = sk.apply(F)
    assert len(set(leaf.tolist())) == k
    assert len(set(zip(labels.tolist(), leaf.tolist()))) == k


# ---------------------------------------------------------------- spectral clustering (Section 4.1)
def test_spectral_embedding_matches_normalised_laplacian():
    """The embedding's eigenvalues are 1 - (smallest eigenvalues of scipy's
    normalised Laplacian); the top one is exactly 1 with eigenvector D^1/2 1."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(5)
    X = rng.random((30, 6))
    A = osel.rbf_affinity(X, 0.7)
    assert np.all(np.diag(A) == 0) and np.allclose(A, A.T)
    U, w = osel.spectral_embedding(A, 4)
    L = csgraph.laplacian(A, normed=True)
    lw = np.linalg.eigvalsh(L)
    assert np.allclose(np.sort(1.0 - w), lw[:4], atol=1e-12)
    assert w[0] == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(np.linalg.norm(U, axis=1), 1.0)
    # the top eigenvector of S is D^1/2 1 (normalised): rows of U before scaling
    d = A.sum(axis=1)
    S = A / np.sqrt(d)[:, None] / np.sqrt(d)[None, :]
    v = np.sqrt(d) / np.linalg.norm(np.sqrt(d))
    assert np.allclose(S @ v, v, atol=1e-12)


def test_spectral_partition_separates_distant_blobs():
    """Three far-apart blobs: the graph has three (numerically) disconnected
    components, eigenvalue 1 has multiplicity 3 and the partition is the blobs."""
    rng = np.random.default_rng(6)
    centres = np.array([[0.0] * 5, [10.0] * 5, [0.0, 10.0, 0.0, 10.0, 0.0]])
    truth = np.repeat(np.arange(3), 12)
    X = centres[truth] + 0.05 * rng.standard_normal((36, 5))
    U, w = osel.spectral_embedding(osel.rbf_affinity(X, 1.0), 3)
    assert np.allclose(w, 1.0, atol=1e-9)
    u = rng.random((4, 3))
    labels, inertia = osel.spectral_partition(X, 3, 1.0, u)
    assert len(set(zip(labels.tolist(), truth.tolist()))) == 3
    assert inertia < 1e-6


def test_cluster_geomean_centres():
    X = np.array([[1.0, 0.5], [0.25, 1.0], [0.5, 0.5], [1.0, 0.0]])
    labels = np.array([0, 0, 1, 1])
    C = osel.cluster_geomean_centres(X, labels, 3, floor=1e-6)
    assert C[0] == pytest.approx([0.5, math.sqrt(0.5)], rel=1e-15)
    assert C[1] == pytest.approx([math.sqrt(0.5), math.sqrt(0.5e-6)], rel=1e-15)
    assert np.all(C[2] == 0)  # empty cluster


# ---------------------------------------------------------------- random-forest trees (Section 5.1 classifiers)
def test_selector_features_by_hand():
    """The sizes pass through; the fifth column is the number of outputs."""
    F = osel.selector_features([[3, 5, 7, 2], [4096, 4096, 16, 16]])
    assert F.shape == (2, 5)
    assert F[0].tolist() == [3, 5, 7, 2, 30]
    assert F[1].tolist() == [4096, 4096, 16, 16, 4096 * 4096 * 16]  # 2^28: exact in FP64


def test_best_labels_by_hand():
    """Position in the deployed list of the fastest deployed column, first on ties."""
    perf = np.array([[1.0, 5.0, 5.0, 0.0], [9.0, 2.0, 3.0, 0.0], [0.0, 0.0, 0.0, 0.0]])
    assert osel.best_labels(perf, [2, 1]).tolist() == [0, 0, 0]  # 5 vs 5: first; 3 vs 2; all zero: first
    assert osel.best_labels(perf, [1, 0]).tolist() == [0, 1, 0]
    assert osel.best_labels(perf, [3, 0, 2]).tolist() == [2, 1, 0]


def test_feature_subset_by_hand():
    # step 0 swaps entries 0 and 0 + 5 % 4 = 1 -> [1, 0, 2, 3]; step 1 swaps 1 and 1 + 7 % 3 = 2 -> [1, 2, 0, 3]
    assert osel.feature_subset(np.array([5, 7, 0, 0]), 4, 2) == [1, 2]
    assert osel.feature_subset(np.array([0, 0, 0, 0]), 4, 1) == [0]
    assert osel.feature_subset(np.array([3, 9, 9, 9]), 4, 4) == [0, 1, 2, 3]


def test_random_forest_tree_restricts_features():
    rng = np.random.default_rng(12)
    F = rng.permutation(4000)[:4 * 120].reshape(120, 4).astype(float)
    y = (F[:, 0] > 2000).astype(int)  # only feature 0 separates the classes
    full = osel.tree_train(F, y, 2)
    assert full[0]["feature"] == 0 and len(full) == 3
    # all features allowed: identical to the plain tree whatever the draws
    draws = rng.integers(0, 2 ** 32, (4096, 4), dtype=np.uint64).astype(np.uint32)
    assert osel.tree_train(F, y, 2, max_features=4, draws=draws) == full
    # root limited to features {1, 2}: its split is the best one over those two alone
    d = draws.copy()
    d[0] = [5, 7, 0, 0]
    nodes = osel.tree_train(F, y, 2, max_features=2, draws=d)
    want = osel.best_split(F, y, 2, 1, features=[1, 2])
    assert (nodes[0]["feature"], nodes[0]["threshold"]) == want[:2]
    for j, nd in enumerate(nodes):
        if nd["feature"] >= 0:
            assert nd["feature"] in osel.feature_subset(d[j], 4, 2)
