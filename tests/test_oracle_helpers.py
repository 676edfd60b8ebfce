"""Direct pins for the oracle's helper functions.

Each helper is also reached through a pinned caller (k-means, the trees, the
convolution, the MLP, the BF16 split).  Here each one is checked on its own,
against closed forms, brute force on tiny inputs, or a library routine.  A
mistake then fails next to where it was made."""
import itertools

import numpy as np
import pytest

from oracle import bf16 as ob
from oracle import mlp as om
from oracle import select as osel
from oracle import vgg as ov


# ---------------------------------------------------------------- k-means helpers (Section 3.4)
def test_sq_dist_closed_forms():
    assert osel.sq_dist(np.array([3.0, 0.0]), np.array([0.0, 4.0])) == 25.0  # 3-4-5 triangle
    assert osel.sq_dist(np.array([1.5, -2.0, 7.0]), np.array([1.5, -2.0, 7.0])) == 0.0
    rng = np.random.default_rng(3)
    for _ in range(20):
        x, c = rng.standard_normal(9), rng.standard_normal(9)
        assert osel.sq_dist(x, c) == pytest.approx(np.linalg.norm(x - c) ** 2, rel=1e-13)
        assert osel.sq_dist(x, c) == osel.sq_dist(c, x)


def test_assign_matches_brute_force_distance_matrix():
    cdist = pytest.importorskip("scipy.spatial.distance").cdist
    rng = np.random.default_rng(11)
    X, C = rng.standard_normal((40, 5)), rng.standard_normal((6, 5))
    labels, inertia = osel.assign(X, C)
    D = cdist(X, C, "sqeuclidean")
    assert np.array_equal(labels, np.argmin(D, axis=1))
    assert inertia == pytest.approx(D.min(axis=1).sum(), rel=1e-12)


def test_assign_breaks_ties_to_the_lowest_index():
    C = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0]])
    X = np.array([[0.0, 0.0],    # equidistant from all three: centre 0
                  [0.0, -1.0],   # equidistant from centres 0 and 1: centre 0
                  [-0.5, 0.5]])  # equidistant from centres 1 and 2: centre 1
    labels, inertia = osel.assign(X, C)
    assert labels.tolist() == [0, 0, 1]
    assert inertia == pytest.approx(1.0 + 2.0 + 0.5, rel=1e-15)


# ---------------------------------------------------------------- decision-tree helpers (Section 4)
def test_gini_closed_forms():
    g = osel.gini_ordered(np.array([[7, 0, 0], [3, 3, 3], [5, 5, 0], [1, 3, 0]]), np.array([7, 9, 10, 4]))
    assert g[0] == 0.0                                       # pure node
    assert g[1] == pytest.approx(1.0 - 1.0 / 3.0, rel=1e-15)  # uniform over 3 classes
    assert g[2] == pytest.approx(0.5, rel=1e-15)              # two equal classes
    assert g[3] == pytest.approx(2 * 0.25 * 0.75, rel=1e-15)  # 2 p (1 - p)


def test_gini_broadcasts_over_leading_dimensions():
    rng = np.random.default_rng(5)
    counts = rng.integers(0, 9, size=(4, 6, 3))
    n = counts.sum(axis=-1) + 1  # any positive totals
    g = osel.gini_ordered(counts, n)
    assert g.shape == (4, 6)
    for i, j in itertools.product(range(4), range(6)):
        p = counts[i, j] / n[i, j]
        assert g[i, j] == pytest.approx(1.0 - float(np.sum(p * p)), rel=1e-14, abs=1e-15)


def test_gini_equals_scikit_learn_root_impurity():
    tree = pytest.importorskip("sklearn.tree")
    y = np.array([0] * 5 + [1] * 9 + [2] * 2)
    X = np.arange(len(y), dtype=np.float64).reshape(-1, 1)
    clf = tree.DecisionTreeClassifier(max_depth=1, random_state=0).fit(X, y)
    counts = np.bincount(y, minlength=3)
    assert osel.gini_ordered(counts, len(y)) == pytest.approx(clf.tree_.impurity[0], rel=1e-12)


def _sse(Y):
    """Summed squared error about the mean, written as n x (per-output variance)."""
    return 0.0 if len(Y) == 0 else float(len(Y) * np.var(Y, axis=0).sum())


def test_regression_split_matches_brute_force():
    rng = np.random.default_rng(17)
    F = rng.integers(0, 50, size=(24, 3)).astype(np.float64) / 8.0
    Y = rng.standard_normal((24, 4))
    idx = np.arange(24)
    gain, f, thr = osel.regression_split(F, Y, idx)
    best = None
    for ff in range(3):
        vals = sorted(set(F[:, ff]))
        for a, b in zip(vals[:-1], vals[1:]):
            t = (a + b) / 2.0
            g = _sse(Y) - _sse(Y[F[:, ff] <= t]) - _sse(Y[F[:, ff] > t])
            if best is None or g > best[0] + 1e-12:
                best = (g, ff, t)
    assert gain == pytest.approx(best[0], rel=1e-10)
    assert (f, thr) == (best[1], best[2])


def test_regression_split_finds_a_planted_step():
    rng = np.random.default_rng(23)
    F = rng.uniform(0.0, 1.0, size=(60, 3))
    Y = np.where(F[:, [1]] > 0.6, 5.0, -5.0) + 0.01 * rng.standard_normal((60, 2))
    gain, f, thr = osel.regression_split(F, Y, np.arange(60))
    lo, hi = F[F[:, 1] <= 0.6, 1].max(), F[F[:, 1] > 0.6, 1].min()
    assert f == 1
    assert thr == (lo + hi) / 2.0
    assert osel.regression_split(F, Y, np.array([7])) is None  # one sample: no split


def test_regression_split_equals_scikit_learn_stump():
    tree = pytest.importorskip("sklearn.tree")
    rng = np.random.default_rng(29)
    F = rng.permutation(np.arange(40, dtype=np.float64)).reshape(20, 2) / 4.0  # distinct, float32-exact
    Y = rng.standard_normal((20, 3))
    gain, f, thr = osel.regression_split(F, Y, np.arange(20))
    reg = tree.DecisionTreeRegressor(max_depth=1, random_state=0).fit(F, Y)
    assert f == reg.tree_.feature[0]
    left = F[:, f] <= thr
    assert np.array_equal(left, F[:, reg.tree_.feature[0]] <= reg.tree_.threshold[0])


# ---------------------------------------------------------------- VGG16 im2col
def test_im2col_gathers_the_zero_padded_neighbourhood():
    N, H, W, C = 2, 3, 4, 2
    x = np.arange(1, N * H * W * C + 1, dtype=np.float64).reshape(N, H, W, C)
    cols = ov.im2col3x3(x)
    assert cols.shape == (N * H * W, 9 * C)
    for n, h, w in itertools.product(range(N), range(H), range(W)):
        row = cols[(n * H + h) * W + w]
        for kh, kw, c in itertools.product(range(3), range(3), range(C)):
            hh, ww = h + kh - 1, w + kw - 1
            want = x[n, hh, ww, c] if 0 <= hh < H and 0 <= ww < W else 0.0
            assert row[(kh * 3 + kw) * C + c] == want


# ---------------------------------------------------------------- MLP parameter layout
def test_pack_unpack_round_trip_and_layout():
    assert om.N_PARAMS == 7 * 64 + 64 + 64 * 64 + 64 + 64 * 8 + 8 == 5192
    theta = np.arange(om.N_PARAMS, dtype=np.float64)
    parts = om.unpack(theta)
    assert [p.shape for p in parts] == [tuple(s) for s in om.SIZES]
    assert parts[0][0, 1] == 1.0 and parts[1][0] == 7 * 64  # row-major, in layer order
    assert np.array_equal(om.pack(parts), theta)


# ---------------------------------------------------------------- BF16 decoding
def test_bf16_bits_to_f32_matches_torch_and_closed_forms():
    assert ob.bf16_bits_to_f32(np.array([0x3F80, 0xC000, 0x0000, 0x8000, 0x7F80], np.uint16)).tolist() == \
        [1.0, -2.0, 0.0, -0.0, float("inf")]
    assert ob.bf16_bits_to_f32(np.array([0x0001], np.uint16))[0] == np.float32(2.0 ** -133)  # smallest subnormal
    torch = pytest.importorskip("torch")
    bits = np.arange(0, 1 << 16, 7, dtype=np.uint16)
    ref = torch.from_numpy(bits.view(np.int16).copy()).view(torch.bfloat16).float().numpy()
    got = ob.bf16_bits_to_f32(bits)
    finite = np.isfinite(ref)
    assert np.array_equal(got[finite], ref[finite])
    assert np.array_equal(np.isnan(got), np.isnan(ref))
