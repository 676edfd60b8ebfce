"""The constants the paper prints, read from tests/golden/paper_constants.json."""
import json
import os

import numpy as np

from oracle import select as osel

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_sigmoid_points():
    g = GOLD["sigmoid"]
    for x, fx in g["points"]:
        assert abs(osel.normalise(np.array([[x, 1.0]]), "sigmoid")[0, 0] - fx) < 1e-12
    for x, bound in g["below"]:
        assert osel.normalise(np.array([[x, 1.0]]), "sigmoid")[0, 0] < bound


def test_cutoffs_act_at_the_printed_threshold():
    """Section 3.4: the raw cutoff zeroes every configuration below 90 % of the
    size's best and leaves the others as they are; the standard cutoff then
    rescales [0.9, 1] onto [0, 1]."""
    t = GOLD["raw_cutoff"]["threshold"]
    row = np.array([[0.5, t - 1e-9, t, (1 + t) / 2, 1.0]]) * 7.0  # throughputs; best 7
    raw = osel.normalise(row, "raw_cutoff")[0]
    assert np.array_equal(raw, [0.0, 0.0, t, (1 + t) / 2, 1.0])
    std = osel.normalise(row, "standard_cutoff")[0]
    assert np.allclose(std, [0.0, 0.0, 0.0, 0.5, 1.0], atol=1e-12)


def _depth_and_leaf_sizes(nodes):
    depth, sizes = {0: 0}, []
    for j, nd in enumerate(nodes):
        if nd["feature"] < 0:
            sizes.append(nd["n"])
        else:
            depth[nd["left"]] = depth[nd["right"]] = depth[j] + 1
    return max(depth.values()), sizes


def test_trees_follow_the_printed_limits():
    """Section 5.1: tree A grows until its leaves are pure, B stops at depth 6
    with at least 3 sizes per leaf, C at depth 3 with at least 4.  On labels
    that need many splits (a period-3 pattern along one feature) each tree
    reaches exactly its printed limits."""
    F = np.arange(96, dtype=np.float64).reshape(-1, 1)
    y = (np.arange(96) // 2) % 3
    for name in "ABC":
        max_depth, min_leaf = GOLD["trees"][name]
        assert list(osel.TREES[name]) == [max_depth, min_leaf]
        nodes = osel.tree_train(F, y, 3, max_depth, min_leaf)
        depth, leaves = _depth_and_leaf_sizes(nodes)
        assert min(leaves) >= min_leaf and sum(leaves) == 96
        if max_depth is None:  # grown until pure
            pred = osel.tree_predict(nodes, F)
            assert np.array_equal(pred, y) and depth > 6
        else:
            assert depth == max_depth


def test_config_space_keeps_the_papers_tile_values():
    """Section 3: per-thread tile rows and columns take the values {1, 2, 4, 8};
    of the paper's ten work-group shapes the library keeps the six with at
    least 8 threads along each side (a one-wide block cannot coalesce its
    loads), and the ten give 640 configurations."""
    g = GOLD["config_space"]
    assert len(g["tile_values"]) ** 3 == g["n_tile_configs"]
    assert g["n_tile_configs"] * len(g["work_groups"]) == g["n_configs"]
    from paper_2008_13145_gb300 import build
    build.build_library()
    from paper_2008_13145_gb300 import kselect as ks
    tm, tn, wg = set(), set(), set()
    for cid in range(576):
        _, a, b, wx, wy, *_ = ks.config_params(cid)
        tm.add(a); tn.add(b); wg.add((wx, wy))
    assert sorted(tm) == g["tile_values"] and sorted(tn) == g["tile_values"]
    assert wg == {tuple(w) for w in g["work_groups"] if min(w) >= 8}
