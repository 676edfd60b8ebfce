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


def test_cutoff_and_trees():
    assert osel.CUTOFF == GOLD["raw_cutoff"]["threshold"]
    for name in "ABC":
        assert list(osel.TREES[name]) == GOLD["trees"][name]


def test_paper_config_space_size():
    g = GOLD["config_space"]
    assert len(g["tile_values"]) ** 3 == g["n_tile_configs"]
    assert g["n_tile_configs"] * len(g["work_groups"]) == g["n_configs"]
