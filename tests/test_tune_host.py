"""Host-side parts of the tuning driver: merging the shards of a sweep (one
box's part each, Section 3.1's data collection split by shape index) and the
seeded group descriptions of the grouped selector."""
import json

import numpy as np

from paper_2008_13145_gb300 import tune
from paper_2008_13145_gb300 import workloads as wl


def fake_record(i, sh, ids):
    return {"i": i, "shape": [sh.M, sh.N, sh.K, sh.batch, sh.transA, sh.transB], "precision": 0,
            "config_ids": ids, "ms": [0.1 * (i + 1) + 0.01 * j for j in range(len(ids))], "status": [0] * len(ids)}


def test_merge_shards_restores_the_sweep(tmp_path):
    shapes = wl.shape_grid(20, 3)
    ids = [5, 7, 9]
    paths = []
    for k in range(3):  # three shards, index % 3 == k, written out of order
        p = tmp_path / f"s{k}.jsonl"
        with open(p, "w") as f:
            for i in reversed(range(k, 20, 3)):
                f.write(json.dumps(fake_record(i, shapes[i], ids)) + "\n")
        paths.append(str(p))
    dup = tmp_path / "dup.jsonl"  # a resumed shard repeating a record: the first one wins
    dup.write_text(json.dumps({**fake_record(4, shapes[4], ids), "ms": [9.0, 9.0, 9.0]}) + "\n")
    merged = tmp_path / "m.jsonl"
    assert tune.merge_sweeps(paths + [str(dup)], str(merged)) == 20
    recs, got_shapes, perf = tune.load_sweep(str(merged))
    assert got_shapes == shapes and [r["i"] for r in recs] == list(range(20))
    want = np.array([[sh.flops / (ms * 1e6) for ms in fake_record(i, sh, ids)["ms"]] for i, sh in enumerate(shapes)])
    assert np.allclose(perf, want, rtol=1e-12)


def test_group_specs_and_features():
    a, b = tune.group_specs(50), tune.group_specs(50)
    assert a == b and len(a) == 50
    assert all(c in tune.GROUP_COUNTS and (lo, hi) in tune.GROUP_RANGES for c, lo, hi, _ in a)
    probs = [dict(M=m, N=n, K=k) for m, n, k in [(5, 9, 2), (1, 3, 8), (7, 4, 6), (3, 1, 1)]]
    assert tune.group_features(probs) == [3, 3, 2, 4]  # lower medians and the count
