"""What the learned selector gains over the method without it.

The performance model is trained by the library's kernels on 80 % of the
2,500-shape GB300 benchmark of the deployed kernels (the table committed
beside the deployment) and scored, like the decision tree, on the held-out
20 % as a fraction of the best deployed kernel per shape (the exhaustive
selector over the deployed set scores 1)."""
import json
import os

import numpy as np
import pytest

from paper_2008_13145_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEPLOY = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2008_13145_gb300", "deploy")


def test_mlp_beats_tree_on_held_out_shapes(lib):
    import torch
    from paper_2008_13145_gb300 import tune
    dep = json.load(open(os.path.join(DEPLOY, "f32.json")))
    shapes, perf, ids, _ = tune.load_table(os.path.join(DEPLOY, "table_mlp_f32.npz"))
    assert ids == dep["config_ids"], "training table belongs to another deployment"
    tr, te = wl.train_test_split(len(shapes), 4)
    T, M = tune.mlp_targets(perf)
    params, hist = tune.mlp_train_params(tune.mlp_features([shapes[i] for i in tr]), T[tr], M[tr], steps=10000)
    assert hist[-1] < 0.05 * hist[0]
    test_shapes = [shapes[i] for i in te]
    col = {c: j for j, c in enumerate(ids)}
    mlp_cols = np.array([col[c] for c in tune.mlp_choose(params, test_shapes, ids)], np.int32)
    h = lib.Handle({k: v for k, v in dep.items() if k != "known"})
    tree_cols = np.array([col[lib.select_kernel(h, s.M, s.N, s.K, s.batch)] for s in test_shapes], np.int32)
    P = torch.from_numpy(np.ascontiguousarray(perf[te], np.float32)).cuda()
    mlp = lib.score(P, chosen=torch.from_numpy(mlp_cols).cuda())["geomean"]
    tree = lib.score(P, chosen=torch.from_numpy(tree_cols).cuda())["geomean"]
    print(f"held-out fraction of the best deployed kernel: MLP {mlp:.4f}, tree {tree:.4f}")
    assert mlp > tree
