"""What the learned selector gains over the method without it.

The performance model is trained by the library's kernels on 80 % of the
2,500-shape GB300 benchmark of the deployed kernels (the table committed
beside the deployment) and scored, like the decision tree, on the held-out
20 % as a fraction of the best deployed kernel per shape (the exhaustive
selector over the deployed set scores 1).

The gain is printed, not assumed.  On the earlier deployments it was positive
(+3.1, +0.2 and +0.9 points); on the set deployed from the current sweep table
the tree already reaches 0.951 and the network ties it (0.944-0.955 over
weight-initialisation seeds, a training loss 140x below its start), so the
assertion allows the seed-to-seed spread of 0.005 below the tree and requires
the network to pick, on geometric mean, a kernel within 7 % of the best
deployed one.
"""
import json
import os

import numpy as np
import pytest

from paper_2008_13145_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEPLOY = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2008_13145_gb300", "deploy")
SEED_SPREAD = 0.005


def test_mlp_against_tree_on_held_out_shapes(lib):
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
    print(f"held-out fraction of the best deployed kernel: MLP {mlp:.4f}, tree {tree:.4f}, gain {mlp - tree:+.4f}")
    assert mlp >= tree - SEED_SPREAD
    assert mlp >= 0.93
