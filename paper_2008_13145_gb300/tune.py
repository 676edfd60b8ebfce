"""Tuning driver: benchmark every configuration over a shape grid, prune the
set by k-means, train the runtime classifier, and write a deployment.

Each numeric step runs in the library (GPU kernels for benchmarking,
normalisation, clustering and scoring; the library's host code for CART and
representatives); this module sequences the calls and reads/writes files.

    python -m paper_2008_13145_gb300.tune sweep  --precision f32 --n 1000 --seed 1 --out sweep_f32.jsonl
    python -m paper_2008_13145_gb300.tune deploy --sweep sweep_f32.jsonl --k 8 --tree B --out f32.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
DEPLOY_DIR = os.path.join(HERE, "deploy")
TREES = {"A": (None, 1), "B": (6, 3), "C": (3, 4)}  # Section 5.1: (max depth, min samples per leaf)


def _ks():
    from . import kselect
    return kselect


def ld_multiple(precision: int) -> int:
    return 8 if precision == 2 else 4


def alloc_inputs(shape: wl.Shape, precision: int, seed: int, device="cuda"):
    """Device buffers (A, B, C, lda, ldb, ldc) for one shape, A and B uniform[-1,1)
    from the library's counter-based fill (BF16 for the BF16 family)."""
    import torch
    ks = _ks()
    m = ld_multiple(precision)
    ar, ac = shape.stored_a()
    br, bc = shape.stored_b()
    lda, ldb, ldc = wl.round_up(ac, m), wl.round_up(bc, m), wl.round_up(shape.N, 4)
    A = torch.empty(shape.batch * ar * lda, device=device)
    B = torch.empty(shape.batch * br * ldb, device=device)
    ks.fill_uniform(A, shape.batch * ar, ac, lda, 1, 2 * seed + 1)
    ks.fill_uniform(B, shape.batch * br, bc, ldb, 1, 2 * seed + 2)
    if precision == 2:
        A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
    C = torch.empty(shape.batch * shape.M * ldc, device=device)
    return A, B, C, lda, ldb, ldc


SPLIT_BASE = 2000  # ids of the FP32 split-K kind: SPLIT_BASE + base config


# ---------------------------------------------------------------- Section 3.1
def sweep(shapes: list[wl.Shape], precision: int, out_path: str, seed: int = 0, refine_ratio: float = 2.0,
          min_total_ms: float = 2.0, config_ids: list[int] | None = None, log=sys.stderr,
          shard: tuple[int, int] = (0, 1)) -> np.ndarray | None:
    """Benchmark every config on every shape; append one JSON line per shape
    to out_path and skip shapes already there (resume; a partial last line, as a
    sweep killed while writing leaves it, is dropped and its shape re-run).
    Returns GFLOP/s (n x c).
    With shard = (k, n) only the shapes with index % n == k are run (one box's
    part of a sweep split over several; `merge_sweeps` joins the files) and
    None is returned."""
    import torch
    ks = _ks()
    ids = list(config_ids) if config_ids is not None else ks.config_ids(precision)
    done = {}
    if os.path.exists(out_path):
        with open(out_path) as f:
            text = f.read()
        lines = text.split("\n")
        keep = []
        for line in lines:
            if not line.strip():
                continue
            try:
                r = json.loads(line)
            except json.JSONDecodeError:
                break  # only the last line can be partial; everything after it is dropped
            keep.append(line)
            if r["config_ids"] == ids:
                done[r["i"]] = r
        if len(keep) != sum(1 for x in lines if x.strip()) or (text and not text.endswith("\n")):
            with open(out_path, "w") as f:
                f.write("".join(x + "\n" for x in keep))
    t0 = time.time()
    with open(out_path, "a") as f:
        for i, sh in enumerate(shapes):
            if i in done or i % shard[1] != shard[0]:
                continue
            A, B, C, lda, ldb, ldc = alloc_inputs(sh, precision, seed + i)
            ms, st = ks.benchmark_configs(ids, sh.transA, sh.transB, sh.M, sh.N, sh.K, A, lda, B, ldb, C, ldc,
                                          sh.batch, refine_ratio=refine_ratio, min_total_ms=min_total_ms)
            rec = {"i": i, "shape": [sh.M, sh.N, sh.K, sh.batch, sh.transA, sh.transB], "precision": precision,
                   "config_ids": ids, "ms": [round(float(x), 6) for x in ms], "status": [int(s) for s in st]}
            f.write(json.dumps(rec) + "\n")
            f.flush()
            done[i] = rec
            del A, B, C
            if log and (i % 50 == 0 or i == len(shapes) - 1):
                best = max(sh.flops / (m * 1e9) for m, s in zip(ms, st) if s == 0 and m > 0) if any(
                    s == 0 for s in st) else 0.0
                log.write(f"[sweep] {i + 1}/{len(shapes)} {sh} best {best:.1f} TFLOP/s  {time.time() - t0:.0f}s\n")
                log.flush()
        torch.cuda.synchronize()
    if shard[1] > 1:
        return None
    return table_from_records([done[i] for i in range(len(shapes))], shapes)


def merge_sweeps(paths: list[str], out_path: str) -> int:
    """Concatenate sweep files (shards of one sweep, or a resumed run) into one,
    one record per shape index (the first one seen wins); returns the count."""
    seen = {}
    for p in paths:
        for line in open(p):
            if line.strip():
                r = json.loads(line)
                seen.setdefault(r["i"], line.strip())
    with open(out_path, "w") as f:
        for i in sorted(seen):
            f.write(seen[i] + "\n")
    return len(seen)


def table_from_records(records, shapes) -> np.ndarray:
    """GFLOP/s per (shape, config); failed configs are 0 (Section 3 reading: a
    configuration that cannot run a size has no throughput)."""
    perf = np.zeros((len(records), len(records[0]["ms"])))
    for r, (rec, sh) in enumerate(zip(records, shapes)):
        ms = np.asarray(rec["ms"], np.float64)
        ok = (np.asarray(rec["status"]) == 0) & (ms > 0)
        perf[r, ok] = sh.flops / (ms[ok] * 1e6)
    return perf


def load_sweep(path: str):
    recs = [json.loads(l) for l in open(path) if l.strip()]
    recs.sort(key=lambda r: r["i"])
    shapes = [wl.Shape(int(r["shape"][0]), int(r["shape"][1]), int(r["shape"][2]), int(r["shape"][3]),
                       r["shape"][4], r["shape"][5]) for r in recs]
    return recs, shapes, table_from_records(recs, shapes)


def save_table(path: str, shapes, perf, config_ids, precision):
    np.savez_compressed(path, perf=perf.astype(np.float32), config_ids=np.asarray(config_ids, np.int32),
                        shapes=np.array([[s.M, s.N, s.K, s.batch, s.transA == "T", s.transB == "T"] for s in shapes],
                                        np.int64), precision=precision)


def load_table(path: str):
    z = np.load(path)
    shapes = [wl.Shape(int(a), int(b), int(c), int(d), "NT"[int(e)], "NT"[int(f)]) for a, b, c, d, e, f in z["shapes"]]
    return shapes, z["perf"].astype(np.float64), [int(x) for x in z["config_ids"]], int(z["precision"])


def combine_tables(paths: list[str], out_path: str, precision: int) -> None:
    """Concatenate sweep tables of the same shapes column-wise (a precision
    class whose candidates span several kernel families)."""
    tabs = [load_table(p) for p in paths]
    shapes = tabs[0][0]
    for t in tabs[1:]:
        assert t[0] == shapes, "tables cover different shapes"
    perf = np.concatenate([t[1] for t in tabs], axis=1)
    ids = [c for t in tabs for c in t[2]]
    save_table(out_path, shapes, perf, ids, precision)


# ---------------------------------------------------------------- Sections 3.4 and 4
def kmeans_draws(n_init: int, k: int, seed: int) -> np.ndarray:
    """The seeding draws (uint32) the clustering consumes: an input, not computed by it."""
    return wl.rng_for(seed, 31).integers(0, 2 ** 32, (n_init, k), dtype=np.uint64).astype(np.uint32)


def prune(perf_train: np.ndarray, k: int, seed: int = 0, norm: str = "standard", n_init: int = 10) -> dict:
    """k-means over the normalised performance vectors of the training sizes;
    the deployed set is each centre's best configuration (Sections 3.4, 4.1-4.2)."""
    import torch
    ks = _ks()
    P = torch.from_numpy(np.ascontiguousarray(perf_train, np.float32)).cuda()
    X = torch.empty_like(P)
    ks.normalise(P, X, norm)
    n, d = X.shape
    cen = torch.empty((k, d), device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    inertia, iters = ks.kmeans(X, k, kmeans_draws(n_init, k, seed), cen, lab)
    cols = ks.representatives(cen.cpu().numpy(), lab.cpu().numpy(), dedupe=True)
    return {"cols": [int(c) for c in cols], "inertia": inertia, "iters": iters,
            "labels": lab.cpu().numpy().tolist()}


def prune_pca(perf_train: np.ndarray, k: int, seed: int = 0, norm: str = "standard", n_init: int = 10,
              var_frac: float = 0.95, r_max: int = 32) -> dict:
    """PCA + k-means pruning (Section 4.1): k-means in the space of the leading
    principal components that explain `var_frac` of the variance; each centre
    is mapped back to a performance vector before taking its best configuration."""
    import torch
    ks = _ks()
    P = torch.from_numpy(np.ascontiguousarray(perf_train, np.float32)).cuda()
    X = torch.empty_like(P)
    ks.normalise(P, X, norm)
    n, d = X.shape
    r_max = min(r_max, d, n - 1)
    V0 = torch.from_numpy(wl.rng_for(seed, 51).standard_normal((d, r_max)).astype(np.float32)).cuda()
    mean, V = torch.empty(d, device="cuda"), torch.empty((d, r_max), device="cuda")
    ev, tot = ks.pca(X, r_max, V0, mean, V)
    r = int(min(r_max, np.searchsorted(np.cumsum(ev) / tot, var_frac - 1e-12) + 1))
    Vr, Y = torch.empty((d, r), device="cuda"), torch.empty((n, r), device="cuda")
    ks.pca(X, r, V0[:, :r].contiguous(), mean, Vr, Y)
    cen = torch.empty((k, r), device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    inertia, iters = ks.kmeans(Y, k, kmeans_draws(n_init, k, seed), cen, lab)
    back = torch.empty((k, d), device="cuda")
    ks.pca_backproject(cen, Vr, mean, back)
    cols = ks.representatives(back.cpu().numpy(), lab.cpu().numpy(), dedupe=True)
    return {"cols": [int(c) for c in cols], "inertia": inertia, "iters": iters, "components": r,
            "explained": float(np.sum(ev[:r]) / tot), "labels": lab.cpu().numpy().tolist()}


def prune_spectral(perf_train: np.ndarray, k: int, seed: int = 0, norm: str = "standard", n_init: int = 10,
                   iters: int = 300, oversample: int = 10) -> dict:
    """Spectral clustering pruning (Section 4.1): k-means on the spectral
    coordinates of the RBF similarity graph of the normalised performance
    vectors, gamma = 1 / (2 x total per-configuration variance) (one over the
    mean squared distance between two sizes); clusters give labels only, so each
    deployed configuration is the best of its cluster's geometric-mean vector
    (Section 4.2)."""
    import torch
    ks = _ks()
    P = torch.from_numpy(np.ascontiguousarray(perf_train, np.float32)).cuda()
    X = torch.empty_like(P)
    ks.normalise(P, X, norm)
    n, d = X.shape
    var = X.double().var(dim=0, unbiased=False).sum().item()
    gamma = 1.0 / (2.0 * var) if var > 0 else 1.0
    r = min(n, k + oversample)
    V0 = torch.from_numpy(wl.rng_for(seed, 71).standard_normal((n, r)).astype(np.float32)).cuda()
    U = torch.empty((n, k), device="cuda")
    ev = ks.spectral_embedding(X, gamma, k, V0, U, iters)
    cen = torch.empty((k, k), device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    inertia, it = ks.kmeans(U, k, kmeans_draws(n_init, k, seed), cen, lab)
    gm = torch.empty((k, d), device="cuda")
    ks.cluster_geomean(X, lab, k, gm)
    cols = ks.representatives(gm.cpu().numpy(), lab.cpu().numpy(), dedupe=True)
    return {"cols": [int(c) for c in cols], "inertia": inertia, "iters": it, "gamma": gamma,
            "eigenvalues": [float(v) for v in ev], "labels": lab.cpu().numpy().tolist()}


def prune_tree(perf_train: np.ndarray, shapes_train, k: int, norm: str = "standard") -> dict:
    """Decision-tree pruning (Section 4.1): a regression tree from the sizes to
    the normalised performance vectors with at most k leaves; each leaf's mean
    vector stands for its sizes and gives one deployed configuration."""
    import torch
    ks = _ks()
    P = torch.from_numpy(np.ascontiguousarray(perf_train, np.float32)).cuda()
    X = torch.empty_like(P)
    ks.normalise(P, X, norm)
    labels, centres = ks.tree_regress(features(shapes_train), X.cpu().numpy(), k)
    cols = ks.representatives(centres, labels, dedupe=True)
    return {"cols": [int(c) for c in cols], "inertia": None, "leaves": int(centres.shape[0]),
            "labels": labels.tolist()}


def prune_by(method: str, perf_train: np.ndarray, shapes_train, k: int, seed: int = 0, norm: str = "standard"):
    if method == "kmeans":
        return prune(perf_train, k, seed, norm)
    if method == "pca":
        return prune_pca(perf_train, k, seed, norm)
    if method == "spectral":
        return prune_spectral(perf_train, k, seed, norm)
    if method == "tree":
        return prune_tree(perf_train, shapes_train, k, norm)
    raise ValueError(method)


def features(shapes) -> np.ndarray:
    """The selector's feature rows of the sizes (computed by the library)."""
    return _ks().selector_features([[s.M, s.N, s.K, s.batch] for s in shapes])


def train_tree(perf_train: np.ndarray, shapes_train, cols: list[int], tree: str = "B") -> list[dict]:
    """Section 5.1: label each training size with its best deployed kernel and fit the tree."""
    ks = _ks()
    y = ks.best_labels(perf_train, cols)
    depth, leaf = TREES[tree]
    return ks.tree_train(features(shapes_train), y, len(cols), depth, leaf)


def evaluate(perf_test: np.ndarray, shapes_test, deployment: dict, all_ids: list[int]) -> dict:
    """Section 4.3 scores on held-out sizes, computed by the library's score kernel."""
    import torch
    ks = _ks()
    h = ks.Handle(deployment)
    col_of = {cid: j for j, cid in enumerate(all_ids)}
    chosen = np.array([col_of[ks.select_kernel(h, s.M, s.N, s.K, s.batch)] for s in shapes_test], np.int32)
    P = torch.from_numpy(np.ascontiguousarray(perf_test, np.float32)).cuda()
    dep_cols = [col_of[c] for c in deployment["config_ids"]]
    return {"deployed_max": ks.score(P, dep_cols),
            "tree": ks.score(P, dep_cols, chosen=torch.from_numpy(chosen).cuda()),
            "exhaustive": ks.score(P),
            "chosen_cols": chosen.tolist()}


def train_forest(perf_train: np.ndarray, shapes_train, cols: list[int], n_trees: int = 16, max_features: int = 2,
                 seed: int = 0) -> list[list[dict]]:
    """Random-forest selector (Tables 1-2's RandomForest as a runtime classifier):
    n_trees type-A trees, each on a bootstrap of the training sizes with
    max_features of the selector's features per node, all draws seeded inputs."""
    ks = _ks()
    y = ks.best_labels(perf_train, cols)
    F = features(shapes_train)
    rng = wl.rng_for(seed, 91)
    boot = rng.integers(0, len(y), (n_trees, len(y)))
    draws = rng.integers(0, 2 ** 32, (n_trees, 8192, ks.TREE_FEATURES), dtype=np.uint64).astype(np.uint32)
    return [ks.tree_train_rf(F[boot[b]], y[boot[b]], len(cols), max_features, draws[b], None, 1)
            for b in range(n_trees)]


def forest_deploy(deploy_path: str, table_path: str, n_trees: int = 16, seed: int = 0, split_seed: int = 1) -> dict:
    """The deployment at deploy_path (same deployed kernels, known table and MLP)
    with a random forest trained on the same training sizes as its selector."""
    shapes, perf, ids, _ = load_table(table_path)
    dep = json.load(open(deploy_path))
    tr, te = wl.train_test_split(len(shapes), split_seed)
    col_of = {cid: j for j, cid in enumerate(ids)}
    cols = [col_of[c] for c in dep["config_ids"]]
    out = {k: v for k, v in dep.items() if k != "meta"}
    out["forest"] = train_forest(perf[tr], [shapes[i] for i in tr], cols, n_trees, seed=seed)
    ev = evaluate(perf[te], [shapes[i] for i in te], {k: v for k, v in out.items() if k != "known"}, ids)
    out["meta"] = {**dep.get("meta", {}), "selector": f"random forest, {n_trees} trees, 2 of 4 features per node",
                   "forest_seed": seed,
                   "scores": {key: v for key, v in ev.items() if key != "chosen_cols"}}
    return out


def retree(deploy_path: str, table_path: str, split_seed: int = 1) -> dict:
    """The deployment at deploy_path with its tree retrained (same deployed
    kernels, known table, MLP and tree type) on the table's training sizes,
    and its held-out scores recomputed."""
    ks = _ks()
    shapes, perf, ids, _ = load_table(table_path)
    dep = json.load(open(deploy_path))
    tr, te = wl.train_test_split(len(shapes), split_seed)
    col_of = {cid: j for j, cid in enumerate(ids)}
    cols = [col_of[c] for c in dep["config_ids"]]
    tree = dep.get("meta", {}).get("tree", "B")
    out = {k: v for k, v in dep.items() if k != "meta"}
    out["nodes"] = train_tree(perf[tr], [shapes[i] for i in tr], cols, tree)
    out.pop("forest", None)
    ev = evaluate(perf[te], [shapes[i] for i in te], {k: v for k, v in out.items() if k != "known"}, ids)
    meta = dict(dep.get("meta", {}))
    import torch
    topn = [int(c) for c in ks.top_n(perf[tr].astype(np.float32), len(cols))]
    ev["top_n"] = ks.score(torch.from_numpy(np.ascontiguousarray(perf[te], np.float32)).cuda(), topn)
    meta["scores"] = {key: v for key, v in ev.items() if key != "chosen_cols"}
    meta["features"] = "M, N, K, batch, M*N*batch"
    out["meta"] = meta
    return out


def deploy(table_path: str, k: int, tree: str, seed: int, norm: str = "standard", split_seed: int = 1,
           method: str = "kmeans") -> dict:
    shapes, perf, ids, precision = load_table(table_path)
    tr, te = wl.train_test_split(len(shapes), split_seed)
    pr = prune_by(method, perf[tr], [shapes[i] for i in tr], k, seed, norm)
    nodes = train_tree(perf[tr], [shapes[i] for i in tr], pr["cols"], tree)
    dep = {"precision": precision, "config_ids": [ids[c] for c in pr["cols"]], "nodes": nodes}
    ev = evaluate(perf[te], [shapes[i] for i in te], dep, ids)
    # Benchmarked (training) sizes keep their exhaustive-best kernel at run time.
    ks = _ks()
    best = ks.best_labels(perf[tr], list(range(len(ids))))
    dep["known"] = [[shapes[i].M, shapes[i].N, shapes[i].K, shapes[i].batch, ids[int(b)]] for i, b in zip(tr, best)]
    topn = [int(c) for c in ks.top_n(perf[tr].astype(np.float32), len(pr["cols"]))]
    import torch
    ev["top_n"] = ks.score(torch.from_numpy(np.ascontiguousarray(perf[te], np.float32)).cuda(), topn)
    dep["meta"] = {"k": k, "tree": tree, "norm": norm, "method": method, "kmeans_seed": seed, "split_seed": split_seed,
                   "n_train": len(tr), "n_test": len(te), "inertia": pr["inertia"],
                   "features": "M, N, K, batch, M*N*batch",
                   "scores": {key: v for key, v in ev.items() if key != "chosen_cols"}}
    return dep


# ---------------------------------------------------------------- learned selector
def shape_rows(shapes, dtype: int = 0) -> np.ndarray:
    return np.array([[s.M, s.N, s.K, s.batch, s.transA == "T", s.transB == "T", dtype] for s in shapes], np.int64)


def mlp_features(shapes, dtype: int = 0):
    """Model inputs (device, n x 7), computed by the library's feature kernel."""
    import torch
    ks = _ks()
    sh = torch.from_numpy(shape_rows(shapes, dtype)).cuda()
    X = torch.empty((len(shapes), 7), device="cuda")
    ks.mlp_features(sh, X)
    return X


def mlp_targets(perf: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per deployed kernel, the log of its throughput relative to the fastest
    deployed kernel for the size, and the mask of measured entries (computed
    by the library's targets kernel)."""
    import torch
    ks = _ks()
    P = torch.from_numpy(np.ascontiguousarray(perf, np.float32)).cuda()
    T, M = torch.empty_like(P), torch.empty_like(P)
    ks.mlp_targets(P, T, M)
    return T.cpu().numpy(), M.cpu().numpy()


def mlp_init(seed: int) -> np.ndarray:
    """He-uniform weights from seeded draws (the draws are the model's input), zero biases."""
    from . import kselect as ks
    u = wl.rng_for(seed, 41).random(ks.MLP_PARAMS)
    sizes = [(7, 64), (64,), (64, 64), (64,), (64, 8), (8,)]
    out, o = [], 0
    for sz in sizes:
        n = int(np.prod(sz))
        out.append((2 * u[o:o + n] - 1) * np.sqrt(6.0 / sz[0]) if len(sz) == 2 else np.zeros(n))
        o += n
    return np.concatenate(out).astype(np.float32)


def mlp_train_params(X, T, mask, steps=10000, lr=3e-3, seed=0, log=None) -> tuple[np.ndarray, list]:
    """Full-batch Adam training by the library's kernels; returns (params, loss history)."""
    import torch
    ks = _ks()
    P = torch.from_numpy(mlp_init(seed)).cuda()
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    hist = torch.empty(steps, device="cuda")
    Xd = X if isinstance(X, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Td, Md = (torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for a in (T, mask))
    ks.mlp_train(P, Xd, Td, Md, m, v, 0, steps, lr=lr, loss_hist=hist)
    h = hist.cpu().numpy().tolist()
    return P.cpu().numpy(), h


def mlp_choose(params: np.ndarray, shapes, config_ids) -> np.ndarray:
    """Config ids the batched selection kernel picks for these shapes."""
    import torch
    ks = _ks()
    h = ks.Handle({"precision": ks.family_of(config_ids[0]), "config_ids": config_ids, "nodes": [],
                   "mlp_params": params})
    sh = torch.from_numpy(shape_rows(shapes)).cuda()
    out = torch.empty(len(shapes), dtype=torch.int32, device="cuda")
    ks.select_kernels_batched(h, sh, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def mlp_study(deploy_path: str, sweep_path: str, n: int = 2500, seed: int = 4, steps: int = 10000) -> dict:
    """Learned selector over the deployed set: sweep n seed-`seed` shapes over
    the deployed kernels, train on 80 %, compare MLP, tree and exhaustive on
    the held-out 20 % (fractions of the best deployed kernel)."""
    import torch
    ks = _ks()
    dep = json.load(open(deploy_path))
    ids = dep["config_ids"]
    shapes = wl.shape_grid(n, seed)
    if sweep_path.endswith(".npz"):  # a table of this sweep saved earlier
        t_shapes, perf, t_ids, _ = load_table(sweep_path)
        assert t_ids == ids and t_shapes == shapes, "the table belongs to another deployment or grid"
    else:
        perf = sweep(shapes, dep["precision"], sweep_path, config_ids=ids)
    tr, te = wl.train_test_split(n, seed)
    X = mlp_features([shapes[i] for i in tr])
    T, M = mlp_targets(perf)
    params, hist = mlp_train_params(X, T[tr], M[tr], steps=steps)
    te_shapes = [shapes[i] for i in te]
    col = {c: j for j, c in enumerate(ids)}
    mlp_cols = np.array([col[c] for c in mlp_choose(params, te_shapes, ids)], np.int32)
    h = ks.Handle(dep)
    tree_cols = np.array([col[ks.select_kernel(h, s.M, s.N, s.K, s.batch)] for s in te_shapes], np.int32)
    P = torch.from_numpy(np.ascontiguousarray(perf[te], np.float32)).cuda()
    res = {"n_train": len(tr), "n_test": len(te), "loss_first": hist[0], "loss_last": hist[-1],
           "mlp": ks.score(P, chosen=torch.from_numpy(mlp_cols).cuda()),
           "tree": ks.score(P, chosen=torch.from_numpy(tree_cols).cuda()),
           "exhaustive_deployed": ks.score(P)}
    return {"params": params.tolist(), "study": res}


# ---------------------------------------------------------------- pruning study (Figures 5-6 analogue)
def pruning_study(table_path: str, k_values=range(4, 16), seed: int = 0, split_seed: int = 1) -> dict:
    """Held-out deployed-set maximum (geometric mean of the best deployed
    kernel's fraction of the per-shape optimum) for k-means, PCA + k-means,
    spectral clustering and decision-tree pruning under each normalisation of
    Section 3.4 and for the Top-N baseline, k = 4..15."""
    import torch
    ks = _ks()
    shapes, perf, ids, _ = load_table(table_path)
    tr, te = wl.train_test_split(len(shapes), split_seed)
    s_tr = [shapes[i] for i in tr]
    P = torch.from_numpy(np.ascontiguousarray(perf[te], np.float32)).cuda()
    methods = {"kmeans": "kmeans", "pca_kmeans": "pca", "spectral": "spectral", "tree": "tree"}
    out = {"k": list(k_values), "top_n": []}
    for key in methods:
        out[key] = {}
    for norm in ("standard", "raw_cutoff", "standard_cutoff", "sigmoid"):
        for key, method in methods.items():
            out[key][norm] = [ks.score(P, prune_by(method, perf[tr], s_tr, k, seed, norm)["cols"])["geomean"]
                              for k in k_values]
    out["top_n"] = [ks.score(P, [int(c) for c in ks.top_n(perf[tr].astype(np.float32), k)])["geomean"]
                    for k in k_values]
    return out


# ---------------------------------------------------------------- classifiers (Tables 1-2 analogue)
def classifier_study(table_path: str, k_values=(5, 6, 8, 15), seed: int = 0, split_seed: int = 1,
                     n_bag: int = 16, mlp_steps: int = 10000) -> dict:
    """For each deployed-set size k (PCA + k-means selection, as in Section 5),
    the held-out geometric-mean fraction of the per-shape optimum reached by:
    decision trees A/B/C, 1/3/7 nearest neighbours on the performance model's
    features, bagged trees (n_bag bootstrap trees of type A, majority vote, from
    seeded draws), a random forest (the same bootstraps, each node limited to 2
    of the selector's features) and, for k <= 8, the MLP performance model."""
    import torch
    ks = _ks()
    shapes, perf, ids, prec = load_table(table_path)
    tr, te = wl.train_test_split(len(shapes), split_seed)
    s_tr, s_te = [shapes[i] for i in tr], [shapes[i] for i in te]
    P = torch.from_numpy(np.ascontiguousarray(perf[te], np.float32)).cuda()
    X_tr, X_te = mlp_features(s_tr), mlp_features(s_te)
    F_tr, F_te = features(s_tr), features(s_te)
    rng = wl.rng_for(seed, 61)
    boot = rng.integers(0, len(tr), (n_bag, len(tr)))
    rf_draws = wl.rng_for(seed, 81).integers(0, 2 ** 32, (n_bag, 8192, ks.TREE_FEATURES),
                                             dtype=np.uint64).astype(np.uint32)
    out = {"k": list(k_values), "deployed_max": [], "classifiers": {}}

    def add(name, cols_chosen):
        out["classifiers"].setdefault(name, []).append(
            ks.score(P, chosen=torch.from_numpy(np.asarray(cols_chosen, np.int32)).cuda())["geomean"])

    def tree_predict(nodes, F):
        hh = ks.Handle({"precision": prec, "config_ids": cfg_ids, "nodes": nodes})
        col = {c: j for j, c in enumerate(cfg_ids)}
        return np.array([col[ks.select_kernel(hh, int(f[0]), int(f[1]), int(f[2]), int(f[3]))] for f in F])

    for k in k_values:
        cols = prune_pca(perf[tr], k, seed)["cols"]
        cfg_ids = [ids[c] for c in cols]
        y = ks.best_labels(perf[tr], cols)
        out["deployed_max"].append(ks.score(P, cols)["geomean"])
        for name, (depth, leaf) in TREES.items():
            add(f"DecisionTree{name}", [cols[j] for j in tree_predict(ks.tree_train(F_tr, y, k, depth, leaf), F_te)])
        yd = torch.from_numpy(y).cuda()
        for nn in (1, 3, 7):
            pred = torch.empty(len(te), dtype=torch.int32, device="cuda")
            ks.knn(X_tr, yd, X_te, nn, pred)
            add(f"{nn}NearestNeighbor", [cols[j] for j in pred.cpu().numpy()])
        votes = np.zeros((len(te), k), np.int64)
        rf_votes = np.zeros((len(te), k), np.int64)
        for b in range(n_bag):
            nodes = ks.tree_train(F_tr[boot[b]], y[boot[b]], k, None, 1)
            votes[np.arange(len(te)), tree_predict(nodes, F_te)] += 1
            rf = ks.tree_train_rf(F_tr[boot[b]], y[boot[b]], k, 2, rf_draws[b], None, 1)
            rf_votes[np.arange(len(te)), tree_predict(rf, F_te)] += 1
        add("BaggedTrees", [cols[j] for j in np.argmax(votes, axis=1)])
        add("RandomForest", [cols[j] for j in np.argmax(rf_votes, axis=1)])
        if k <= 8:
            T, M = mlp_targets(np.pad(perf[tr][:, cols], ((0, 0), (0, 8 - k))))
            params, _ = mlp_train_params(X_tr, T, M, steps=mlp_steps, seed=seed)
            col = {c: j for j, c in enumerate(cfg_ids)}
            add("MLP", [cols[col[c]] for c in mlp_choose(params, s_te, cfg_ids)])
        else:
            out["classifiers"].setdefault("MLP", []).append(None)
    return out


# ---------------------------------------------------------------- grouped launch (autotuned tile shape)
def grouped_workload(family: int, n: int = 256, seed: int = 3, data_seed: int = 500, lo: int = 32, hi: int = 4096):
    """Device buffers of an uneven group (M, N, K log-uniform in [lo, hi]), K-contiguous operands."""
    probs, keep = [], []
    for i, sh in enumerate(wl.grouped_problems(n, seed, lo, hi)):
        A, B, C, lda, ldb, ldc = alloc_inputs(sh, family, data_seed + i)
        keep.append((A, B, C))
        probs.append(dict(M=sh.M, N=sh.N, K=sh.K, transA="N", transB="T", A=A, lda=lda, B=B, ldb=ldb, C=C, ldc=ldc))
    flops = sum(2 * q["M"] * q["N"] * q["K"] for q in probs)
    return probs, keep, flops


def time_grouped_graph(plan, reps: int = 10, warmup: int = 2) -> float:
    """Mean ms of one replay of a CUDA graph holding one grouped launch."""
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.run(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(s)
    for _ in range(warmup):
        g.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def grouped_tune(families=("tf32", "bf16", "f32x3")) -> dict:
    """The benchmark step of the method applied to the grouped launch: every
    tile configuration of a family timed on the group; the fastest is deployed."""
    ks = _ks()
    out = {}
    for name in families:
        fam = ks.PRECISIONS[name]
        probs, keep, flops = grouped_workload(fam)
        res = []
        for cid in ks.config_ids(fam):
            plan = ks.GroupedPlan(cid, probs)
            ms = time_grouped_graph(plan)
            plan.close()
            res.append({"config": cid, "params": ks.config_params(cid), "ms": ms, "tflops": flops / (ms * 1e9)})
        best = max(res, key=lambda r: r["tflops"])
        out[name] = {"config": best["config"], "tflops": best["tflops"], "gflop": flops / 1e9, "all": res}
        del keep
    return out


# ---------------------------------------------------------------- grouped tile-shape selector
GROUP_COUNTS = (16, 32, 64, 128, 256)
GROUP_RANGES = ((32, 512), (64, 1024), (128, 2048), (32, 4096), (256, 4096))


def group_specs(n_groups: int = 100, seed: int = 11) -> list[tuple[int, int, int, int]]:
    """Seeded groups (problem count, lo, hi, problem seed): the count and the
    log-uniform size range of each group drawn from the sets above."""
    rng = wl.rng_for(seed, 101)
    return [(int(GROUP_COUNTS[rng.integers(len(GROUP_COUNTS))]), *GROUP_RANGES[rng.integers(len(GROUP_RANGES))],
             1000 + g) for g in range(n_groups)]


def group_features(problems) -> list[int]:
    """(median M, median N, median K, count), lower medians, as gemm_grouped_select reads them."""
    c = len(problems)
    med = lambda v: sorted(v)[(c - 1) // 2]
    return [med([q["M"] for q in problems]), med([q["N"] for q in problems]), med([q["K"] for q in problems]), c]


def grouped_sweep(family: str, specs, out_path: str, reps: int = 5, log=sys.stderr) -> tuple[np.ndarray, np.ndarray]:
    """The benchmark step on groups: every tile config of the family timed on
    every group (CUDA-graph replay of one grouped launch).  Resumable JSONL.
    Returns (TFLOP/s n_groups x configs, features n_groups x 4)."""
    ks = _ks()
    fam = ks.PRECISIONS[family]
    ids = ks.config_ids(fam)
    done = {}
    if os.path.exists(out_path):
        for line in open(out_path):
            if line.strip():
                r = json.loads(line)
                done[r["g"]] = r
    t0 = time.time()
    with open(out_path, "a") as f:
        for g, (count, lo, hi, seed) in enumerate(specs):
            if g in done:
                continue
            probs, keep, flops = grouped_workload(fam, count, seed, 700 + g, lo, hi)
            tf = []
            for cid in ids:
                plan = ks.GroupedPlan(cid, probs)
                tf.append(flops / (time_grouped_graph(plan, reps=reps) * 1e9))
                plan.close()
            rec = {"g": g, "spec": [count, lo, hi, seed], "features": group_features(probs), "config_ids": ids,
                   "tflops": tf}
            f.write(json.dumps(rec) + "\n")
            f.flush()
            done[g] = rec
            del keep
            if log and (g % 20 == 0 or g == len(specs) - 1):
                log.write(f"[grouped sweep {family}] {g + 1}/{len(specs)}  {time.time() - t0:.0f}s\n")
                log.flush()
    recs = [done[g] for g in range(len(specs))]
    return np.array([r["tflops"] for r in recs]), np.array([r["features"] for r in recs], np.float64)


def grouped_study(family: str, sweep_path: str, n_groups: int = 100, k: int = 4, tree: str = "B", seed: int = 0,
                  split_seed: int = 1) -> dict:
    """Benchmark, prune and classify on groups: the grouped sweep, k-means over
    the standard-normalised per-group vectors, a tree on the group features;
    held-out groups scored against the per-group best tile config."""
    import torch
    ks = _ks()
    specs = group_specs(n_groups)
    perf, F = grouped_sweep(family, specs, sweep_path)
    ids = ks.config_ids(ks.PRECISIONS[family])
    tr, te = wl.train_test_split(n_groups, split_seed)
    pr = prune(perf[tr], k, seed)
    y = ks.best_labels(perf[tr], pr["cols"])
    depth, leaf = TREES[tree]
    nodes = ks.tree_train(ks.selector_features(F[tr]), y, len(pr["cols"]), depth, leaf)
    dep = {"precision": ks.PRECISIONS[family], "config_ids": [ids[c] for c in pr["cols"]], "nodes": nodes}
    h = ks.Handle(dep)
    col = {c: j for j, c in enumerate(ids)}
    chosen = [col[ks.select_kernel(h, *map(int, F[i]))] for i in te]
    P = torch.from_numpy(np.ascontiguousarray(perf[te], np.float32)).cuda()
    scores = {"deployed_max": ks.score(P, pr["cols"]),
              "tree": ks.score(P, pr["cols"], chosen=torch.from_numpy(np.asarray(chosen, np.int32)).cuda()),
              "single_best": ks.score(P, [int(np.argmax(np.exp(np.mean(np.log(perf[tr] / perf[tr].max(1, keepdims=True)),
                                                                       axis=0))))])}
    return {"selector": dep, "scores": scores, "n_groups": n_groups, "n_train": len(tr), "n_test": len(te),
            "features": "median M, median N, median K, problem count", "specs": [list(x) for x in specs]}


def grouped_deploy(grouped_path: str, studies: dict[str, str]) -> dict:
    """grouped.json with each family's group classifier: "config" becomes the
    selector's choice for the 256-problem reference group (M, N, K
    log-uniform in [32, 4096], seed 3), "exhaustive_config" keeps the fastest
    config timed on that group."""
    ks = _ks()
    out = json.load(open(grouped_path))
    ref = [dict(M=s.M, N=s.N, K=s.K) for s in wl.grouped_problems(256, 3)]
    for fam, path in studies.items():
        st = json.load(open(path))
        h = ks.Handle(st["selector"])
        entry = out[fam]
        entry.setdefault("exhaustive_config", entry["config"])
        entry["config"] = ks.select_kernel(h, *group_features(ref))
        entry["selector"] = st["selector"]
        entry["selector_scores"] = st["scores"]
        entry["selector_groups"] = {"n_groups": st["n_groups"], "features": st["features"]}
    return out


# ---------------------------------------------------------------- VGG16 layers (Section 6)
def vgg_study(deploy_path: str, sweep_path: str, batches=(1, 16), layout: str = "nhwc") -> dict:
    """Per VGG16 GEMM (im2col convolutions and FC layers): the throughput of the
    kernel the deployed tree selects against the layer's exhaustive best over
    the whole family, and the layer-time-weighted totals."""
    return network_study("vgg16", deploy_path, sweep_path, batches, layout)


def network_study(net: str, deploy_path: str, sweep_path: str, batches=(1, 16), layout: str = "nhwc") -> dict:
    """vgg_study for any network of workloads.NETWORKS: each distinct GEMM of the
    forward pass is benchmarked over every config once; layers that repeat a GEMM
    count once per occurrence in the totals."""
    ks = _ks()
    dep = json.load(open(deploy_path))
    prec = dep["precision"]
    ids = ks.config_ids(prec)
    make = wl.NETWORKS[net]
    layers = [(b, name, sh) for b in batches
              for name, sh in (make(b, layout) if net == "vgg16" else make(b))]
    uniq = {}
    for _, _, sh in layers:
        uniq.setdefault(sh, len(uniq))
    perf_u = sweep(list(uniq), prec, sweep_path, seed=77, config_ids=ids)
    shapes = [sh for _, _, sh in layers]
    perf = perf_u[[uniq[sh] for sh in shapes]]
    h = ks.Handle(dep)
    col = {c: j for j, c in enumerate(ids)}
    mlp = mlp_choose(np.asarray(dep["mlp_params"], np.float32), shapes, dep["config_ids"]) \
        if dep.get("mlp_params") else None
    rows, tot = [], {}
    for i, ((b, name, sh), p) in enumerate(zip(layers, perf)):
        sel = ks.select_kernel(h, sh.M, sh.N, sh.K, sh.batch)
        best = int(np.argmax(p))
        r = {"batch": b, "layer": name, "M": sh.M, "N": sh.N, "K": sh.K, "selected": sel,
             "selected_tflops": p[col[sel]] / 1e3, "best": ids[best], "best_tflops": p[best] / 1e3,
             "ratio": p[col[sel]] / p[best] if p[best] > 0 else 0.0}
        t = tot.setdefault(b, [0.0, 0.0, 0.0, 0.0])
        t[0] += sh.flops / (p[col[sel]] * 1e6)  # ms with the tree's kernel
        t[1] += sh.flops / (p[best] * 1e6)      # ms with the per-layer best
        t[2] += sh.flops
        if mlp is not None:
            m = int(mlp[i])
            r.update({"mlp_selected": m, "mlp_tflops": p[col[m]] / 1e3, "mlp_ratio": p[col[m]] / p[best]})
            t[3] += sh.flops / (p[col[m]] * 1e6)
        rows.append(r)
    totals = {}
    for b, v in tot.items():
        totals[str(b)] = {"selected_ms": v[0], "exhaustive_ms": v[1], "ratio": v[1] / v[0],
                          "selected_tflops": v[2] / (v[0] * 1e9),
                          "distinct_selected": len({r["selected"] for r in rows if r["batch"] == b})}
        if mlp is not None:
            totals[str(b)].update({"mlp_ms": v[3], "mlp_ratio": v[1] / v[3]})
    return {"layers": rows, "totals": totals}


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    s = sub.add_parser("sweep")
    s.add_argument("--precision", default="f32")
    s.add_argument("--n", type=int, default=1000)
    s.add_argument("--seed", type=int, default=1)
    s.add_argument("--out", required=True)
    s.add_argument("--table", default=None)
    s.add_argument("--kind", default="all", choices=["all", "base", "split"],
                   help="FP32 only: every config, the 576 base configs, or the split-K kind")
    s.add_argument("--shard", default="0/1", help="k/n: run the shapes with index % n == k")
    mg = sub.add_parser("merge")
    mg.add_argument("--sweeps", nargs="+", required=True)
    mg.add_argument("--n", type=int, default=1000)
    mg.add_argument("--seed", type=int, default=1)
    mg.add_argument("--table", required=True)
    ml = sub.add_parser("mlp")
    ml.add_argument("--deploy", required=True)
    ml.add_argument("--sweep", required=True)
    ml.add_argument("--n", type=int, default=2500)
    ml.add_argument("--steps", type=int, default=10000)
    ml.add_argument("--out", required=True)
    cb = sub.add_parser("combine")
    cb.add_argument("--tables", nargs="+", required=True)
    cb.add_argument("--precision", default="f32")
    cb.add_argument("--out", required=True)
    cl = sub.add_parser("classifiers")
    cl.add_argument("--table", required=True)
    cl.add_argument("--out", required=True)
    st = sub.add_parser("study")
    st.add_argument("--table", required=True)
    st.add_argument("--out", required=True)
    gr = sub.add_parser("grouped")
    gr.add_argument("--out", required=True)
    gs = sub.add_parser("grouped_select")
    gs.add_argument("--family", required=True, choices=["tf32", "bf16", "f32x3"])
    gs.add_argument("--sweep", required=True)
    gs.add_argument("--groups", type=int, default=100)
    gs.add_argument("--k", type=int, default=4)
    gs.add_argument("--out", required=True)
    gd = sub.add_parser("grouped_deploy")
    gd.add_argument("--grouped", required=True)
    gd.add_argument("--studies", nargs="+", required=True, help="family=path pairs")
    gd.add_argument("--out", required=True)
    vg = sub.add_parser("vgg")
    vg.add_argument("--deploy", required=True)
    vg.add_argument("--sweep", required=True)
    vg.add_argument("--out", required=True)
    vg.add_argument("--layout", default="nhwc", choices=["nhwc", "batched"])
    fo = sub.add_parser("forest")
    fo.add_argument("--deploy", required=True)
    fo.add_argument("--table", required=True)
    fo.add_argument("--trees", type=int, default=16)
    fo.add_argument("--out", required=True)
    nw = sub.add_parser("network")
    nw.add_argument("--net", required=True, choices=sorted(wl.NETWORKS))
    nw.add_argument("--deploy", required=True)
    nw.add_argument("--sweep", required=True)
    nw.add_argument("--out", required=True)
    rt = sub.add_parser("retree")
    rt.add_argument("--deploy", required=True)
    rt.add_argument("--table", required=True)
    rt.add_argument("--out", required=True)
    d = sub.add_parser("deploy")
    d.add_argument("--table", required=True)
    d.add_argument("--k", type=int, default=8)
    d.add_argument("--tree", default="B")
    d.add_argument("--norm", default="standard")
    d.add_argument("--seed", type=int, default=0)
    d.add_argument("--method", default="kmeans", choices=["kmeans", "pca", "spectral", "tree"])
    d.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    ks = _ks()
    if a.cmd == "combine":
        combine_tables(a.tables, a.out, ks.PRECISIONS[a.precision])
        return
    if a.cmd == "classifiers":
        r = classifier_study(a.table)
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
        print(json.dumps(r))
        return
    if a.cmd == "study":
        r = pruning_study(a.table)
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
        print(json.dumps(r))
        return
    if a.cmd == "merge":
        merged = a.table + ".jsonl"
        count = merge_sweeps(a.sweeps, merged)
        recs, shapes, perf = load_sweep(merged)
        assert count == a.n and shapes == wl.shape_grid(a.n, a.seed), "shards do not cover the grid"
        save_table(a.table, shapes, perf, recs[0]["config_ids"], int(recs[0]["precision"]))
        print(json.dumps({"shapes": count, "table": a.table}))
        return
    if a.cmd == "grouped_deploy":
        r = grouped_deploy(a.grouped, dict(x.split("=", 1) for x in a.studies))
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
        print(json.dumps({k: {"config": v["config"], "exhaustive_config": v["exhaustive_config"]}
                          for k, v in r.items()}, indent=1))
        return
    if a.cmd == "grouped_select":
        r = grouped_study(a.family, a.sweep, a.groups, a.k)
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
        print(json.dumps({"config_ids": r["selector"]["config_ids"], "scores": r["scores"]}, indent=1))
        return
    if a.cmd == "grouped":
        r = grouped_tune()
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
        print(json.dumps({k: {"config": v["config"], "tflops": v["tflops"]} for k, v in r.items()}, indent=1))
        return
    if a.cmd == "retree":
        r = retree(a.deploy, a.table)
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
        print(json.dumps(r["meta"]["scores"], indent=1))
        return
    if a.cmd == "forest":
        r = forest_deploy(a.deploy, a.table, a.trees)
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
        print(json.dumps(r["meta"]["scores"], indent=1))
        return
    if a.cmd == "network":
        r = network_study(a.net, a.deploy, a.sweep)
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
        print(json.dumps(r["totals"], indent=1))
        return
    if a.cmd == "vgg":
        r = vgg_study(a.deploy, a.sweep, layout=a.layout)
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
        print(json.dumps(r["totals"], indent=1))
        return
    if a.cmd == "mlp":
        r = mlp_study(a.deploy, a.sweep, a.n, steps=a.steps)
        dep = json.load(open(a.deploy))
        dep["mlp_params"] = r["params"]
        dep.setdefault("meta", {})["mlp_study"] = r["study"]
        with open(a.out, "w") as f:
            json.dump(dep, f, indent=1)
        print(json.dumps(r["study"], indent=1))
        return
    if a.cmd == "sweep":
        prec = ks.PRECISIONS[a.precision]
        shapes = wl.shape_grid(a.n, a.seed)
        ids = ks.config_ids(prec)
        if a.kind != "all":
            ids = [c for c in ids if (c >= SPLIT_BASE) == (a.kind == "split")]
        k, n = (int(x) for x in a.shard.split("/"))
        perf = sweep(shapes, prec, a.out, config_ids=ids, shard=(k, n))
        if a.table and perf is not None:
            save_table(a.table, shapes, perf, ids, prec)
    else:
        dep = deploy(a.table, a.k, a.tree, a.seed, a.norm, method=a.method)
        with open(a.out, "w") as f:
            json.dump(dep, f, indent=1)
        print(json.dumps(dep["meta"]["scores"], indent=1))


if __name__ == "__main__":
    main()
