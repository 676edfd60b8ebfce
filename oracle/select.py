"""FP64 oracle of the pruning and selection pipeline -- TEST INFRASTRUCTURE ONLY.

Each function follows the paper's steps in its own order and notation:

* normalisations        -- Section 3.4 ("Normalization method")
* k-means pruning       -- Section 4.1 (k-means clustering of the normalised
                           performance vectors, one point per set of sizes)
* representatives       -- Section 4.2 (best configuration of each centroid;
                           geometric mean of a cluster when only labels exist)
* Top-N                 -- Section 4.2 (the configurations that are best most often)
* score                 -- Section 4.3 (geometric mean, over held-out sizes, of the
                           best selected configuration's normalised performance)
* decision tree         -- Section 5.1 (classifier from sizes to a deployed kernel;
                           trees A, B, C differ in depth and leaf-size limits)
* PCA variance          -- Section 3.3

Readings where the paper is silent (each is listed with its reason in the
design notes of the repository): k-means++ seeding with the uniform draws
passed in; Lloyd's iterations with scikit-learn's stopping rule (centre shift
below tol times the mean per-dimension variance); an empty cluster keeps its
previous centre; distance ties go to the lowest centre index; duplicate
representatives are replaced by the best unused configuration, clusters taken
in descending size; CART with Gini impurity, thresholds at midpoints of
consecutive distinct values, features scanned in order and the first best split
kept, leaves labelled by majority with the lowest class on ties.
"""
from __future__ import annotations

import numpy as np

NORMALISATIONS = ("standard", "raw_cutoff", "standard_cutoff", "sigmoid")
CUTOFF = 0.9


# ----------------------------------------------------------------------------- Section 3.4
def normalise(perf: np.ndarray, mode: str = "standard") -> np.ndarray:
    """Per set of sizes (row), map throughputs to [0, 1].

    standard:        divide by the row's best throughput.
    raw_cutoff:      standard, then values below 0.9 set to 0 (others unchanged).
    standard_cutoff: raw cutoff, then rescaled so [0.9, 1] spans [0, 1].
    sigmoid:         f(x) = 1 / (1 + exp(50 (0.85 - x))) of the standard value.
    A row whose best throughput is 0 (every configuration failed) maps to 0.
    """
    perf = np.asarray(perf, np.float64)
    best = perf.max(axis=1, keepdims=True)
    x = np.zeros_like(perf)
    ok = best[:, 0] > 0
    x[ok] = perf[ok] / best[ok]
    if mode == "standard":
        return x
    if mode == "raw_cutoff":
        return np.where(x < CUTOFF, 0.0, x)
    if mode == "standard_cutoff":
        return np.where(x < CUTOFF, 0.0, (x - CUTOFF) / (1.0 - CUTOFF))
    if mode == "sigmoid":
        return 1.0 / (1.0 + np.exp(50.0 * (0.85 - x)))
    raise ValueError(mode)


# ----------------------------------------------------------------------------- Section 4.1
def sq_dist(x: np.ndarray, c: np.ndarray) -> float:
    d = x - c
    return float(np.dot(d, d))


def kmeanspp_init(X: np.ndarray, k: int, u: np.ndarray) -> np.ndarray:
    """k-means++ seeding (Arthur & Vassilvitskii 2007) driven by k uniform draws u in [0, 1).

    First centre: point floor(u[0] * n).  Centre c >= 1: the first point i
    whose running sum of D(x)^2 (squared distance to the nearest chosen centre)
    exceeds u[c] times the total; if the total is 0, point floor(u[c] * n).
    """
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    idx = [min(int(u[0] * n), n - 1)]
    d2 = np.array([sq_dist(X[i], X[idx[0]]) for i in range(n)])
    for c in range(1, k):
        total = d2.sum()
        if total > 0:
            target = u[c] * total
            run = 0.0
            pick = n - 1
            for i in range(n):
                run += d2[i]
                if run > target:
                    pick = i
                    break
        else:
            pick = min(int(u[c] * n), n - 1)
        idx.append(pick)
        d2 = np.minimum(d2, np.array([sq_dist(X[i], X[pick]) for i in range(n)]))
    return X[idx].copy()


def assign(X: np.ndarray, centres: np.ndarray) -> tuple[np.ndarray, float]:
    """Nearest centre per point (lowest index on ties) and the total squared distance."""
    n, k = X.shape[0], centres.shape[0]
    labels = np.empty(n, np.int64)
    inertia = 0.0
    for i in range(n):
        best, bd = 0, sq_dist(X[i], centres[0])
        for c in range(1, k):
            d = sq_dist(X[i], centres[c])
            if d < bd:
                best, bd = c, d
        labels[i] = best
        inertia += bd
    return labels, inertia


def lloyd(X: np.ndarray, centres: np.ndarray, max_iter: int = 300, tol: float = 1e-4):
    """Lloyd's iterations from the given centres.

    Each iteration assigns every point to its nearest centre, then moves each
    centre to the mean of its points (an empty cluster keeps its centre).  It
    stops after the update whose total squared centre shift is <= tol times the
    mean per-dimension variance of X, or after max_iter updates.  Labels and
    inertia are then recomputed against the final centres.
    Returns (centres, labels, inertia, n_iter).
    """
    X = np.asarray(X, np.float64)
    C = np.array(centres, np.float64, copy=True)
    tol_abs = tol * float(np.mean(np.var(X, axis=0)))
    it = 0
    for it in range(1, max_iter + 1):
        labels, _ = assign(X, C)
        newC = C.copy()
        for c in range(C.shape[0]):
            members = X[labels == c]
            if len(members):
                newC[c] = members.mean(axis=0)
        shift = float(np.sum((newC - C) ** 2))
        C = newC
        if shift <= tol_abs:
            break
    labels, inertia = assign(X, C)
    return C, labels, inertia, it


def kmeans(X: np.ndarray, k: int, uniforms: np.ndarray, max_iter: int = 300, tol: float = 1e-4):
    """Best of n_init = len(uniforms) seeded runs (lowest inertia; first on ties).
    uniforms: (n_init, k) draws in [0, 1).  Returns (centres, labels, inertia, run)."""
    best = None
    for r in range(uniforms.shape[0]):
        C0 = kmeanspp_init(X, k, uniforms[r])
        C, labels, inertia, _ = lloyd(X, C0, max_iter, tol)
        if best is None or inertia < best[2]:
            best = (C, labels, inertia, r)
    return best


def brute_force_partition(X: np.ndarray, k: int) -> tuple[float, np.ndarray]:
    """Global minimum of the k-means objective over every assignment of the n
    points to k non-empty clusters (n small).  Used only to pin ``kmeans``."""
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    best = (np.inf, None)
    labels = np.zeros(n, np.int64)

    def rec(i, used):
        nonlocal best
        if i == n:
            if used != k:
                return
            cost = 0.0
            for c in range(k):
                m = X[labels == c]
                cost += float(((m - m.mean(axis=0)) ** 2).sum())
            if cost < best[0]:
                best = (cost, labels.copy())
            return
        # canonical labelling: point i joins an existing cluster or opens the next one
        for c in range(min(used + 1, k)):
            labels[i] = c
            rec(i + 1, max(used, c + 1))

    rec(0, 0)
    return best


# ----------------------------------------------------------------------------- Section 4.2
def representatives(centres: np.ndarray, labels: np.ndarray, dedupe: bool = True) -> np.ndarray:
    """Deployed configuration per cluster: the best configuration of its centre.

    Clusters are taken in descending size (lower index first on ties); with
    ``dedupe`` a cluster whose best configuration is already taken gets its best
    unused one, so k clusters give k distinct configurations.  Returns config
    column indices, in cluster-size order.
    """
    k, d = centres.shape
    sizes = np.bincount(labels, minlength=k)
    order = sorted(range(k), key=lambda c: (-sizes[c], c))
    chosen: list[int] = []
    for c in order:
        ranking = sorted(range(d), key=lambda j: (-centres[c, j], j))
        if dedupe:
            pick = next(j for j in ranking if j not in chosen)
        else:
            pick = ranking[0]
            if pick in chosen:
                continue
        chosen.append(pick)
    return np.array(chosen, np.int64)


def cluster_geomean_representatives(Xnorm: np.ndarray, labels: np.ndarray, k: int,
                                    floor: float = 1e-6) -> np.ndarray:
    """For label-only clusterings: the best configuration of each cluster's
    geometric-mean performance vector (values clamped at ``floor``)."""
    out = []
    for c in range(k):
        m = Xnorm[labels == c]
        if len(m) == 0:
            continue
        g = np.exp(np.mean(np.log(np.maximum(m, floor)), axis=0))
        out.append(int(np.argmax(g)))
    return np.array(sorted(set(out), key=out.index), np.int64)


def top_n(perf: np.ndarray, n: int) -> np.ndarray:
    """The n configurations that are best for the most sets of sizes (lowest
    index wins ties, in both the per-row best and the counts).  If fewer than n
    configurations are ever best, the rest are filled by highest mean
    standard-normalised performance."""
    best = np.argmax(perf, axis=1)
    counts = np.bincount(best, minlength=perf.shape[1])
    order = sorted(range(perf.shape[1]), key=lambda j: (-counts[j], j))
    chosen = [j for j in order if counts[j] > 0][:n]
    if len(chosen) < n:
        mean = normalise(perf, "standard").mean(axis=0)
        for j in sorted(range(perf.shape[1]), key=lambda j: (-mean[j], j)):
            if len(chosen) == n:
                break
            if j not in chosen:
                chosen.append(j)
    return np.array(chosen, np.int64)


# ----------------------------------------------------------------------------- Section 4.3
def score(perf: np.ndarray, deployed: np.ndarray | None = None, chosen: np.ndarray | None = None,
          floor: float = 1e-6) -> dict:
    """Fraction of optimal performance over the rows of ``perf`` (held-out sizes).

    Per row the ratio is perf[s, pick] / max_c perf[s, c], where pick is
    ``chosen[s]`` (a classifier's choice) or, when ``chosen`` is None, the best
    of the ``deployed`` columns (the deployed set's attainable maximum), or
    every column when both are None (the exhaustive selector, ratio 1).
    Returns the geometric mean (ratios clamped at ``floor``), the arithmetic
    mean and the number clamped.
    """
    perf = np.asarray(perf, np.float64)
    best = perf.max(axis=1)
    if chosen is not None:
        got = perf[np.arange(perf.shape[0]), np.asarray(chosen, np.int64)]
    elif deployed is not None:
        got = perf[:, np.asarray(deployed, np.int64)].max(axis=1)
    else:
        got = best
    ratio = np.where(best > 0, got / np.where(best > 0, best, 1.0), 0.0)
    clamped = int(np.sum(ratio < floor))
    r = np.maximum(ratio, floor)
    return {"geomean": float(np.exp(np.mean(np.log(r)))), "mean": float(np.mean(ratio)),
            "clamped": clamped, "ratios": ratio}


# ----------------------------------------------------------------------------- Section 5.1
def gini_ordered(counts: np.ndarray, n) -> np.ndarray:
    """1 - sum_c (counts_c / n)^2 with the class sum taken in class order, so
    that two splits with equal counts give bit-identical impurities.
    ``counts`` is (..., n_classes), ``n`` broadcasts against its leading dims."""
    n = np.asarray(n, np.float64)
    s = np.zeros(counts.shape[:-1], np.float64)
    for c in range(counts.shape[-1]):
        p = counts[..., c] / n
        s = s + p * p
    return 1.0 - s


def best_split(F: np.ndarray, y: np.ndarray, n_classes: int, min_leaf: int, features=None):
    """Lowest weighted child Gini, (n_L G_L + n_R G_R) / n, over every
    (feature, midpoint threshold) whose two sides each hold >= min_leaf
    samples.  Features in column order (only those in ``features`` when given),
    thresholds ascending; the first best is kept.  Returns (feature, threshold,
    weighted impurity) or None."""
    n = len(y)
    best = None
    for f in (range(F.shape[1]) if features is None else sorted(features)):
        order = np.argsort(F[:, f], kind="stable")
        xs = F[order, f]
        onehot = np.zeros((n, n_classes))
        onehot[np.arange(n), y[order]] = 1.0
        cum = np.cumsum(onehot, axis=0)            # class counts of the first i+1 sorted samples
        pos = np.nonzero(xs[:-1] < xs[1:])[0]      # split between sorted positions i and i+1
        nl = (pos + 1).astype(np.float64)
        nr = n - nl
        ok = (nl >= min_leaf) & (nr >= min_leaf)
        pos, nl, nr = pos[ok], nl[ok], nr[ok]
        if len(pos) == 0:
            continue
        cl = cum[pos]
        cr = cum[-1] - cl
        w = (nl * gini_ordered(cl, nl) + nr * gini_ordered(cr, nr)) / n
        j = int(np.argmin(w))
        if best is None or w[j] < best[2]:
            best = (f, (float(xs[pos[j]]) + float(xs[pos[j] + 1])) / 2.0, float(w[j]))
    return best


def selector_features(sizes) -> np.ndarray:
    """Section 5.1: the classifier maps the matrix sizes to a deployed kernel.
    Its feature row here is the sizes and the number of outputs, (M, N, K,
    batch, M * N * batch): one more function of the sizes, which a
    depth-limited tree of axis-aligned splits cannot form (a reading of
    "matrix sizes").  sizes: n x 4 (M, N, K, batch)."""
    s = np.asarray(sizes, np.float64).reshape(-1, 4)
    return np.column_stack([s, s[:, 0] * s[:, 1] * s[:, 3]])


def best_labels(perf: np.ndarray, cols) -> np.ndarray:
    """Section 5.1: each training size is labelled with the deployed kernel
    that ran it fastest -- the position j in ``cols`` of the largest
    perf[i, cols[j]], the first such j on ties."""
    perf = np.asarray(perf, np.float64)
    out = np.empty(perf.shape[0], np.int64)
    for i in range(perf.shape[0]):
        best = 0
        for j in range(len(cols)):
            if perf[i, cols[j]] > perf[i, cols[best]]:
                best = j
        out[i] = best
    return out


def feature_subset(draw_row: np.ndarray, n_features: int, m: int) -> list[int]:
    """The m features a random-forest node may split on: the first m entries of a
    partial Fisher-Yates shuffle of 0..n_features-1 in which step t swaps entry t
    with entry t + draw_row[t] mod (n_features - t) (uint32 draws passed in)."""
    order = list(range(n_features))
    for t in range(m):
        j = t + int(draw_row[t]) % (n_features - t)
        order[t], order[j] = order[j], order[t]
    return sorted(order[:m])


def tree_train(F: np.ndarray, y: np.ndarray, n_classes: int, max_depth: int | None = None,
               min_leaf: int = 1, max_features: int | None = None, draws: np.ndarray | None = None) -> list[dict]:
    """CART classification tree, nodes in depth-first preorder.

    A node is a leaf when it is pure, is at max_depth, or has no admissible
    split; otherwise it splits at ``best_split`` (x[feature] <= threshold goes
    left).  Leaf label: majority class, lowest class on ties.  Every node
    records its majority label.  With ``max_features`` < the feature count (a
    random-forest tree), node j may only split on ``feature_subset(draws[j])``
    and becomes a leaf when none of those features splits it.
    """
    F = np.asarray(F, np.float64)
    y = np.asarray(y, np.int64)
    nodes: list[dict] = []
    subsample = max_features is not None and max_features < F.shape[1]

    def grow(idx, depth):
        counts = np.bincount(y[idx], minlength=n_classes)
        node = {"feature": -1, "threshold": 0.0, "left": -1, "right": -1,
                "label": int(np.argmax(counts)), "n": int(len(idx))}
        me = len(nodes)
        nodes.append(node)
        if counts.max() == len(idx) or (max_depth is not None and depth >= max_depth):
            return me
        feats = feature_subset(draws[me], F.shape[1], max_features) if subsample else None
        s = best_split(F[idx], y[idx], n_classes, min_leaf, feats)
        if s is None:
            return me
        f, t, _ = s
        go_left = F[idx, f] <= t
        node["feature"], node["threshold"] = int(f), float(t)
        node["left"] = grow(idx[go_left], depth + 1)
        node["right"] = grow(idx[~go_left], depth + 1)
        return me

    if len(y):
        grow(np.arange(len(y)), 0)
    return nodes


def tree_predict(nodes: list[dict], F: np.ndarray) -> np.ndarray:
    F = np.asarray(F, np.float64)
    out = np.empty(F.shape[0], np.int64)
    for i in range(F.shape[0]):
        j = 0
        while nodes[j]["feature"] >= 0:
            j = nodes[j]["left"] if F[i, nodes[j]["feature"]] <= nodes[j]["threshold"] else nodes[j]["right"]
        out[i] = nodes[j]["label"]
    return out


def knn_predict(train: np.ndarray, labels: np.ndarray, query: np.ndarray, k: int) -> np.ndarray:
    """k nearest neighbours by squared Euclidean distance (ties to the lower
    training index); majority label, ties to the label met first in
    nearest-first order."""
    train = np.asarray(train, np.float64)
    out = np.empty(len(query), np.int64)
    for q, x in enumerate(np.asarray(query, np.float64)):
        d = ((train - x) ** 2).sum(axis=1)
        nn = sorted(range(len(train)), key=lambda i: (d[i], i))[:k]
        best, count = None, 0
        for i in nn:
            c = sum(1 for j in nn if labels[j] == labels[i])
            if c > count:
                best, count = labels[i], c
        out[q] = best
    return out


TREES = {"A": (None, 1), "B": (6, 3), "C": (3, 4)}  # (max_depth, min samples per leaf), Section 5.1


# ----------------------------------------------------------------------------- Section 3.3
def pca_explained_variance(X: np.ndarray) -> np.ndarray:
    """Fraction of total variance per principal component (descending), from the
    eigenvalues of the sample covariance."""
    X = np.asarray(X, np.float64)
    Xc = X - X.mean(axis=0)
    cov = Xc.T @ Xc / max(X.shape[0] - 1, 1)
    ev = np.linalg.eigvalsh(cov)[::-1]
    ev = np.maximum(ev, 0.0)
    return ev / ev.sum() if ev.sum() > 0 else ev


def pca_top(X: np.ndarray, r: int):
    """Mean, the r largest eigenvalues (descending) and unit eigenvectors (d x r)
    of the sample covariance, and its trace (the total variance)."""
    X = np.asarray(X, np.float64)
    mean = X.mean(axis=0)
    Xc = X - mean
    cov = Xc.T @ Xc / max(X.shape[0] - 1, 1)
    w, v = np.linalg.eigh(cov)
    order = np.argsort(w)[::-1][:r]
    return mean, w[order], v[:, order], float(np.trace(cov))


def components_for(explained: np.ndarray, frac: float) -> int:
    return int(np.searchsorted(np.cumsum(explained), frac - 1e-12) + 1)


# ----------------------------------------------------------------------------- Section 4.1, decision tree
def leaf_sse(Y: np.ndarray) -> float:
    """Sum over outputs of the squared deviations from the leaf mean."""
    if len(Y) == 0:
        return 0.0
    return float(np.sum((Y - Y.mean(axis=0)) ** 2))


GAIN_TIE = 1e-9  # gains within this relative distance of the best count as ties


def regression_split(F: np.ndarray, Y: np.ndarray, idx: np.ndarray):
    """Best split of the samples `idx` for a multi-output regression tree: the
    (feature, midpoint threshold) with the largest drop of summed squared error,
    features in order and thresholds ascending, the first best kept (a later
    candidate must beat it by more than GAIN_TIE relative, so that splits giving
    the same partition through different features tie whatever the rounding).
    Returns (gain, feature, threshold) or None when no split separates the samples."""
    parent = leaf_sse(Y[idx])
    best = None
    for f in range(F.shape[1]):
        vals = np.unique(F[idx, f])
        for a, b in zip(vals[:-1], vals[1:]):
            thr = (a + b) / 2.0
            left = idx[F[idx, f] <= thr]
            right = idx[F[idx, f] > thr]
            gain = parent - leaf_sse(Y[left]) - leaf_sse(Y[right])
            if best is None or gain > best[0] * (1 + GAIN_TIE):
                best = (gain, f, thr)
    return best


def tree_regression_partition(F: np.ndarray, Y: np.ndarray, max_leaves: int):
    """Section 4.1 "Decision tree": a regression tree from the sizes F (n x 4) to
    the normalised performance vectors Y (n x d), limited to `max_leaves` leaves.

    Grown best-first: while there are fewer than max_leaves leaves, split the
    leaf whose best split removes the most squared error (lowest leaf index on
    ties, within GAIN_TIE).  Growth stops when no split removes more than 1e-12 of the root's
    squared error (rounding noise of leaves that are already constant).  A split
    leaf keeps its index for the left part and the right part becomes a new last
    leaf.  Returns (labels: leaf index per sample, centres: mean of Y per leaf)."""
    n = len(F)
    leaves = [np.arange(n)]
    splits = [regression_split(F, Y, leaves[0])]
    tol = 1e-12 * leaf_sse(Y)
    while len(leaves) < max_leaves:
        i = None
        for j, s in enumerate(splits):
            if s is not None and s[0] > tol and (i is None or s[0] > splits[i][0] * (1 + GAIN_TIE)):
                i = j
        if i is None:
            break
        _, f, thr = splits[i]
        idx = leaves[i]
        left, right = idx[F[idx, f] <= thr], idx[F[idx, f] > thr]
        leaves[i] = left
        leaves.append(right)
        splits[i] = regression_split(F, Y, left)
        splits.append(regression_split(F, Y, right))
    labels = np.empty(n, np.int64)
    centres = np.empty((len(leaves), Y.shape[1]))
    for j, idx in enumerate(leaves):
        labels[idx] = j
        centres[j] = Y[idx].mean(axis=0)
    return labels, centres


# ----------------------------------------------------------------------------- Section 4.1, spectral clustering
def rbf_affinity(X: np.ndarray, gamma: float) -> np.ndarray:
    """Similarity graph as an adjacency matrix: A_ij = exp(-gamma |x_i - x_j|^2), zero diagonal."""
    n = len(X)
    A = np.empty((n, n))
    for i in range(n):
        A[i] = np.exp(-gamma * np.sum((X - X[i]) ** 2, axis=1))
    np.fill_diagonal(A, 0.0)
    return A


def spectral_embedding(A: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Coordinates from the Laplacian of the adjacency matrix: the k eigenvectors
    of the normalised Laplacian L = I - D^-1/2 A D^-1/2 with the smallest
    eigenvalues (equivalently the largest of S = D^-1/2 A D^-1/2), each row then
    scaled to unit length.  A row with zero degree (an isolated size) gets
    D^-1/2 = 0, and a zero row of the embedding stays zero.
    Returns (rows n x k, eigenvalues of S, descending)."""
    d = A.sum(axis=1)
    s = np.zeros_like(d)
    s[d > 0] = 1.0 / np.sqrt(d[d > 0])
    S = A * s[:, None] * s[None, :]
    w, V = np.linalg.eigh(S)
    order = np.argsort(-w, kind="stable")[:k]
    U = V[:, order]
    nrm = np.linalg.norm(U, axis=1, keepdims=True)
    U = np.divide(U, nrm, out=np.zeros_like(U), where=nrm > 0)
    return U, w[order]


def spectral_partition(X: np.ndarray, k: int, gamma: float, uniforms: np.ndarray):
    """Section 4.1 "Spectral clustering": k-means (same seeding draws as the
    direct k-means) on the spectral coordinates of the RBF similarity graph.
    Returns (labels, inertia in the embedding)."""
    U, _ = spectral_embedding(rbf_affinity(X, gamma), k)
    _, labels, inertia, _ = kmeans(U, k, uniforms)
    return labels, inertia


def cluster_geomean_centres(X: np.ndarray, labels: np.ndarray, k: int, floor: float = 1e-6) -> np.ndarray:
    """Section 4.2 for label-only clusterings: each cluster's geometric-mean
    performance vector (values clamped at ``floor``); an empty cluster gives zeros.
    The deployed configurations are then `representatives` of these centres."""
    out = np.zeros((k, X.shape[1]))
    for c in range(k):
        m = X[labels == c]
        if len(m):
            out[c] = np.exp(np.mean(np.log(np.maximum(m, floor)), axis=0))
    return out
