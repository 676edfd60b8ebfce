"""GPU parity of the pruning pipeline kernels against the FP64 oracle.

Normalisation and scores are FP32 on the GPU: relative tolerance 1e-6 (a few
FP32 ulps through one division and, for the sigmoid, one exp).  k-means runs
in FP32 with the same seeding draws as the oracle: on separated clusters the
labels must agree exactly and the inertia to 1e-4 relative (FP32 sums of
~10^4 squared distances)."""
import numpy as np
import pytest

from oracle import select as osel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.mark.parametrize("mode", osel.NORMALISATIONS)
def test_normalise(lib, torch, mode):
    rng = np.random.default_rng(1)
    perf = (rng.random((333, 576)) ** 4 * 50).astype(np.float32)
    perf[5] = 0.0
    perf[7, :10] = 0.0
    out = torch.empty(perf.shape, device="cuda")
    lib.normalise(torch.from_numpy(perf).cuda(), out, mode)
    got = out.cpu().numpy().astype(np.float64)
    want = osel.normalise(perf.astype(np.float64), mode)
    assert np.allclose(got, want, rtol=1e-6, atol=1e-6)
    if mode != "sigmoid":  # an all-zero row maps to exact zeros (the sigmoid maps it to f(0) ~ 3.5e-19)
        assert np.all(got[5] == 0.0)


def planted(n_per, k, d, spread, seed):
    rng = np.random.default_rng(seed)
    centres = rng.random((k, d))
    X = np.concatenate([c + spread * rng.standard_normal((n_per, d)) for c in centres])
    return X.astype(np.float32)


@pytest.mark.parametrize("k,d,seed", [(3, 5, 0), (4, 64, 1), (8, 576, 2), (15, 200, 3)])
def test_kmeans_matches_oracle(lib, torch, k, d, seed):
    X = planted(25, k, d, 0.02, seed)
    n = X.shape[0]
    draws = np.random.default_rng(seed + 10).integers(0, 2 ** 32, (10, k), dtype=np.uint64).astype(np.uint32)
    cen = torch.empty((k, d), device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    inertia, iters = lib.kmeans(torch.from_numpy(X).cuda(), k, draws, cen, lab)
    C, labels, ref_inertia, _ = osel.kmeans(X.astype(np.float64), k, draws.astype(np.float64) / 2.0 ** 32)
    assert np.array_equal(lab.cpu().numpy(), labels)
    assert inertia == pytest.approx(ref_inertia, rel=1e-4)
    assert np.allclose(cen.cpu().numpy(), C, atol=1e-5)


def test_kmeans_seeding_picks_same_points(lib, torch):
    X = planted(10, 4, 8, 0.05, 7)
    draws = np.random.default_rng(3).integers(0, 2 ** 32, (1, 4), dtype=np.uint64).astype(np.uint32)
    cen = torch.empty((4, 8), device="cuda")
    lab = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    lib.kmeans(torch.from_numpy(X).cuda(), 4, draws, cen, lab, max_iter=1, tol=0.0)
    C0 = osel.kmeanspp_init(X.astype(np.float64), 4, draws[0].astype(np.float64) / 2.0 ** 32)
    C1, _, _, _ = osel.lloyd(X.astype(np.float64), C0, max_iter=1, tol=0.0)
    assert np.allclose(cen.cpu().numpy(), C1, atol=1e-5)


@pytest.mark.parametrize("which", ["deployed", "chosen", "all"])
def test_score(lib, torch, which):
    rng = np.random.default_rng(4)
    perf = (rng.random((200, 64)) ** 2).astype(np.float32)
    perf[3, :] = 0.0
    tp = torch.from_numpy(perf).cuda()
    dep = [3, 17, 40, 63]
    chosen = rng.choice(dep, 200).astype(np.int32)
    if which == "deployed":
        got = lib.score(tp, dep)
        want = osel.score(perf.astype(np.float64), deployed=np.array(dep))
    elif which == "chosen":
        got = lib.score(tp, dep, chosen=torch.from_numpy(chosen).cuda())
        want = osel.score(perf.astype(np.float64), chosen=chosen)
    else:
        got = lib.score(tp)
        want = osel.score(perf.astype(np.float64))
    assert got["geomean"] == pytest.approx(want["geomean"], rel=1e-5)
    assert got["mean"] == pytest.approx(want["mean"], rel=1e-5)
    assert got["clamped"] == want["clamped"]


@pytest.mark.parametrize("k", [1, 3, 7])
def test_knn_matches_oracle(lib, torch, k):
    rng = np.random.default_rng(k)
    train = rng.random((400, 7)).astype(np.float32)
    labels = rng.integers(0, 5, 400).astype(np.int32)
    query = rng.random((300, 7)).astype(np.float32)
    out = torch.empty(300, dtype=torch.int32, device="cuda")
    lib.knn(torch.from_numpy(train).cuda(), torch.from_numpy(labels).cuda(), torch.from_numpy(query).cuda(), k, out)
    want = osel.knn_predict(train.astype(np.float64), labels, query.astype(np.float64), k)
    assert np.array_equal(out.cpu().numpy(), want)


# ---------------------------------------------------------------- spectral clustering (Section 4.1)
def blobs(seed, n_per=40, k=4, d=12, spread=0.15):
    rng = np.random.default_rng(seed)
    centres = rng.random((k, d)) * 3
    truth = np.repeat(np.arange(k), n_per)
    X = centres[truth] + spread * rng.standard_normal((k * n_per, d))
    return X.astype(np.float32), truth


@pytest.mark.parametrize("seed", [0, 1])
def test_spectral_embedding_matches_oracle(lib, torch, seed):
    """Eigenvalues to 2e-4; the embedding through the rotation-invariant Gram
    matrix U U^T (eigenvectors are fixed only up to sign and, within a
    multiple eigenvalue, rotation) to 2e-3."""
    X, _ = blobs(seed)
    n, k, r = X.shape[0], 4, 12
    gamma = 1.0 / (2.0 * X.astype(np.float64).var(axis=0).sum())
    V0 = np.random.default_rng(50 + seed).standard_normal((n, r)).astype(np.float32)
    U = torch.empty((n, k), device="cuda")
    ev = lib.spectral_embedding(torch.from_numpy(X).cuda(), gamma, k, torch.from_numpy(V0).cuda(), U, iters=300)
    Uo, wo = osel.spectral_embedding(osel.rbf_affinity(X.astype(np.float64), gamma), k)
    assert np.allclose(ev, wo, atol=2e-4), (ev, wo)
    Ug = U.cpu().numpy().astype(np.float64)
    assert np.allclose(np.linalg.norm(Ug, axis=1), 1.0, atol=1e-5)
    assert np.allclose(Ug @ Ug.T, Uo @ Uo.T, atol=2e-3)


def test_spectral_partition_recovers_blobs(lib, torch):
    X, truth = blobs(3)
    n, k = X.shape[0], 4
    gamma = 1.0 / (2.0 * X.astype(np.float64).var(axis=0).sum())
    V0 = np.random.default_rng(9).standard_normal((n, 14)).astype(np.float32)
    U = torch.empty((n, k), device="cuda")
    lib.spectral_embedding(torch.from_numpy(X).cuda(), gamma, k, torch.from_numpy(V0).cuda(), U, iters=300)
    cen = torch.empty((k, k), device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    draws = np.random.default_rng(4).integers(0, 2 ** 32, (10, k), dtype=np.uint64).astype(np.uint32)
    lib.kmeans(U, k, draws, cen, lab)
    got = lab.cpu().numpy()
    assert len(set(zip(got.tolist(), truth.tolist()))) == k
    ref, _ = osel.spectral_partition(X.astype(np.float64), k, gamma, draws / 2.0 ** 32)
    assert len(set(zip(got.tolist(), ref.tolist()))) == k


def test_cluster_geomean_matches_oracle(lib, torch):
    rng = np.random.default_rng(8)
    X = (rng.random((300, 50)) ** 2).astype(np.float32)
    X[:20, :5] = 0.0  # clamped at the floor
    labels = rng.integers(0, 6, 300).astype(np.int32)
    labels[labels == 4] = 3  # cluster 4 empty
    out = torch.full((6, 50), 7.0, device="cuda")
    lib.cluster_geomean(torch.from_numpy(X).cuda(), torch.from_numpy(labels).cuda(), 6, out, floor=1e-6)
    want = osel.cluster_geomean_centres(X.astype(np.float64), labels, 6, floor=1e-6)
    assert np.allclose(out.cpu().numpy(), want, rtol=2e-6, atol=0)
    assert np.all(out.cpu().numpy()[4] == 0)
