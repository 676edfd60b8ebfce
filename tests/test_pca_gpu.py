"""GPU PCA (covariance by the library's FP32 GEMM, subspace iteration,
Rayleigh-Ritz) against the FP64 eigen-decomposition of the oracle.

Tolerances: eigenvalues 1e-4 relative and the total variance 1e-5 relative
(FP32 covariance sums); eigenvectors compared through |v_gpu . v_ref| >= 1 - 1e-4
for components separated from their neighbours."""
import numpy as np
import pytest

from oracle import select as osel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def planted(n, d, spectrum, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    Z = rng.standard_normal((n, d)) * np.sqrt(np.r_[spectrum, np.full(d - len(spectrum), 1e-4)])
    return (Z @ Q.T + rng.random(d)).astype(np.float32)


@pytest.mark.parametrize("n,d,r", [(300, 40, 5), (800, 576, 12)])
def test_pca_matches_eigh(lib, torch, n, d, r):
    spectrum = [10.0 / (1 + i) ** 1.2 for i in range(r + 4)]
    X = planted(n, d, spectrum, seed=d)
    V0 = np.random.default_rng(1).standard_normal((d, r)).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    mean, V, Y = torch.empty(d, device="cuda"), torch.empty((d, r), device="cuda"), torch.empty((n, r), device="cuda")
    ev, tot = lib.pca(t(X), r, t(V0), mean, V, Y, iters=200)
    rm, rw, rv, rtot = osel.pca_top(X.astype(np.float64), r)
    assert tot == pytest.approx(rtot, rel=1e-5)
    assert np.allclose(ev, rw, rtol=1e-4)
    assert np.allclose(mean.cpu().numpy(), rm, atol=1e-5)
    Vg = V.cpu().numpy().astype(np.float64)
    assert np.allclose(Vg.T @ Vg, np.eye(r), atol=1e-4)
    assert np.all(np.abs(np.sum(Vg * rv, axis=0)) >= 1 - 1e-4)
    Xc = X.astype(np.float64) - rm
    assert np.allclose(Y.cpu().numpy(), Xc @ Vg, atol=1e-3)


def test_backproject(lib, torch):
    rng = np.random.default_rng(3)
    cent, V, mean = rng.random((4, 3)), rng.random((50, 3)), rng.random(50)
    out = torch.empty((4, 50), device="cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    lib.pca_backproject(t(cent), t(V), t(mean), out)
    assert np.allclose(out.cpu().numpy(), mean + cent @ V.T, atol=1e-5)
