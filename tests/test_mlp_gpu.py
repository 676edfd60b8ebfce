"""GPU parity of the learned selector's kernels (forward, loss/gradient, Adam,
graph-replayed training, batched selection) against the FP64 oracle.

FP32 against FP64: forward outputs to 1e-5 (relative to the output scale);
gradients to 1e-4 of the largest gradient entry; one Adam step to 1e-6
absolute in the parameters.  Argmax decisions are compared where the top two
predictions differ by more than 1e-3."""
import numpy as np
import pytest

from oracle import mlp as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def data(n, seed):
    rng = np.random.default_rng(seed)
    M, N, K = (np.exp(rng.uniform(np.log(16), np.log(4096), n)).round() for _ in range(3))
    b = rng.choice([1, 2, 4, 8, 16], n)
    ta, tb = rng.integers(0, 2, n), rng.integers(0, 2, n)
    X = om.features(M, N, K, b, ta, tb, np.zeros(n))
    T = rng.normal(3.0, 1.0, (n, 8))
    mask = (rng.random((n, 8)) > 0.1).astype(np.float64)
    shapes = np.stack([M, N, K, b, ta, tb, np.zeros(n)], 1).astype(np.int64)
    return X, T, mask, shapes


def params(seed):
    return om.init_params(np.random.default_rng(seed).random(om.N_PARAMS)) + \
        0.01 * np.random.default_rng(seed + 1).standard_normal(om.N_PARAMS)


def dev(torch, x, dtype=None):
    import torch as t
    return t.from_numpy(np.ascontiguousarray(x, dtype or np.float32)).cuda()


def test_forward(lib, torch):
    X, _, _, _ = data(1000, 0)
    th = params(1)
    Y = torch.empty((1000, 8), device="cuda")
    lib.mlp_forward(dev(torch, th), dev(torch, X), Y)
    ref, _ = om.forward(th.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    got = Y.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [1, 31, 32, 1000, 2003])
def test_loss_and_gradient(lib, torch, n):
    X, T, mask, _ = data(n, 2)
    th = params(3).astype(np.float32).astype(np.float64)
    X32, T32 = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    g = torch.empty(om.N_PARAMS, device="cuda")
    loss = torch.empty(1, device="cuda")
    lib.mlp_loss_grad(dev(torch, th), dev(torch, X32), dev(torch, T32), dev(torch, mask), g, loss)
    ref_loss, ref_g = om.loss_and_grad(th, X32, T32, mask)
    assert loss.item() == pytest.approx(ref_loss, rel=1e-5)
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg - ref_g)) <= 1e-4 * np.max(np.abs(ref_g))


def test_adam_step(lib, torch):
    rng = np.random.default_rng(4)
    th = rng.standard_normal(om.N_PARAMS).astype(np.float32).astype(np.float64)
    g = rng.standard_normal(om.N_PARAMS).astype(np.float32).astype(np.float64)
    m = (0.1 * rng.standard_normal(om.N_PARAMS)).astype(np.float32).astype(np.float64)
    v = (0.1 * rng.random(om.N_PARAMS)).astype(np.float32).astype(np.float64)
    P, M, V = dev(torch, th), dev(torch, m), dev(torch, v)
    lib.mlp_adam_step(P, dev(torch, g), M, V, 7, lr=1e-2)
    rt, rm, rv = om.adam_step(th, g, m, v, 7, lr=1e-2)
    assert np.max(np.abs(P.cpu().numpy() - rt)) <= 1e-6
    assert np.max(np.abs(M.cpu().numpy() - rm)) <= 1e-6 and np.max(np.abs(V.cpu().numpy() - rv)) <= 1e-6


def test_training_matches_oracle_and_decreases_loss(lib, torch):
    X, T, mask, _ = data(500, 5)
    X32, T32 = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    th = params(6).astype(np.float32).astype(np.float64)
    P = dev(torch, th)
    M = torch.zeros(om.N_PARAMS, device="cuda")
    V = torch.zeros(om.N_PARAMS, device="cuda")
    hist = torch.empty(5, device="cuda")
    lib.mlp_train(P, dev(torch, X32), dev(torch, T32), dev(torch, mask), M, V, 0, 5, lr=1e-3, loss_hist=hist)
    rth, rm, rv = th.copy(), np.zeros(om.N_PARAMS), np.zeros(om.N_PARAMS)
    ref_hist = []
    for t in range(1, 6):
        l, g = om.loss_and_grad(rth, X32, T32, mask)
        ref_hist.append(l)
        rth, rm, rv = om.adam_step(rth, g, rm, rv, t, lr=1e-3)
    assert np.allclose(hist.cpu().numpy(), ref_hist, rtol=1e-4)
    # Adam moves each parameter by about lr per step whatever the gradient's
    # size, so entries whose gradient is at FP32 noise level may step the other
    # way: bound those by 2 lr per step, and require the rest to agree.
    d = np.abs(P.cpu().numpy() - rth)
    assert d.max() <= 2 * 1e-3 * 5 and np.mean(d <= 1e-5) >= 0.95
    hist2 = torch.empty(300, device="cuda")
    lib.mlp_train(P, dev(torch, X32), dev(torch, T32), dev(torch, mask), M, V, 5, 300, lr=1e-2, loss_hist=hist2)
    h = hist2.cpu().numpy()
    assert h[-1] < 0.5 * h[0]


def test_batched_selection(lib, torch):
    _, _, _, shapes = data(4096, 7)
    th = params(8)
    ids = [3, 77, 150, 301, 400, 450, 500, 575]
    h = lib.Handle({"precision": 0, "config_ids": ids, "nodes": [], "mlp_params": th})
    out = torch.empty(4096, dtype=torch.int32, device="cuda")
    pred = torch.empty((4096, 8), device="cuda")
    lib.select_kernels_batched(h, dev(torch, shapes, np.int64), out, pred)
    torch.cuda.synchronize()
    X = om.features(*[shapes[:, i] for i in range(7)])
    y, pick = om.predict_select(th.astype(np.float32).astype(np.float64), X)
    assert np.max(np.abs(pred.cpu().numpy() - y)) <= 1e-4 * max(1.0, np.abs(y).max())
    srt = np.sort(y, axis=1)
    clear = (srt[:, -1] - srt[:, -2]) > 1e-3
    got = out.cpu().numpy()
    assert np.array_equal(got[clear], np.array(ids)[pick[clear]])
    assert set(got.tolist()) <= set(ids)


def test_features_kernel(lib, torch):
    _, _, _, shapes = data(777, 9)
    X = torch.empty((777, 7), device="cuda")
    lib.mlp_features(dev(torch, shapes, np.int64), X)
    ref = om.features(*[shapes[:, i] for i in range(7)])
    assert np.max(np.abs(X.cpu().numpy() - ref)) <= 1e-6


def test_targets_kernel(lib, torch):
    """log(perf / row max) and the measured mask, against the FP64 oracle: rows
    with unmeasured (0) kernels, a row with none measured, and a throughput
    range of nine decades."""
    rng = np.random.default_rng(11)
    perf = np.exp(rng.uniform(-3, 18, (513, 8))).astype(np.float32)
    perf[rng.random((513, 8)) < 0.2] = 0.0
    perf[7] = 0.0
    T = torch.empty((513, 8), device="cuda")
    mask = torch.empty((513, 8), device="cuda")
    lib.mlp_targets(dev(torch, perf), T, mask)
    rT, rmask = om.targets(perf.astype(np.float64))
    assert np.array_equal(mask.cpu().numpy(), rmask)
    assert np.max(np.abs(T.cpu().numpy() - rT)) <= 1e-5
