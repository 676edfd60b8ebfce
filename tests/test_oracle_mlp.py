"""Pins for the FP64 MLP and BF16 oracles."""
import numpy as np
import pytest

from oracle import bf16 as ob
from oracle import mlp as om


def test_param_count():
    assert om.N_PARAMS == 7 * 64 + 64 + 64 * 64 + 64 + 64 * 8 + 8 == 5192


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = om.init_params(rng.random(om.N_PARAMS)) + 0.01 * rng.standard_normal(om.N_PARAMS)
    X = rng.random((16, 7))
    T = rng.standard_normal((16, 8))
    mask = (rng.random((16, 8)) > 0.2).astype(float)
    _, g = om.loss_and_grad(theta, X, T, mask)
    idx = rng.choice(om.N_PARAMS, 200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(om.N_PARAMS)
        e[i] = h
        lp, _ = om.loss_and_grad(theta + e, X, T, mask)
        lm, _ = om.loss_and_grad(theta - e, X, T, mask)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_zero_weights_closed_form():
    theta = np.zeros(om.N_PARAMS)
    b3 = np.arange(8, dtype=float)
    theta[-8:] = b3
    X = np.random.default_rng(1).random((5, 7))
    T = np.zeros((5, 8))
    y, _ = om.forward(theta, X)
    assert np.array_equal(y, np.tile(b3, (5, 1)))
    loss, g = om.loss_and_grad(theta, X, T)
    assert loss == pytest.approx(np.mean(b3 ** 2))
    assert np.allclose(g[-8:], 2 * b3 / 8)
    assert np.all(g[:-8] == 0)


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    theta, m, v = om.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.1, eps=0.0 + 1e-30)
    assert np.allclose(theta[:3], -0.1 * np.sign(g[:3]), rtol=1e-12)
    assert theta[3] == 0.0


def test_select_respects_mask():
    theta = np.zeros(om.N_PARAMS)
    theta[-8:] = [5, 1, 7, 7, 0, 0, 0, 9]
    allowed = np.array([[1, 1, 1, 1, 1, 1, 1, 0]], bool)
    _, pick = om.predict_select(theta, np.zeros((1, 7)), allowed)
    assert pick[0] == 2


def test_features():
    f = om.features(4096, 16, 1, 16, 1, 0, 3)
    assert np.allclose(f, [1.0, 4 / 12, 0.0, 1.0, 1.0, 0.0, 1.0])


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.standard_normal(10000).astype(np.float32) * 10.0 ** rng.integers(-20, 20, 10000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.4e38, 1e-40, -np.inf, np.inf],
                                 np.float32)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ob.to_bf16_bits(x), ref)


def test_bf16_split_error():
    x = np.random.default_rng(3).uniform(-1, 1, 100000).astype(np.float32)
    hi, lo = ob.split_bf16(x)
    # x - hi is exact in binary32 (Sterbenz), and |x - hi - lo| <= 2^-8 |x - hi| <= 2^-16 |x|
    r = x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64)
    assert np.all(np.abs(r) <= 2.0 ** -16 * np.abs(x.astype(np.float64)))
    assert np.array_equal(ob.round_bf16(hi), hi) and np.array_equal(ob.round_bf16(lo), lo)


def test_targets_by_hand_and_scale_invariance():
    """log(perf / row max) on measured entries: the fastest kernel gets 0, one at
    half its speed log(1/2); unmeasured entries are masked; a size that ran twice
    as fast everywhere has the same targets (only relative speed is learned)."""
    perf = np.array([[2.0, 4.0, 0.0, 1.0], [0.0, 0.0, 0.0, 0.0], [3.0, 3.0, 3.0, 3.0]])
    T, mask = om.targets(perf)
    assert np.allclose(T[0], [np.log(0.5), 0.0, 0.0, np.log(0.25)], rtol=0, atol=1e-15)
    assert mask[0].tolist() == [1, 1, 0, 1] and mask[1].tolist() == [0, 0, 0, 0] and T[1].tolist() == [0, 0, 0, 0]
    assert T[2].tolist() == [0, 0, 0, 0]
    T2, mask2 = om.targets(perf * 2.0)
    assert np.allclose(T2, T, rtol=0, atol=1e-15) and np.array_equal(mask2, mask)
