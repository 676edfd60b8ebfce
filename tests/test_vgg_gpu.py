"""VGG16 inference through the library against the FP64 oracle forward pass.

Layer kernels (im2col, bias/ReLU, pooling) must match exactly; whole networks
within a relative error of the logits (max |difference| / max |logit|) of
1e-4 (narrow network) and 1e-3 (full VGG16: 16 FP32 GEMM layers, K up to 25088)."""
import json
import os

import numpy as np
import pytest

from oracle import vgg as ov
from paper_2008_13145_gb300 import vgg
from paper_2008_13145_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEPLOY = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2008_13145_gb300", "deploy")


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def test_layer_kernels_exact(lib, torch):
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 6, 8, 5)).astype(np.float32)
    tx = torch.from_numpy(x).cuda()
    col = torch.full((2 * 6 * 8, 48), 9.0, device="cuda")
    lib.im2col3x3(tx, 2, 6, 8, 5, col, 48)
    got = col.cpu().numpy()
    assert np.array_equal(got[:, :45], ov.im2col3x3(x.astype(np.float64)).astype(np.float32))
    assert np.all(got[:, 45:] == 9.0)
    pooled = torch.empty((2, 3, 4, 5), device="cuda")
    lib.maxpool2x2(tx, 2, 6, 8, 5, pooled)
    assert np.array_equal(pooled.cpu().numpy(), ov.maxpool2x2(x.astype(np.float64)).astype(np.float32))
    y = rng.standard_normal((7, 12)).astype(np.float32)
    b = rng.standard_normal(10).astype(np.float32)
    ty = torch.from_numpy(y).cuda()
    lib.bias_act(ty, 7, 10, 12, torch.from_numpy(b).cuda(), True)
    want = y.copy()
    want[:, :10] = np.maximum(y[:, :10] + b, 0)
    assert np.array_equal(ty.cpu().numpy(), want)


def test_layer_kernels_exact_vector_paths(lib, torch):
    """Channel counts and leading dimensions that are multiples of 4 take the
    16-byte paths; results must be the same bits as the oracle's."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, 6, 10, 8)).astype(np.float32)
    tx = torch.from_numpy(x).cuda()
    col = torch.full((3 * 6 * 10, 76), 9.0, device="cuda")
    lib.im2col3x3(tx, 3, 6, 10, 8, col, 76)
    got = col.cpu().numpy()
    assert np.array_equal(got[:, :72], ov.im2col3x3(x.astype(np.float64)).astype(np.float32))
    assert np.all(got[:, 72:] == 9.0)
    pooled = torch.empty((3, 3, 5, 8), device="cuda")
    lib.maxpool2x2(tx, 3, 6, 10, 8, pooled)
    assert np.array_equal(pooled.cpu().numpy(), ov.maxpool2x2(x.astype(np.float64)).astype(np.float32))
    y = rng.standard_normal((9, 16)).astype(np.float32)
    b = rng.standard_normal(12).astype(np.float32)
    for relu in (True, False):
        ty = torch.from_numpy(y).cuda()
        lib.bias_act(ty, 9, 12, 16, torch.from_numpy(b).cuda(), relu)
        want = y.copy()
        want[:, :12] = y[:, :12] + b
        if relu:
            want[:, :12] = np.maximum(want[:, :12], 0)
        assert np.array_equal(ty.cpu().numpy(), want)


def run_net(lib, torch, batch, width_div, hw, classes, deploy="f32.json", layout="nhwc", with_logits=False):
    h = lib.Handle(json.load(open(os.path.join(DEPLOY, deploy))))
    net = vgg.VGG16(h, batch, width_div, hw, classes, layout=layout)
    x = np.abs(wl.normal_matrix(batch * hw * hw, 3, 3, 1, 5, 0, 1.0)[0]).reshape(batch, hw, hw, 3)
    xin = x if layout == "nhwc" else np.ascontiguousarray(x.transpose(0, 3, 1, 2))
    got = net.forward(torch.from_numpy(xin).cuda()).cpu().numpy()
    want = ov.forward(net.plan, vgg.make_weights(net.plan), x.astype(np.float64))
    rel = np.max(np.abs(got - want)) / np.max(np.abs(want))
    return (rel, got) if with_logits else rel


def test_narrow_network(lib, torch):
    assert run_net(lib, torch, 2, 16, 32, 10) <= 1e-4


def test_full_vgg16_batch1(lib, torch):
    assert run_net(lib, torch, 1, 1, 224, 1000) <= 1e-3


def test_narrow_network_mixed_deployment(lib, torch):
    """The FP32-input class that mixes SIMT and split-BF16 x3 kernels."""
    assert run_net(lib, torch, 2, 16, 32, 10, "f32mix.json") <= 1e-4


def test_nchw_layer_kernels_exact(lib, torch):
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 5, 6, 7)).astype(np.float32)  # NCHW
    col = torch.full((2 * 6 * 7, 48), 9.0, device="cuda")
    lib.im2col3x3_nchw(torch.from_numpy(x).cuda(), 2, 5, 6, 7, col, 48)
    got = col.cpu().numpy()
    want = ov.im2col3x3(x.transpose(0, 2, 3, 1).astype(np.float64)).astype(np.float32)
    assert np.array_equal(got[:, :45], want) and np.all(got[:, 45:] == 9.0)
    y = rng.standard_normal((2, 5, 42)).astype(np.float32)
    b = rng.standard_normal(5).astype(np.float32)
    ty = torch.from_numpy(y).cuda()
    lib.bias_act_nchw(ty, 2, 5, 42, torch.from_numpy(b).cuda(), True)
    assert np.array_equal(ty.cpu().numpy(), np.maximum(y + b[None, :, None], 0))


def test_gemm_batched_layout_matches_oracle_and_nhwc(lib, torch):
    """The paper's GEMM-batched layout (per image Cout x HW, shared weights) gives
    the oracle's logits and, up to rounding, the NHWC variant's."""
    rel_b, logits_b = run_net(lib, torch, 3, 16, 32, 10, layout="batched", with_logits=True)
    rel_n, logits_n = run_net(lib, torch, 3, 16, 32, 10, layout="nhwc", with_logits=True)
    assert rel_b <= 1e-4 and rel_n <= 1e-4
    assert np.max(np.abs(logits_b - logits_n)) <= 2e-4 * np.max(np.abs(logits_n))


def test_gemm_batched_layout_mixed_deployment(lib, torch):
    assert run_net(lib, torch, 2, 16, 32, 10, deploy="f32mix.json", layout="batched") <= 1e-4
