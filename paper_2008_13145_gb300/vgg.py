"""VGG16 inference on the library (Section 6 analogue).

NHWC activations; every 3x3 convolution is im2col + the library's GEMM (the
handle's selector picks the kernel per layer) + fused bias/ReLU; 2x2 max
pooling; three fully connected layers.  Weights are synthetic He-normal draws
(the paper's pretrained Keras weights are not available), biases small normal
draws.  ``width_div`` and ``hw`` shrink the network for tests.
"""
from __future__ import annotations

import numpy as np

from . import workloads as wl

CFG = [64, 64, "M", 128, 128, "M", 256, 256, 256, "M", 512, 512, 512, "M", 512, 512, 512, "M"]
FC = [4096, 4096, 1000]


def layer_plan(width_div: int = 1, hw: int = 224, classes: int = 1000):
    """[("conv", H, Cin, Cout) | ("pool", H, C) | ("fc", Kin, Nout, relu)] for the network."""
    plan, c, h = [], 3, hw
    for v in CFG:
        if v == "M":
            plan.append(("pool", h, c))
            h //= 2
        else:
            co = max(v // width_div, 1)
            plan.append(("conv", h, c, co))
            c = co
    fin = h * h * c
    for i, f in enumerate(FC):
        fo = classes if i == len(FC) - 1 else max(f // width_div, 1)
        plan.append(("fc", fin, fo, i < len(FC) - 1))
        fin = fo
    return plan


def make_weights(plan, seed: int = 7):
    """Host float32 weights: conv (Cout, 9 Cin), fc (Nout, Kin), He-normal; biases N(0, 0.05^2)."""
    ws = []
    for i, layer in enumerate(plan):
        if layer[0] == "conv":
            _, _, ci, co = layer
            W = wl.normal_matrix(co, 9 * ci, 9 * ci, 1, seed, 2 * i, np.sqrt(2.0 / (9 * ci)))[0]
            b = wl.normal_matrix(1, co, co, 1, seed, 2 * i + 1, 0.05)[0, 0]
            ws.append((W, b))
        elif layer[0] == "fc":
            _, kin, nout, _ = layer
            W = wl.normal_matrix(nout, kin, kin, 1, seed, 2 * i, np.sqrt(2.0 / kin))[0]
            b = wl.normal_matrix(1, nout, nout, 1, seed, 2 * i + 1, 0.05)[0, 0]
            ws.append((W, b))
        else:
            ws.append(None)
    return ws


def flops(plan, batch: int) -> int:
    f = 0
    for layer in plan:
        if layer[0] == "conv":
            _, h, ci, co = layer
            f += 2 * batch * h * h * 9 * ci * co
        elif layer[0] == "fc":
            f += 2 * batch * layer[1] * layer[2]
    return f


def nchw_fc1(W1: np.ndarray, hw: int, c: int) -> np.ndarray:
    """The first FC layer's weights for an NCHW flatten (c, h, w): the same layer
    as W1 on the NHWC flatten (h, w, c), so both layouts compute the same logits."""
    nout = W1.shape[0]
    return np.ascontiguousarray(W1.reshape(nout, hw, hw, c).transpose(0, 3, 1, 2).reshape(nout, -1))


class VGG16:
    """Device weights plus activation buffers for one batch size.

    layout "nhwc": one GEMM per convolution with M = batch x H x W, N = Cout
    (the im2col rows of all images at once).  layout "batched": the paper's
    GEMM-batched form, per image M = Cout, N = H x W, batch = images, the
    weights shared by a zero batch stride; activations NCHW."""

    def __init__(self, handle, batch: int, width_div: int = 1, hw: int = 224, classes: int = 1000, seed: int = 7,
                 layout: str = "nhwc"):
        import torch
        assert layout in ("nhwc", "batched")
        self.plan = layer_plan(width_div, hw, classes)
        self.handle, self.batch, self.layout = handle, batch, layout
        host = make_weights(self.plan, seed)
        if layout == "batched":
            fc1 = next(i for i, layer in enumerate(self.plan) if layer[0] == "fc")
            last = [layer for layer in self.plan[:fc1] if layer[0] == "pool"][-1]
            side, chans = last[1] // 2, last[2]
            host[fc1] = (nchw_fc1(host[fc1][0], side, chans), host[fc1][1])
        self.weights = [None if w is None else (torch.from_numpy(w[0]).cuda(), torch.from_numpy(w[1]).cuda())
                        for w in host]
        biggest_act, biggest_col = 0, 0
        for layer in self.plan:
            if layer[0] == "conv":
                _, h, ci, co = layer
                biggest_act = max(biggest_act, batch * h * h * max(ci, co))
                biggest_col = max(biggest_col, batch * h * h * wl.round_up(9 * ci, 4))
            elif layer[0] == "fc":
                biggest_act = max(biggest_act, batch * max(layer[1], layer[2]))
        self.act = [torch.empty(biggest_act, device="cuda"), torch.empty(biggest_act, device="cuda")]
        self.col = torch.empty(biggest_col, device="cuda")
        self.flops = flops(self.plan, batch)

    def forward(self, x, stream=None):
        """x: device (batch, hw, hw, 3) NHWC float32 (the "batched" layout takes
        (batch, 3, hw, hw) NCHW); returns the logits tensor (batch, classes)."""
        from . import kselect as ks
        n = self.batch
        cur = x.reshape(-1)
        nxt = 0
        for layer, w in zip(self.plan, self.weights):
            out = self.act[nxt]
            if self.layout == "batched" and layer[0] != "fc":
                if layer[0] == "conv":
                    _, h, ci, co = layer
                    K, ldk = 9 * ci, wl.round_up(9 * ci, 4)
                    ks.im2col3x3_nchw(cur, n, ci, h, h, self.col, ldk, stream)
                    ks.gemm_strided_batched(self.handle, "N", "T", co, h * h, K, 1.0, w[0], K, 0, self.col, ldk,
                                            h * h * ldk, 0.0, out, h * h, co * h * h, n, stream)
                    ks.bias_act_nchw(out, n, co, h * h, w[1], True, stream)
                else:
                    _, h, c = layer
                    ks.maxpool2x2(cur, n * c, h, h, 1, out, stream)
                cur, nxt = out, 1 - nxt
                continue
            if layer[0] == "conv":
                _, h, ci, co = layer
                M, K = n * h * h, 9 * ci
                ldk = wl.round_up(K, 4)
                ks.im2col3x3(cur, n, h, h, ci, self.col, ldk, stream)
                ks.gemm(self.handle, "N", "T", M, co, K, 1.0, self.col, ldk, w[0], K, 0.0, out, co, 1, stream)
                ks.bias_act(out, M, co, co, w[1], True, stream)
            elif layer[0] == "pool":
                _, h, c = layer
                ks.maxpool2x2(cur, n, h, h, c, out, stream)
            else:
                _, kin, nout, relu = layer
                ks.gemm(self.handle, "N", "T", n, nout, kin, 1.0, cur, kin, w[0], kin, 0.0, out, nout, 1, stream)
                ks.bias_act(out, n, nout, nout, w[1], relu, stream)
            cur, nxt = out, 1 - nxt
        return cur[: n * self.plan[-1][2]].view(n, self.plan[-1][2])
