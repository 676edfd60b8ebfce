"""FP64 oracle of the VGG16 forward pass (Section 6) -- TEST INFRASTRUCTURE ONLY.

NHWC activations.  A 3x3 convolution with padding 1 is evaluated as the
im2col matrix (rows = output pixels, columns ordered (kh, kw, c)) times the
transposed weights (Cout x 9 Cin), a library matmul serving as the product;
``conv3x3_direct`` is the definition written as loops, used to pin it.
"""
from __future__ import annotations

import numpy as np


def im2col3x3(x: np.ndarray) -> np.ndarray:
    N, H, W, C = x.shape
    xp = np.zeros((N, H + 2, W + 2, C))
    xp[:, 1:-1, 1:-1, :] = x
    cols = [xp[:, kh:kh + H, kw:kw + W, :] for kh in range(3) for kw in range(3)]
    return np.concatenate(cols, axis=3).reshape(N * H * W, 9 * C)


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    N, H, Wd, _ = x.shape
    return (im2col3x3(x) @ np.asarray(W, np.float64).T + b).reshape(N, H, Wd, -1)


def conv3x3_direct(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[n,h,w,o] = b[o] + sum_{kh,kw,c} x[n,h+kh-1,w+kw-1,c] W[o,(kh*3+kw)*C+c] (zero padding)."""
    N, H, Wd, C = x.shape
    O = W.shape[0]
    out = np.zeros((N, H, Wd, O))
    for n in range(N):
        for h in range(H):
            for w in range(Wd):
                for o in range(O):
                    s = b[o]
                    for kh in range(3):
                        for kw in range(3):
                            hh, ww = h + kh - 1, w + kw - 1
                            if 0 <= hh < H and 0 <= ww < Wd:
                                for c in range(C):
                                    s += x[n, hh, ww, c] * W[o, (kh * 3 + kw) * C + c]
                    out[n, h, w, o] = s
    return out


def maxpool2x2(x: np.ndarray) -> np.ndarray:
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).max(axis=(2, 4))


def forward(plan, weights, x: np.ndarray) -> np.ndarray:
    """Logits (N, classes) in FP64 for the plan/weights of the library's VGG16."""
    a = np.asarray(x, np.float64)
    for layer, w in zip(plan, weights):
        if layer[0] == "conv":
            a = np.maximum(conv3x3(a, w[0], np.asarray(w[1], np.float64)), 0.0)
        elif layer[0] == "pool":
            a = maxpool2x2(a)
        else:
            a = a.reshape(a.shape[0], -1) @ np.asarray(w[0], np.float64).T + np.asarray(w[1], np.float64)
            if layer[3]:
                a = np.maximum(a, 0.0)
    return a
