"""FP64 oracle of the MLP performance model -- TEST INFRASTRUCTURE ONLY.

The learned selector predicts, from a GEMM's sizes, the log-throughput of each
deployed kernel relative to the fastest deployed kernel for those sizes (the
log of Section 3.4's standard-normalised performance) and picks the best.  It
replaces the paper's MLP classifier (Section 5.1, Tables 1-2) by a regressor
over the deployed set.

Network: 7 inputs -> 64 ReLU -> 64 ReLU -> 8 linear outputs.  Parameters are
one flat vector in the order W1 (7x64, row = input), b1 (64), W2 (64x64),
b2 (64), W3 (64x8), b3 (8): 5192 values.  Loss: mean squared error over the
measured (mask = 1) outputs.  Optimiser: Adam (Kingma & Ba 2015) with bias
correction.  The ReLU derivative at 0 is taken as 0.

Features of a GEMM (M, N, K, batch, transA, transB, dtype):
    [log2 M / 12, log2 N / 12, log2 K / 12, log2 batch / 4, transA, transB, dtype / 3]
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 7, 64, 8
SIZES = [(N_IN, N_H), (N_H,), (N_H, N_H), (N_H,), (N_H, N_OUT), (N_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SIZES)


def unpack(theta: np.ndarray):
    out, o = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], np.float64).reshape(s))
        o += n
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in parts])


def features(M, N, K, batch, transA, transB, dtype) -> np.ndarray:
    M, N, K, batch = (np.asarray(v, np.float64) for v in (M, N, K, batch))
    return np.stack([np.log2(M) / 12.0, np.log2(N) / 12.0, np.log2(K) / 12.0, np.log2(batch) / 4.0,
                     np.asarray(transA, np.float64), np.asarray(transB, np.float64),
                     np.asarray(dtype, np.float64) / 3.0], axis=-1)


def targets(perf):
    """Training targets and mask of a throughput table (rows = sizes, columns =
    deployed kernels, 0 = not measured): log(perf / row max) where measured,
    else 0 with mask 0 -- Section 3.4's standard normalisation, in log space."""
    perf = np.asarray(perf, np.float64)
    mask = (perf > 0).astype(np.float64)
    T = np.zeros_like(perf)
    for i in range(perf.shape[0]):
        mx = perf[i].max()
        for j in range(perf.shape[1]):
            if perf[i, j] > 0:
                T[i, j] = np.log(perf[i, j] / mx)
    return T, mask


def forward(theta, X):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, np.float64)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, T, mask=None):
    """Returns (loss, gradient) of the masked mean squared error."""
    _, _, W2, _, W3, _ = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    T = np.asarray(T, np.float64)
    m = np.ones_like(T) if mask is None else np.asarray(mask, np.float64)
    cnt = m.sum()
    r = (y - T) * m
    loss = float((r * r).sum() / cnt)
    dy = 2.0 * r / cnt
    dW3 = h2.T @ dy
    db3 = dy.sum(0)
    dz2 = (dy @ W3.T) * (z2 > 0)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)
    dW1 = X.T @ dz1
    db1 = dz1.sum(0)
    return loss, pack([dW1, db1, dW2, db2, dW3, db3])


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based).  Returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def predict_select(theta, X, allowed=None):
    """Predicted outputs and, per row, the index of the largest allowed output
    (lowest index on ties)."""
    y, _ = forward(theta, X)
    if allowed is not None:
        y = np.where(np.asarray(allowed, bool), y, -np.inf)
    return y, np.argmax(y, axis=1)


def init_params(uniforms: np.ndarray) -> np.ndarray:
    """He-uniform weights from N_PARAMS uniform[0, 1) draws; biases 0."""
    parts, o = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        u = np.asarray(uniforms[o:o + n], np.float64)
        if len(s) == 2:
            lim = np.sqrt(6.0 / s[0])
            parts.append(((2.0 * u - 1.0) * lim).reshape(s))
        else:
            parts.append(np.zeros(s))
        o += n
    return pack(parts)
