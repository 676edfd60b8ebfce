"""Seeded synthetic workloads: shape grids and input matrices.

This module holds recipes and random draws only, none of the method's
arithmetic, so that both the CUDA path (tests, bench) and the CPU oracle can be
fed from it without sharing any computation.

Recipes (all from a counter-based Philox stream seeded per workload):

* ``single_gemm_256``: one row-major NN GEMM, M = N = K = 256, alpha = 1,
  beta = 0, A then B drawn i.i.d. uniform[-1, 1] from seed 0.
* ``shape_grid``: the tuning grid, n shapes with M, N, K log-uniform in
  [lo, hi] (rounded to integers), batch uniform in {1, 2, 4, 8, 16} and
  transA / transB uniform in {N, T}.  The paper's own size sets come from
  VGG, ResNet and MobileNet layers (Section 3, "The dataset"); they are not
  available here, and this grid stands in for them.
* ``vgg16_layers``: the 13 3x3 convolutions of VGG16 lowered by im2col
  (M = H*W*batch, K = 9*Cin, N = Cout) and the three fully connected layers
  (M = batch), following the network used in Section 6.
* ``grouped_problems``: uneven groups of GEMMs with M, N, K log-uniform.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BATCH_CHOICES = (1, 2, 4, 8, 16)


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    """A Philox generator for (seed, stream); streams separate independent draws."""
    return np.random.Generator(np.random.Philox(key=[seed, stream]))


def round_up(x: int, m: int) -> int:
    return ((int(x) + m - 1) // m) * m


@dataclasses.dataclass(frozen=True)
class Shape:
    M: int
    N: int
    K: int
    batch: int = 1
    transA: str = "N"
    transB: str = "N"

    @property
    def flops(self) -> int:
        return 2 * self.M * self.N * self.K * self.batch

    def stored_a(self) -> tuple[int, int]:
        """(rows, cols) of A as stored (row-major)."""
        return (self.M, self.K) if self.transA == "N" else (self.K, self.M)

    def stored_b(self) -> tuple[int, int]:
        return (self.K, self.N) if self.transB == "N" else (self.N, self.K)


def log_uniform_int(rng: np.random.Generator, lo: int, hi: int, n: int) -> np.ndarray:
    v = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(np.int64)
    return np.clip(v, lo, hi)


def shape_grid(n: int = 1000, seed: int = 1, lo: int = 16, hi: int = 4096) -> list[Shape]:
    """The tuning grid: M, N, K drawn (in that order) log-uniform, then batch, transA, transB."""
    rng = rng_for(seed)
    M = log_uniform_int(rng, lo, hi, n)
    N = log_uniform_int(rng, lo, hi, n)
    K = log_uniform_int(rng, lo, hi, n)
    batch = rng.choice(np.array(BATCH_CHOICES), n)
    ta = rng.integers(0, 2, n)
    tb = rng.integers(0, 2, n)
    return [Shape(int(M[i]), int(N[i]), int(K[i]), int(batch[i]),
                  "NT"[int(ta[i])], "NT"[int(tb[i])]) for i in range(n)]


def train_test_split(n: int, seed: int, train_frac: float = 0.8) -> tuple[np.ndarray, np.ndarray]:
    """Seeded split of shape indices; the paper does not state its ratio, 80/20 is used."""
    perm = rng_for(seed, 7).permutation(n)
    n_train = int(round(train_frac * n))
    return np.sort(perm[:n_train]), np.sort(perm[n_train:])


def vgg16_layers(batch: int, layout: str = "nhwc") -> list[tuple[str, Shape]]:
    """VGG16 GEMMs.  layout "nhwc": activations (im2col rows of all images) are
    A (M = batch x H x W by K, 'N'); weights are stored output-channel-major
    (N x K), so op(B) = B^T ('T').  layout "batched" (the GEMM-batched form of
    Section 6): per image, weights A (Cout x K, 'N') times the image's im2col
    rows B (H W x K, 'T'), batch = images.  FC layers are the same in both."""
    convs = [("conv1_1", 224, 3, 64), ("conv1_2", 224, 64, 64),
             ("conv2_1", 112, 64, 128), ("conv2_2", 112, 128, 128),
             ("conv3_1", 56, 128, 256), ("conv3_2", 56, 256, 256), ("conv3_3", 56, 256, 256),
             ("conv4_1", 28, 256, 512), ("conv4_2", 28, 512, 512), ("conv4_3", 28, 512, 512),
             ("conv5_1", 14, 512, 512), ("conv5_2", 14, 512, 512), ("conv5_3", 14, 512, 512)]
    if layout == "batched":
        out = [(name, Shape(cout, hw * hw, 9 * cin, batch, "N", "T")) for name, hw, cin, cout in convs]
    else:
        out = [(name, Shape(hw * hw * batch, cout, 9 * cin, 1, "N", "T")) for name, hw, cin, cout in convs]
    out += [("fc6", Shape(batch, 4096, 25088, 1, "N", "T")),
            ("fc7", Shape(batch, 4096, 4096, 1, "N", "T")),
            ("fc8", Shape(batch, 1000, 4096, 1, "N", "T"))]
    return out


def _lowered(name: str, out_hw: int, k: int, cin: int, cout: int, batch: int) -> tuple[str, Shape]:
    """A k x k convolution as an im2col GEMM: M = output pixels x images, N = Cout, K = k^2 Cin."""
    return name, Shape(out_hw * out_hw * batch, cout, k * k * cin, 1, "N", "T")


def resnet50_layers(batch: int) -> list[tuple[str, Shape]]:
    """ResNet-50 (v1.5: stride 2 on the 3x3 convolution of each downsampling block),
    224 x 224 input, every convolution lowered by im2col plus the FC layer.  Repeated
    blocks repeat their GEMMs (the per-layer list, as a forward pass runs it)."""
    out = [_lowered("conv1", 112, 7, 3, 64, batch)]
    cin = 64
    for stage, (width, blocks, hw) in enumerate([(64, 3, 56), (128, 4, 28), (256, 6, 14), (512, 3, 7)], start=2):
        for b in range(blocks):
            in_hw = hw * 2 if (b == 0 and stage > 2) else hw
            tag = f"conv{stage}_{b + 1}"
            out.append(_lowered(tag + "a", in_hw, 1, cin, width, batch))
            out.append(_lowered(tag + "b", hw, 3, width, width, batch))
            out.append(_lowered(tag + "c", hw, 1, width, 4 * width, batch))
            if b == 0:
                out.append(_lowered(tag + "_down", hw, 1, cin, 4 * width, batch))
            cin = 4 * width
    out.append(("fc", Shape(batch, 1000, 2048, 1, "N", "T")))
    return out


def mobilenet_v1_layers(batch: int) -> list[tuple[str, Shape]]:
    """MobileNet v1 (width 1.0, 224 x 224): the first 3x3 convolution and the 13
    pointwise (1x1) convolutions as im2col GEMMs, plus the FC layer.  The 3x3
    depthwise convolutions are not matrix multiplies (one 9-tap filter per channel)
    and are left out."""
    pw = [(112, 32, 64), (56, 64, 128), (56, 128, 128), (28, 128, 256), (28, 256, 256), (14, 256, 512)] + \
         [(14, 512, 512)] * 5 + [(7, 512, 1024), (7, 1024, 1024)]
    out = [_lowered("conv1", 112, 3, 3, 32, batch)]
    out += [_lowered(f"pw{i + 1}", hw, 1, cin, cout, batch) for i, (hw, cin, cout) in enumerate(pw)]
    out.append(("fc", Shape(batch, 1000, 1024, 1, "N", "T")))
    return out


NETWORKS = {"vgg16": vgg16_layers, "resnet50": resnet50_layers, "mobilenet_v1": mobilenet_v1_layers}


def grouped_problems(n: int = 256, seed: int = 3, lo: int = 32, hi: int = 4096) -> list[Shape]:
    """Uneven group: M, N, K log-uniform; op(A) = A (M x K), op(B) = B^T with B
    stored N x K, so both operands are K-contiguous."""
    rng = rng_for(seed)
    M = log_uniform_int(rng, lo, hi, n)
    N = log_uniform_int(rng, lo, hi, n)
    K = log_uniform_int(rng, lo, hi, n)
    return [Shape(int(M[i]), int(N[i]), int(K[i]), 1, "N", "T") for i in range(n)]


def uniform_matrix(rows: int, cols: int, ld: int, batch: int, seed: int, stream: int,
                   lo: float = -1.0, hi: float = 1.0, pad_value: float = np.nan) -> np.ndarray:
    """float32 array (batch, rows, ld): i.i.d. uniform[lo, hi) in the first
    ``cols`` columns and ``pad_value`` in the padding, so that a kernel which
    reads padding poisons its result."""
    rng = rng_for(seed, stream)
    out = np.full((batch, rows, ld), pad_value, dtype=np.float32)
    vals = rng.uniform(lo, hi, size=(batch, rows, cols))
    out[:, :, :cols] = vals.astype(np.float32)
    return out


def normal_matrix(rows: int, cols: int, ld: int, batch: int, seed: int, stream: int,
                  std: float, absolute: bool = False, pad_value: float = np.nan) -> np.ndarray:
    """float32 (batch, rows, ld) of N(0, std^2) draws (|.| of them if ``absolute``)."""
    rng = rng_for(seed, stream)
    out = np.full((batch, rows, ld), pad_value, dtype=np.float32)
    vals = rng.normal(0.0, std, size=(batch, rows, cols))
    if absolute:
        vals = np.abs(vals)
    out[:, :, :cols] = vals.astype(np.float32)
    return out


def integer_matrix(rows: int, cols: int, ld: int, batch: int, seed: int, stream: int,
                   bound: int, pad_value: float = np.nan) -> np.ndarray:
    """float32 (batch, rows, ld) of integers uniform in [-bound, bound]."""
    rng = rng_for(seed, stream)
    out = np.full((batch, rows, ld), pad_value, dtype=np.float32)
    out[:, :, :cols] = rng.integers(-bound, bound + 1, size=(batch, rows, cols)).astype(np.float32)
    return out


def gemm_inputs(shape: Shape, seed: int, ld_multiple: int = 4, beta_nonzero: bool = False,
                kind: str = "uniform", bound: int = 8):
    """Seeded A, B, C0 for one shape, each float32 (batch, rows, ld) with ld the
    stored column count rounded up to ``ld_multiple``.  A is drawn first, then B, then C0."""
    ar, ac = shape.stored_a()
    br, bc = shape.stored_b()
    lda, ldb, ldc = round_up(ac, ld_multiple), round_up(bc, ld_multiple), round_up(shape.N, ld_multiple)
    if kind == "uniform":
        A = uniform_matrix(ar, ac, lda, shape.batch, seed, 1)
        B = uniform_matrix(br, bc, ldb, shape.batch, seed, 2)
        C0 = uniform_matrix(shape.M, shape.N, ldc, shape.batch, seed, 3) if beta_nonzero else \
            np.full((shape.batch, shape.M, ldc), np.nan, dtype=np.float32)
    elif kind == "integer":
        A = integer_matrix(ar, ac, lda, shape.batch, seed, 1, bound)
        B = integer_matrix(br, bc, ldb, shape.batch, seed, 2, bound)
        C0 = integer_matrix(shape.M, shape.N, ldc, shape.batch, seed, 3, bound) if beta_nonzero else \
            np.full((shape.batch, shape.M, ldc), np.nan, dtype=np.float32)
    else:
        raise ValueError(kind)
    return A, B, C0


def sample_positions(shape: Shape, n_rows: int, n_cols: int, seed: int) -> np.ndarray:
    """Deterministic sample of output entries (b, i, j) for large-shape checks:
    per batch entry, ``n_rows`` seeded rows x all columns plus ``n_cols``
    seeded columns x all rows (duplicates removed)."""
    rng = rng_for(seed, 11)
    pos = []
    for b in range(shape.batch):
        rows = rng.choice(shape.M, size=min(n_rows, shape.M), replace=False)
        cols = rng.choice(shape.N, size=min(n_cols, shape.N), replace=False)
        for i in rows:
            pos.append(np.stack([np.full(shape.N, b), np.full(shape.N, i), np.arange(shape.N)], 1))
        for j in cols:
            pos.append(np.stack([np.full(shape.M, b), np.arange(shape.M), np.full(shape.M, j)], 1))
    p = np.unique(np.concatenate(pos, 0).astype(np.int64), axis=0)
    return p


def band_positions(shape: Shape, band_m: int, band_n: int, seed: int) -> np.ndarray:
    """Sampled output entries (b, i, j) that meet every band_m x band_n output
    tile: per batch entry, one seeded row inside each band of band_m rows x all
    columns, plus one seeded column inside each band of band_n columns x all
    rows (duplicates removed)."""
    rng = rng_for(seed, 13)
    pos = []
    for b in range(shape.batch):
        for r0 in range(0, shape.M, band_m):
            i = r0 + int(rng.integers(0, min(band_m, shape.M - r0)))
            pos.append(np.stack([np.full(shape.N, b), np.full(shape.N, i), np.arange(shape.N)], 1))
        for c0 in range(0, shape.N, band_n):
            j = c0 + int(rng.integers(0, min(band_n, shape.N - c0)))
            pos.append(np.stack([np.full(shape.M, b), np.arange(shape.M), np.full(shape.M, j)], 1))
    return np.unique(np.concatenate(pos, 0).astype(np.int64), axis=0)
