"""Back-to-back dependent GEMMs on one stream, with no host synchronisation.

Every kernel of the GEMM path is launched with programmatic dependent launch:
it may be scheduled while the previous kernel drains and must wait for it
before touching memory.  A ping-pong chain X_{i+1} = X_i * P_i, each P_i a
permutation matrix and X_0 small integers, is exact in every FP32-storage
family (SIMT, split-K, TF32 with its pre-pass, split-BF16 x3) and has a
closed form: X_0's columns moved by the composed permutation.  Each launch
reads the buffer the previous launch wrote (read after write) and overwrites
the buffer the launch before that read (write after read)."""
import numpy as np
import pytest

from paper_2008_13145_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

M, N = 64, 1536  # X is M x N; every P is N x N
# (config, transB): SIMT staged / direct, split-K kind, TF32 (B through the
# pre-pass when stored K x N) in BN 128 and 256 tiles, x3 in BN 256 tiles
# with 4 and 3 stages.
CHAIN = [(533, "N"), (2533, "T"), (1010, "N"), (369, "T"), (1216, "N"), (2533, "N"), (1016, "T"), (1214, "T"),
         (368, "N")]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def test_dependent_chain_without_sync(lib, torch):
    ks = lib
    split, _ = ks.split_factor(2533, M, N, N, 1)
    assert split > 1, "the chain should contain a split-K launch (partial GEMM + reduction)"
    X0 = wl.integer_matrix(M, N, N, 1, seed=21, stream=1, bound=8)[0]
    rng = np.random.default_rng(22)
    perms = [rng.permutation(N) for _ in CHAIN]
    mats = []
    for perm, (_, tb) in zip(perms, CHAIN):
        P = np.zeros((N, N), np.float32)  # op(B)[k, perm[k]] = 1
        P[np.arange(N), perm] = 1.0
        mats.append(torch.from_numpy(P if tb == "N" else np.ascontiguousarray(P.T)).cuda())
    X = [torch.from_numpy(X0).cuda(), torch.full((M, N), float("nan"), device="cuda")]
    for rep in range(2):
        if rep:
            X[0].copy_(torch.from_numpy(X0))
        torch.cuda.synchronize()
        for i, ((cid, tb), P) in enumerate(zip(CHAIN, mats)):
            src, dst = X[i % 2], X[(i + 1) % 2]
            ks.gemm_with_config(cid, "N", tb, M, N, N, 1.0, src, N, P, N, 0.0, dst, N, 1)
        torch.cuda.synchronize()
        expect = X0.copy()
        for perm in perms:
            nxt = np.empty_like(expect)
            nxt[:, perm] = expect
            expect = nxt
        got = X[len(CHAIN) % 2].cpu().numpy()
        assert np.array_equal(got, expect), f"repetition {rep}: {int((got != expect).sum())} entries differ"
    assert ks.device_status() == 0
