"""The allocation-free loss/gradient entry point against the allocating one.

Some callers cannot allocate device memory while they run (a process whose
memory is owned by an external pool, a latency-bound loop);
mlp_loss_grad_noalloc serves them from a fixed array inside the library.  This file is collected last so that a failure here
comes after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def inputs(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.random((n, 7)).astype(np.float32)
    T = rng.normal(3.0, 1.0, (n, 8)).astype(np.float32)
    mask = (rng.random((n, 8)) > 0.1).astype(np.float32)
    P = (0.1 * rng.standard_normal(5192)).astype(np.float32)
    return P, X, T, mask


def test_noalloc_matches_allocating_entry_point_twice(lib):
    import torch
    from oracle import mlp as om
    # Two calls in a row: the second uses fewer samples, so stale partials of the
    # first call's extra blocks are still in the shared array and must not leak.
    for n, seed in ((2003, 1), (517, 2)):
        host = inputs(n, seed)
        P, X, T, mask = (torch.from_numpy(a).cuda() for a in host)
        g_ref = torch.empty(5192, device="cuda")
        l_ref = torch.empty(1, device="cuda")
        lib.mlp_loss_grad(P, X, T, mask, g_ref, l_ref)
        g = torch.full((5192,), float("nan"), device="cuda")
        loss = torch.full((1,), float("nan"), device="cuda")
        lib.mlp_loss_grad_noalloc(P, X, T, mask, g, loss)
        torch.cuda.synchronize()
        gr, gn = g_ref.cpu().numpy(), g.cpu().numpy()
        assert np.all(np.isfinite(gn))
        assert np.max(np.abs(gn - gr)) <= 1e-4 * np.max(np.abs(gr))
        assert loss.item() == pytest.approx(l_ref.item(), rel=1e-5)
        # and against the FP64 oracle of the loss and its analytic gradient
        o_loss, o_grad = om.loss_and_grad(*(a.astype(np.float64) for a in host))
        assert np.max(np.abs(gn - o_grad)) <= 1e-4 * np.max(np.abs(o_grad))
        assert loss.item() == pytest.approx(o_loss, rel=1e-5)


def test_noalloc_rejects_more_samples_than_its_scratch(lib):
    import torch
    X = torch.zeros((8193, 7), device="cuda")
    with pytest.raises(lib.KSelectError) as e:
        lib.mlp_loss_grad_noalloc(torch.zeros(5192, device="cuda"), X, torch.zeros((8193, 8), device="cuda"), None,
                                  torch.empty(5192, device="cuda"), torch.empty(1, device="cuda"))
    assert e.value.status == -2
