"""Shared helpers for GPU parity tests: output buffers with sentinel guard regions."""
import numpy as np

SENTINEL = 7777.0
GUARD = 64


class Out:
    """C buffer (batch, M, ldc) inside a flat device tensor with guard regions
    before and after it and sentinel values in the ldc padding; for beta == 0
    the valid region starts as NaN, so a kernel that reads C shows up."""

    def __init__(self, torch, C0, beta, N):
        self.batch, self.M, self.ldc = C0.shape
        flat = np.full(GUARD + C0.size + GUARD, SENTINEL, np.float32)
        body = C0.copy()
        body[:, :, N:] = SENTINEL
        if beta == 0:
            body[:, :, :N] = np.nan
        flat[GUARD:GUARD + C0.size] = body.ravel()
        self.flat = torch.from_numpy(flat).cuda()
        self.ptr = self.flat.data_ptr() + 4 * GUARD

    def result(self, N):
        f = self.flat.cpu().numpy()
        assert np.all(f[:GUARD] == SENTINEL), "write before C"
        assert np.all(f[GUARD + self.batch * self.M * self.ldc:] == SENTINEL), "write after C"
        body = f[GUARD:GUARD + self.batch * self.M * self.ldc].reshape(self.batch, self.M, self.ldc)
        assert np.all(body[:, :, N:] == SENTINEL), "write into ldc padding"
        return body[:, :, :N]
