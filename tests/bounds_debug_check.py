"""Run by tests/test_bounds_debug_gpu.py in a child process with
KSELECT_DEBUG_BOUNDS=1, so that the binding loads the bounds-checking debug
build.  Every FP32 config that build instantiates, and its split-K id where it
has one, runs ragged batched products of every transpose (beta != 0, NaN
padding), explicit-stride batches with gaps and a zero stride, and shapes that
split; the device counter of accesses outside the operands' extents must stay
0 and every result must match the FP64 oracle.  Then the checker is shown to
work: with A's declared extent 16 bytes short, accesses are flagged.
Prints one JSON line."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import gemm as og  # noqa: E402
from paper_2008_13145_gb300 import kselect as ks  # noqa: E402
from paper_2008_13145_gb300 import workloads as wl  # noqa: E402


def errors(clear=True):
    v = ks.i32()
    ks.check(ks._lib.kselect_debug_bounds_errors(ks.ctypes.byref(v), int(clear)), "kselect_debug_bounds_errors")
    return v.value


def run(cid, sh, alpha, beta, seed, strided=False):
    A, B, C0 = wl.gemm_inputs(sh, seed=seed, beta_nonzero=beta != 0, ld_multiple=4)
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.from_numpy(np.nan_to_num(C0, nan=0.0) if beta != 0 else np.zeros_like(C0)).cuda()
    if not strided:
        st = ks._lib.gemm_with_config(cid, sh.transA.encode(), sh.transB.encode(), sh.M, sh.N, sh.K, alpha,
                                      tA.data_ptr(), A.shape[2], tB.data_ptr(), B.shape[2], beta, C.data_ptr(),
                                      C0.shape[2], sh.batch, None)
        Aref = A
    else:  # A shared by every entry (stride 0)
        st = ks._lib.gemm_strided_batched_with_config(cid, sh.transA.encode(), sh.transB.encode(), sh.M, sh.N, sh.K,
                                                      alpha, tA.data_ptr(), A.shape[2], 0, tB.data_ptr(), B.shape[2],
                                                      B.shape[1] * B.shape[2], beta, C.data_ptr(), C0.shape[2],
                                                      C0.shape[1] * C0.shape[2], sh.batch, None)
        Aref = np.repeat(A[:1], sh.batch, axis=0)
    if st == -6:
        return None  # not instantiated in the debug build
    ks.check(st, "gemm")
    torch.cuda.synchronize()
    ref, den = og.gemm(sh.transA, sh.transB, sh.M, sh.N, sh.K, alpha, Aref, B, beta, C0 if beta != 0 else None)
    return og.error_ratio(C.cpu().numpy()[:, :, :sh.N], ref, den)


def main():
    errors(clear=True)
    ids = [c for c in ks.config_ids(ks.PREC_F32)]
    worst, cases, configs = 0.0, 0, set()
    shapes = [wl.Shape(37, 45, 29, 2, "N", "N"), wl.Shape(45, 37, 61, 3, "T", "N"), wl.Shape(70, 33, 40, 2, "N", "T"),
              wl.Shape(29, 64, 35, 2, "T", "T"), wl.Shape(40, 56, 1200, 2, "T", "N")]
    for cid in ids:
        for n, sh in enumerate(shapes):
            for strided in (False, True):
                err = run(cid, sh, -0.5, 0.25, 100 + n, strided)
                if err is None:
                    break
                cases += 1
                configs.add(cid)
                worst = max(worst, err)
    found = errors(clear=True)
    # the checker itself: A's extent declared 16 bytes short
    ks.check(ks._lib.kselect_debug_shrink_extents(16, 0, 0), "kselect_debug_shrink_extents")
    probe = next(iter(sorted(configs)))
    run(probe, wl.Shape(64, 64, 64, 1, "N", "N"), 1.0, 0.0, 7)
    flagged = errors(clear=True)
    ks.check(ks._lib.kselect_debug_shrink_extents(0, 0, 0), "kselect_debug_shrink_extents")
    print(json.dumps({"configs": len(configs), "split_configs": sum(c >= 2000 for c in configs), "cases": cases,
                      "out_of_bounds": found, "worst_error_ratio": worst, "negative_control_flagged": flagged}))


if __name__ == "__main__":
    main()
