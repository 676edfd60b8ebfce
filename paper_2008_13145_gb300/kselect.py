"""ctypes binding of libkselect.so, entry point for entry point (argument marshalling only).

Every function takes device buffers as torch tensors (or raw integer device
pointers) and an optional stream (torch.cuda.Stream, raw handle, or None for
torch's current stream).  A non-OK status raises ``KSelectError``.  Importing
this module loads the compiled library and raises if it is missing: there is
no fallback implementation.  With KSELECT_DEBUG_BOUNDS=1 in the environment it
loads the bounds-checking debug build (libkselect_debug.so) instead.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import DEBUG_LIB, LIB

if os.environ.get("KSELECT_DEBUG_BOUNDS") == "1":
    LIB = DEBUG_LIB
if not os.path.exists(LIB):
    raise ImportError(f"{os.path.basename(LIB)} is not built ({LIB}); run __graft_entry__.build() first")

_lib = ctypes.CDLL(LIB)

i32, i64, u64, f32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float, ctypes.c_double
vp, ch = ctypes.c_void_p, ctypes.c_char

GEMM_OK = 0
PREC_F32, PREC_TF32, PREC_BF16, PREC_F32X3 = 0, 1, 2, 3
PRECISIONS = {"f32": PREC_F32, "tf32": PREC_TF32, "bf16": PREC_BF16, "f32x3": PREC_F32X3}
MLP_PARAMS = 5192
TREE_FEATURES = 5  # M, N, K, batch, M * N * batch
MAX_DEPLOYED = 16


class TreeNode(ctypes.Structure):
    _fields_ = [("feature", i32), ("left", i32), ("right", i32), ("label", i32), ("threshold", f64)]


class Problem(ctypes.Structure):
    _fields_ = [("M", i64), ("N", i64), ("K", i64), ("transA", ch), ("transB", ch), ("alpha", f32), ("beta", f32),
                ("A", vp), ("lda", i64), ("B", vp), ("ldb", i64), ("C", vp), ("ldc", i64)]


class HostProblem(ctypes.Structure):
    _fields_ = [("transA", ctypes.c_char), ("transB", ctypes.c_char), ("M", i64), ("N", i64), ("K", i64),
                ("batch", i64), ("alpha", f32), ("beta", f32), ("A_host", vp), ("lda", i64), ("B_host", vp),
                ("ldb", i64), ("C_host", vp), ("ldc", i64), ("A_dev", vp), ("B_dev", vp), ("C_dev", vp)]


class Deployment(ctypes.Structure):
    _fields_ = [("precision", i32), ("n_configs", i32), ("config_ids", ctypes.POINTER(i32)),
                ("n_nodes", i32), ("nodes", ctypes.POINTER(TreeNode)), ("mlp_params", ctypes.POINTER(f32)),
                ("n_known", i32), ("known_sizes", ctypes.POINTER(i64)), ("known_ids", ctypes.POINTER(i32)),
                ("n_trees", i32), ("tree_roots", ctypes.POINTER(i32))]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("gemm_status_string", ctypes.c_char_p, [i32])
_sig("gemm_last_cuda_error", i32, [])
_sig("kselect_debug_bounds_errors", i32, [ctypes.POINTER(i32), i32])
_sig("kselect_debug_shrink_extents", i32, [i64, i64, i64])
_sig("gemm_config_count", i32, [i32])
_sig("gemm_config_id", i32, [i32, i32])
_sig("gemm_config_params", i32, [i32, ctypes.POINTER(i32)])
_sig("gemm_split_choose", i32, [i64, i64, i64, i64, i32, i32, i32, i32, i32, ctypes.POINTER(i32)])
_sig("gemm_split_factor", i32, [i32, i64, i64, i64, i64, ctypes.POINTER(i32)])
_sig("gemm_library_create", i32, [ctypes.POINTER(Deployment), ctypes.POINTER(vp)])
_sig("gemm_library_destroy", None, [vp])
_sig("select_kernel", i32, [vp, i64, i64, i64, i64])
_GEMM_ARGS = [ch, ch, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i64, vp]
_sig("gemm", i32, [vp] + _GEMM_ARGS)
_sig("gemm_with_config", i32, [i32] + _GEMM_ARGS)
_STRIDED_ARGS = [ch, ch, i64, i64, i64, f32, vp, i64, i64, vp, i64, i64, f32, vp, i64, i64, i64, vp]
_sig("gemm_strided_batched", i32, [vp] + _STRIDED_ARGS)
_sig("gemm_strided_batched_with_config", i32, [i32] + _STRIDED_ARGS)
_sig("gemm_host", i32, [vp, ch, ch, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i64, vp, vp, vp, vp])
_sig("gemm_host_pipeline", i32, [vp, i32, ctypes.POINTER(HostProblem), vp])
_sig("gemm_benchmark", i32, [i32, ch, ch, i64, i64, i64, vp, i64, vp, i64, vp, i64, i64, i32, i32, i32, f64,
                             ctypes.POINTER(f64), ctypes.POINTER(i32), vp])
_sig("gemm_error_check", i32, [i64, i64, i64, vp, i64, i64, i64, vp, vp, vp, ctypes.POINTER(f64), vp])
_sig("kselect_fill_uniform", i32, [vp, i64, i64, i64, i64, u64, f32, f32, f32, vp])
_sig("gemm_device_status", i32, [ctypes.POINTER(i32), i32])
_sig("kselect_wait_selftest", i32, [i64, ctypes.POINTER(i32), vp])
_sig("gemm_grouped_plan_create", i32, [i32, i32, ctypes.POINTER(Problem), vp, ctypes.POINTER(vp)])
_sig("gemm_grouped_run", i32, [vp, vp])
_sig("gemm_grouped_plan_destroy", None, [vp])
_sig("gemm_grouped_with_config", i32, [i32, i32, ctypes.POINTER(Problem), vp])
_sig("gemm_grouped", i32, [vp, i32, ctypes.POINTER(Problem), i32, vp])
_sig("gemm_grouped_reserve", i32, [vp, i32, ctypes.POINTER(Problem), i32])
_sig("gemm_grouped_select", i32, [vp, i32, ctypes.POINTER(Problem)])
_sig("mlp_features", i32, [i32, vp, vp, vp])
_sig("mlp_forward", i32, [i32, vp, vp, vp, vp])
_sig("mlp_targets", i32, [i32, i32, vp, vp, vp, vp])
_sig("mlp_loss_grad", i32, [i32, vp, vp, vp, vp, vp, vp, vp])
_sig("mlp_adam_step", i32, [vp, vp, vp, vp, i32, f32, f32, f32, f32, vp])
_sig("mlp_loss_grad_noalloc", i32, [i32, vp, vp, vp, vp, vp, vp, vp])
_sig("mlp_train", i32, [i32, vp, vp, vp, vp, vp, vp, i32, i32, f32, f32, f32, f32, vp, vp])
_sig("select_kernels_batched", i32, [vp, i32, vp, vp, vp, vp])
_sig("gemm_benchmark_configs", i32, [i32, ctypes.POINTER(i32), ch, ch, i64, i64, i64, vp, i64, vp, i64, vp, i64,
                                     i64, i32, i32, i32, f64, f64, ctypes.POINTER(f64), ctypes.POINTER(i32),
                                     ctypes.POINTER(f64), ctypes.POINTER(i32), vp])
_sig("kselect_normalise", i32, [i64, i32, vp, vp, i32, vp])
_sig("kselect_kmeans", i32, [i32, i32, i32, i32, vp, ctypes.POINTER(ctypes.c_uint32), i32, f32, vp, vp,
                             ctypes.POINTER(f64), ctypes.POINTER(i32), vp])
_sig("kselect_pca", i32, [i32, i32, vp, i32, i32, vp, vp, vp, vp, ctypes.POINTER(f64), ctypes.POINTER(f64), vp])
_sig("kselect_pca_backproject", i32, [i32, i32, i32, vp, vp, vp, vp, vp])
_sig("kselect_score", i32, [i32, i32, vp, i32, ctypes.POINTER(i32), vp, f32, ctypes.POINTER(f64), vp])
_sig("kselect_im2col3x3", i32, [vp, i32, i32, i32, i32, vp, i64, vp])
_sig("kselect_bias_act", i32, [vp, i64, i32, i64, vp, i32, vp])
_sig("kselect_maxpool2x2", i32, [vp, i32, i32, i32, i32, vp, vp])
_sig("kselect_im2col3x3_nchw", i32, [vp, i32, i32, i32, i32, vp, i64, vp])
_sig("kselect_bias_act_nchw", i32, [vp, i32, i32, i64, vp, i32, vp])
_sig("kselect_knn", i32, [i32, i32, i32, vp, vp, vp, i32, vp, vp])
_sig("kselect_representatives", i32, [i32, i32, ctypes.POINTER(f32), i32, ctypes.POINTER(i32), i32,
                                      ctypes.POINTER(i32), ctypes.POINTER(i32)])
_sig("kselect_top_n", i32, [i32, i32, ctypes.POINTER(f32), i32, ctypes.POINTER(i32)])
_sig("kselect_spectral_embedding", i32, [i32, i32, vp, f32, i32, i32, i32, vp, vp, ctypes.POINTER(f64), vp])
_sig("kselect_cluster_geomean", i32, [i32, i32, vp, vp, i32, f32, vp, vp])
_sig("kselect_tree_regress", i32, [i32, i32, ctypes.POINTER(f64), ctypes.POINTER(f32), i32, ctypes.POINTER(i32),
                                   ctypes.POINTER(f32), ctypes.POINTER(i32)])
_sig("kselect_tree_train_rf", i32, [i32, ctypes.POINTER(f64), ctypes.POINTER(i32), i32, i32, i32, i32,
                                    ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(TreeNode), i32, ctypes.POINTER(i32)])
_sig("kselect_selector_features", i32, [i32, ctypes.POINTER(i64), ctypes.POINTER(f64)])
_sig("kselect_best_labels", i32, [i32, i32, ctypes.POINTER(f64), i32, ctypes.POINTER(i32), ctypes.POINTER(i32)])
_sig("kselect_tree_train", i32, [i32, ctypes.POINTER(f64), ctypes.POINTER(i32), i32, i32, i32,
                                 ctypes.POINTER(TreeNode), i32, ctypes.POINTER(i32)])


class KSelectError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.gemm_status_string(status).decode()
        if status == -4:
            msg += f" (cudaError {_lib.gemm_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [{status}]")


def check(status: int, where: str) -> None:
    if status != GEMM_OK:
        raise KSelectError(status, where)


def ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _c(t: str) -> bytes:
    return t.encode() if isinstance(t, str) else t


# ---------------------------------------------------------------- config space
def config_count(precision: int) -> int:
    n = _lib.gemm_config_count(precision)
    if n < 0:
        raise KSelectError(n, "gemm_config_count")
    return n


def config_id(precision: int, index: int) -> int:
    r = _lib.gemm_config_id(precision, index)
    if r < 0:
        raise KSelectError(r, "gemm_config_id")
    return r


def config_ids(precision: int) -> list[int]:
    return [config_id(precision, i) for i in range(config_count(precision))]


def family_of(cid: int) -> int:
    return config_params(cid)[0]


def config_params(cid: int) -> list[int]:
    out = (i32 * 8)()
    check(_lib.gemm_config_params(cid, out), "gemm_config_params")
    return list(out)


def split_choose(M, N, K, batch, BM, BN, BK, resident_ctas_per_sm, sm_count) -> tuple[int, int]:
    """(split factor, K per split) of the split-K kind's host cost model."""
    kc = i32()
    r = _lib.gemm_split_choose(M, N, K, batch, BM, BN, BK, resident_ctas_per_sm, sm_count, ctypes.byref(kc))
    if r < 0:
        raise KSelectError(r, "gemm_split_choose")
    return r, kc.value


def split_factor(cid: int, M, N, K, batch) -> tuple[int, int]:
    """(split factor, K per split) config `cid` uses for these sizes on the current device."""
    kc = i32()
    r = _lib.gemm_split_factor(cid, M, N, K, batch, ctypes.byref(kc))
    if r < 0:
        raise KSelectError(r, "gemm_split_factor")
    return r, kc.value


# ---------------------------------------------------------------- handle
class Handle:
    """An immutable library handle built from a deployment dict:
    {"precision": int, "config_ids": [...], "nodes": [{"feature", "threshold",
    "left", "right", "label"}, ...], "mlp_params": [5192 floats] | None,
    "known": [[M, N, K, batch, config id], ...] | None,
    "forest": [[nodes of tree 0], [nodes of tree 1], ...] | None}.
    With "forest", its trees (each with node indices local to itself) replace
    "nodes" and vote."""

    def __init__(self, deployment: dict):
        ids = list(deployment["config_ids"])
        nodes = deployment.get("nodes") or []
        roots = []
        if deployment.get("forest"):
            nodes = []
            for tree in deployment["forest"]:
                base = len(nodes)
                roots.append(base)
                nodes += [{**n, "left": n["left"] + base if n["feature"] >= 0 else -1,
                           "right": n["right"] + base if n["feature"] >= 0 else -1} for n in tree]
        self._roots = (i32 * max(len(roots), 1))(*roots)
        mlp = deployment.get("mlp_params")
        self._ids = (i32 * max(len(ids), 1))(*ids)
        self._nodes = (TreeNode * max(len(nodes), 1))(
            *[TreeNode(int(n["feature"]), int(n["left"]), int(n["right"]), int(n["label"]),
                       float(n["threshold"])) for n in nodes])
        self._mlp = (f32 * MLP_PARAMS)(*np.asarray(mlp, np.float32)) if mlp is not None else None
        known = deployment.get("known") or []  # rows (M, N, K, batch, config id)
        self._ksz = (i64 * max(4 * len(known), 1))(*[int(v) for r in known for v in r[:4]])
        self._kid = (i32 * max(len(known), 1))(*[int(r[4]) for r in known])
        d = Deployment(int(deployment["precision"]), len(ids), self._ids, len(nodes), self._nodes,
                       self._mlp if self._mlp is not None else None, len(known), self._ksz, self._kid,
                       len(roots), self._roots)
        h = vp()
        check(_lib.gemm_library_create(ctypes.byref(d), ctypes.byref(h)), "gemm_library_create")
        self.value = h.value
        self.precision = int(deployment["precision"])
        self.ids = ids

    def close(self):
        if self.value:
            _lib.gemm_library_destroy(self.value)
            self.value = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def select_kernel(handle: Handle, M: int, N: int, K: int, batch: int = 1) -> int:
    r = _lib.select_kernel(handle.value, M, N, K, batch)
    if r < 0:
        raise KSelectError(r, "select_kernel")
    return r


# ---------------------------------------------------------------- GEMM
def gemm(handle: Handle, transA: str, transB: str, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, batch=1,
         stream=None) -> None:
    check(_lib.gemm(handle.value, _c(transA), _c(transB), M, N, K, alpha, ptr(A), lda, ptr(B), ldb, beta,
                    ptr(C), ldc, batch, stream_handle(stream)), "gemm")


def gemm_host(handle: Handle, transA: str, transB: str, M, N, K, alpha, A_host, lda, B_host, ldb, beta, C_host, ldc,
              batch, A_dev, B_dev, C_dev, stream=None) -> None:
    """gemm() on host buffers (pinned torch tensors or raw host pointers) through device staging buffers."""
    check(_lib.gemm_host(handle.value, _c(transA), _c(transB), M, N, K, alpha, ptr(A_host), lda, ptr(B_host), ldb,
                         beta, ptr(C_host), ldc, batch, ptr(A_dev), ptr(B_dev), ptr(C_dev), stream_handle(stream)),
          "gemm_host")


def gemm_with_config(cid: int, transA: str, transB: str, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, batch=1,
                     stream=None) -> None:
    check(_lib.gemm_with_config(cid, _c(transA), _c(transB), M, N, K, alpha, ptr(A), lda, ptr(B), ldb, beta,
                                ptr(C), ldc, batch, stream_handle(stream)), "gemm_with_config")


def host_problems(problems: list[dict]):
    """ctypes array of gemm_host_problem_t from dicts with the gemm_host arguments
    (transA, transB, M, N, K, batch, alpha, beta, A_host, lda, B_host, ldb, C_host,
    ldc, A_dev, B_dev, C_dev); keep the result alive while the call is queued."""
    arr = (HostProblem * len(problems))()
    for q, p in zip(arr, problems):
        q.transA, q.transB = _c(p["transA"]), _c(p["transB"])
        q.M, q.N, q.K, q.batch = p["M"], p["N"], p["K"], p.get("batch", 1)
        q.alpha, q.beta = p.get("alpha", 1.0), p.get("beta", 0.0)
        q.A_host, q.lda, q.B_host, q.ldb = ptr(p["A_host"]), p["lda"], ptr(p["B_host"]), p["ldb"]
        q.C_host, q.ldc = ptr(p["C_host"]), p["ldc"]
        q.A_dev, q.B_dev, q.C_dev = ptr(p["A_dev"]), ptr(p["B_dev"]), ptr(p["C_dev"])
    return arr


def gemm_host_pipeline(handle: Handle, problems, stream=None) -> None:
    """problems: a list of dicts (see host_problems) or its ctypes array."""
    arr = problems if isinstance(problems, ctypes.Array) else host_problems(problems)
    check(_lib.gemm_host_pipeline(handle.value, len(arr), arr, stream_handle(stream)), "gemm_host_pipeline")


def gemm_strided_batched(h, transA: str, transB: str, M, N, K, alpha, A, lda, strideA, B, ldb, strideB, beta, C,
                         ldc, strideC, batch=1, stream=None) -> None:
    check(_lib.gemm_strided_batched(h.value, _c(transA), _c(transB), M, N, K, alpha,
                                    ptr(A), lda, strideA, ptr(B), ldb, strideB, beta, ptr(C), ldc, strideC, batch,
                                    stream_handle(stream)), "gemm_strided_batched")


def gemm_strided_batched_with_config(cid: int, transA: str, transB: str, M, N, K, alpha, A, lda, strideA, B, ldb,
                                     strideB, beta, C, ldc, strideC, batch=1, stream=None) -> None:
    check(_lib.gemm_strided_batched_with_config(cid, _c(transA), _c(transB), M, N, K, alpha, ptr(A), lda, strideA,
                                                ptr(B), ldb, strideB, beta, ptr(C), ldc, strideC, batch,
                                                stream_handle(stream)), "gemm_strided_batched_with_config")


def gemm_status(cid: int, transA: str, transB: str, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, batch=1,
                stream=None) -> int:
    """gemm_with_config returning the raw status instead of raising."""
    return _lib.gemm_with_config(cid, _c(transA), _c(transB), M, N, K, alpha, ptr(A), lda, ptr(B), ldb, beta,
                                 ptr(C), ldc, batch, stream_handle(stream))


def gemm_benchmark(cid: int, transA: str, transB: str, M, N, K, A, lda, B, ldb, C, ldc, batch=1, warmup=2,
                   min_reps=3, max_reps=50, min_total_ms=2.0, stream=None, with_reps=False):
    """(status, mean ms per launch[, launches timed]); a non-OK status is
    returned, not raised, so that a sweep can record configs that cannot run
    as failed."""
    out, reps = f64(), i32()
    st = _lib.gemm_benchmark(cid, _c(transA), _c(transB), M, N, K, ptr(A), lda, ptr(B), ldb, ptr(C), ldc, batch,
                             warmup, min_reps, max_reps, min_total_ms, ctypes.byref(out), ctypes.byref(reps),
                             stream_handle(stream))
    return (st, out.value, reps.value) if with_reps else (st, out.value)


def error_check(C, Cref, den, rows=0, cols=0, batch=0, ldc=0, strideC=0, pos=None, stream=None) -> float:
    """Max |C - Cref| / den on the GPU in FP64 (full mode, or sampled when ``pos`` is given)."""
    out = f64()
    n = 0 if pos is None else pos.shape[0]
    check(_lib.gemm_error_check(rows, cols, batch, ptr(C), ldc, strideC, n, ptr(pos), ptr(Cref), ptr(den),
                                ctypes.byref(out), stream_handle(stream)), "gemm_error_check")
    return out.value


def wait_selftest(limit_ns: int, stream=None) -> int:
    """Runs the bounded-wait test hook; returns 1 if the never-arriving barrier completed, else 0."""
    w = i32()
    check(_lib.kselect_wait_selftest(limit_ns, ctypes.byref(w), stream_handle(stream)), "kselect_wait_selftest")
    return w.value


def device_status(clear: bool = True) -> int:
    """The tensor-core status word (0 = no bounded wait gave up); synchronises the device."""
    v = i32()
    st = _lib.gemm_device_status(ctypes.byref(v), int(clear))
    if st not in (GEMM_OK, -5):
        raise KSelectError(st, "gemm_device_status")
    return v.value


def fill_uniform(dst, rows, cols, ld, batch, seed, lo=-1.0, hi=1.0, pad=0.0, stream=None) -> None:
    check(_lib.kselect_fill_uniform(ptr(dst), rows, cols, ld, batch, seed, lo, hi, pad, stream_handle(stream)),
          "kselect_fill_uniform")


def _arr(a, dtype, ctype):
    a = np.ascontiguousarray(a, dtype)
    return a, a.ctypes.data_as(ctypes.POINTER(ctype))


def benchmark_configs(cids, transA, transB, M, N, K, A, lda, B, ldb, C, ldc, batch=1, warmup=1, min_reps=2,
                      max_reps=50, min_total_ms=2.0, refine_ratio=2.0, stream=None, details=False):
    """Section 3.1 over a config list: (ms per launch, status) arrays, plus
    (pass-1 probe ms, launches averaged) with details=True."""
    ids, pids = _arr(cids, np.int32, i32)
    ms = np.zeros(len(ids), np.float64)
    st = np.zeros(len(ids), np.int32)
    probe = np.zeros(len(ids), np.float64)
    reps = np.zeros(len(ids), np.int32)
    check(_lib.gemm_benchmark_configs(len(ids), pids, _c(transA), _c(transB), M, N, K, ptr(A), lda, ptr(B), ldb,
                                      ptr(C), ldc, batch, warmup, min_reps, max_reps, min_total_ms, refine_ratio,
                                      ms.ctypes.data_as(ctypes.POINTER(f64)), st.ctypes.data_as(ctypes.POINTER(i32)),
                                      probe.ctypes.data_as(ctypes.POINTER(f64)),
                                      reps.ctypes.data_as(ctypes.POINTER(i32)), stream_handle(stream)),
          "gemm_benchmark_configs")
    return (ms, st, probe, reps) if details else (ms, st)


NORM_MODES = {"standard": 0, "raw_cutoff": 1, "standard_cutoff": 2, "sigmoid": 3}


def normalise(perf, out, mode="standard", stream=None) -> None:
    n_rows, n_cols = perf.shape
    check(_lib.kselect_normalise(n_rows, n_cols, ptr(perf), ptr(out), NORM_MODES[mode], stream_handle(stream)),
          "kselect_normalise")


def kmeans(X, k: int, draws: np.ndarray, centres_out, labels_out, max_iter=300, tol=1e-4, stream=None):
    """Returns (inertia, iterations); draws is (n_init, k) uint32."""
    n, d = X.shape
    dr, pdr = _arr(draws, np.uint32, ctypes.c_uint32)
    inertia, iters = f64(), i32()
    check(_lib.kselect_kmeans(n, d, k, dr.shape[0], ptr(X), pdr, max_iter, tol, ptr(centres_out), ptr(labels_out),
                              ctypes.byref(inertia), ctypes.byref(iters), stream_handle(stream)), "kselect_kmeans")
    return inertia.value, iters.value


def pca(X, r: int, V0, mean_out, V_out, Y_out=None, iters: int = 60, stream=None):
    """Returns (eigenvalues (r,), total variance); fills mean_out, V_out and optionally Y_out."""
    n, d = X.shape
    ev = np.zeros(r, np.float64)
    tot = f64()
    check(_lib.kselect_pca(n, d, ptr(X), r, iters, ptr(V0), ptr(mean_out), ptr(V_out), ptr(Y_out),
                           ev.ctypes.data_as(ctypes.POINTER(f64)), ctypes.byref(tot), stream_handle(stream)),
          "kselect_pca")
    return ev, tot.value


def pca_backproject(cent, V, mean, out, stream=None) -> None:
    k, r = cent.shape
    check(_lib.kselect_pca_backproject(k, V.shape[0], r, ptr(cent), ptr(V), ptr(mean), ptr(out), stream_handle(stream)),
          "kselect_pca_backproject")


def score(perf, deployed_cols=None, chosen=None, floor=1e-6, stream=None) -> dict:
    n_rows, n_cols = perf.shape
    dep = list(deployed_cols) if deployed_cols is not None else []
    d, pd = _arr(dep if dep else [0], np.int32, i32)
    out = (f64 * 3)()
    check(_lib.kselect_score(n_rows, n_cols, ptr(perf), len(dep), pd, ptr(chosen), floor, out,
                             stream_handle(stream)), "kselect_score")
    return {"geomean": out[0], "mean": out[1], "clamped": int(out[2])}


def im2col3x3(x, N, H, W, C, out, ld, stream=None) -> None:
    check(_lib.kselect_im2col3x3(ptr(x), N, H, W, C, ptr(out), ld, stream_handle(stream)), "kselect_im2col3x3")


def bias_act(y, rows, cols, ld, bias, relu=True, stream=None) -> None:
    check(_lib.kselect_bias_act(ptr(y), rows, cols, ld, ptr(bias), int(relu), stream_handle(stream)), "kselect_bias_act")


def maxpool2x2(x, N, H, W, C, out, stream=None) -> None:
    check(_lib.kselect_maxpool2x2(ptr(x), N, H, W, C, ptr(out), stream_handle(stream)), "kselect_maxpool2x2")


def im2col3x3_nchw(x, N, C, H, W, out, ld, stream=None) -> None:
    check(_lib.kselect_im2col3x3_nchw(ptr(x), N, C, H, W, ptr(out), ld, stream_handle(stream)),
          "kselect_im2col3x3_nchw")


def bias_act_nchw(y, N, C, HW, bias, relu=True, stream=None) -> None:
    check(_lib.kselect_bias_act_nchw(ptr(y), N, C, HW, ptr(bias), int(relu), stream_handle(stream)),
          "kselect_bias_act_nchw")


def knn(train, labels, query, k: int, out, stream=None) -> None:
    """k-nearest-neighbour labels of the query rows (device tensors)."""
    check(_lib.kselect_knn(train.shape[0], query.shape[0], train.shape[1], ptr(train), ptr(labels), ptr(query), k,
                           ptr(out), stream_handle(stream)), "kselect_knn")


def spectral_embedding(X, gamma: float, k: int, V0, U_out, iters: int = 200, stream=None) -> np.ndarray:
    """Unit-length spectral coordinates (U_out, n x k) of the rows of X; V0 (n x r) the
    starting block.  Returns the k leading eigenvalues of D^-1/2 A D^-1/2."""
    n, d = X.shape
    r = V0.shape[1]
    ev = (f64 * k)()
    check(_lib.kselect_spectral_embedding(n, d, ptr(X), gamma, k, r, iters, ptr(V0), ptr(U_out), ev,
                                          stream_handle(stream)), "kselect_spectral_embedding")
    return np.array(ev[:])


def cluster_geomean(X, labels, k: int, out, floor: float = 1e-6, stream=None) -> None:
    check(_lib.kselect_cluster_geomean(X.shape[0], X.shape[1], ptr(X), ptr(labels), k, floor, ptr(out),
                                       stream_handle(stream)), "kselect_cluster_geomean")


def tree_regress(features: np.ndarray, Y: np.ndarray, max_leaves: int) -> tuple[np.ndarray, np.ndarray]:
    """Regression-tree partition of the sizes (host): (labels, leaf-mean centres)."""
    n, d = Y.shape
    F, pf = _arr(features, np.float64, f64)
    assert F.shape == (n, TREE_FEATURES)
    Yc, py = _arr(Y, np.float32, f32)
    labels = np.zeros(n, np.int32)
    centres = np.zeros((max_leaves, d), np.float32)
    nl = i32()
    check(_lib.kselect_tree_regress(n, d, pf, py, max_leaves, labels.ctypes.data_as(ctypes.POINTER(i32)),
                                    centres.ctypes.data_as(ctypes.POINTER(f32)), ctypes.byref(nl)),
          "kselect_tree_regress")
    return labels, centres[:nl.value].copy()


def representatives(centres: np.ndarray, labels: np.ndarray, dedupe=True) -> np.ndarray:
    k, d = centres.shape
    c, pc = _arr(centres, np.float32, f32)
    lab, pl = _arr(labels, np.int32, i32)
    out = np.zeros(k, np.int32)
    cnt = i32()
    check(_lib.kselect_representatives(k, d, pc, len(lab), pl, int(dedupe), out.ctypes.data_as(ctypes.POINTER(i32)),
                                       ctypes.byref(cnt)), "kselect_representatives")
    return out[:cnt.value].copy()


def top_n(perf: np.ndarray, n: int) -> np.ndarray:
    p, pp = _arr(perf, np.float32, f32)
    out = np.zeros(n, np.int32)
    check(_lib.kselect_top_n(p.shape[0], p.shape[1], pp, n, out.ctypes.data_as(ctypes.POINTER(i32))), "kselect_top_n")
    return out


def selector_features(sizes) -> np.ndarray:
    """(n, TREE_FEATURES) feature rows of (M, N, K, batch) sizes, as the tree reads them."""
    s = np.ascontiguousarray(np.asarray(sizes, np.int64).reshape(-1, 4))
    out = np.zeros((s.shape[0], TREE_FEATURES), np.float64)
    check(_lib.kselect_selector_features(s.shape[0], s.ctypes.data_as(ctypes.POINTER(i64)),
                                         out.ctypes.data_as(ctypes.POINTER(f64))), "kselect_selector_features")
    return out


def best_labels(perf: np.ndarray, cols) -> np.ndarray:
    """Per row of perf, the index into cols of its best column (lowest on ties)."""
    P, pP = _arr(perf, np.float64, f64)
    c, pc = _arr(cols, np.int32, i32)
    out = np.zeros(P.shape[0], np.int32)
    check(_lib.kselect_best_labels(P.shape[0], P.shape[1], pP, len(c), pc, out.ctypes.data_as(ctypes.POINTER(i32))),
          "kselect_best_labels")
    return out


def tree_train(features: np.ndarray, labels: np.ndarray, n_classes: int, max_depth=None, min_leaf=1,
               max_nodes=8192) -> list[dict]:
    F, pF = _arr(features, np.float64, f64)
    assert F.ndim == 2 and F.shape[1] == TREE_FEATURES
    y, py = _arr(labels, np.int32, i32)
    nodes = (TreeNode * max_nodes)()
    cnt = i32()
    check(_lib.kselect_tree_train(F.shape[0], pF, py, n_classes, -1 if max_depth is None else max_depth, min_leaf,
                                  nodes, max_nodes, ctypes.byref(cnt)), "kselect_tree_train")
    return [{"feature": nodes[j].feature, "threshold": nodes[j].threshold, "left": nodes[j].left,
             "right": nodes[j].right, "label": nodes[j].label} for j in range(cnt.value)]


def tree_train_rf(features: np.ndarray, labels: np.ndarray, n_classes: int, max_features: int, draws: np.ndarray,
                  max_depth=None, min_leaf=1, max_nodes=8192) -> list[dict]:
    """One random-forest tree; draws: (>= max_nodes, TREE_FEATURES) uint32, row j for node j."""
    F, pF = _arr(features, np.float64, f64)
    assert F.ndim == 2 and F.shape[1] == TREE_FEATURES
    y, py = _arr(labels, np.int32, i32)
    d = np.ascontiguousarray(draws, np.uint32)
    assert d.ndim == 2 and d.shape[1] == TREE_FEATURES and d.shape[0] >= max_nodes
    nodes = (TreeNode * max_nodes)()
    cnt = i32()
    check(_lib.kselect_tree_train_rf(F.shape[0], pF, py, n_classes, -1 if max_depth is None else max_depth, min_leaf,
                                     max_features, d.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), nodes,
                                     max_nodes, ctypes.byref(cnt)), "kselect_tree_train_rf")
    return [{"feature": nodes[j].feature, "threshold": nodes[j].threshold, "left": nodes[j].left,
             "right": nodes[j].right, "label": nodes[j].label} for j in range(cnt.value)]


# ---------------------------------------------------------------- grouped GEMM
def grouped_select(handle: Handle, problems) -> int:
    """Config id the handle's group classifier picks for these problems (dicts as for GroupedPlan)."""
    arr = _problems(problems)
    r = _lib.gemm_grouped_select(handle.value, len(problems), arr)
    if r < 0:
        raise KSelectError(r, "gemm_grouped_select")
    return r


def _problems(problems):
    """problems: iterable of dicts with M, N, K, transA, transB, alpha, beta, A, lda, B, ldb, C, ldc."""
    arr = (Problem * len(problems))()
    for i, q in enumerate(problems):
        arr[i] = Problem(q["M"], q["N"], q["K"], _c(q.get("transA", "N")), _c(q.get("transB", "T")),
                         q.get("alpha", 1.0), q.get("beta", 0.0), ptr(q["A"]), q["lda"], ptr(q["B"]), q["ldb"],
                         ptr(q["C"]), q["ldc"])
    return arr


class GroupedPlan:
    """A validated group with device-resident descriptors; run() only launches (graph-capturable)."""

    def __init__(self, cid: int, problems, stream=None):
        self._arr = _problems(problems)
        h = vp()
        check(_lib.gemm_grouped_plan_create(cid, len(problems), self._arr, stream_handle(stream), ctypes.byref(h)),
              "gemm_grouped_plan_create")
        self.value = h.value

    def run(self, stream=None) -> None:
        check(_lib.gemm_grouped_run(self.value, stream_handle(stream)), "gemm_grouped_run")

    def close(self):
        if self.value:
            _lib.gemm_grouped_plan_destroy(self.value)
            self.value = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm_grouped_with_config(cid: int, problems, stream=None) -> None:
    """One-shot grouped launch with an explicit config (plans, runs, synchronises)."""
    arr = _problems(problems)
    check(_lib.gemm_grouped_with_config(cid, len(problems), arr, stream_handle(stream)), "gemm_grouped_with_config")


def gemm_grouped(handle: Handle, problems, precision: int, stream=None) -> None:
    """The group's tile config picked by the handle's group selector, launched
    asynchronously on `stream` (capturable once the handle's workspace fits)."""
    arr = _problems(problems)
    check(_lib.gemm_grouped(handle.value, len(problems), arr, precision, stream_handle(stream)), "gemm_grouped")


def gemm_grouped_reserve(handle: Handle, problems, precision: int) -> None:
    arr = _problems(problems)
    check(_lib.gemm_grouped_reserve(handle.value, len(problems), arr, precision), "gemm_grouped_reserve")


# ---------------------------------------------------------------- learned selector
def mlp_features(shapes, X, stream=None) -> None:
    check(_lib.mlp_features(shapes.shape[0], ptr(shapes), ptr(X), stream_handle(stream)), "mlp_features")


def mlp_targets(perf, T, mask, stream=None) -> None:
    """Targets and mask (n x d, device) from a device throughput table."""
    check(_lib.mlp_targets(perf.shape[0], perf.shape[1], ptr(perf), ptr(T), ptr(mask), stream_handle(stream)),
          "mlp_targets")


def mlp_forward(params, X, Y, stream=None) -> None:
    check(_lib.mlp_forward(X.shape[0], ptr(params), ptr(X), ptr(Y), stream_handle(stream)), "mlp_forward")


def _check_mlp_loss_args(where, params, X, T, mask, grad, loss) -> int:
    """The C entry points take raw pointers and n: a tensor of the wrong shape,
    type, layout or device would be read out of bounds on the GPU, so every
    argument is checked here first (GEMM_ERR_INVALID_ARG).  Returns n."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else None

    def ok(t, shape):
        return (isinstance(t, torch.Tensor) and t.dtype == torch.float32 and t.is_contiguous()
                and t.device == dev and tuple(t.shape) == shape)

    n = X.shape[0] if isinstance(X, torch.Tensor) and X.dim() == 2 else -1
    good = (n >= 1 and ok(params, (MLP_PARAMS,)) and ok(X, (n, 7)) and ok(T, (n, 8))
            and (mask is None or ok(mask, (n, 8))) and ok(grad, (MLP_PARAMS,)) and ok(loss, (1,)))
    if not good:
        raise KSelectError(-1, f"{where}: params and grad must be ({MLP_PARAMS},), X (n, 7), T and mask (n, 8), "
                               f"loss (1,): float32, contiguous, on the current CUDA device")
    return n


def mlp_loss_grad(params, X, T, mask, grad, loss, stream=None) -> None:
    n = _check_mlp_loss_args("mlp_loss_grad", params, X, T, mask, grad, loss)
    check(_lib.mlp_loss_grad(n, ptr(params), ptr(X), ptr(T), ptr(mask), ptr(grad), ptr(loss),
                             stream_handle(stream)), "mlp_loss_grad")


def mlp_loss_grad_noalloc(params, X, T, mask, grad, loss, stream=None) -> None:
    """mlp_loss_grad without device allocation (fixed in-library scratch, n <= 8192)."""
    n = _check_mlp_loss_args("mlp_loss_grad_noalloc", params, X, T, mask, grad, loss)
    check(_lib.mlp_loss_grad_noalloc(n, ptr(params), ptr(X), ptr(T), ptr(mask), ptr(grad), ptr(loss),
                                     stream_handle(stream)), "mlp_loss_grad_noalloc")


def mlp_adam_step(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    check(_lib.mlp_adam_step(ptr(params), ptr(grad), ptr(m), ptr(v), t, lr, beta1, beta2, eps, stream_handle(stream)),
          "mlp_adam_step")


def mlp_train(params, X, T, mask, m, v, t0, steps, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, loss_hist=None,
              stream=None) -> None:
    check(_lib.mlp_train(X.shape[0], ptr(params), ptr(X), ptr(T), ptr(mask), ptr(m), ptr(v), t0, steps, lr, beta1,
                         beta2, eps, ptr(loss_hist), stream_handle(stream)), "mlp_train")


def select_kernels_batched(handle: Handle, shapes, ids_out, pred=None, stream=None) -> None:
    """shapes: (n, 7) int64 device tensor (M, N, K, batch, transA, transB, dtype)."""
    check(_lib.select_kernels_batched(handle.value, shapes.shape[0], ptr(shapes), ptr(ids_out), ptr(pred),
                                      stream_handle(stream)), "select_kernels_batched")


def exported_symbols() -> list[str]:
    """Names of the C-ABI entry points this binding expects."""
    return ["gemm_status_string", "gemm_last_cuda_error", "kselect_debug_bounds_errors",
            "kselect_debug_shrink_extents", "gemm_config_count", "gemm_config_id",
            "gemm_config_params", "gemm_split_choose", "gemm_split_factor", "gemm_library_create", "gemm_library_destroy", "select_kernel", "gemm",
            "gemm_with_config", "gemm_host_pipeline", "gemm_strided_batched", "gemm_strided_batched_with_config", "gemm_host", "gemm_benchmark", "gemm_error_check", "kselect_fill_uniform",
            "gemm_benchmark_configs", "gemm_device_status", "kselect_wait_selftest", "kselect_normalise", "kselect_kmeans", "kselect_score",
            "kselect_im2col3x3", "kselect_bias_act", "kselect_maxpool2x2", "kselect_im2col3x3_nchw", "kselect_bias_act_nchw", "kselect_knn", "kselect_representatives", "kselect_top_n", "kselect_tree_regress", "kselect_tree_train", "kselect_tree_train_rf", "kselect_spectral_embedding", "kselect_cluster_geomean", "kselect_pca", "kselect_pca_backproject", "mlp_features", "mlp_forward", "mlp_loss_grad",
            "mlp_adam_step", "mlp_loss_grad_noalloc", "mlp_train", "select_kernels_batched", "gemm_grouped_plan_create", "gemm_grouped_run",
            "gemm_grouped_plan_destroy", "gemm_grouped", "gemm_grouped_with_config", "gemm_grouped_reserve",
            "gemm_grouped_select", "kselect_selector_features", "kselect_best_labels", "mlp_targets"]
