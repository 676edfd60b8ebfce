"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/*.h, decodes its config space, validates deployments and
arguments, and walks the decision tree exactly like the oracle's tree."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from oracle import select as osel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ks():
    from paper_2008_13145_gb300 import build
    build.build_library()
    from paper_2008_13145_gb300 import kselect
    return kselect


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(ks):
    lib = ctypes.CDLL(ks.LIB)
    names = declared_functions()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(ks.exported_symbols()) <= names


def test_simt_config_space(ks):
    assert ks.config_count(ks.PREC_F32) == 576 + 192
    ids = ks.config_ids(ks.PREC_F32)
    assert ids[:576] == list(range(576))
    seen, split = set(), []
    for cid in ids:
        fam, tm, tn, wx, wy, bk, staged, splitk = ks.config_params(cid)
        assert fam == 0 and tm in (1, 2, 4, 8) and tn in (1, 2, 4, 8) and bk in (8, 16, 32) and staged in (0, 1)
        assert (wx, wy) in [(8, 8), (16, 16), (32, 8), (8, 32), (16, 8), (8, 16)]
        assert splitk == (cid >= 2000)
        if splitk:
            split.append((tm, tn, wx, wy, bk, staged))
            assert ks.config_params(cid - 2000)[:7] == [fam, tm, tn, wx, wy, bk, staged]
        else:
            seen.add((tm, tn, wx, wy, bk, staged))
    assert len(seen) == 576
    # the split-K kind: every staged config with BK 16 or 32, once, ids ascending
    assert sorted(set(split)) == sorted(c for c in seen if c[5] == 1 and c[4] in (16, 32))
    assert len(split) == 192 and ids[576:] == sorted(ids[576:])
    for bad in (2000, 2001, 2002, 2000 + 576, 576, 1999):  # unstaged or BK 8 bases, out of range
        with pytest.raises(ks.KSelectError):
            ks.config_params(bad)


def test_split_choice_invariants(ks):
    """The split-K kind's host cost model on GB300-like figures (152 SMs)."""
    # a full-GPU product never splits
    assert ks.split_choose(4096, 4096, 4096, 1, 64, 64, 32, 4, 152) == (1, 4096)
    # K too short for a first split of 4 K-steps and a second one
    assert ks.split_choose(64, 64, 192, 1, 64, 64, 32, 4, 152) == (1, 192)
    assert ks.split_choose(64, 64, 193, 1, 64, 64, 32, 4, 152) == (2, 128)
    for (M, N, K, b, BM, BN, BK) in [(64, 64, 8192, 1, 64, 64, 32), (37, 45, 2000, 2, 32, 32, 16),
                                    (300, 200, 3945, 8, 64, 32, 32), (323, 312, 3945, 8, 64, 64, 32),
                                    (100, 100, 100000, 1, 128, 64, 16)]:
        S, kc = ks.split_choose(M, N, K, b, BM, BN, BK, 4, 152)
        assert 2 <= S <= 16, (M, N, K, S)
        nk = -(-K // BK)
        assert kc % BK == 0 and kc // BK >= 4
        assert S == -(-nk // (kc // BK))  # every split non-empty
        assert (S - 1) * kc < K <= S * kc
        assert b * S <= 65535 and S * b * M * (-(-N // 4) * 4) * 4 <= 256 << 20
    # batch x S stays within the grid's z limit
    S, _ = ks.split_choose(8, 8, 4096, 65535, 64, 64, 32, 4, 152)
    assert S == 1
    S, _ = ks.split_choose(8, 8, 4096, 60000, 64, 64, 32, 4, 152)
    assert S == 1
    # the partial-tile workspace stays within 256 MB
    S, _ = ks.split_choose(4000, 4000, 1 << 20, 1, 4096, 4096, 32, 1, 1)
    assert S == 1 or S * 4000 * 4000 * 4 <= 256 << 20
    # no occupancy information, or degenerate sizes: no split
    assert ks.split_choose(64, 64, 8192, 1, 64, 64, 32, 0, 152)[0] == 1
    assert ks.split_choose(0, 64, 8192, 1, 64, 64, 32, 4, 152)[0] == 1
    assert ks.split_choose(64, 64, 0, 1, 64, 64, 32, 4, 152) == (1, 0)
    for bad in [(-1, 64, 64, 1, 64, 64, 32, 4, 152), (64, 64, 64, 1, 0, 64, 32, 4, 152),
                (64, 64, 1 << 31, 1, 64, 64, 32, 4, 152)]:
        with pytest.raises(ks.KSelectError):
            ks.split_choose(*bad)


def test_tc_config_space(ks):
    for prec in (ks.PREC_TF32, ks.PREC_BF16, ks.PREC_F32X3):
        ids = ks.config_ids(prec)
        assert len(ids) == 9 and len(set(ids)) == 9
        assert ids == [1000 + 100 * (prec - 1) + 2 * i for i in range(9)]
        combos = {tuple(ks.config_params(c)[1:6]) for c in ids}
        assert len(combos) == 9
        for c in ids:
            p = ks.config_params(c)
            assert p[0] == prec and p[1] == 128 and p[2] in (64, 128, 256) and p[4] in (2, 3, 4)
            assert p[3] == (32 if prec == ks.PREC_TF32 else 64) and p[5] == 0
            # the odd slot after each id is reserved: no kernel
            with pytest.raises(ks.KSelectError) as e:
                ks.config_params(c + 1)
            assert e.value.status == -6
    with pytest.raises(ks.KSelectError):
        ks.config_params(999)


def nodes_to_dicts(nodes):
    return [{"feature": n["feature"], "threshold": n["threshold"], "left": n["left"], "right": n["right"],
             "label": n["label"]} for n in nodes]


def test_select_kernel_walks_the_tree_like_the_oracle(ks):
    rng = np.random.default_rng(0)
    S = np.exp(rng.uniform(np.log(16), np.log(4096), (300, 4))).round()
    S[:, 3] = rng.choice([1, 2, 4, 8, 16], 300)
    F = osel.selector_features(S)
    # labels that depend on the output count, so the trees split on it
    y = (rng.integers(0, 3, 300) + (F[:, 4] > np.median(F[:, 4])) * 2).astype(np.int64)
    for depth, leaf in osel.TREES.values():
        nodes = osel.tree_train(F, y, 5, depth, leaf)
        assert any(n["feature"] == 4 for n in nodes)
        ids = [3, 77, 150, 301, 575]
        h = ks.Handle({"precision": ks.PREC_F32, "config_ids": ids, "nodes": nodes_to_dicts(nodes)})
        St = np.exp(rng.uniform(np.log(16), np.log(4096), (500, 4))).round()
        St[:, 3] = rng.choice([1, 2, 4, 8, 16], 500)
        want = osel.tree_predict(nodes, osel.selector_features(St))
        got = [ks.select_kernel(h, *map(int, s)) for s in St]
        assert got == [ids[w] for w in want]


def test_deployment_validation(ks):
    ok = {"precision": 0, "config_ids": [1, 2], "nodes": [
        {"feature": 0, "threshold": 100.5, "left": 1, "right": 2, "label": 0},
        {"feature": -1, "threshold": 0, "left": -1, "right": -1, "label": 0},
        {"feature": -1, "threshold": 0, "left": -1, "right": -1, "label": 1}]}
    h = ks.Handle(ok)
    assert ks.select_kernel(h, 100, 5, 5, 1) == 1 and ks.select_kernel(h, 101, 5, 5, 1) == 2
    bad_label = {**ok, "nodes": [dict(ok["nodes"][0]), ok["nodes"][1], {**ok["nodes"][2], "label": 2}]}
    cyc = {**ok, "nodes": [{**ok["nodes"][0], "left": 0}, ok["nodes"][1], ok["nodes"][2]]}
    oob = {**ok, "nodes": [{**ok["nodes"][0], "right": 7}, ok["nodes"][1], ok["nodes"][2]]}
    for bad, code in ((bad_label, -1), (cyc, -1), (oob, -1)):
        with pytest.raises(ks.KSelectError) as e:
            ks.Handle(bad)
        assert e.value.status == code
    with pytest.raises(ks.KSelectError) as e:
        ks.Handle({"precision": 0, "config_ids": [1, 1002], "nodes": []})
    assert e.value.status == -6
    with pytest.raises(ks.KSelectError) as e:
        ks.Handle({"precision": 0, "config_ids": [], "nodes": []})
    assert e.value.status == -6
    # an FP32-input handle may mix the SIMT and split-BF16 x3 families, not TF32 or BF16
    assert ks.Handle({"precision": 0, "config_ids": [5, 1202], "nodes": []}).ids == [5, 1202]
    with pytest.raises(ks.KSelectError):
        ks.Handle({"precision": 3, "config_ids": [1102], "nodes": []})
    # benchmarked sizes take their measured best kernel, the rest the tree's choice
    hk = ks.Handle({**ok, "known": [[100, 5, 5, 1, 77], [7, 8, 9, 2, 1202], [100, 5, 5, 1, 3]]})
    assert ks.select_kernel(hk, 100, 5, 5, 1) == 77 and ks.select_kernel(hk, 7, 8, 9, 2) == 1202
    assert ks.select_kernel(hk, 100, 5, 5, 2) == 1 and ks.select_kernel(hk, 101, 5, 5, 1) == 2
    with pytest.raises(ks.KSelectError):
        ks.Handle({**ok, "known": [[1, 1, 1, 1, 1002]]})
    h0 = ks.Handle({"precision": 0, "config_ids": [42], "nodes": []})
    assert ks.select_kernel(h0, 1, 1, 1, 1) == 42


def test_argument_validation_needs_no_device(ks):
    fake = 1 << 20  # never dereferenced: validation fails before any launch
    args = dict(M=4, N=4, K=4, alpha=1.0, A=fake, lda=4, B=fake, ldb=4, beta=0.0, C=fake, ldc=4, batch=1)

    def st(**kw):
        a = {**args, **kw}
        return ks.gemm_status(0, kw.get("ta", "N"), kw.get("tb", "N"), a["M"], a["N"], a["K"], a["alpha"], a["A"],
                              a["lda"], a["B"], a["ldb"], a["beta"], a["C"], a["ldc"], a["batch"], stream=0)

    assert st(ta="X") == -1
    assert st(M=-1) == -1
    assert st(lda=3) == -1
    assert st(ta="T", lda=3) == -1
    assert st(ldc=3) == -1
    assert st(A=0) == -1
    assert st(C=0) == -1
    assert st(batch=70000) == -2
    assert st(M=1 << 31) == -2
    assert st(M=0, A=0, B=0, C=0) == 0  # empty: no-op
    assert st(batch=0) == 0
    assert ks.gemm_status(5000, "N", "N", 4, 4, 4, 1.0, fake, 4, fake, 4, 0.0, fake, 4, 1, stream=0) == -6

    def strided(sa, sb, sc, batch=3, cid=0):
        return ks._lib.gemm_strided_batched_with_config(cid, b"N", b"N", 4, 4, 4, 1.0, fake, 4, sa, fake, 4, sb, 0.0,
                                                       fake, 4, sc, batch, None)
    assert strided(-1, 16, 16) == -1
    assert strided(16, -4, 16) == -1
    assert strided(16, 16, 15) == -1  # batch entries would overlap in C
    assert strided(0, 0, 0, batch=1, cid=5000) == -6
    assert strided(0, 16, 16, batch=0) == 0  # empty: no-op

    # the host pipeline validates every problem before it enqueues anything
    h = ks.Handle({"precision": 0, "config_ids": [369], "nodes": []})
    good = dict(transA="N", transB="N", M=4, N=4, K=4, lda=4, ldb=4, ldc=4, A_host=fake, B_host=fake, C_host=fake,
                A_dev=fake, B_dev=fake, C_dev=fake)
    for bad in (dict(lda=3), dict(transA="Q"), dict(C_host=0), dict(M=-1), dict(C_dev=0)):
        arr = ks.host_problems([good, {**good, **bad}])
        assert ks._lib.gemm_host_pipeline(h.value, 2, arr, None) == -1, bad
    assert ks._lib.gemm_host_pipeline(h.value, -1, None, None) == -1
    assert ks._lib.gemm_host_pipeline(None, 0, None, None) == -1


def test_mlp_wrappers_reject_bad_arguments_before_any_launch(ks):
    """The loss/gradient wrappers check shapes, type, layout and device before
    passing raw pointers on (GEMM_ERR_INVALID_ARG, nothing launched).  Host
    tensors are never on the current CUDA device, so even the well-shaped set
    is refused here."""
    import torch
    good = dict(params=torch.zeros(5192), X=torch.zeros(4, 7), T=torch.zeros(4, 8), mask=None,
                grad=torch.zeros(5192), loss=torch.zeros(1))
    bad = [dict(good, params=torch.zeros(5191)), dict(good, X=torch.zeros(4, 6)), dict(good, T=torch.zeros(5, 8)),
           dict(good, mask=torch.zeros(4, 7)), dict(good, X=torch.zeros(4, 7, dtype=torch.float64)),
           dict(good, X=torch.zeros(7, 4).t()), dict(good, loss=torch.zeros(2)), dict(good, X=torch.zeros(0, 7))]
    for fn in (ks.mlp_loss_grad, ks.mlp_loss_grad_noalloc):
        for args in bad + [good]:
            with pytest.raises(ks.KSelectError) as e:
                fn(**args)
            assert e.value.status == -1
