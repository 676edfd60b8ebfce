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
    assert ks.config_count(ks.PREC_F32) == 576
    seen = set()
    for cid in ks.config_ids(ks.PREC_F32):
        fam, tm, tn, wx, wy, bk, staged, _ = ks.config_params(cid)
        assert fam == 0 and tm in (1, 2, 4, 8) and tn in (1, 2, 4, 8) and bk in (8, 16, 32) and staged in (0, 1)
        assert (wx, wy) in [(8, 8), (16, 16), (32, 8), (8, 32), (16, 8), (8, 16)]
        seen.add((tm, tn, wx, wy, bk, staged))
    assert len(seen) == 576


def test_tc_config_space(ks):
    for prec in (ks.PREC_TF32, ks.PREC_BF16, ks.PREC_F32X3):
        ids = ks.config_ids(prec)
        assert len(ids) == 18 and len(set(ids)) == 18
        combos = {tuple(ks.config_params(c)[1:6]) for c in ids}
        assert len(combos) == 18
        for c in ids:
            p = ks.config_params(c)
            assert p[0] == prec and p[1] == 128 and p[2] in (64, 128, 256) and p[4] in (2, 3, 4)
            assert p[3] == (32 if prec == ks.PREC_TF32 else 64) and p[5] in (0, 1)
    with pytest.raises(ks.KSelectError):
        ks.config_params(999)


def nodes_to_dicts(nodes):
    return [{"feature": n["feature"], "threshold": n["threshold"], "left": n["left"], "right": n["right"],
             "label": n["label"]} for n in nodes]


def test_select_kernel_walks_the_tree_like_the_oracle(ks):
    rng = np.random.default_rng(0)
    F = np.exp(rng.uniform(np.log(16), np.log(4096), (300, 4))).round()
    F[:, 3] = rng.choice([1, 2, 4, 8, 16], 300)
    y = rng.integers(0, 5, 300)
    for depth, leaf in osel.TREES.values():
        nodes = osel.tree_train(F, y, 5, depth, leaf)
        ids = [3, 77, 150, 301, 575]
        h = ks.Handle({"precision": ks.PREC_F32, "config_ids": ids, "nodes": nodes_to_dicts(nodes)})
        Ft = np.exp(rng.uniform(np.log(16), np.log(4096), (500, 4))).round()
        Ft[:, 3] = rng.choice([1, 2, 4, 8, 16], 500)
        want = osel.tree_predict(nodes, Ft)
        got = [ks.select_kernel(h, *map(int, f)) for f in Ft]
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
        ks.Handle({"precision": 0, "config_ids": [1, 1001], "nodes": []})
    assert e.value.status == -6
    with pytest.raises(ks.KSelectError) as e:
        ks.Handle({"precision": 0, "config_ids": [], "nodes": []})
    assert e.value.status == -6
    # an FP32-input handle may mix the SIMT and split-BF16 x3 families, not TF32 or BF16
    assert ks.Handle({"precision": 0, "config_ids": [5, 1201], "nodes": []}).ids == [5, 1201]
    with pytest.raises(ks.KSelectError):
        ks.Handle({"precision": 3, "config_ids": [1101], "nodes": []})
    # benchmarked sizes take their measured best kernel, the rest the tree's choice
    hk = ks.Handle({**ok, "known": [[100, 5, 5, 1, 77], [7, 8, 9, 2, 1201], [100, 5, 5, 1, 3]]})
    assert ks.select_kernel(hk, 100, 5, 5, 1) == 77 and ks.select_kernel(hk, 7, 8, 9, 2) == 1201
    assert ks.select_kernel(hk, 100, 5, 5, 2) == 1 and ks.select_kernel(hk, 101, 5, 5, 1) == 2
    with pytest.raises(ks.KSelectError):
        ks.Handle({**ok, "known": [[1, 1, 1, 1, 1001]]})
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
