"""Index files on the GPU: an index saved and loaded back into a fresh index holds the same stores,
graph and entry point byte for byte and answers every query identically (inner product and
Euclidean indices, LVQ-8 and FP16 secondaries, the float32 baseline); a damaged file leaves the
target index untouched."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import gpu_index, small_problem, t

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


@pytest.fixture(scope="module")
def pb():
    return small_problem(oracle, n=2000, D=48, d=16, m=200, seed=21)


def _same_index(a, b):
    ia, ib = a.info(), b.info()
    for k in ("n", "D", "d", "primary_bits", "secondary_bits", "primary_stride", "secondary_stride", "R", "entry",
              "mu2"):
        assert ia[k] == ib[k], k
    assert torch.equal(a.primary_records(), b.primary_records())
    if ia["secondary_bits"]:
        assert torch.equal(a.secondary_records(), b.secondary_records())
    if ia["R"]:
        ga, ea = a.get_graph()
        gb, eb = b.get_graph()
        assert ea == eb and torch.equal(ga, gb)


def _same_answers(a, b, Q, P, **kw):
    ia, sa = a.search(Q, P, **kw)
    ib, sb = b.search(Q, P, **kw)
    assert torch.equal(ia, ib) and torch.equal(sa, sb)


def test_round_trip_lvq(lv, pb, tmp_path):
    a = gpu_index(lv, pb)
    path = str(tmp_path / "a.lvi")
    a.save(path)
    info = lv.leanvec_index_file_check(path)
    assert info["n"] == 2000 and info["R"] == pb["graph"].shape[1] and info["entry"] == pb["entry"]
    b = lv.Index(0).load(path)
    _same_index(a, b)
    _same_answers(a, b, t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48, width=2)


def test_round_trip_l2_fp16_and_float32(lv, pb, tmp_path):
    X, P = t(pb["X"]), t(pb["P"])
    a = lv.Index(0, metric=lv.METRIC_L2).encode(X, P, 8, 16)
    a.build_graph(R=16, L_build=32, alpha=1.2, batch=512)
    path = str(tmp_path / "l2.lvi")
    a.save(path)
    b = lv.Index(0).load(path)  # the metric comes from the file
    _same_index(a, b)
    _same_answers(a, b, t(pb["Q"]), P, k=10, L=40, rerank=40)
    f = lv.Index(0).encode_fp32(X)
    g, e = a.get_graph()
    f.set_graph(g, e)
    path = str(tmp_path / "f32.lvi")
    f.save(path)
    h = lv.Index(0).load(path)
    _same_index(f, h)
    _same_answers(f, h, t(pb["Q"]), None, k=10, L=40)


def test_damaged_file_leaves_the_index_unchanged(lv, pb, tmp_path):
    a = gpu_index(lv, pb)
    path = tmp_path / "a.lvi"
    a.save(str(path))
    raw = bytearray(path.read_bytes())
    raw[200] ^= 1
    bad = tmp_path / "bad.lvi"
    bad.write_bytes(bytes(raw))
    b = gpu_index(lv, pb)
    with pytest.raises(lv.LeanVecError) as e:
        b.load(str(bad))
    assert e.value.code == -7
    _same_index(a, b)
    with pytest.raises(lv.LeanVecError):
        lv.Index(0).save(str(tmp_path / "empty.lvi"))  # an index without a store
