"""Two queries per warp (beam_half_kernel): the same search as one query per warp.

The half-warp kernel runs the same rounds on the same beam with the same scorer arithmetic (the
per-query constants summed in the same order), so ids, scores and expansion counts are equal bit
for bit to those of one query per warp -- for LVQ-8 and LVQ-4 primaries, both metrics, widths 1
and 2, a tiny visited cache (many forgotten ids), ragged candidate steps (width * R not a multiple
of 64), per-query descriptors and sub-batches.  Only the re-score counts may differ (the two
caches forget different ids).  The 16-bit tags of its visited cache are exact up to
n = 65535 * slots / 4; the largest such n is searched, one more id is refused."""
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
    return small_problem(oracle, n=3000, D=64, d=16, m=600)


def _same(lv, idx, Q, P, **kw):
    a = idx.search(Q, P, stats=True, queries_per_warp=1, **kw)
    b = idx.search(Q, P, stats=True, queries_per_warp=2, **kw)
    idx.sync_status()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert torch.equal(a[2][:, 0], b[2][:, 0])
    return b


def _qp(pb):
    return pb["Q"].astype(np.float64) @ pb["P"].T.astype(np.float64)


@pytest.mark.parametrize("W", [1, 2])
@pytest.mark.parametrize("hs", [0, 64, 128])
@pytest.mark.parametrize("L,r", [(16, 16), (48, 48), (100, 0)])
def test_half_warp_equals_one_query_per_warp(lv, pb, W, hs, L, r):
    idx = gpu_index(lv, pb)
    if hs and hs < 2 * ((L + 31) // 32 * 32):
        hs = 0  # raised to 2 x Lcap anyway
    ids, sc, st = _same(lv, idx, t(pb["Q"]), t(pb["P"]), k=10, L=L, rerank=r, width=W, hash_slots=hs)
    ref = oracle.search(pb["graph"], pb["entry"], _qp(pb), k=10, L=L, rerank=r, prim=pb["prim"], sec=pb["sec"],
                        qs=pb["Q"].astype(np.float64), width=W)
    ids = ids.cpu().numpy()
    assert (ids == ref["ids"]).mean() >= 0.99
    same = np.all(ids == ref["ids"], axis=1)
    assert np.all(st[:, 1].cpu().numpy()[same] >= ref["scored"][same])


def test_half_warp_descriptors_and_budget(lv, pb):
    idx = gpu_index(lv, pb)
    m = pb["Q"].shape[0]
    rng = np.random.default_rng(21)
    k = rng.choice([1, 5, 10], m)
    L = np.maximum(rng.integers(10, 120, m), k)
    r = np.minimum(L, rng.integers(0, 80, m))
    desc = t(np.stack([k, L, r, rng.integers(0, 60, m)], 1).astype(np.int32))
    for W in (1, 2):
        _same(lv, idx, t(pb["Q"]), t(pb["P"]), k=10, L=128, rerank=128, desc=desc, width=W)


@pytest.mark.parametrize("R", [24, 48, 64])
def test_half_warp_ragged_steps(lv, R):
    """width * R = 48, 96, 128: the visited test's steps of 64 ids cut through a parent's row (or
    hold both parents' ids), so two lanes of one step can meet the same id."""
    sub = small_problem(oracle, n=2500, D=48, d=24, m=300, seed=23, R=R, Lb=64)
    idx = gpu_index(lv, sub)
    for hs in (0, 64):
        _same(lv, idx, t(sub["Q"]), t(sub["P"]), k=10, L=32, rerank=32, width=2, hash_slots=hs)


def test_half_warp_lvq4_and_l2(lv):
    sub = small_problem(oracle, n=2000, D=64, d=40, m=200, seed=24, bits=4)
    idx = gpu_index(lv, sub)
    for W in (1, 2):
        _same(lv, idx, t(sub["Q"]), t(sub["P"]), k=10, L=40, rerank=40, width=W)
    # L2 (the norm chunk read after the constants chunk), LVQ-8 and LVQ-4 primaries
    for bits in (8, 4):
        idx2 = lv.Index(0, metric=lv.METRIC_L2)
        idx2.encode(t(sub["X"]), t(sub["P"]), bits, 8)
        idx2.set_graph(t(sub["graph"]), -1)
        for W in (1, 2):
            _same(lv, idx2, t(sub["Q"]), t(sub["P"]), k=10, L=40, rerank=40, width=W)


def test_half_warp_wide_primary(lv):
    """d = 240 (4 chunks per lane of the scorer, the largest LVQ-8 primary)."""
    sub = small_problem(oracle, n=1500, D=256, d=240, m=100, seed=25)
    idx = gpu_index(lv, sub)
    _same(lv, idx, t(sub["Q"]), t(sub["P"]), k=10, L=32, rerank=32, width=2)


def test_half_warp_sub_batches(lv, pb):
    """12000 queries: more than one wave of the 40 query slots per SM, not a multiple of it, so two
    sub-batches on two streams; equal to batches of 100."""
    Q = np.concatenate([pb["Q"]] * 20)
    idx = gpu_index(lv, pb)
    Qd, P = t(Q), t(pb["P"])
    ids, sc, st = idx.search(Qd, P, k=10, L=48, rerank=48, width=2, stats=True, queries_per_warp=2)
    assert idx.info()["last_search_kernels"] == 1 + 2 * 2
    parts = [idx.search(Qd[s:s + 100].contiguous(), P, k=10, L=48, rerank=48, width=2, queries_per_warp=2)
             for s in range(0, Q.shape[0], 100)]
    assert torch.equal(ids, torch.cat([p[0] for p in parts])) and torch.equal(sc, torch.cat([p[1] for p in parts]))
    one = idx.search(Qd, P, k=10, L=48, rerank=48, width=2, queries_per_warp=1)
    assert torch.equal(ids, one[0]) and torch.equal(sc, one[1])


def test_half_warp_tag_limit(lv):
    """With 64 visited-cache slots (16 buckets) a tag is x >> 4: n = 65535 * 16 is the largest store
    whose tags all stay below the empty mark 0xFFFF.  Random graph, queries near the top ids: the
    two kernels agree; one more record and two queries per warp are refused."""
    n, D, d, R = 65535 * 16, 32, 16, 16
    rng = np.random.default_rng(26)
    X = rng.standard_normal((n + 1, D), dtype=np.float32)
    P = np.linalg.qr(rng.standard_normal((D, D)))[0][:d].astype(np.float32)
    Q = X[n - 200:n] + 0.05 * rng.standard_normal((200, D), dtype=np.float32)
    g = oracle.random_graph(n, R, 26)
    idx = lv.Index(0).encode(t(X[:n]), t(P), 8, 8)
    idx.set_graph(t(g), n - 1)
    ids, _, _ = _same(lv, idx, t(Q), t(P), k=10, L=16, rerank=16, width=2, hash_slots=64)
    assert (ids.cpu().numpy() >= n - 65536).any()  # the walk reaches the largest tags
    g1 = oracle.random_graph(n + 1, R, 27)
    idx1 = lv.Index(0).encode(t(X), t(P), 8, 8)
    idx1.set_graph(t(g1), n)
    with pytest.raises(lv.LeanVecError):
        idx1.search(t(Q), t(P), k=10, L=16, rerank=16, width=2, hash_slots=64, queries_per_warp=2)
    a = idx1.search(t(Q), t(P), k=10, L=16, rerank=16, width=2, hash_slots=64)
    b = idx1.search(t(Q), t(P), k=10, L=16, rerank=16, width=2, hash_slots=64, queries_per_warp=1)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])  # the default is one query per warp


def test_half_warp_errors(lv, pb):
    idx = gpu_index(lv, pb)
    Q, P = t(pb["Q"]), t(pb["P"])
    for kw in (dict(width=4), dict(width=2, warps_per_query=2), dict(width=3)):
        with pytest.raises(lv.LeanVecError):
            idx.search(Q, P, k=10, L=48, queries_per_warp=2, **kw)
    with pytest.raises(lv.LeanVecError):
        idx.search(Q, P, k=10, L=48, queries_per_warp=3)
    fp = lv.Index(0).encode_fp32(t(pb["X"]))
    fp.set_graph(t(pb["graph"]), pb["entry"])
    with pytest.raises(lv.LeanVecError):
        fp.search(Q, None, k=10, L=48, queries_per_warp=2)
