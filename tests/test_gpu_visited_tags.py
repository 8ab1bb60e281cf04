"""The visited cache of 16-bit tags (buckets of 8) against the one of 32-bit ids (buckets of 4)
and the oracle's exact visited set.

A tag names its id exactly, so the cache never reports an unvisited id as visited; it may forget
ids (a full bucket is overwritten, or two ids of one step take the same free slot), which only
costs re-scores: the beam, hence every result, is the one of an exact visited set."""
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
    return small_problem(oracle, n=3000, D=64, d=16, m=300)


def _qp(pb):
    return pb["Q"].astype(np.float64) @ pb["P"].T.astype(np.float64)


@pytest.mark.parametrize("W,T", [(1, 1), (2, 1), (4, 1), (2, 2)])
def test_tags_and_ids_same_result(lv, pb, W, T):
    """Identical ids, scores and expansion counts with either slot width, from a cache that
    forgets often (64 / 128 slots) to one that forgets nothing; the oracle's ids."""
    idx = gpu_index(lv, pb)
    ref = oracle.search(pb["graph"], pb["entry"], _qp(pb), k=10, L=48, rerank=48, prim=pb["prim"], sec=pb["sec"],
                        qs=pb["Q"].astype(np.float64), width=W)
    kw = dict(k=10, L=48, rerank=48, width=W, warps_per_query=T, stats=True)
    for hs in (0, 128, 8192):
        a, sa, ta = idx.search(t(pb["Q"]), t(pb["P"]), hash_slots=hs, visited_bits=32, **kw)
        b, sb, tb = idx.search(t(pb["Q"]), t(pb["P"]), hash_slots=hs, visited_bits=16, **kw)
        c, sc, tc = idx.search(t(pb["Q"]), t(pb["P"]), hash_slots=hs, **kw)  # default: ids
        idx.sync_status()
        assert torch.equal(a, b) and torch.equal(sa, sb) and torch.equal(ta[:, 0], tb[:, 0])
        assert torch.equal(a, c) and torch.equal(sa, sc) and torch.equal(ta[:, 0], tc[:, 0])
        if T == 1:  # (a team's warps test ids concurrently: its re-score count varies from run to run)
            assert torch.equal(ta, tc)
        assert (b.cpu().numpy() == ref["ids"]).mean() >= 0.99
    # the smallest cache the beam allows (2 x 64 slots for L = 48: 16 buckets of 8 tags)
    a, sa = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48, width=W, warps_per_query=T, hash_slots=64,
                       visited_bits=16)
    assert (a.cpu().numpy() == ref["ids"]).mean() >= 0.99


def test_tags_rescore_little(lv, pb):
    """Width 1 with 8192 tag slots for at most a few hundred visits per query (no bucket of 8
    overflows): the oracle's hop counts, and never fewer scored records than the oracle's distinct
    visited nodes (a cache that reported an unvisited id as visited would score fewer); the few
    extra are ids that another id of the same step wrote over (same bucket, same free slot).  In
    the same bytes, 8-way buckets of tags overflow less than 4-way buckets of ids: with 512 bytes
    per query (32 buckets for about 170 visits) the tags score fewer records."""
    idx = gpu_index(lv, pb)
    ref = oracle.search(pb["graph"], pb["entry"], _qp(pb), k=10, L=48, prim=pb["prim"])
    _, _, st = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, hash_slots=8192, visited_bits=16, stats=True)
    st = st.cpu().numpy()
    np.testing.assert_array_equal(st[:, 0], ref["hops"])
    assert (st[:, 1] >= ref["scored"]).all()
    assert (st[:, 1] - ref["scored"]).sum() <= 0.01 * ref["scored"].sum()
    _, _, s16 = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, stats=True, hash_slots=256, visited_bits=16)
    _, _, s32 = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, stats=True, hash_slots=128, visited_bits=32)
    assert s16[:, 1].sum().item() < s32[:, 1].sum().item()
    assert (s16[:, 1].cpu().numpy() >= ref["scored"]).all()


def test_tags_other_scorers(lv, pb):
    """LVQ-4 primaries and full-dimensional float32 records: the same answers with either slot width."""
    sub = small_problem(oracle, n=2000, D=48, d=16, m=100, bits=4, seed=2)
    idx = gpu_index(lv, sub)
    for W in (1, 2):
        a, sa = idx.search(t(sub["Q"]), t(sub["P"]), k=10, L=40, rerank=40, width=W, visited_bits=32, hash_slots=128)
        b, sb = idx.search(t(sub["Q"]), t(sub["P"]), k=10, L=40, rerank=40, width=W, visited_bits=16, hash_slots=128)
        assert torch.equal(a, b) and torch.equal(sa, sb)
    f = lv.Index(0).encode_fp32(t(pb["X"])).set_graph(t(pb["graph"]), pb["entry"])
    for W in (1, 2):
        a, sa = f.search(t(pb["Q"]), None, k=10, L=32, width=W, visited_bits=32, hash_slots=64)
        b, sb = f.search(t(pb["Q"]), None, k=10, L=32, width=W, visited_bits=16, hash_slots=64)
        f.sync_status()
        assert torch.equal(a, b) and torch.equal(sa, sb)


def test_tags_errors(lv, pb):
    """A slot width other than 0, 16 or 32 is refused, and so are 16-bit tags that cannot name every
    id: with 64 slots (8 buckets) the tags of n = 600,000 ids run past 0xFFFE."""
    idx = gpu_index(lv, pb)
    with pytest.raises(lv.LeanVecError):
        idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=16, visited_bits=8)
    n, d = 600_000, 16
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((n, d)).astype(np.float32)
    big = lv.Index(0).set_primary(t(Y), t(Y.mean(0)), 8, d)
    big.set_graph(t(rng.integers(0, n, (n, 4)).astype(np.int32)), 0)
    P = np.eye(d, dtype=np.float32)
    Q = rng.standard_normal((8, d)).astype(np.float32)
    with pytest.raises(lv.LeanVecError):
        big.search(t(Q), t(P), k=4, L=16, hash_slots=64, visited_bits=16)
    # 32-bit ids for that cache; tags in the default one (2048 slots: n <= 16.7 M)
    a, _ = big.search(t(Q), t(P), k=4, L=16, hash_slots=64)
    b, _ = big.search(t(Q), t(P), k=4, L=16, visited_bits=16)
    big.sync_status()
    assert torch.equal(a, b)
