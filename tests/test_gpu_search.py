"""GPU beam search + rerank against the oracle on the same seeded inputs and graph.

Tolerances: scores within 1e-4 * ||q'|| * ||x_hat|| (FP32 path); ids >= 99 %
identical position by position; recall@10 against brute force within 0.002."""
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


def _qp(pb, Q=None):
    Q = pb["Q"] if Q is None else Q
    return Q.astype(np.float64) @ pb["P"].T.astype(np.float64)


def _check_scores(ids, scores, ref_dec, qv, tol=1e-4):
    """scores of returned ids agree with the FP64 decoded inner products."""
    for j in range(ids.shape[0]):
        sel = ids[j] >= 0
        u = ids[j][sel]
        exact = ref_dec[u] @ qv[j]
        bound = tol * np.linalg.norm(qv[j]) * np.linalg.norm(ref_dec[u], axis=1)
        assert np.all(np.abs(scores[j][sel] - exact) <= bound), (j, np.abs(scores[j][sel] - exact).max())


def test_primary_scores_full_window(lv, pb):
    """L >= n: the beam holds every reachable node; the GPU primary scores of the
    returned ids match FP64 decode-then-dot."""
    n = 400
    sub = small_problem(oracle, n=n, D=48, d=12, m=20, seed=3)
    idx = gpu_index(lv, sub)
    qp = _qp(sub)
    ids, sc = idx.search(t(sub["Q"]), t(sub["P"]), k=n, L=n, rerank=0)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    _check_scores(ids, sc, sub["prim"].decode(), qp)
    ref = oracle.search(sub["graph"], sub["entry"], qp, k=n, L=n, prim=sub["prim"])
    for j in range(20):
        assert set(ids[j][ids[j] >= 0].tolist()) == set(ref["ids"][j][ref["ids"][j] >= 0].tolist())


def test_rerank_scores_full_window(lv):
    n = 300
    sub = small_problem(oracle, n=n, D=200, d=24, m=16, seed=4)  # D = 200: ragged secondary chunk
    idx = gpu_index(lv, sub)
    ids, sc = idx.search(t(sub["Q"]), t(sub["P"]), k=50, L=n, rerank=n)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    _check_scores(ids, sc, sub["sec"].decode(), sub["Q"].astype(np.float64))
    ref = oracle.search(sub["graph"], sub["entry"], _qp(sub), k=50, L=n, rerank=n, prim=sub["prim"], sec=sub["sec"],
                        qs=sub["Q"].astype(np.float64))
    assert (ids == ref["ids"]).mean() >= 0.99


@pytest.mark.parametrize("L,r", [(16, 16), (40, 40), (100, 60)])
def test_ids_match_oracle(lv, pb, L, r):
    idx = gpu_index(lv, pb)
    ids, sc, st = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=L, rerank=r, stats=True)
    idx.sync_status()
    ids = ids.cpu().numpy()
    ref = oracle.search(pb["graph"], pb["entry"], _qp(pb), k=10, L=L, rerank=r, prim=pb["prim"], sec=pb["sec"],
                        qs=pb["Q"].astype(np.float64))
    same = (ids == ref["ids"]).mean()
    assert same >= 0.99, same
    truth, _ = oracle.bruteforce(pb["X"], pb["Q"], 10)
    assert abs(oracle.recall(ids, truth, 10) - oracle.recall(ref["ids"], truth, 10)) <= 0.002
    _check_scores(ids, sc.cpu().numpy(), pb["sec"].decode(), pb["Q"].astype(np.float64))
    st = st.cpu().numpy()
    # expansions equal the oracle's (exact beam), scored counts are >= (forgotten ids are rescored)
    assert np.abs(st[:, 0] - ref["hops"]).mean() <= 0.5
    assert np.all(st[:, 1] >= 1)


@pytest.mark.parametrize("W,mh", [(1, 20), (2, 25), (2, 36), (4, 30), (3, 31)])
def test_expansion_budget_matches_oracle(lv, pb, W, mh):
    """max_hops below the unlimited search's hop count (about 50 here): the last round is cut to
    the remaining budget on both sides, so the beams, the reranked ids and the hop counts agree."""
    idx = gpu_index(lv, pb)
    ref = oracle.search(pb["graph"], pb["entry"], _qp(pb), k=10, L=48, rerank=48, prim=pb["prim"], sec=pb["sec"],
                        qs=pb["Q"].astype(np.float64), width=W, max_hops=mh)
    assert ref["hops"].max() <= mh and (ref["hops"] == mh).mean() > 0.5  # the budget binds
    ids, sc, st = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48, width=W, max_hops=mh, stats=True)
    ids = ids.cpu().numpy()
    assert (ids == ref["ids"]).mean() >= 0.99
    hops = st[:, 0].cpu().numpy()
    assert hops.max() <= mh
    assert np.abs(hops - ref["hops"]).mean() <= 0.5


@pytest.mark.parametrize("W", [2, 4])
def test_search_width_matches_oracle(lv, pb, W):
    """Expanding the W best unexpanded members per round: same result as the oracle's
    width-W rule, also with a tiny visited cache (cross-parent forgotten ids)."""
    idx = gpu_index(lv, pb)
    ref = oracle.search(pb["graph"], pb["entry"], _qp(pb), k=10, L=48, rerank=48, prim=pb["prim"], sec=pb["sec"],
                        qs=pb["Q"].astype(np.float64), width=W)
    for hs in (0, 128):
        ids, sc, st = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48, width=W, stats=True, hash_slots=hs)
        ids = ids.cpu().numpy()
        assert (ids == ref["ids"]).mean() >= 0.99
        assert np.abs(st[:, 0].cpu().numpy() - ref["hops"]).mean() <= 0.5
    with pytest.raises(lv.LeanVecError):
        idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, width=5)


@pytest.mark.parametrize("W,T", [(2, 2), (4, 2), (4, 4)])
def test_warps_per_query_same_result(lv, pb, W, T):
    """A team of T warps per query expands the same parents per round as one warp:
    identical ids, scores and expansion counts (also with a tiny visited cache, where
    the warps' concurrent tests let shared neighbours through twice, and with uneven
    per-query descriptors)."""
    idx = gpu_index(lv, pb)
    for hs in (0, 128):
        a, sa, ta = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48, width=W, stats=True, hash_slots=hs)
        b, sb, tb = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48, width=W, stats=True, hash_slots=hs,
                               warps_per_query=T)
        idx.sync_status()
        assert torch.equal(a, b) and torch.equal(sa, sb)
        assert torch.equal(ta[:, 0], tb[:, 0])
    m = pb["Q"].shape[0]
    rng = np.random.default_rng(7)
    k = rng.choice([1, 5, 10], m)
    L = np.maximum(rng.integers(10, 80, m), k)
    r = np.minimum(L, rng.integers(0, 60, m))
    desc = t(np.stack([k, L, r, rng.integers(0, 40, m)], 1).astype(np.int32))
    a, sa = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=80, rerank=80, desc=desc, width=W)
    b, sb = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=80, rerank=80, desc=desc, width=W, warps_per_query=T,
                       warps_per_block=4)
    assert torch.equal(a, b) and torch.equal(sa, sb)


def test_warps_per_query_errors(lv, pb):
    idx = gpu_index(lv, pb)
    for W, T, wpb in ((2, 4, 0), (4, 3, 0), (3, 2, 0), (2, 2, 3)):
        with pytest.raises(lv.LeanVecError):
            idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, width=W, warps_per_query=T, warps_per_block=wpb)


def test_fp16_secondary_encode_and_rerank(lv, pb):
    """FP16 secondaries (secondary_bits = 16): records are x rounded to IEEE half (bit-exact against
    numpy, padding zero); the rerank over them matches the oracle's FP64 scores of the same halves."""
    idx = lv.Index(0).encode(t(pb["X"]), t(pb["P"]), 8, 16)
    inf = idx.info()
    D = pb["D"]
    assert inf["secondary_bits"] == 16 and inf["secondary_stride"] == (2 * D + 31) // 32 * 32
    rec = idx.secondary_records().cpu().numpy()
    X16 = pb["X"].astype(np.float16)
    np.testing.assert_array_equal(rec[:, :2 * D].copy().view(np.uint16), X16.view(np.uint16))
    assert (rec[:, 2 * D:] == 0).all()
    # the oracle's primaries (same n: the FP16 secondary store stays) and graph
    idx.set_primary(t(pb["Y"]), t(pb["mu_p"]), pb["bits"], D).set_graph(t(pb["graph"]), pb["entry"])
    assert idx.info()["secondary_bits"] == 16
    ids, sc = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48)
    ref = oracle.search(pb["graph"], pb["entry"], _qp(pb), k=10, L=48, rerank=48, prim=pb["prim"],
                        sec_vecs=X16.astype(np.float32), qs=pb["Q"].astype(np.float64))
    ids = ids.cpu().numpy()
    assert (ids == ref["ids"]).mean() >= 0.99
    _check_scores(ids, sc.cpu().numpy(), X16.astype(np.float64), pb["Q"].astype(np.float64))
    # the no-allocation entry point reranks the same way
    ids2, sc2 = idx.search_noalloc(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48)
    assert (ids2.cpu().numpy() == ref["ids"]).mean() >= 0.99


def test_small_hash_still_exact(lv, pb):
    """A tiny visited cache forgets often; the beam (hence the result) is unchanged."""
    idx = gpu_index(lv, pb)
    a, _ = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=64, rerank=32, hash_slots=128)
    b, _ = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=64, rerank=32, hash_slots=8192)
    assert torch.equal(a, b)


def test_uneven_batch_descriptors(lv, pb):
    idx = gpu_index(lv, pb)
    m = pb["Q"].shape[0]
    rng = np.random.default_rng(5)
    k = rng.choice([1, 5, 10], m)
    L = np.maximum(rng.integers(10, 80, m), k)
    r = np.minimum(L, rng.integers(0, 60, m))
    desc = np.stack([k, L, r, np.zeros(m, int)], 1).astype(np.int32)
    ids, sc = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=80, rerank=80, desc=t(desc), ldo=10)
    idx.sync_status()
    ref = oracle.search(pb["graph"], pb["entry"], _qp(pb), k=10, L=80, rerank=80, prim=pb["prim"], sec=pb["sec"],
                        qs=pb["Q"].astype(np.float64), desc=desc)
    ids = ids.cpu().numpy()
    valid = np.arange(10)[None, :] < k[:, None]
    assert (ids[valid] == ref["ids"][valid]).mean() >= 0.99
    assert np.all(ids[~valid] == -1)


def test_unreachable_padding_and_max_hops(lv):
    sub = small_problem(oracle, n=200, D=32, d=8, m=8, seed=6)
    g = np.full_like(sub["graph"], -1)
    g[0, :2] = [1, 2]
    sub2 = dict(sub, graph=g, entry=0)
    idx = gpu_index(lv, sub2)
    ids, sc = idx.search(t(sub["Q"]), t(sub["P"]), k=5, L=10, rerank=10)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    assert (ids[:, 3:] == -1).all() and np.isinf(sc[:, 3:]).all() and (sc[:, 3:] < 0).all()
    assert set(ids[0, :3].tolist()) == {0, 1, 2}
    idx2 = gpu_index(lv, sub)
    _, _, st = idx2.search(t(sub["Q"]), t(sub["P"]), k=5, L=30, rerank=0, max_hops=3, stats=True)
    assert (st[:, 0].cpu().numpy() <= 3).all()


def test_repeated_and_out_of_range_ids_in_user_graph(lv):
    sub = small_problem(oracle, n=300, D=32, d=8, m=10, seed=7)
    g = sub["graph"].copy()
    g[:, -1] = g[:, 0]  # repeated id in every row
    idx = gpu_index(lv, dict(sub, graph=g))
    ids, _ = idx.search(t(sub["Q"]), t(sub["P"]), k=5, L=20, rerank=20)
    ref = oracle.search(g, sub["entry"], _qp(sub), k=5, L=20, rerank=20, prim=sub["prim"], sec=sub["sec"],
                        qs=sub["Q"].astype(np.float64))
    assert (ids.cpu().numpy() == ref["ids"]).mean() >= 0.99
    g2 = sub["graph"].copy()
    g2[3, 0] = 10 ** 6
    with pytest.raises(lv.LeanVecError):
        gpu_index(lv, dict(sub, graph=g2)).sync_status()


def test_float32_baseline_matches_oracle(lv, pb):
    idx = lv.Index(0)
    idx.encode_fp32(t(pb["X"])).set_graph(t(pb["graph"]), pb["entry"])
    ids, sc = idx.search(t(pb["Q"]), None, k=10, L=40)
    ids = ids.cpu().numpy()
    ref = oracle.search(pb["graph"], pb["entry"], pb["Q"].astype(np.float64), k=10, L=40, prim_vecs=pb["X"])
    assert (ids == ref["ids"]).mean() >= 0.99
    Xd = pb["X"].astype(np.float64)
    _check_scores(ids, sc.cpu().numpy(), Xd, pb["Q"].astype(np.float64))
    a, sa = idx.search(t(pb["Q"]), None, k=10, L=40, width=2)
    b, sb = idx.search(t(pb["Q"]), None, k=10, L=40, width=2, warps_per_query=2)
    assert torch.equal(a, b) and torch.equal(sa, sb)


def test_lvq4_primary(lv):
    sub = small_problem(oracle, n=2000, D=64, d=32, m=100, seed=8, bits=4)
    idx = gpu_index(lv, sub)
    ids, sc = idx.search(t(sub["Q"]), t(sub["P"]), k=10, L=40, rerank=40)
    ref = oracle.search(sub["graph"], sub["entry"], _qp(sub), k=10, L=40, rerank=40, prim=sub["prim"], sec=sub["sec"],
                        qs=sub["Q"].astype(np.float64))
    assert (ids.cpu().numpy() == ref["ids"]).mean() >= 0.99


def test_argument_errors(lv, pb):
    idx = gpu_index(lv, pb)
    with pytest.raises(lv.LeanVecError):
        idx.search(t(pb["Q"]), t(pb["P"]), k=20, L=10)  # k > L
    with pytest.raises(lv.LeanVecError):
        idx.search(t(pb["Q"]), t(pb["P"]), k=5, L=1000)  # L > 512
    empty = lv.Index(0)
    with pytest.raises(lv.LeanVecError):
        empty.search(t(pb["Q"]), t(pb["P"]), k=5, L=10)
    ids, sc = idx.search(t(pb["Q"][:0]), t(pb["P"]), k=5, L=10)
    assert ids.shape == (0, 5)


def test_cuda_graph_replay_and_autotune(lv, pb):
    """Batching form: an uneven batch captured once in a CUDA graph and replayed gives the
    eager result; the autotuner's choice (queries per warp, launch shape, visited cache) does not
    change it."""
    idx = gpu_index(lv, pb)
    m = pb["Q"].shape[0]
    rng = np.random.default_rng(11)
    k = rng.choice([1, 5, 10], m)
    L = np.maximum(rng.integers(10, 96, m), k)
    desc = t(np.stack([k, L, L, np.zeros(m, int)], 1).astype(np.int32))
    Q, P = t(pb["Q"]), t(pb["P"])
    eager = idx.search(Q, P, k=10, L=96, rerank=96, desc=desc, ldo=10)
    tune = lv.autotune(idx, Q, P, k=10, L=96, rerank=96, desc=desc)
    assert tune["best"] is not None and len(tune["table"]) >= 2
    g = lv.SearchGraph(idx, Q, P, k=10, L=96, rerank=96, desc=desc, hash_slots=tune["best"]["hash_slots"],
                       warps_per_block=tune["best"]["warps_per_block"],
                       queries_per_warp=tune["best"]["queries_per_warp"])
    for _ in range(3):
        ids, sc = g.replay()
        torch.cuda.synchronize()
        assert torch.equal(ids, eager[0])
        assert torch.equal(sc, eager[1])


def test_sub_batches_match_small_batches(lv):
    """m = 12000 is above one wave of resident query slots and not a multiple of it: the queries
    past the last whole wave run as a second launch on a second stream.  Every query is computed
    independently, so ids, scores and counters equal those of batches of 100 (one launch each),
    also when the search is captured in a CUDA graph; and the ids agree with the oracle."""
    sub = small_problem(oracle, n=3000, D=64, d=16, m=12000, seed=11)
    idx = gpu_index(lv, sub)
    Q, P = t(sub["Q"]), t(sub["P"])
    ids, sc, st = idx.search(Q, P, k=10, L=48, rerank=48, width=2, stats=True)
    # fp32 projection, then beam + rerank for each of the two sub-batches
    assert idx.info()["last_search_kernels"] == 1 + 2 * 2
    parts = [idx.search(Q[s:s + 100].contiguous(), P, k=10, L=48, rerank=48, width=2, stats=True)
             for s in range(0, 12000, 100)]
    assert idx.info()["last_search_kernels"] == 1 + 2
    torch.testing.assert_close(ids, torch.cat([p[0] for p in parts]), rtol=0, atol=0)
    torch.testing.assert_close(sc, torch.cat([p[1] for p in parts]), rtol=0, atol=0)
    torch.testing.assert_close(st, torch.cat([p[2] for p in parts]), rtol=0, atol=0)
    g = lv.SearchGraph(idx, Q, P, k=10, L=48, rerank=48, width=2)
    gi, gs = g.replay()
    torch.cuda.synchronize()
    torch.testing.assert_close(gi, ids, rtol=0, atol=0)
    torch.testing.assert_close(gs, sc, rtol=0, atol=0)
    ref = oracle.search(sub["graph"], sub["entry"], _qp(sub), k=10, L=48, rerank=48, prim=sub["prim"],
                        sec=sub["sec"], qs=sub["Q"].astype(np.float64), width=2)
    assert (ids.cpu().numpy() == ref["ids"]).mean() >= 0.99
    # per-query descriptors (k, L, rerank, max_hops) follow their queries into the second sub-batch
    rng = np.random.default_rng(3)
    kk = rng.integers(1, 11, 12000)
    LL = np.maximum(kk, rng.integers(8, 65, 12000))
    desc = np.stack([kk, LL, LL, rng.integers(0, 40, 12000)], 1).astype(np.int32)
    dids, dsc = idx.search(Q, P, k=10, L=64, rerank=64, desc=t(desc), width=2)
    dparts = [idx.search(Q[s:s + 100].contiguous(), P, k=10, L=64, rerank=64, desc=t(desc[s:s + 100]), width=2)
              for s in range(0, 12000, 100)]
    torch.testing.assert_close(dids, torch.cat([p[0] for p in dparts]), rtol=0, atol=0)
    torch.testing.assert_close(dsc, torch.cat([p[1] for p in dparts]), rtol=0, atol=0)


def test_autotune_target_d(lv):
    """The target-d autotuner: for each d, the smallest L of the grid whose recall@10 reaches the
    target under the given graph, and the fastest such d; recall checked against the oracle's
    brute force (the caller's ground truth)."""
    sub = small_problem(oracle, n=3000, D=64, d=16, m=500, seed=12)
    truth, _ = oracle.bruteforce(sub["X"], sub["Q"], 10)
    X, Q = t(sub["X"]), t(sub["Q"])
    tune = lv.autotune_target_d(X, Q, torch.from_numpy(truth).cuda(), t(sub["graph"]), sub["entry"], ds=(8, 16, 32),
                                target=0.5, L_grid=(16, 32, 64, 128, 256), projection=lv.PREC_FP32, width=1)
    assert [r["d"] for r in tune["table"]] == [8, 16, 32]
    for r in tune["table"]:
        if r["L"] is not None:
            assert r["recall"] >= 0.5 and r["qps"] > 0
    assert tune["best"] is not None and tune["best"]["qps"] == max(r["qps"] or 0 for r in tune["table"])
    # the reported recall is that of the search at the chosen L, recomputed here
    b = tune["best"]
    idx = lv.Index(0).encode(X, b["A"], 8, 8, precision=lv.PREC_BF16).set_graph(t(sub["graph"]), sub["entry"])
    ids = idx.search(Q, b["A"], k=10, L=b["L"], rerank=b["L"], width=1)[0].cpu().numpy()
    assert abs(oracle.recall(ids, truth, 10) - b["recall"]) < 1e-6


@pytest.mark.parametrize("batch", [0, 70, 300])
def test_search_host_matches_search(lv, pb, batch):
    """leanvec_search_host: pinned host queries in, host results out, in batches of `batch` rows
    (a ragged last batch at 70; one batch at 0 and 300) with the copies of neighbouring batches
    on the index's copy streams; the results equal a device search of each batch, bit for bit,
    and the oracle's ids; a second call reuses the staging slots."""
    idx = gpu_index(lv, pb)
    P = t(pb["P"])
    Qh = torch.from_numpy(pb["Q"]).pin_memory()
    m = Qh.shape[0]
    for _ in range(2):
        ids_h, sc_h = idx.search_host(Qh, P, k=10, L=48, rerank=48, width=2, batch=batch)
        torch.cuda.synchronize()
        bt = batch or m
        for q0 in range(0, m, bt):
            ids, sc = idx.search(t(pb["Q"][q0:q0 + bt]), P, k=10, L=48, rerank=48, width=2)
            torch.testing.assert_close(ids_h[q0:q0 + bt], ids.cpu(), rtol=0, atol=0)
            torch.testing.assert_close(sc_h[q0:q0 + bt], sc.cpu(), rtol=0, atol=0)
    idx.sync_status()
    ref = oracle.search(pb["graph"], pb["entry"], _qp(pb), k=10, L=48, rerank=48, prim=pb["prim"], sec=pb["sec"],
                        qs=pb["Q"].astype(np.float64), width=2)
    assert (ids_h.numpy() == ref["ids"]).mean() >= 0.99


def test_search_host_descriptors(lv, pb):
    """Per-query descriptors from host memory across batch boundaries: the same results as the
    device search with the same descriptors."""
    idx = gpu_index(lv, pb)
    P = t(pb["P"])
    m = pb["Q"].shape[0]
    rng = np.random.default_rng(12)
    L = rng.integers(12, 64, m).astype(np.int32)
    k = np.minimum(rng.choice([1, 5, 10], m), L).astype(np.int32)
    desc = np.stack([k, L, L, np.zeros(m, np.int32)], axis=1).astype(np.int32)
    ids_h, sc_h = idx.search_host(torch.from_numpy(pb["Q"]).pin_memory(), P, k=10, L=64, ldo=10,
                                  desc=torch.from_numpy(desc), batch=128, width=2)
    torch.cuda.synchronize()
    ids, sc = idx.search(t(pb["Q"]), P, k=10, L=64, ldo=10, desc=t(desc), width=2)
    torch.testing.assert_close(ids_h, ids.cpu(), rtol=0, atol=0)
    torch.testing.assert_close(sc_h, sc.cpu(), rtol=0, atol=0)
    idx.sync_status()


def test_autotune_uneven_graph_matches_eager(lv, pb):
    """The batching form's autotuner: every plan (caller's order, longest first, beam-width
    classes each with its own capacity and timed knobs), run from one CUDA-graph replay, returns
    the same ids and scores, bit for bit, as one eager launch over the whole batch; each plan covers
    every query once and the winner is the fastest."""
    idx = gpu_index(lv, pb)
    Q, P = t(pb["Q"]), t(pb["P"])
    m = Q.shape[0]
    rng = np.random.default_rng(21)
    L = rng.integers(10, 200, m)
    k = np.minimum(rng.choice([1, 5, 10], m), L)
    desc = t(np.stack([k, L, L, np.zeros(m, int)], 1).astype(np.int32))
    ref_ids, ref_sc = idx.search(Q, P, k=10, L=200, rerank=200, desc=desc, ldo=10, width=2)
    tuned = lv.autotune_uneven(idx, Q, P, desc, ldo=10, width=2, bounds=(32, 64, 128, 200), reps=1)
    assert tuned["plans"][tuned["plan"]] == min(tuned["plans"].values())
    assert len(tuned["plan_launches"]["classes"]) >= 3
    for name in ("one", "longest", "classes"):
        plan = {"order": tuned["plan_orders"][name], "classes": tuned["plan_launches"][name]}
        assert sorted(plan["order"].tolist()) == list(range(m))
        assert sum(c["queries"] for c in plan["classes"]) == m
        for c in plan["classes"]:
            assert c["beam_capacity"] % 32 == 0 and c["L_max"] <= c["beam_capacity"]
            assert c["warps_per_query"] in (1, 2)
        g = lv.UnevenGraph(idx, Q, P, desc, plan, ldo=10, width=2)
        for _ in range(2):
            ids, sc = g.replay()
            torch.cuda.synchronize()
            torch.testing.assert_close(g.unsorted(ids), ref_ids, rtol=0, atol=0)
            torch.testing.assert_close(g.unsorted(sc), ref_sc, rtol=0, atol=0)
    idx.sync_status()
