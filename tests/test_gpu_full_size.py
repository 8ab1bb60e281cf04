"""The search at full size, id-1M-768 (10^6 x 768 database, 10^4 queries, d = 160, LVQ-8 primaries
and secondaries, R = 64), in the launch configuration the benchmark times: one call for the 10^4
queries (two sub-batches on two streams), k = 10, L = rerank = 152, max_hops = 76 (the calibrated
expansion budget), width 2.

The oracle computes every input the GPU search gets: the LeanVec-ID projection (FP64 eigenvectors
of a 10^5-row second moment), the projected database in FP64 rounded to float32, the FP64 means,
the LVQ stores, and the graph (its counter-based SplitMix64 random R-regular graph: a full-size
Vamana build is out of the oracle's reach in a test, and the search's arithmetic does not depend
on how the graph was made).  Sampled queries are then searched by the oracle one by one and
compared element by element with the GPU's answers; for the benchmark's bf16 query projection
the oracle applies the same operand rounding (``oracle.rounding``) before its FP64 projection."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import t
from oracle import fit, rounding

pytestmark = pytest.mark.gpu

N, M, D, d, R = 1_000_000, 10_000, 768, 160, 64
K, L, MAXH, W = 10, 152, 76, 2
SAMPLE = 64


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


@pytest.fixture(scope="module")
def problem():
    Xg, Qg, _ = workloads.make_workload_torch("anisotropic", N, M, D, 1000, cfg=2, device=torch.device("cuda", 0),
                                              m_learn=0)
    X, Q = Xg.cpu().numpy(), Qg.cpu().numpy()
    del Xg, Qg
    rows = workloads.subsample_rows(N, 100_000, 2)
    P = fit.fit_id(fit.second_moment(X[rows]), d).astype(np.float32)
    P64 = P.astype(np.float64)
    Y = np.empty((N, d), np.float32)
    sx = np.zeros(D, np.float64)
    sy = np.zeros(d, np.float64)
    for s in range(0, N, 100_000):
        x64 = X[s:s + 100_000].astype(np.float64)
        y = x64 @ P64.T
        Y[s:s + 100_000] = y
        sx += x64.sum(axis=0)
        sy += Y[s:s + 100_000].astype(np.float64).sum(axis=0)
    mu_s = (sx / N).astype(np.float32)
    mu_p = (sy / N).astype(np.float32)
    prim = oracle.lvq_encode(Y, mu_p, 8)
    sec = oracle.lvq_encode(X, mu_s, 8)
    graph = oracle.random_graph(N, R, 5002)
    return dict(X=X, Q=Q, P=P, Y=Y, mu_p=mu_p, mu_s=mu_s, prim=prim, sec=sec, graph=graph, entry=0)


def _decode_rows(lvq, ids):
    return (lvq.mean[None, :].astype(np.float64) + lvq.lower[ids, None].astype(np.float64)
            + lvq.delta[ids, None].astype(np.float64) * lvq.codes[ids].astype(np.float64))


def test_id_1m_768_sampled_parity(lv, problem):
    pb = problem
    idx = lv.Index(0)
    idx.set_primary(t(pb["Y"]), t(pb["mu_p"]), 8, D)
    idx.set_secondary(t(pb["X"]), t(pb["mu_s"]))
    idx.set_graph(t(pb["graph"]), pb["entry"])
    Qd, Pd = t(pb["Q"]), t(pb["P"])
    ids, sc = idx.search(Qd, Pd, k=K, L=L, rerank=L, max_hops=MAXH, width=W, projection=lv.PREC_FP32)
    idx.sync_status()
    # projection, then beam + rerank for each of the two sub-batches
    assert idx.info()["last_search_kernels"] == 1 + 2 * 2
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    s = np.sort(np.random.default_rng(7).choice(M, SAMPLE, replace=False))
    Qs = pb["Q"][s].astype(np.float64)
    ref = oracle.search(pb["graph"], pb["entry"], Qs @ pb["P"].astype(np.float64).T, k=K, L=L, rerank=L,
                        prim=pb["prim"], sec=pb["sec"], qs=Qs, max_hops=MAXH, width=W)
    assert (ids[s] == ref["ids"]).mean() >= 0.99
    assert np.all(ref["hops"] <= MAXH)
    # each returned score is the decoded secondary inner product of its id (FP32 path bound)
    for j, qi in enumerate(s):
        dec = _decode_rows(pb["sec"], ids[qi])
        exact = dec @ Qs[j]
        bound = 1e-4 * np.linalg.norm(Qs[j]) * np.linalg.norm(dec, axis=1)
        assert np.all(np.abs(sc[qi] - exact) <= bound)
        assert np.all(np.diff(sc[qi]) <= 0)
        assert len(set(ids[qi].tolist())) == K
    # the benchmark's bf16 query projection: the oracle searches with the projection of the same
    # bf16-rounded operands (computed in FP64), and the ids must agree as for the float32 path
    ids_b, sc_b = idx.search(Qd, Pd, k=K, L=L, rerank=L, max_hops=MAXH, width=W, projection=lv.PREC_BF16)
    idx.sync_status()
    ids_b, sc_b = ids_b.cpu().numpy(), sc_b.cpu().numpy()
    ref_b = oracle.search(pb["graph"], pb["entry"], rounding.project(pb["Q"][s], pb["P"], "bf16"), k=K, L=L,
                          rerank=L, prim=pb["prim"], sec=pb["sec"], qs=Qs, max_hops=MAXH, width=W)
    assert (ids_b[s] == ref_b["ids"]).mean() >= 0.99
    for j, qi in enumerate(s):
        dec = _decode_rows(pb["sec"], ids_b[qi])
        bound = 1e-4 * np.linalg.norm(Qs[j]) * np.linalg.norm(dec, axis=1)
        assert np.all(np.abs(sc_b[qi] - dec @ Qs[j]) <= bound)


def test_id_1m_768_graph_build_properties(lv, problem):
    """The GPU build at full size on the oracle's primaries with the benchmark's build parameters
    (R = 64, L_build = 128, unit-L2 rule at alpha 1.02, two passes, batches of 65536): properties
    that hold at any size -- ids in range, no self loops or repeats, padding only at the end of a
    row, at least 99 % of the nodes reachable from the entry -- and a search over it that finds at least 0.8 of the
    exact FP64 top 10 of the sampled queries (the search parity itself is the test above)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    pb = problem
    idx = lv.Index(0)
    idx.set_primary(t(pb["Y"]), t(pb["mu_p"]), 8, D)
    idx.set_secondary(t(pb["X"]), t(pb["mu_s"]))
    idx.build_graph(R=R, L_build=128, alpha=1.02, passes=2, batch=65536, rule=lv.PRUNE_UNIT_L2)
    idx.sync_status()
    g, entry = idx.get_graph()
    g = g.cpu().numpy()
    assert g.shape == (N, R) and 0 <= entry < N
    assert g.min() >= -1 and g.max() < N
    valid = g >= 0
    assert np.all(valid[:, :-1] | ~valid[:, 1:])  # -1 only after the last id of a row
    assert not np.any(g == np.arange(N, dtype=np.int32)[:, None])
    srt = np.sort(np.where(valid, g, -np.arange(1, R + 1, dtype=np.int32)[None, :]), axis=1)
    assert not np.any(srt[:, 1:] == srt[:, :-1])
    rows, cols = np.nonzero(valid)
    adj = sp.csr_matrix((np.ones(len(rows), np.int8), (rows, g[rows, cols])), shape=(N, N))
    reach = breadth_first_order(adj, entry, directed=True, return_predecessors=False)
    assert len(reach) >= 0.99 * N, len(reach) / N
    s = np.sort(np.random.default_rng(8).choice(M, SAMPLE, replace=False))
    Qd = t(pb["Q"][s])
    ids, _ = idx.search(Qd, t(pb["P"]), k=K, L=L, rerank=L, max_hops=MAXH, width=W, projection=lv.PREC_BF16)
    truth, _ = oracle.bruteforce(pb["X"], pb["Q"][s], K)
    assert oracle.recall(ids.cpu().numpy(), truth, K) >= 0.8
