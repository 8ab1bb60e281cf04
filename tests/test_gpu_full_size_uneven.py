"""The uneven batch at full size, uneven-10M-200 (10^7 x 200 database, OOD queries, LeanVec-OOD
d = 64, LVQ-8 primaries and secondaries, R = 64), in the launch configuration the benchmark
times: 5 x 10^4 queries with per-query k in {1, 10, 100}, L uniform in [20, 300] (L >= k) and
rerank = L, served by one persistent launch replayed from a CUDA graph, width 2.

The oracle computes every input the GPU search gets: the LeanVec-OOD projection (eigenvector
search over the FP64 second moments of a 10^5-row database sample and the 10^4 learning queries),
the projected database in FP64 rounded to float32, the FP64 means, the LVQ stores and its
SplitMix64 random 64-regular graph.  Sampled queries are searched by the oracle one by one with
their own descriptors and compared element by element with the GPU's answers."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import encode_parallel, t
from oracle import fit

pytestmark = pytest.mark.gpu

N, M, D, d, R = 10_000_000, 50_000, 200, 64, 64
SAMPLE = 96


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


@pytest.fixture(scope="module")
def problem():
    Xg, Qg, Qlg = workloads.make_workload_torch("anisotropic", N, M, D, 1000, cfg=5, device=torch.device("cuda", 0),
                                                ood=True, m_learn=10_000)
    X, Q, Ql = Xg.cpu().numpy(), Qg.cpu().numpy(), Qlg.cpu().numpy()
    del Xg, Qg, Qlg
    rows = workloads.subsample_rows(N, 100_000, 5)
    es = fit.eigsearch(fit.second_moment(Ql), fit.second_moment(X[rows]), Ql.shape[0], len(rows), d)
    P = es["P"].astype(np.float32)
    P64 = P.astype(np.float64)
    Y = np.empty((N, d), np.float32)
    sx = np.zeros(D, np.float64)
    sy = np.zeros(d, np.float64)
    for s in range(0, N, 500_000):
        x64 = X[s:s + 500_000].astype(np.float64)
        Y[s:s + 500_000] = x64 @ P64.T
        sx += x64.sum(axis=0)
        sy += Y[s:s + 500_000].astype(np.float64).sum(axis=0)
    mu_s = (sx / N).astype(np.float32)
    mu_p = (sy / N).astype(np.float32)
    prim = encode_parallel(oracle, Y, mu_p, 8)
    sec = encode_parallel(oracle, X, mu_s, 8)
    graph = oracle.random_graph(N, R, 5005)
    kl = workloads.uneven_batch(M, seed=workloads.SEED_TEST_QUERIES + 55)
    desc = np.stack([kl[:, 0], kl[:, 1], kl[:, 1], np.zeros(M, np.int32)], 1).astype(np.int32)
    return dict(X=X, Q=Q, P=P, Y=Y, mu_p=mu_p, mu_s=mu_s, prim=prim, sec=sec, graph=graph, entry=0, desc=desc)


def test_uneven_10m_200_sampled_parity(lv, problem):
    pb = problem
    idx = lv.Index(0)
    idx.set_primary(t(pb["Y"]), t(pb["mu_p"]), 8, D)
    idx.set_secondary(t(pb["X"]), t(pb["mu_s"]))
    idx.set_graph(t(pb["graph"]), pb["entry"])
    desc = pb["desc"]
    kmax, Lmax = int(desc[:, 0].max()), int(desc[:, 1].max())
    g = lv.SearchGraph(idx, t(pb["Q"]), t(pb["P"]), k=kmax, L=Lmax, rerank=Lmax, desc=t(desc), width=2,
                       projection=lv.PREC_FP32)
    ids, sc = g.replay()
    torch.cuda.synchronize()
    idx.sync_status()
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    s = np.sort(np.random.default_rng(9).choice(M, SAMPLE, replace=False))
    Qs = pb["Q"][s].astype(np.float64)
    ref = oracle.search(pb["graph"], pb["entry"], Qs @ pb["P"].astype(np.float64).T, k=kmax, L=Lmax,
                        rerank=Lmax, prim=pb["prim"], sec=pb["sec"], qs=Qs, desc=desc[s], width=2)
    k = desc[s, 0]
    valid = np.arange(kmax)[None, :] < k[:, None]
    assert (ids[s][valid] == ref["ids"][valid]).mean() >= 0.99
    assert np.all(ids[s][~valid] == -1)
    for j, qi in enumerate(s):
        got = ids[qi, :k[j]]
        lvq = pb["sec"]
        dec = (lvq.mean[None, :].astype(np.float64) + lvq.lower[got, None].astype(np.float64)
               + lvq.delta[got, None].astype(np.float64) * lvq.codes[got].astype(np.float64))
        bound = 1e-4 * np.linalg.norm(Qs[j]) * np.linalg.norm(dec, axis=1)
        assert np.all(np.abs(sc[qi, :k[j]] - dec @ Qs[j]) <= bound)
