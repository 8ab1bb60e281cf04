"""The OOD search at full size, ood-1M-512 (10^6 x 512 database, 10^4 shifted test queries, d = 128,
LVQ-8 primaries and secondaries, R = 64), in the launch configuration the benchmark times for it:
10^4 queries in one call (two sub-batches), k = 10, L = rerank = max_hops = 320 (the beam at which
the OOD projections reach recall 0.90), width 2.

The oracle computes every input the GPU search gets: the LeanVec-OOD projection by eigenvector
search (FP64 second moments of a 10^5-row database sample and the 10^4 learning queries, bounded
Brent over beta), the projected database in FP64 rounded to float32, the FP64 means, the LVQ
stores and its SplitMix64 random 64-regular graph.  Sampled queries are searched by the oracle one
by one and compared element by element with the GPU's answers."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import t
from oracle import fit

pytestmark = pytest.mark.gpu

N, M, D, d, R = 1_000_000, 10_000, 512, 128, 64
K, L, W = 10, 320, 2
SAMPLE = 64


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


@pytest.fixture(scope="module")
def problem():
    Xg, Qg, Qlg = workloads.make_workload_torch("anisotropic", N, M, D, 1000, cfg=3, device=torch.device("cuda", 0),
                                                ood=True, m_learn=M)
    X, Q, Ql = Xg.cpu().numpy(), Qg.cpu().numpy(), Qlg.cpu().numpy()
    del Xg, Qg, Qlg
    rows = workloads.subsample_rows(N, 100_000, 3)
    es = fit.eigsearch(fit.second_moment(Ql), fit.second_moment(X[rows]), Ql.shape[0], len(rows), d)
    P = es["P"].astype(np.float32)
    P64 = P.astype(np.float64)
    Y = np.empty((N, d), np.float32)
    sx = np.zeros(D, np.float64)
    sy = np.zeros(d, np.float64)
    for s in range(0, N, 100_000):
        x64 = X[s:s + 100_000].astype(np.float64)
        Y[s:s + 100_000] = x64 @ P64.T
        sx += x64.sum(axis=0)
        sy += Y[s:s + 100_000].astype(np.float64).sum(axis=0)
    mu_s = (sx / N).astype(np.float32)
    mu_p = (sy / N).astype(np.float32)
    prim = oracle.lvq_encode(Y, mu_p, 8)
    sec = oracle.lvq_encode(X, mu_s, 8)
    graph = oracle.random_graph(N, R, 5003)
    return dict(X=X, Q=Q, P=P, Y=Y, mu_p=mu_p, mu_s=mu_s, prim=prim, sec=sec, graph=graph, entry=0)


def test_ood_1m_512_sampled_parity(lv, problem):
    pb = problem
    idx = lv.Index(0)
    idx.set_primary(t(pb["Y"]), t(pb["mu_p"]), 8, D)
    idx.set_secondary(t(pb["X"]), t(pb["mu_s"]))
    idx.set_graph(t(pb["graph"]), pb["entry"])
    ids, sc = idx.search(t(pb["Q"]), t(pb["P"]), k=K, L=L, rerank=L, max_hops=L, width=W, projection=lv.PREC_FP32)
    idx.sync_status()
    assert idx.info()["last_search_kernels"] == 1 + 2 * 2
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    s = np.sort(np.random.default_rng(11).choice(M, SAMPLE, replace=False))
    Qs = pb["Q"][s].astype(np.float64)
    ref = oracle.search(pb["graph"], pb["entry"], Qs @ pb["P"].astype(np.float64).T, k=K, L=L, rerank=L,
                        prim=pb["prim"], sec=pb["sec"], qs=Qs, max_hops=L, width=W)
    assert (ids[s] == ref["ids"]).mean() >= 0.99
    lvq = pb["sec"]
    for j, qi in enumerate(s):
        got = ids[qi]
        dec = (lvq.mean[None, :].astype(np.float64) + lvq.lower[got, None].astype(np.float64)
               + lvq.delta[got, None].astype(np.float64) * lvq.codes[got].astype(np.float64))
        bound = 1e-4 * np.linalg.norm(Qs[j]) * np.linalg.norm(dec, axis=1)
        assert np.all(np.abs(sc[qi] - dec @ Qs[j]) <= bound)
        assert np.all(np.diff(sc[qi]) <= 0)
        assert len(set(got.tolist())) == K
