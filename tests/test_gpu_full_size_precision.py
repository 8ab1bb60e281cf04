"""The precision form at full size, prec-10M-768 (10^7 x 768 database, 10,000 mixture components,
d = 160 LVQ-4 primaries and LVQ-8 secondaries, R = 64), in the launch configuration the benchmark
times: 10^5 queries in one call (sub-batches on two streams), k = 10, L = rerank = 512, no expansion
budget, width 2.

The oracle computes every input the GPU search gets: the LeanVec-ID projection (FP64 eigenvectors
of a 10^5-row second moment), the projected database in FP64 rounded to float32, the FP64 means,
the LVQ-4 / LVQ-8 stores and its SplitMix64 random 64-regular graph.  Sampled queries are searched
by the oracle one by one.  With the FP32 query projection the ids must agree element by element;
with the benchmark's e4m3 projection (per-row scales) the oracle applies the same operand rounding
(``oracle.rounding``) before its FP64 projection and the ids must agree likewise; every returned
score is the exact rerank score of its id, scores are sorted and ids distinct."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import encode_parallel, t
from oracle import fit, rounding

pytestmark = pytest.mark.gpu

N, M, D, d, R = 10_000_000, 100_000, 768, 160, 64
K, L, W = 10, 512, 2
SAMPLE = 48


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


@pytest.fixture(scope="module")
def problem():
    Xg, Qg, _ = workloads.make_workload_torch("anisotropic", N, M, D, 10_000, cfg=4, device=torch.device("cuda", 0),
                                              m_learn=0)
    X, Q = Xg.cpu().numpy(), Qg.cpu().numpy()
    del Xg, Qg
    torch.cuda.empty_cache()
    rows = workloads.subsample_rows(N, 100_000, 4)
    P = fit.fit_id(fit.second_moment(X[rows]), d).astype(np.float32)
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
    prim = encode_parallel(oracle, Y, mu_p, 4)
    sec = encode_parallel(oracle, X, mu_s, 8)
    graph = oracle.random_graph(N, R, 5004)
    return dict(X=X, Q=Q, P=P, Y=Y, mu_p=mu_p, mu_s=mu_s, prim=prim, sec=sec, graph=graph, entry=0)


def _check_scores(pb, ids, sc, s, Qs):
    lvq = pb["sec"]
    for j, qi in enumerate(s):
        got = ids[qi]
        dec = (lvq.mean[None, :].astype(np.float64) + lvq.lower[got, None].astype(np.float64)
               + lvq.delta[got, None].astype(np.float64) * lvq.codes[got].astype(np.float64))
        bound = 1e-4 * np.linalg.norm(Qs[j]) * np.linalg.norm(dec, axis=1)
        assert np.all(np.abs(sc[qi] - dec @ Qs[j]) <= bound)
        assert np.all(np.diff(sc[qi]) <= 0)
        assert len(set(got.tolist())) == K


def test_precision_10m_768_sampled_parity(lv, problem):
    pb = problem
    idx = lv.Index(0)
    idx.set_primary(t(pb["Y"]), t(pb["mu_p"]), 4, D)
    Xd = t(pb["X"])
    idx.set_secondary(Xd, t(pb["mu_s"]))
    del Xd
    torch.cuda.empty_cache()
    idx.set_graph(t(pb["graph"]), pb["entry"])
    Qd, Pd = t(pb["Q"]), t(pb["P"])
    ids, sc = idx.search(Qd, Pd, k=K, L=L, rerank=L, width=W, projection=lv.PREC_FP32)
    idx.sync_status()
    assert idx.info()["last_search_kernels"] == 1 + 2 * 2
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    s = np.sort(np.random.default_rng(10).choice(M, SAMPLE, replace=False))
    Qs = pb["Q"][s].astype(np.float64)
    ref = oracle.search(pb["graph"], pb["entry"], Qs @ pb["P"].astype(np.float64).T, k=K, L=L, rerank=L,
                        prim=pb["prim"], sec=pb["sec"], qs=Qs, width=W)
    assert (ids[s] == ref["ids"]).mean() >= 0.99
    _check_scores(pb, ids, sc, s, Qs)
    ids8, sc8 = idx.search(Qd, Pd, k=K, L=L, rerank=L, width=W, projection=lv.PREC_FP8)
    idx.sync_status()
    ids8, sc8 = ids8.cpu().numpy(), sc8.cpu().numpy()
    _check_scores(pb, ids8, sc8, s, Qs)
    # the e4m3 projection: the oracle searches with the projection of the same per-row scaled
    # e4m3 operands (computed in FP64), and the ids must agree as for the float32 path
    ref8 = oracle.search(pb["graph"], pb["entry"], rounding.project(pb["Q"][s], pb["P"], "e4m3"), k=K, L=L,
                         rerank=L, prim=pb["prim"], sec=pb["sec"], qs=Qs, width=W)
    assert (ids8[s] == ref8["ids"]).mean() >= 0.99
    # each e4m3-projected query is within 2e-2 of the unrounded FP64 projection, per coordinate
    # relative to ||q|| ||a||
    P64 = pb["P"].astype(np.float64)
    err = np.abs(rounding.project(pb["Q"][s], pb["P"], "e4m3") - Qs @ P64.T)
    assert np.all(err <= 2e-2 * np.linalg.norm(Qs, axis=1)[:, None] * np.linalg.norm(P64, axis=1)[None, :])
