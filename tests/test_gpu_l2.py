"""The Euclidean metric on the GPU against the oracle's L2 reading (scores 2 <q, x> - ||x||^2 with
the original vectors' squared norms; build score -||y_a - y_b||^2; entry nearest the mean):
records bit-exact (codes, constants, self scores N), squared norms within one float32 ulp,
graphs bit-exact, search ids >= 99 % identical and recall within 0.002."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import t, unpack_records

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


def _mixture(n, m, D, comps, seed):
    """Gaussian mixture with unequal norms (no normalisation: the L2 setting)."""
    rng = np.random.default_rng(seed)
    means = rng.standard_normal((comps, D)) * 2.0
    X = means[rng.integers(0, comps, n)] + rng.standard_normal((n, D)) * rng.uniform(0.3, 1.0, (n, 1))
    Q = means[rng.integers(0, comps, m)] + rng.standard_normal((m, D)) * 0.6
    return X.astype(np.float32), Q.astype(np.float32)


def _l2_records(rec, dim, bits):
    co = (dim if bits == 8 else (dim + 1) // 2 + 0)
    co = (co + 15) // 16 * 16
    base = unpack_records(rec, dim, bits)
    nrm = np.ascontiguousarray(rec[:, co + 16:co + 32]).view(np.float32)
    return base, nrm


@pytest.mark.parametrize("dim,bits", [(32, 8), (160, 8), (64, 4), (100, 4)])
def test_l2_records(lv, dim, bits):
    rng = np.random.default_rng(dim + bits)
    n, D = 700, 2 * dim
    X = rng.standard_normal((n, D)).astype(np.float32) * rng.uniform(0.5, 2, (n, 1)).astype(np.float32)
    Y = X[:, :dim].copy()
    mu = oracle.mean_fp32(Y)
    idx = lv.Index(0, metric=lv.METRIC_L2).set_primary(t(Y), t(mu), bits, D)
    rec = idx.primary_records().cpu().numpy()
    co = ((dim if bits == 8 else (dim + 1) // 2) + 15) // 16 * 16
    assert rec.shape[1] == (co + 32 + 31) // 32 * 32
    ref = oracle.lvq_encode(Y, mu, bits)
    (codes, delta, lower, G, H, pad, tail), nrm = _l2_records(rec, dim, bits)
    np.testing.assert_array_equal(codes, ref.codes)
    np.testing.assert_array_equal(delta, ref.delta)
    np.testing.assert_array_equal(lower, ref.lower)
    bs = oracle.BuildStore(ref, metric=1)
    np.testing.assert_array_equal(G, bs.G)
    np.testing.assert_array_equal(nrm[:, 0], bs.N)                # N = <y, y>, bit-exact
    np.testing.assert_array_equal(nrm[:, 1], bs.N)                # ||x||^2 defaults to N
    assert not nrm[:, 2:].any()
    # the original vectors set ||x||^2 in both stores
    idx.set_secondary(t(X))
    rec = idx.primary_records().cpu().numpy()
    _, nrm = _l2_records(rec, dim, bits)
    want = oracle.sqnorms_fp32(X)
    assert np.all(np.abs(nrm[:, 1] - want) <= np.spacing(want))
    srec = idx.secondary_records().cpu().numpy()
    _, snrm = _l2_records(srec, D, 8)
    assert np.all(np.abs(snrm[:, 1] - want) <= np.spacing(want))


def _prims(n, d, bits, seed):
    rng = np.random.default_rng(seed)
    means = rng.standard_normal((15, d)) * 2
    Y = (means[rng.integers(0, 15, n)] + rng.standard_normal((n, d))).astype(np.float32)
    mu = oracle.mean_fp32(Y)
    return Y, mu, oracle.lvq_encode(Y, mu, bits)


@pytest.mark.parametrize("n,d,bits,R,Lb,alpha,batch", [
    (600, 16, 8, 8, 16, 1.2, 1),
    (900, 24, 8, 16, 32, 1.2, 64),
    (800, 24, 4, 12, 24, 1.2, 100),
    (777, 40, 8, 32, 64, 1.3, 128),     # R > 32, ragged sizes
    (400, 256, 8, 16, 32, 1.2, 50),     # long records: a whole warp per record
])
def test_l2_build_bit_exact(lv, n, d, bits, R, Lb, alpha, batch):
    Y, mu, q = _prims(n, d, bits, seed=n + d)
    g_ref, e_ref = oracle.vamana_build(q, R=R, L_build=Lb, alpha=alpha, passes=2, batch=batch, seed=42, metric=1)
    idx = lv.Index(0, metric=lv.METRIC_L2).set_primary(t(Y), t(mu), bits, d)
    idx.build_graph(R=R, L_build=Lb, alpha=alpha, passes=2, batch=batch, seed=42)
    idx.sync_status()
    g, e = idx.get_graph()
    assert e == e_ref
    np.testing.assert_array_equal(g.cpu().numpy(), g_ref)


@pytest.fixture(scope="module")
def pb():
    from oracle import fit
    X, Q = _mixture(3000, 300, 64, 25, 7)
    d = 16
    P = fit.fit_id(fit.second_moment(X), d).astype(np.float32)
    Y = (X.astype(np.float64) @ P.T.astype(np.float64)).astype(np.float32)
    mu_p, mu_s = oracle.mean_fp32(Y), oracle.mean_fp32(X)
    prim = oracle.lvq_encode(Y, mu_p, 8)
    sec = oracle.lvq_encode(X, mu_s, 8)
    graph, entry = oracle.vamana_build(prim, R=16, L_build=32, alpha=1.2, passes=2, batch=256, seed=5000, metric=1)
    return dict(X=X, Q=Q, P=P, Y=Y, mu_p=mu_p, mu_s=mu_s, prim=prim, sec=sec, graph=graph, entry=entry,
                nrm=oracle.sqnorms_fp32(X))


def _check_l2_scores(ids, scores, dec, qv, nrm, tol=1e-4):
    for j in range(ids.shape[0]):
        sel = ids[j] >= 0
        u = ids[j][sel]
        exact = 2.0 * (dec[u] @ qv[j]) - nrm[u].astype(np.float64)
        bound = 2 * tol * np.linalg.norm(qv[j]) * np.linalg.norm(dec[u], axis=1) + 4 * np.spacing(nrm[u])
        assert np.all(np.abs(scores[j][sel] - exact) <= bound), (j, np.abs(scores[j][sel] - exact).max())


@pytest.mark.parametrize("W", [1, 2])
def test_l2_search_and_rerank_match_oracle(lv, pb, W):
    idx = lv.Index(0, metric=lv.METRIC_L2)
    idx.set_primary(t(pb["Y"]), t(pb["mu_p"]), 8, 64).set_secondary(t(pb["X"]), t(pb["mu_s"]))
    idx.set_graph(t(pb["graph"]), pb["entry"])
    Qd = pb["Q"].astype(np.float64)
    qp = Qd @ pb["P"].T.astype(np.float64)
    for L, r in ((40, 0), (64, 64)):
        ids, sc = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=L, rerank=r, width=W)
        idx.sync_status()
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
        ref = oracle.search(pb["graph"], pb["entry"], qp, k=10, L=L, rerank=r, prim=pb["prim"], sec=pb["sec"],
                            qs=Qd, metric=1, sqnorm=pb["nrm"], width=W)
        assert (ids == ref["ids"]).mean() >= 0.99
        truth, _ = oracle.bruteforce(pb["X"], pb["Q"], 10, metric=1)
        assert abs(oracle.recall(ids, truth, 10) - oracle.recall(ref["ids"], truth, 10)) <= 0.002
        if r:
            _check_l2_scores(ids, sc, pb["sec"].decode(), Qd, pb["nrm"])
        else:
            _check_l2_scores(ids, sc, pb["prim"].decode(), qp, pb["nrm"])
    # the no-allocation entry point gives the same ids
    a, _ = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48)
    b, _ = idx.search_noalloc(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48)
    assert torch.equal(a, b)


def test_l2_fp16_secondaries_and_fp32_baseline(lv, pb):
    X16 = pb["X"].astype(np.float16).astype(np.float32)
    idx = lv.Index(0, metric=lv.METRIC_L2).encode(t(pb["X"]), t(pb["P"]), 8, 16)
    idx.set_primary(t(pb["Y"]), t(pb["mu_p"]), 8, 64).set_graph(t(pb["graph"]), pb["entry"])
    Qd = pb["Q"].astype(np.float64)
    qp = Qd @ pb["P"].T.astype(np.float64)
    ids, sc = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48)
    ids = ids.cpu().numpy()
    # primary ||x||^2 = N after set_primary (no original vectors given): the oracle uses the same
    nrm_prim = oracle.BuildStore(pb["prim"], metric=1).N
    ref = oracle.search(pb["graph"], pb["entry"], qp, k=10, L=48, rerank=48, prim=pb["prim"], sec_vecs=X16, qs=Qd,
                        metric=1, sqnorm=nrm_prim)
    assert (ids == ref["ids"]).mean() >= 0.99
    # FP16 rerank scores: 2 <q, x16> - ||x16||^2 of the halves themselves
    for j in range(ids.shape[0]):
        u = ids[j]
        exact = 2.0 * (X16[u].astype(np.float64) @ Qd[j]) - (X16[u].astype(np.float64) ** 2).sum(1)
        assert np.all(np.abs(sc.cpu().numpy()[j] - exact) <= 1e-4 * (1 + np.abs(exact)))
    # full-dimensional float32 records with the L2 metric
    base = lv.Index(0, metric=lv.METRIC_L2).encode_fp32(t(pb["X"])).set_graph(t(pb["graph"]), pb["entry"])
    ids2, _ = base.search(t(pb["Q"]), None, k=10, L=40)
    ref2 = oracle.search(pb["graph"], pb["entry"], Qd, k=10, L=40, prim_vecs=pb["X"], metric=1)
    assert (ids2.cpu().numpy() == ref2["ids"]).mean() >= 0.99


def test_l2_set_metric_errors(lv, pb):
    idx = lv.Index(0).set_primary(t(pb["Y"]), t(pb["mu_p"]), 8, 64)
    with pytest.raises(lv.LeanVecError):
        lv._native.check(lv._native.lib().leanvec_set_metric(idx.handle, 1))
    with pytest.raises(lv.LeanVecError):
        lv.Index(0, metric=3)
