"""Pins for the oracle's Euclidean metric: scores are 2 <q, x> - ||x||^2, which ranks like
-||q - x||^2 (the query's norm is constant per query); the build score is -||y_a - y_b||^2
between decoded primaries in the fixed FP32 arithmetic; the entry point is the primary nearest
the mean."""
import numpy as np
import pytest

import oracle
import workloads


@pytest.fixture(scope="module")
def oracle_lib():
    return oracle


def _data(n, D, seed, scale=True):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, D)) * (rng.uniform(0.5, 2.0, (n, 1)) if scale else 1.0)
    return X.astype(np.float32)


def test_sqnorms_fp64(oracle_lib):
    X = _data(50, 33, 1)
    np.testing.assert_array_equal(oracle_lib.sqnorms_fp32(X),
                                  np.array([np.dot(x.astype(np.float64), x.astype(np.float64)) for x in X],
                                           np.float64).astype(np.float32))


def test_l2_bruteforce_against_numpy_distances(oracle_lib):
    X, Q = _data(300, 20, 2), _data(7, 20, 3)
    ids, sc = oracle_lib.bruteforce(X, Q, 10, metric=1)
    Xd, Qd = X.astype(np.float64), Q.astype(np.float64)
    for j in range(Q.shape[0]):
        dist = ((Xd - Qd[j]) ** 2).sum(1)
        order = np.lexsort((np.arange(X.shape[0]), dist))[:10]
        np.testing.assert_array_equal(ids[j], order)
        # score = ||q||^2 - ||q - x||^2
        np.testing.assert_allclose(sc[j], (Qd[j] @ Qd[j]) - dist[order], rtol=0, atol=1e-9)


def _connected_graph(n, R, seed):
    rng = np.random.default_rng(seed)
    g = np.full((n, R), -1, np.int32)
    for i in range(n):
        nb = [(i + 1) % n] + list(rng.choice(n, R - 1, replace=False))
        nb = list(dict.fromkeys(u for u in nb if u != i))[:R]
        g[i, :len(nb)] = nb
    return g


def test_l2_full_window_search_is_bruteforce(oracle_lib):
    """Raw fp32 primaries, L = n, no projection: the beam holds every node and the top k is the
    exact Euclidean top k."""
    n, D = 150, 12
    X, Q = _data(n, D, 4), _data(5, D, 5)
    res = oracle_lib.search(_connected_graph(n, 4, 6), 0, Q.astype(np.float64), k=8, L=n, prim_vecs=X, metric=1)
    bf, bsc = oracle_lib.bruteforce(X, Q, 8, metric=1)
    np.testing.assert_array_equal(res["ids"], bf)
    np.testing.assert_allclose(res["scores"], bsc, rtol=0, atol=1e-9)


def test_l2_lvq_scores_use_the_original_norms(oracle_lib):
    """LVQ primaries: the L2 score is 2 <q', decode(y)> - ||x||^2 with the stored original norm."""
    n, D, d = 80, 16, 6
    X, Q = _data(n, D, 7), _data(4, D, 8)
    P = np.linalg.qr(np.random.default_rng(9).standard_normal((D, d)))[0].T
    Y = (X.astype(np.float64) @ P.T).astype(np.float32)
    prim = oracle_lib.lvq_encode(Y, oracle_lib.mean_fp32(Y), 8)
    nrm = oracle_lib.sqnorms_fp32(X)
    qp = Q.astype(np.float64) @ P.T
    res = oracle_lib.search(_connected_graph(n, 4, 10), 0, qp, k=n, L=n, prim=prim, metric=1, sqnorm=nrm,
                            want_beam=True)
    dec = prim.decode()
    for j in range(4):
        ids = res["beam_ids"][j]
        exact = 2.0 * (dec[ids] @ qp[j]) - nrm[ids].astype(np.float64)
        np.testing.assert_allclose(res["beam_scores"][j], exact, rtol=0, atol=1e-9)


def _prims(oracle_lib, n, d, bits, seed):
    X = _data(n, d, seed)
    return oracle_lib.lvq_encode(X, oracle_lib.mean_fp32(X), bits)


@pytest.mark.parametrize("bits", [8, 4])
def test_l2_build_score_is_negative_squared_distance(oracle_lib, bits):
    q = _prims(oracle_lib, 60, 24, bits, 11)
    bs = oracle_lib.BuildStore(q, metric=1)
    dec = q.decode()
    nrm = (dec * dec).sum(1)
    for a, b in [(0, 1), (3, 17), (59, 2), (8, 8)]:
        s = bs.score(a, b)
        exact = -((dec[a] - dec[b]) ** 2).sum()
        assert abs(float(s) - exact) <= 16 * 2.0 ** -24 * (nrm[a] + nrm[b]), (a, b, s, exact)
        assert bs.score(a, b) == bs.score(b, a)  # symmetric bit for bit
    assert bs.score(5, 5) == 0.0


def test_l2_entry_is_the_primary_nearest_the_mean(oracle_lib):
    q = _prims(oracle_lib, 200, 16, 8, 12)
    bs = oracle_lib.BuildStore(q, metric=1)
    dec = q.decode()
    mu = q.mean.astype(np.float64)
    d2 = ((dec - mu) ** 2).sum(1)
    assert bs.entry() == int(np.argmin(d2))


def test_l2_prune_keeps_vamana_invariant(oracle_lib):
    """Kept neighbours satisfy Vamana's rule on squared distances: for kept p_i before p_j,
    alpha d(p_i, p_j) > d(p, p_j) (else p_j would have been dropped)."""
    q = _prims(oracle_lib, 120, 12, 8, 13)
    bs = oracle_lib.BuildStore(q, metric=1)
    dec = q.decode().astype(np.float64)
    p, alpha = 0, 1.2
    pool = list(range(1, 120))
    kept = bs.robust_prune(p, pool, alpha, 16)
    assert 0 < len(kept) <= 16 and len(set(kept)) == len(kept) and p not in kept

    def d(a, b):
        return ((dec[a] - dec[b]) ** 2).sum()
    for i in range(len(kept)):
        for j in range(i + 1, len(kept)):
            assert alpha * d(kept[i], kept[j]) >= d(p, kept[j]) * (1 - 1e-5)
    # the first kept one is the nearest pool member
    assert kept[0] == min(pool, key=lambda u: (d(p, u), u))


def test_l2_build_invariants_and_search_quality(oracle_lib):
    rng = np.random.default_rng(14)
    n, D = 1200, 16
    means = rng.standard_normal((12, D)) * 3
    X = (means[rng.integers(0, 12, n)] + rng.standard_normal((n, D))).astype(np.float32)
    q = oracle_lib.lvq_encode(X, oracle_lib.mean_fp32(X), 8)
    g, e = oracle_lib.vamana_build(q, R=16, L_build=32, alpha=1.2, passes=2, batch=128, seed=15, metric=1)
    assert g.shape == (n, 16)
    for i in range(n):
        row = g[i][g[i] >= 0]
        assert i not in row and len(set(row.tolist())) == len(row)
    Q = (means[rng.integers(0, 12, 50)] + rng.standard_normal((50, D))).astype(np.float32)
    nrm = oracle_lib.sqnorms_fp32(X)
    res = oracle_lib.search(g, e, Q.astype(np.float64), k=10, L=64, prim=q, metric=1, sqnorm=nrm)
    truth, _ = oracle_lib.bruteforce(X, Q, 10, metric=1)
    assert oracle_lib.recall(res["ids"], truth, 10) >= 0.9
