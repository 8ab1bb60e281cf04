"""Pins for the oracle's LVQ, scores, beam search, rerank and brute force.

Each check ties the oracle to something other than itself: hand-worked LVQ
examples, the LVQ error bound, closed-form score identities, brute force on tiny
inputs, and the L >= n property of best-first search."""
import json
import os

import numpy as np
import pytest

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def test_lvq_worked_examples(oracle_lib):
    g = json.load(open(os.path.join(HERE, "golden", "lvq_worked_examples.json")))
    for case in g["cases"]:
        y = np.array([case["y"]], np.float32)
        mean = np.array(case["mean"], np.float32)
        q = oracle_lib.lvq_encode(y, mean, case["bits"])
        assert q.codes[0].tolist() == case["codes"]
        assert q.delta[0] == pytest.approx(case["delta"], rel=1e-6, abs=1e-12)
        assert q.lower[0] == pytest.approx(case["lower"], rel=1e-6, abs=1e-7)


@pytest.mark.parametrize("bits", [8, 4, 2])
def test_lvq_error_bound_and_extremes(oracle_lib, bits):
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((300, 37)).astype(np.float32)
    mean = oracle_lib.mean_fp32(Y)
    q = oracle_lib.lvq_encode(Y, mean, bits)
    V = (Y.astype(np.float64) - mean.astype(np.float64))
    dec = q.decode() - mean.astype(np.float64)[None, :]
    err = np.abs(dec - V)
    bound = q.delta.astype(np.float64)[:, None] / 2 + 4e-7 * (np.abs(V) + 1)
    assert np.all(err <= bound)
    levels = (1 << bits) - 1
    # the minimum coordinate maps to code 0 and the maximum to the top code
    assert np.all(q.codes[np.arange(300), np.argmin(V, axis=1)] == 0)
    assert np.all(q.codes[np.arange(300), np.argmax(V, axis=1)] == levels)
    assert q.codes.max() <= levels


def test_primary_score_formula(oracle_lib):
    """<q', decode(c)> equals c_q + l * sum(q') + delta * <q', c> (decode is affine)."""
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((50, 16)).astype(np.float32)
    mean = oracle_lib.mean_fp32(Y)
    q = oracle_lib.lvq_encode(Y, mean, 8)
    qp = rng.standard_normal(16)
    direct = q.decode() @ qp
    formula = (qp @ mean.astype(np.float64) + q.lower.astype(np.float64) * qp.sum()
               + q.delta.astype(np.float64) * (q.codes.astype(np.float64) @ qp))
    np.testing.assert_allclose(direct, formula, rtol=1e-12, atol=1e-12)


def _connected_graph(n, R, seed):
    import oracle
    g = oracle.random_graph(n, R, seed)
    # add a ring so that every node is reachable from every other
    g[:, 0] = (np.arange(n) + 1) % n
    return g


def _reachable(graph, entry):
    seen = {entry}
    st = [entry]
    while st:
        p = st.pop()
        for u in graph[p]:
            if u >= 0 and u not in seen:
                seen.add(int(u))
                st.append(int(u))
    return seen


def test_beam_search_full_window_equals_bruteforce(oracle_lib):
    """With L >= n, best-first search scores every node reachable from the entry, so
    its top-k equals the brute-force top-k of the same score over those nodes."""
    rng = np.random.default_rng(11)
    n, D, m = 200, 24, 12
    Y = rng.standard_normal((n, D)).astype(np.float32)
    mean = oracle_lib.mean_fp32(Y)
    q = oracle_lib.lvq_encode(Y, mean, 8)
    g = oracle_lib.random_graph(n, 4, 5)
    entry = 3
    reach = np.array(sorted(_reachable(g, entry)))
    qp = rng.standard_normal((m, D))
    res = oracle_lib.search(g, entry, qp, k=10, L=n, prim=q, want_beam=True)
    dec = q.decode()
    for j in range(m):
        s = dec[reach] @ qp[j]
        order = np.lexsort((reach, -s))
        np.testing.assert_array_equal(res["ids"][j], reach[order[:10]])
        np.testing.assert_allclose(res["scores"][j], s[order[:10]], rtol=1e-12)
        assert res["beam_ids"][j, len(reach):].tolist() == [-1] * (n - len(reach))


def test_search_width_full_window_and_python_replay(oracle_lib):
    """Any search width explores every reachable node when L >= n; at small L the C
    oracle equals a direct Python replay of the width-W rule."""
    rng = np.random.default_rng(16)
    n, D = 150, 12
    X = rng.standard_normal((n, D)).astype(np.float32)
    g = _connected_graph(n, 5, 3)
    qp = rng.standard_normal((6, D))
    full1 = oracle_lib.search(g, 0, qp, k=10, L=n, prim_vecs=X)
    for W in (2, 4):
        fullW = oracle_lib.search(g, 0, qp, k=10, L=n, prim_vecs=X, width=W)
        np.testing.assert_array_equal(fullW["ids"], full1["ids"])
    S = qp @ X.astype(np.float64).T
    for W in (1, 3):
        res = oracle_lib.search(g, 0, qp, k=5, L=12, prim_vecs=X, width=W)
        for j in range(6):
            C = {0: S[j, 0]}
            exp, vis = set(), {0}
            while True:
                order = sorted(C, key=lambda u: (-C[u], u))
                par = [u for u in order if u not in exp][:W]
                if not par:
                    break
                exp.update(par)
                for p in par:
                    for u in g[p]:
                        if u >= 0 and u not in vis:
                            vis.add(int(u))
                            C[int(u)] = S[j, u]
                C = {u: C[u] for u in sorted(C, key=lambda u: (-C[u], u))[:12]}
            top = sorted(C, key=lambda u: (-C[u], u))[:5]
            assert res["ids"][j].tolist() == top


def test_identity_projection_exact_search(oracle_lib):
    """A = B = I at d = D with raw fp32 primaries: the full-window search equals the
    exact brute force over X (Sec. 2: the approximation becomes an identity)."""
    rng = np.random.default_rng(12)
    n, D = 150, 16
    X = workloads.unit_rows(rng.standard_normal((n, D)))
    Q = workloads.unit_rows(rng.standard_normal((9, D)))
    g = _connected_graph(n, 5, 9)
    A = np.eye(D)
    res = oracle_lib.search(g, 0, Q.astype(np.float64) @ A.T, k=7, L=n, prim_vecs=X)
    bf_ids, bf_sc = oracle_lib.bruteforce(X, Q, 7)
    np.testing.assert_array_equal(res["ids"], bf_ids)
    np.testing.assert_allclose(res["scores"], bf_sc, rtol=1e-12)


def test_bruteforce_against_numpy(oracle_lib):
    rng = np.random.default_rng(13)
    X = rng.standard_normal((300, 20)).astype(np.float32)
    Q = rng.standard_normal((15, 20)).astype(np.float32)
    X[17] = X[5]  # an exact tie: the smaller id must come first
    Q[0] = X[5]
    ids, sc = oracle_lib.bruteforce(X, Q, 10)
    S = Q.astype(np.float64) @ X.astype(np.float64).T
    for j in range(15):
        order = np.lexsort((np.arange(300), -S[j]))[:10]
        np.testing.assert_array_equal(ids[j], order)
    assert ids[0, 0] == 5 and ids[0, 1] == 17


def test_rerank_uses_secondary_scores(oracle_lib):
    """The rerank returns the top-k of the secondary score among the top-r primary
    candidates; with r = L >= n that is the brute-force top-k of the secondary."""
    rng = np.random.default_rng(14)
    n, D, d = 120, 32, 6
    Y = workloads.unit_rows(rng.standard_normal((n, D)))
    mean = oracle_lib.mean_fp32(Y)
    sec = oracle_lib.lvq_encode(Y, mean, 8)
    P = np.linalg.qr(rng.standard_normal((D, d)))[0].T
    Yp = (Y.astype(np.float64) @ P.T).astype(np.float32)
    prim = oracle_lib.lvq_encode(Yp, oracle_lib.mean_fp32(Yp), 8)
    g = _connected_graph(n, 4, 2)
    Q = workloads.unit_rows(rng.standard_normal((5, D))).astype(np.float64)
    res = oracle_lib.search(g, 0, Q @ P.T, k=5, L=n, rerank=n, prim=prim, sec=sec, qs=Q)
    dec = sec.decode()
    for j in range(5):
        s = dec @ Q[j]
        order = np.lexsort((np.arange(n), -s))[:5]
        np.testing.assert_array_equal(res["ids"][j], order)
    # recall@10 of the primary alone is below the reranked recall (Sec. 3 "Re-ranking")
    assert res["ids"].shape == (5, 5)


def test_rerank_with_raw_secondary_vectors(oracle_lib):
    """Raw secondary vectors (the FP16 secondaries' exact values): with r = L >= n the result is the
    brute-force top-k of <q, x16> over all nodes, i.e. numpy on the half-rounded vectors."""
    rng = np.random.default_rng(16)
    n, D, d = 100, 24, 5
    X = workloads.unit_rows(rng.standard_normal((n, D))).astype(np.float32)
    X16 = X.astype(np.float16).astype(np.float32)  # IEEE round to nearest even, exact widening
    assert np.abs(X16 - X).max() <= 2.0 ** -11 * np.abs(X).max() * 1.0001
    P = np.linalg.qr(rng.standard_normal((D, d)))[0].T
    Yp = (X.astype(np.float64) @ P.T).astype(np.float32)
    prim = oracle_lib.lvq_encode(Yp, oracle_lib.mean_fp32(Yp), 8)
    Q = workloads.unit_rows(rng.standard_normal((4, D))).astype(np.float64)
    res = oracle_lib.search(_connected_graph(n, 4, 3), 0, Q @ P.T, k=6, L=n, rerank=n, prim=prim, sec_vecs=X16, qs=Q)
    for j in range(4):
        s = X16.astype(np.float64) @ Q[j]
        order = np.lexsort((np.arange(n), -s))[:6]
        np.testing.assert_array_equal(res["ids"][j], order)
        np.testing.assert_allclose(res["scores"][j], s[order], rtol=0, atol=1e-12)


def test_padding_and_max_hops(oracle_lib):
    rng = np.random.default_rng(15)
    n, D = 30, 8
    X = rng.standard_normal((n, D)).astype(np.float32)
    g = np.full((n, 3), -1, np.int32)
    g[0, :2] = [1, 2]  # entry reaches only {0, 1, 2}
    res = oracle_lib.search(g, 0, rng.standard_normal((2, D)), k=5, L=10, prim_vecs=X)
    assert (res["ids"][:, 3:] == -1).all() and np.isinf(res["scores"][:, 3:]).all()
    assert set(res["ids"][0, :3].tolist()) == {0, 1, 2}
    res2 = oracle_lib.search(_connected_graph(n, 3, 1), 0, rng.standard_normal((2, D)), k=3, L=10,
                             prim_vecs=X, max_hops=2)
    assert (res2["hops"] <= 2).all()


def test_recall_definition(oracle_lib):
    found = np.array([[1, 2, 3, 4], [5, 6, -1, -1]])
    truth = np.array([[4, 3, 9, 8], [5, 6, 7, 8]])
    assert oracle_lib.recall(found, truth, 4) == pytest.approx((2 + 2) / 8)


def test_encode_parallel_equals_one_call(oracle_lib):
    """The threaded block encode the full-size GPU tests use for the oracle's stores gives the
    codes and constants of one oracle call (blocks of unequal length, both widths)."""
    from gpu_util import encode_parallel
    rng = np.random.default_rng(21)
    Y = rng.standard_normal((1003, 37)).astype(np.float32)
    mu = Y.astype(np.float64).mean(axis=0).astype(np.float32)
    for bits in (4, 8):
        one = oracle_lib.lvq_encode(Y, mu, bits)
        par = encode_parallel(oracle_lib, Y, mu, bits, parts=7)
        assert np.array_equal(one.codes, par.codes)
        assert np.array_equal(one.delta, par.delta) and np.array_equal(one.lower, par.lower)
