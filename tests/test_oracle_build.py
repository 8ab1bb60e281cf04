"""Pins for the oracle's build score, RobustPrune and batch-synchronous Vamana."""
import numpy as np
import pytest

import workloads


def _primaries(oracle_lib, n=80, d=12, bits=8, seed=21):
    rng = np.random.default_rng(seed)
    Y = workloads.unit_rows(rng.standard_normal((n, d)))
    return oracle_lib.lvq_encode(Y, oracle_lib.mean_fp32(Y), bits)


def test_splitmix_reference_values(oracle_lib):
    """SplitMix64 (Steele, Lea, Flood 2014) from state 0: the first outputs of the
    published generator are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F."""
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [oracle_lib.splitmix(0, 0, k) for k in range(3)] == expect


def test_build_score_matches_fp64_decode(oracle_lib):
    q = _primaries(oracle_lib)
    bs = oracle_lib.BuildStore(q)
    mu_fix = np.rint(q.mean.astype(np.float64) * 2.0 ** 20) / 2.0 ** 20
    dec = (mu_fix[None, :] + q.lower.astype(np.float64)[:, None]
           + q.delta.astype(np.float64)[:, None] * q.codes.astype(np.float64))
    for a, b in [(0, 1), (5, 5), (7, 70), (33, 12), (79, 0)]:
        ref = float(dec[a] @ dec[b])
        got = float(bs.score(a, b))
        assert got == pytest.approx(ref, rel=2e-5, abs=2e-6)
        assert bs.score(a, b) == bs.score(b, a)  # symmetric bit for bit


def test_robust_prune_unit_l2_rule(oracle_lib):
    """Rule 1 is the L2 rule alpha |p*-p'|^2 <= |p-p'|^2 on unit-norm vectors, written with
    s = <.,.> (|a-b|^2 = 2 - 2 s): brute-force replay with explicit squared distances."""
    rng = np.random.default_rng(30)
    Y = workloads.unit_rows(rng.standard_normal((50, 6)))
    q = oracle_lib.lvq_encode(Y, np.zeros(6, np.float32), 8)
    bs = oracle_lib.BuildStore(q)
    a = 1.3
    out = bs.robust_prune(0, list(range(1, 50)), a, 10, float(np.float32(a) - np.float32(1.0)))
    s = lambda i, j: float(bs.score(i, j))
    order = sorted(range(1, 50), key=lambda u: (-s(0, u), u))
    kept, alive = [], list(order)
    while alive and len(kept) < 10:
        p = alive.pop(0)
        kept.append(p)
        # squared distances of (approximately) unit vectors from the same scores
        alive = [u for u in alive if not (a * (2 - 2 * s(p, u)) <= 2 - 2 * s(0, u) + 1e-6)]
    # the float32 rule and the distance replay agree away from rounding ties
    assert len(set(out.tolist()) ^ set(kept)) <= 1


def test_robust_prune_invariants(oracle_lib):
    q = _primaries(oracle_lib, n=60)
    bs = oracle_lib.BuildStore(q)
    p = 4
    pool = [i for i in range(60) if i != p]
    for alpha in (1.0, 0.95):
        out = bs.robust_prune(p, pool, alpha, 8)
        assert len(out) <= 8 and len(set(out.tolist())) == len(out) and p not in out
        # kept nodes never dominate one another (selection order)
        for i in range(len(out)):
            for j in range(i + 1, len(out)):
                assert not (np.float32(alpha) * bs.score(out[i], out[j]) >= bs.score(p, out[j]))
        # brute force: replay the rule directly
        order = sorted(pool, key=lambda u: (-float(bs.score(p, u)), u))
        alive = list(order)
        kept = []
        while alive and len(kept) < 8:
            s = alive.pop(0)
            kept.append(s)
            alive = [u for u in alive if not (np.float32(alpha) * bs.score(s, u) >= bs.score(p, u))]
        assert out.tolist() == kept


def _python_sequential_vamana(oracle_lib, q, R, L, alpha, passes, seed, rule=0, metric=0):
    """Textbook sequential Vamana (one node at a time), written independently of the
    C batch build: greedy search from the entry, prune, add reverse edges and prune
    any neighbour that overflows."""
    bs = oracle_lib.BuildStore(q, metric)
    n = q.codes.shape[0]
    G = [list(int(u) for u in row if u >= 0) for row in oracle_lib.random_graph(n, R, seed)]
    entry = bs.entry()
    perm = oracle_lib.permutation(n, seed)

    def search(p):
        C = [(float(bs.score(p, entry)), entry)]
        expanded, visited = set(), {entry}
        while True:
            cand = [c for c in C if c[1] not in expanded]
            if not cand:
                return C
            best = min(cand, key=lambda c: (-c[0], c[1]))
            expanded.add(best[1])
            for u in G[best[1]]:
                if u not in visited:
                    visited.add(u)
                    C.append((float(bs.score(p, u)), u))
            C = sorted(C, key=lambda c: (-c[0], c[1]))[:L]

    for t in range(passes):
        a = 1.0 if t < passes - 1 else alpha
        sh = float(np.float32(a) - np.float32(1.0)) if rule else 0.0
        for p in perm:
            p = int(p)
            pool = [u for _, u in search(p) if u != p]
            for u in G[p]:
                if u != p and u not in pool:
                    pool.append(u)
            G[p] = bs.robust_prune(p, pool, a, R, sh).tolist()
            for u in G[p]:
                if p not in G[u] and u != p:
                    G[u].append(p)
                    if len(G[u]) > R:
                        G[u] = bs.robust_prune(u, G[u], a, R, sh).tolist()
    out = np.full((n, R), -1, np.int32)
    for i, row in enumerate(G):
        out[i, :len(row)] = row
    return out, entry


@pytest.mark.parametrize("bits,rule,alpha,metric", [(8, 0, 0.95, 0), (4, 0, 0.95, 0), (8, 1, 1.2, 0),
                                                     (8, 0, 1.2, 1), (4, 0, 1.2, 1)])
def test_batch_one_equals_sequential_vamana(oracle_lib, bits, rule, alpha, metric):
    q = _primaries(oracle_lib, n=70, d=10, bits=bits, seed=22)
    g, e = oracle_lib.vamana_build(q, R=6, L_build=12, alpha=alpha, passes=2, batch=1, seed=77, rule=rule,
                                   metric=metric)
    g2, e2 = _python_sequential_vamana(oracle_lib, q, 6, 12, alpha, 2, 77, rule=rule, metric=metric)
    assert e == e2
    np.testing.assert_array_equal(g, g2)


def test_batched_build_invariants_and_quality(oracle_lib):
    rng = np.random.default_rng(23)
    n, D = 1500, 24
    means = rng.standard_normal((12, D))
    X = workloads.unit_rows(means[rng.integers(0, 12, n)] + 0.3 * rng.standard_normal((n, D)))
    q = oracle_lib.lvq_encode(X, oracle_lib.mean_fp32(X), 8)
    R = 12
    g, entry = oracle_lib.vamana_build(q, R=R, L_build=24, alpha=1.0, passes=2, batch=64, seed=5)
    for i in range(n):
        row = g[i][g[i] >= 0]
        assert len(row) <= R and i not in row and len(set(row.tolist())) == len(row)
        assert (g[i][len(row):] == -1).all()  # padding only at the end
    # deterministic
    g_again, _ = oracle_lib.vamana_build(q, R=R, L_build=24, alpha=1.0, passes=2, batch=64, seed=5)
    np.testing.assert_array_equal(g, g_again)
    # the graph is navigable: recall@10 of a modest beam on ID queries is high
    Q = workloads.unit_rows(means[rng.integers(0, 12, 50)] + 0.3 * rng.standard_normal((50, D)))
    truth, _ = oracle_lib.bruteforce(X, Q, 10)
    res = oracle_lib.search(g, entry, Q.astype(np.float64), k=10, L=40, prim_vecs=X)
    assert oracle_lib.recall(res["ids"], truth, 10) >= 0.9


def test_ip_entry_is_argmax_of_decoded_primary_dot_mean(oracle_lib):
    """Inner product: the entry point is argmax_i <mu, decoded y_i> (the primary with the largest
    inner product with the dataset mean), ties to the smaller id; checked against an independent
    FP64 argmax of the decoded primaries, including a planted tie."""
    rng = np.random.default_rng(44)
    Y = workloads.unit_rows(rng.standard_normal((300, 10)) + np.linspace(0, 2, 10)[None, :])
    q = oracle_lib.lvq_encode(Y, oracle_lib.mean_fp32(Y), 8)
    dec = q.decode().astype(np.float64)
    mu = q.mean.astype(np.float64)
    v = dec @ mu
    top2 = np.sort(v)[-2:]
    assert top2[1] - top2[0] > 1e-4 * np.abs(v).max()  # a unique maximum by a clear margin
    assert oracle_lib.BuildStore(q).entry() == int(np.argmax(v))
    assert oracle_lib.BuildStore(q).entry() != int(np.argmin(v))
    # a tie: the best record copied to a smaller and to a larger id -> the smallest id wins
    b = int(np.argmax(v))
    for dup in (0, 299):
        if dup == b:
            continue
        c2, d2, l2 = q.codes.copy(), q.delta.copy(), q.lower.copy()
        c2[dup], d2[dup], l2[dup] = c2[b], d2[b], l2[b]
        q2 = oracle_lib.LVQ(c2, d2, l2, q.mean, 8)
        assert oracle_lib.BuildStore(q2).entry() == min(dup, b)
