"""Pins for the FP64 projection-learning oracle (Sec. 2.1-2.4, App. B, App. C)."""
import numpy as np
import pytest

from oracle import fit


def _data(seed=0, n=400, m=300, D=20, shift=True):
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((D, D)))[0]
    s = np.arange(1, D + 1) ** -1.0
    X = (rng.standard_normal((n, D)) * np.sqrt(s)) @ U.T
    if shift:
        O = np.linalg.qr(rng.standard_normal((D, D)))[0]
        Q = (rng.standard_normal((m, D)) * np.sqrt(s)) @ (U @ O).T + 0.3
    else:
        Q = (rng.standard_normal((m, D)) * np.sqrt(s)) @ U.T
    return X, Q


def _stiefel(rng, d, D):
    return np.linalg.qr(rng.standard_normal((D, d)))[0].T


def test_trace_form_equals_frobenius_form():
    X, Q = _data()
    rng = np.random.default_rng(1)
    KX, KQ = fit.second_moment(X), fit.second_moment(Q)
    for _ in range(3):
        A, B = rng.standard_normal((5, 20)), rng.standard_normal((5, 20))
        assert fit.ood_loss(A, B, KQ, KX) == pytest.approx(fit.ood_loss_frobenius(A, B, Q, X), rel=1e-11)


def test_second_moment_two_ways():
    X, _ = _data(n=50)
    K = fit.second_moment(X)
    K2 = sum(np.outer(x, x) for x in X.astype(np.float64))
    np.testing.assert_allclose(K, K2, rtol=1e-12, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(K) > -1e-10)


def test_pca_reconstruction_equals_discarded_eigenvalues():
    """Problem pca: ||X - M^T M X||_F^2 at the PCA solution = sum of discarded eigenvalues of X X^T."""
    X, _ = _data(n=300)
    KX = fit.second_moment(X)
    for d in (1, 5, 12):
        P, w = fit.top_eigvecs(KX, d)
        np.testing.assert_allclose(P @ P.T, np.eye(d), atol=1e-12)
        assert fit.reconstruction_error(P, X) == pytest.approx(w[d:].sum(), rel=1e-9)


def test_identity_projection_is_exact():
    X, Q = _data()
    KX, KQ = fit.second_moment(X), fit.second_moment(Q)
    I = np.eye(20)
    assert abs(fit.ood_loss(I, I, KQ, KX)) <= 1e-9 * np.trace(KQ @ KX)
    gA, gB = fit.ood_grads(I, I, KQ, KX)
    assert np.abs(gA).max() < 1e-9 and np.abs(gB).max() < 1e-9


def test_gradients_match_central_differences():
    X, Q = _data(D=12, n=100, m=80)
    KX, KQ = fit.second_moment(X), fit.second_moment(Q)
    rng = np.random.default_rng(2)
    A, B = rng.standard_normal((4, 12)) * 0.3, rng.standard_normal((4, 12)) * 0.3
    gA, gB = fit.ood_grads(A, B, KQ, KX)
    eps = 1e-6
    for (M, g, which) in ((A, gA, 0), (B, gB, 1)):
        fd = np.zeros_like(M)
        for i in range(M.shape[0]):
            for j in range(M.shape[1]):
                Mp, Mm = M.copy(), M.copy()
                Mp[i, j] += eps
                Mm[i, j] -= eps
                fp = fit.ood_loss(Mp, B, KQ, KX) if which == 0 else fit.ood_loss(A, Mp, KQ, KX)
                fm = fit.ood_loss(Mm, B, KQ, KX) if which == 0 else fit.ood_loss(A, Mm, KQ, KX)
                fd[i, j] = (fp - fm) / (2 * eps)
        assert np.linalg.norm(fd - g) <= 1e-6 * np.linalg.norm(g)


def test_proposition_1_bound():
    """App. B: f(A, B) <= ||Q||_F^2 ||A^T B X - X||_F^2 for A, B in St(D, d)."""
    X, Q = _data()
    rng = np.random.default_rng(3)
    for _ in range(5):
        A, B = _stiefel(rng, 6, 20), _stiefel(rng, 6, 20)
        lhs = fit.ood_loss_frobenius(A, B, Q, X)
        E = X @ B.T @ A - X
        rhs = np.sum(Q * Q) * np.sum(E * E)
        assert lhs <= rhs * (1 + 1e-12)


def test_lmo_attains_nuclear_norm():
    rng = np.random.default_rng(4)
    C = rng.standard_normal((5, 17))
    S = fit.lmo(C)
    assert np.sum(S * C) == pytest.approx(np.linalg.norm(C, "nuc"), rel=1e-12)
    assert fit.op_norm(S) == pytest.approx(1.0, rel=1e-12)
    # no other point of the ball does better
    for _ in range(20):
        T = rng.standard_normal((5, 17))
        T /= fit.op_norm(T)
        assert np.sum(T * C) <= np.sum(S * C) + 1e-12


def test_frank_wolfe_invariants():
    X, Q = _data()
    KX, KQ = fit.second_moment(X), fit.second_moment(Q)
    res = fit.frank_wolfe(KQ, KX, 6, alpha=0.5)
    assert 2 <= res["iterations"] < 200
    assert fit.op_norm(res["A"]) <= 1 + 1e-12 and fit.op_norm(res["B"]) <= 1 + 1e-12
    assert np.all(res["gaps"] >= -1e-9 * res["loss"][0])
    tr = res["loss"]
    assert tr[-1] < tr[0]
    assert abs(tr[-1] - tr[-2]) / tr[-2] <= 1e-3
    # first step from A0 = B0 = 0 lands on the ID solution for A (zero gradient reading)
    r1 = fit.frank_wolfe(KQ, KX, 6, alpha=0.5, max_iter=1)
    np.testing.assert_allclose(r1["A"], fit.fit_id(KX, 6), atol=1e-12)
    # OOD solution beats the ID solution on the OOD loss
    P = fit.fit_id(KX, 6)
    assert tr[-1] <= fit.ood_loss(P, P, KQ, KX)


def test_line_search_is_quadratic_minimiser():
    X, Q = _data(D=10, n=100, m=90)
    KX, KQ = fit.second_moment(X), fit.second_moment(Q)
    rng = np.random.default_rng(5)
    A, B = _stiefel(rng, 3, 10) * 0.5, _stiefel(rng, 3, 10)
    gA, _ = fit.ood_grads(A, B, KQ, KX)
    S = fit.lmo(-gA)
    g = fit._line_search(gA, S, A, B, KQ, KX, "A")
    f = lambda t: fit.ood_loss(A + t * (S - A), B, KQ, KX)
    # fit the parabola through 3 points and compare its minimiser
    c2 = (f(1.0) - 2 * f(0.5) + f(0.0)) / 0.5
    c1 = (f(1.0) - f(0.0)) - c2
    tstar = float(np.clip(-c1 / (2 * c2), 0, 1))
    assert g == pytest.approx(tstar, abs=1e-9)


def test_eigsearch_endpoints_and_id_invariance():
    X, Q = _data(n=500, m=400)
    KX, KQ = fit.second_moment(X), fit.second_moment(Q)
    d = 5
    P1 = fit.es_projection(KQ, KX, 400, 500, d, 1.0)
    P0 = fit.es_projection(KQ, KX, 400, 500, d, 0.0)
    np.testing.assert_allclose(P1.T @ P1, fit.fit_id(KX, d).T @ fit.fit_id(KX, d), atol=1e-10)
    Pq = fit.top_eigvecs(KQ, d)[0]
    np.testing.assert_allclose(P0.T @ P0, Pq.T @ Pq, atol=1e-10)
    # ID case: K_Q/m = K_X/n exactly -> the subspace does not depend on beta (Sec. 2.4)
    Xs = X[:200]
    Kx = fit.second_moment(Xs)
    Pa = fit.es_projection(2 * Kx, Kx, 400, 200, d, 0.2)
    Pb = fit.es_projection(2 * Kx, Kx, 400, 200, d, 0.9)
    np.testing.assert_allclose(Pa.T @ Pa, Pb.T @ Pb, atol=1e-10)
    res = fit.eigsearch(KQ, KX, 400, 500, d)
    assert 0.0 <= res["beta"] <= 1.0
    assert res["loss"] <= min(fit.ood_loss(P1, P1, KQ, KX), fit.ood_loss(P0, P0, KQ, KX)) + 1e-9
    # ES + FW (line search) refines the ES solution only a little (Sec. 2.4)
    fw = fit.frank_wolfe(KQ, KX, d, A0=res["P"], B0=res["P"], line_search=True)
    assert fw["loss"][-1] <= res["loss"] * (1 + 1e-12)


def test_pair_form_equals_trace_form():
    X, Q = _data(n=120, m=70, D=14)
    KX, KQ = fit.second_moment(X), fit.second_moment(Q)
    rng = np.random.default_rng(6)
    A, B = rng.standard_normal((4, 14)), rng.standard_normal((4, 14))
    L, gA, gB = fit.pair_loss_and_grads(A, B, Q, X)
    nm = 120 * 70
    assert L == pytest.approx(fit.ood_loss(A, B, KQ, KX) / nm, rel=1e-10)
    tA, tB = fit.ood_grads(A, B, KQ, KX)
    np.testing.assert_allclose(gA, tA / nm, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(gB, tB / nm, rtol=1e-10, atol=1e-14)


def test_qualitative_claims_on_shifted_queries():
    """The paper's qualitative claims, reproduced by the oracle on a small shifted-query mixture
    (exhaustive ranking by <A q, B x>, no quantisation): (i) the true top 10 is mostly inside the
    top 50 of the reduced scores but much less inside their top 10, which is what the rerank of
    r > k candidates recovers (Sec. 3, re-ranking); (ii) with queries from another distribution the
    learned OOD projections (eigenvector search, Frank-Wolfe) find more of the true neighbours than
    the ID projection (Sec. 3, the OOD results)."""
    import oracle
    import workloads
    w = workloads.make_workload("anisotropic", 20000, 500, 96, 100, cfg=41, ood=True, m_learn=2000)
    X, Q, Ql = w.X, w.Q, w.Q_learn
    KX, KQ = fit.second_moment(X), fit.second_moment(Ql)
    truth, _ = oracle.bruteforce(X, Q, 10)
    Q64, X64 = Q.astype(np.float64), X.astype(np.float64)

    def recall(A, B, kk):
        s = (Q64 @ A.T) @ (X64 @ B.T).T
        top = np.argsort(-s, axis=1, kind="stable")[:, :kk]
        return np.mean([len(set(top[i].tolist()) & set(truth[i].tolist())) / 10 for i in range(len(Q))])

    d = 16
    P = fit.fit_id(KX, d)
    r10, r50 = recall(P, P, 10), recall(P, P, 50)
    assert r50 >= 2 * r10
    es = fit.eigsearch(KQ, KX, Ql.shape[0], X.shape[0], d)
    fw = fit.frank_wolfe(KQ, KX, d)
    assert recall(es["P"], es["P"], 10) >= r10 + 0.03
    assert recall(fw["A"], fw["B"], 10) >= r10 + 0.03
