"""Second moments, the FP64 Jacobi eigensolver and LeanVec-ID on the GPU against the
FP64 oracle (oracle.fit)."""
import numpy as np
import pytest
import torch

from gpu_util import t
from oracle import fit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


@pytest.mark.parametrize("n,D", [(1, 5), (1000, 64), (4097, 130), (20000, 768)])
def test_second_moment_fp32(lv, n, D):
    rng = np.random.default_rng(n + D)
    X = rng.standard_normal((n, D)).astype(np.float32)
    K = lv.leanvec_second_moment(t(X)).cpu().numpy().astype(np.float64)
    ref = fit.second_moment(X)
    norms = np.linalg.norm(X, axis=0)
    # float32 accumulation of n products: error grows like 2^-24 * sqrt(n) * |X_a| |X_b|
    tol = 4 * 2.0 ** -24 * np.sqrt(max(n, 16)) * np.outer(norms, norms)
    assert np.all(np.abs(K - ref) <= tol)


@pytest.mark.parametrize("D", [2, 7, 64, 129, 512])
def test_eigh_fp64(lv, D):
    rng = np.random.default_rng(D)
    G = rng.standard_normal((D, D))
    K = G @ G.T / D + np.diag(np.linspace(0, 1, D))
    w, V = lv.leanvec_eigh(torch.from_numpy(K).cuda())
    w, V = w.cpu().numpy(), V.cpu().numpy()
    P, wref = fit.top_eigvecs(K, D)
    np.testing.assert_allclose(w, wref, rtol=1e-11, atol=1e-12 * wref[0])
    # eigen-equation and orthonormality in FP64
    assert np.abs(V @ K - w[:, None] * V).max() <= 1e-10 * wref[0]
    assert np.abs(V @ V.T - np.eye(D)).max() <= 1e-11
    # same sign convention as the oracle (for well separated eigenvalues)
    gaps = np.abs(np.diff(wref))
    sep = np.concatenate([[np.inf], gaps]) > 1e-6 * wref[0]
    sep &= np.concatenate([gaps, [np.inf]]) > 1e-6 * wref[0]
    np.testing.assert_allclose(V[sep], P[sep], atol=1e-8)


def _check_top(w, V, K, nout, ortho=1e-11):
    P, wref = fit.top_eigvecs(K, nout)
    np.testing.assert_allclose(w, wref[:nout], rtol=1e-11, atol=1e-12 * abs(wref[0]))
    assert np.abs(V @ K - w[:, None] * V).max() <= 1e-10 * abs(wref[0])
    assert np.abs(V @ V.T - np.eye(nout)).max() <= ortho
    return P, wref


@pytest.mark.parametrize("D,nout", [(8, 3), (64, 16), (129, 40), (512, 160), (768, 160), (300, 299)])
def test_eigh_top_fp64(lv, D, nout):
    """The nout leading eigenpairs by tridiagonal reduction, bisection and inverse iteration: the
    oracle's eigenvalues, the eigen-equation and orthonormality in FP64, the oracle's sign
    convention for separated eigenvalues."""
    rng = np.random.default_rng(D * 3 + nout)
    G = rng.standard_normal((D, D))
    K = G @ G.T / D + np.diag(np.linspace(0, 1, D))
    w, V = lv.leanvec_eigh_top(torch.from_numpy(K).cuda(), nout)
    w, V = w.cpu().numpy(), V.cpu().numpy()
    P, wref = _check_top(w, V, K, nout)
    gaps = np.abs(np.diff(wref))[:nout]
    sep = np.concatenate([[np.inf], gaps[:nout - 1]]) > 1e-6 * wref[0]
    sep &= gaps > 1e-6 * wref[0]
    np.testing.assert_allclose(V[sep], P[sep], atol=1e-8)


def test_eigh_top_close_and_repeated_eigenvalues(lv):
    """A 1/i spectrum (gaps down to 4e-5 of the largest eigenvalue among the leading 160), exactly
    repeated eigenvalues (multiplicities 3 and 2: the computed vectors span the eigenspace), and a
    rank-deficient second moment (40 rows, D = 128, 60 pairs: a cluster of 20 zero eigenvalues)."""
    rng = np.random.default_rng(41)
    D = 768
    Qm, _ = np.linalg.qr(rng.standard_normal((D, D)))
    K = (Qm * (1.0 / np.arange(1, D + 1))) @ Qm.T
    K = (K + K.T) / 2
    w, V = lv.leanvec_eigh_top(torch.from_numpy(K).cuda(), 160)
    _check_top(w.cpu().numpy(), V.cpu().numpy(), K, 160, ortho=1e-10)
    lam = np.concatenate([[3.0, 3.0, 3.0, 2.0, 2.0], np.linspace(1.5, 0.1, 59)])
    Qm, _ = np.linalg.qr(rng.standard_normal((64, 64)))
    K = (Qm * lam) @ Qm.T
    K = (K + K.T) / 2
    w, V = lv.leanvec_eigh_top(torch.from_numpy(K).cuda(), 10)
    w, V = w.cpu().numpy(), V.cpu().numpy()
    _check_top(w, V, K, 10)
    for a, b in ((0, 3), (3, 5)):
        np.testing.assert_allclose(V[a:b].T @ V[a:b], Qm[:, a:b] @ Qm[:, a:b].T, atol=1e-10)
    X = rng.standard_normal((40, 128))
    K = X.T @ X
    w, V = lv.leanvec_eigh_top(torch.from_numpy(K).cuda(), 60)
    w, V = w.cpu().numpy(), V.cpu().numpy()
    _check_top(w, V, K, 60)
    assert np.abs(w[40:]).max() <= 1e-12 * w[0]


def test_fit_id_matches_oracle_subspace(lv):
    import workloads
    w = workloads.make_workload("anisotropic", 20000, 10, 256, 50, cfg=9)
    d = 48
    A = lv.leanvec_fit_id(t(w.X), d).cpu().numpy().astype(np.float64)
    P = fit.fit_id(fit.second_moment(w.X), d)
    # compare the projectors (robust to sign/rotation within degenerate eigenspaces)
    assert np.linalg.norm(A.T @ A - P.T @ P) <= 1e-3 * np.sqrt(d)
    assert np.abs(A @ A.T - np.eye(d)).max() <= 1e-5
