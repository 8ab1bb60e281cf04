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


def test_fit_id_matches_oracle_subspace(lv):
    import workloads
    w = workloads.make_workload("anisotropic", 20000, 10, 256, 50, cfg=9)
    d = 48
    A = lv.leanvec_fit_id(t(w.X), d).cpu().numpy().astype(np.float64)
    P = fit.fit_id(fit.second_moment(w.X), d)
    # compare the projectors (robust to sign/rotation within degenerate eigenspaces)
    assert np.linalg.norm(A.T @ A - P.T @ P) <= 1e-3 * np.sqrt(d)
    assert np.abs(A @ A.T - np.eye(d)).max() <= 1e-5
