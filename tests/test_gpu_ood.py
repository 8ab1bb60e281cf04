"""LeanVec-OOD on the GPU against the FP64 oracle (oracle.fit):
Frank-Wolfe BCD, eigenvector search, ES + FW, the pair-tile loss forward / backward
(differentiation form), its autograd.Function, and the spectral-norm projection."""
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


@pytest.fixture(scope="module")
def data():
    import workloads
    w = workloads.make_workload("anisotropic", 6000, 2000, 64, 40, cfg=31, ood=True, m_learn=3000)
    X, Ql = w.X, w.Q_learn
    return X, Ql, fit.second_moment(X), fit.second_moment(Ql)


def test_frank_wolfe_matches_oracle(lv, data):
    X, Q, KX, KQ = data
    d = 12
    A, B, rep = lv.leanvec_fit_ood(t(X), t(Q), d, method=lv.FIT_FW, alpha=0.5, tol=1e-3)
    ref = fit.frank_wolfe(KQ, KX, d, alpha=0.5, tol=1e-3)
    A, B = A.cpu().numpy().astype(np.float64), B.cpu().numpy().astype(np.float64)
    f = fit.ood_loss(A, B, KQ, KX)
    # same reading of Algorithm 1 -> same trajectory up to float32 gradient rounding
    assert abs(rep["iterations"] - ref["iterations"]) <= 2
    assert f == pytest.approx(ref["loss"][-1], rel=2e-3)
    assert rep["loss"] == pytest.approx(f, rel=1e-4)
    assert np.linalg.norm(A - ref["A"]) <= 2e-2 * np.linalg.norm(ref["A"])
    assert fit.op_norm(A) <= 1 + 1e-4 and fit.op_norm(B) <= 1 + 1e-4
    tr = rep["loss_trace"]
    assert len(tr) == rep["iterations"] + 1 and tr[-1] < tr[0]


def test_eigenvector_search_matches_oracle(lv, data):
    X, Q, KX, KQ = data
    d = 12
    A, B, rep = lv.leanvec_fit_ood(t(X), t(Q), d, method=lv.FIT_ES)
    ref = fit.eigsearch(KQ, KX, Q.shape[0], X.shape[0], d)
    A = A.cpu().numpy().astype(np.float64)
    assert torch.equal(torch.from_numpy(A), torch.from_numpy(B.cpu().numpy().astype(np.float64)))
    assert 0.0 <= rep["beta"] <= 1.0
    f = fit.ood_loss(A, A, KQ, KX)
    # two Brent implementations on a smooth unimodal curve: same minimum value
    assert f == pytest.approx(ref["loss"], rel=1e-4)
    assert abs(rep["beta"] - ref["beta"]) <= 2e-2
    np.testing.assert_allclose(A @ A.T, np.eye(d), atol=1e-5)


def test_es_then_fw_improves_es(lv, data):
    X, Q, KX, KQ = data
    d = 12
    _, _, es = lv.leanvec_fit_ood(t(X), t(Q), d, method=lv.FIT_ES)
    A, B, rep = lv.leanvec_fit_ood(t(X), t(Q), d, method=lv.FIT_ES_FW)
    f = fit.ood_loss(A.cpu().numpy(), B.cpu().numpy(), KQ, KX)
    assert f <= es["loss"] * (1 + 1e-5)
    assert rep["loss0"] == pytest.approx(es["loss"], rel=1e-5)


def test_line_search_and_bf16_second_moments(lv, data):
    X, Q, KX, KQ = data
    A, B, rep = lv.leanvec_fit_ood(t(X), t(Q), 12, method=lv.FIT_FW, line_search=True, precision=lv.PREC_BF16)
    ref = fit.frank_wolfe(KQ, KX, 12, alpha=0.5, tol=1e-3, line_search=True)
    f = fit.ood_loss(A.cpu().numpy(), B.cpu().numpy(), KQ, KX)
    assert f == pytest.approx(ref["loss"][-1], rel=2e-2)


@pytest.mark.parametrize("m,n,D,d", [(70, 130, 24, 5), (300, 1000, 64, 16), (129, 257, 200, 64),
                                     (1000, 5000, 128, 40), (600, 4000, 512, 128), (257, 3000, 256, 160),
                                     (100, 300, 30, 7), (90, 400, 132, 12)])
def test_pair_loss_forward_backward(lv, m, n, D, d):
    """The tensor-core forms: the loss for D % 4 == 0 (tf32x3 tile products), the gradients for
    D % 8 == 0 and d <= 128 with the residual tiles recomputed in TMEM (bf16x3) and contracted
    there (tf32x3) -- ragged row tiles (70, 129), column blocks (130, 257) and K blocks (24, 200),
    d from 5 to 128 (MMA N rounded up to 16), the C3 shape D = 512, d = 128; d = 160, D = 30 and
    D = 132 take the CUDA-core sweeps (also recomputing)."""
    rng = np.random.default_rng(m + n)
    Q = (rng.standard_normal((m, D)) / np.sqrt(D)).astype(np.float32)
    X = (rng.standard_normal((n, D)) / np.sqrt(D)).astype(np.float32)
    A = (rng.standard_normal((d, D)) / np.sqrt(D)).astype(np.float32)
    B = (rng.standard_normal((d, D)) / np.sqrt(D)).astype(np.float32)
    L = lv.leanvec_ood_loss_fwd(t(A), t(B), t(Q), t(X))
    gA, gB = lv.leanvec_ood_loss_bwd(t(A), t(B), t(Q), t(X))
    Lr, gAr, gBr = fit.pair_loss_and_grads(A, B, Q, X)
    assert L == pytest.approx(Lr, rel=1e-5)
    np.testing.assert_allclose(gA.cpu().numpy(), gAr, rtol=0, atol=1e-4 * np.abs(gAr).max())
    np.testing.assert_allclose(gB.cpu().numpy(), gBr, rtol=0, atol=1e-4 * np.abs(gBr).max())
    # equals the closed-form gradient built from K_Q, K_X (Eq. leanvec_gradients) / (n m)
    tA, tB = fit.ood_grads(A, B, fit.second_moment(Q), fit.second_moment(X))
    np.testing.assert_allclose(gA.cpu().numpy(), tA / (n * m), rtol=0, atol=1e-4 * np.abs(tA / (n * m)).max())


def test_pair_loss_backward_large(lv):
    """20000 queries x 30000 database rows (6e8 pairs, whose residual matrix would take 2.4 GB):
    the gradients recompute every residual tile, with many column ranges per pass (partial slots
    summed in order).  Checked against the closed-form gradients built from K_Q and K_X in FP64
    (Eq. leanvec_gradients / (n m))."""
    m, n, D, d = 20000, 30000, 64, 24
    rng = np.random.default_rng(17)
    Q = (rng.standard_normal((m, D)) / np.sqrt(D)).astype(np.float32)
    X = (rng.standard_normal((n, D)) / np.sqrt(D)).astype(np.float32)
    A = (rng.standard_normal((d, D)) / np.sqrt(D)).astype(np.float32)
    B = (rng.standard_normal((d, D)) / np.sqrt(D)).astype(np.float32)
    gA, gB = lv.leanvec_ood_loss_bwd(t(A), t(B), t(Q), t(X))
    KQ, KX = fit.second_moment(Q), fit.second_moment(X)
    tA, tB = fit.ood_grads(A, B, KQ, KX)
    np.testing.assert_allclose(gA.cpu().numpy(), tA / (n * m), rtol=0, atol=1e-4 * np.abs(tA / (n * m)).max())
    np.testing.assert_allclose(gB.cpu().numpy(), tB / (n * m), rtol=0, atol=1e-4 * np.abs(tB / (n * m)).max())
    L = lv.leanvec_ood_loss_fwd(t(A), t(B), t(Q), t(X))
    assert L == pytest.approx(fit.ood_loss(A, B, KQ, KX) / (n * m), rel=1e-5)


def test_autograd_function_and_gradient_optimiser(lv, data):
    X, Q, KX, KQ = data
    d = 12
    Xt, Qt = t(X[:2000]), t(Q[:1000])
    # start from the ID solution of another sample (at the ID solution of the same sample
    # the A-gradient vanishes identically)
    A = torch.nn.Parameter(lv.leanvec_fit_id(t(X[2000:4000]), d))
    B = torch.nn.Parameter(A.detach().clone())
    loss = lv.OODLoss.apply(A, B, Qt, Xt)
    loss.backward()
    ref_L, ref_gA, ref_gB = fit.pair_loss_and_grads(A.detach().cpu().numpy(), B.detach().cpu().numpy(), Q[:1000],
                                                    X[:2000])
    assert float(loss.detach()) == pytest.approx(ref_L, rel=1e-5)
    np.testing.assert_allclose(A.grad.cpu().numpy(), ref_gA, rtol=0, atol=1e-4 * np.abs(ref_gA).max())
    A1, B1, trace = lv.fit_ood_gradient(Xt, Qt, d, steps=30, lr=5e-3)
    assert min(trace) < trace[0] and len(trace) == 31
    assert fit.op_norm(A1.cpu().numpy()) <= 1 + 1e-4


def test_gradient_optimiser_against_frank_wolfe(lv, data):
    """The differentiation form's optimiser on the small shifted-query mixture: Adam on the
    hand-written pair loss (100 steps, lr 1e-2, from LeanVec-ID, projected onto the spectral-norm
    ball) ends with a loss f(A, B) / (n m) -- FP64 trace form from K_Q, K_X -- no larger than
    Frank-Wolfe's (Algorithm 1, alpha 0.5, relative-change stop 1e-3) and at least 10 % below
    LeanVec-ID's; the iterate returned is the best one of its loss trace."""
    X, Q, KX, KQ = data
    d = 12
    n, m = X.shape[0], Q.shape[0]
    Xt, Qt = t(X), t(Q)
    Afw, Bfw, _ = lv.leanvec_fit_ood(Xt, Qt, d, method=lv.FIT_FW, alpha=0.5, tol=1e-3)
    Ag, Bg, trace = lv.fit_ood_gradient(Xt, Qt, d, steps=100, lr=1e-2)
    P = lv.leanvec_fit_id(Xt, d)

    def f(A, B):
        return fit.ood_loss(A.cpu().numpy().astype(np.float64), B.cpu().numpy().astype(np.float64), KQ, KX) / (n * m)

    l_fw, l_g, l_id = f(Afw, Bfw), f(Ag, Bg), f(P, P)
    assert l_g <= l_fw, (l_g, l_fw)
    assert l_g <= 0.9 * l_id, (l_g, l_id)
    assert min(trace) == pytest.approx(l_g, rel=1e-4)
    assert fit.op_norm(Ag.cpu().numpy()) <= 1 + 1e-4 and fit.op_norm(Bg.cpu().numpy()) <= 1 + 1e-4


def test_spectral_clip(lv):
    rng = np.random.default_rng(9)
    A = rng.standard_normal((10, 40)).astype(np.float32)
    out = lv.leanvec_spectral_clip(t(A).contiguous()).cpu().numpy().astype(np.float64)
    U, s, Vt = np.linalg.svd(A.astype(np.float64), full_matrices=False)
    ref = U @ np.diag(np.minimum(s, 1.0)) @ Vt
    np.testing.assert_allclose(out, ref, atol=1e-5)
    small = (A / 100).astype(np.float32)
    np.testing.assert_allclose(lv.leanvec_spectral_clip(t(small).contiguous()).cpu().numpy(), small, atol=1e-7)
