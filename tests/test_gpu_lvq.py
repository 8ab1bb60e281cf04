"""GPU LVQ encoding, column mean and projection against the oracle.
LVQ codes, constants and the build-score terms G, H are bit-exact."""
import numpy as np
import pytest

import oracle
from gpu_util import t, unpack_records

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


@pytest.mark.parametrize("dim,bits", [(32, 8), (160, 8), (100, 8), (768, 8), (200, 8), (160, 4), (33, 4), (64, 4),
                                      (1, 8)])
def test_lvq_bit_exact(lv, dim, bits):
    rng = np.random.default_rng(dim * 10 + bits)
    n = 1037
    Y = rng.standard_normal((n, dim)).astype(np.float32) * 0.2
    Y[5] = 0.125  # constant row: delta = 0, all codes 0
    Y[6, :] = Y[6, 0]
    mean = oracle.mean_fp32(Y)
    rec = lv.leanvec_lvq_encode(t(Y), t(mean), bits).cpu().numpy()
    assert rec.shape == (n, lv.leanvec_record_stride(dim, bits))
    ref = oracle.lvq_encode(Y, mean, bits)
    codes, delta, lower, G, H, pad, tail = unpack_records(rec, dim, bits)
    np.testing.assert_array_equal(codes, ref.codes)
    np.testing.assert_array_equal(delta, ref.delta)
    np.testing.assert_array_equal(lower, ref.lower)
    bs = oracle.BuildStore(ref)
    np.testing.assert_array_equal(G, bs.G)
    np.testing.assert_array_equal(H, bs.H)
    if pad is not None:
        assert not pad.any()
    assert not tail.any()


def test_column_mean(lv):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((5001, 77)).astype(np.float32)
    got = lv.leanvec_column_mean(t(X)).cpu().numpy()
    ref = X.astype(np.float64).mean(axis=0)
    assert np.abs(got - ref).max() <= 1e-7


@pytest.mark.parametrize("n,D,d,ldy", [(1, 8, 3, 3), (300, 128, 32, 32), (1000, 768, 160, 160), (77, 200, 64, 80)])
def test_projection_fp32(lv, n, D, d, ldy):
    rng = np.random.default_rng(n + D)
    X = rng.standard_normal((n, D)).astype(np.float32)
    P = rng.standard_normal((d, D)).astype(np.float32)
    Y = lv.leanvec_project(t(X), t(P), ldy=ldy).cpu().numpy()
    ref = X.astype(np.float64) @ P.T.astype(np.float64)
    scale = np.linalg.norm(X, axis=1)[:, None] * np.linalg.norm(P, axis=1)[None, :]
    assert np.all(np.abs(Y[:, :d] - ref) <= 1e-5 * scale)
    assert not Y[:, d:].any()
