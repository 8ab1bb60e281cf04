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


@pytest.mark.parametrize("dim,bits,n", [(32, 8, 1037), (160, 8, 1037), (100, 8, 1037), (768, 8, 1037),
                                        (200, 8, 1037), (160, 4, 1037), (33, 4, 1037), (64, 4, 1037), (1, 8, 1037),
                                        (1100, 8, 300), (1024, 4, 300), (16, 8, 40000), (12, 4, 40000)])
def test_lvq_bit_exact(lv, dim, bits, n):
    """dim % 4 == 0 takes the 16-byte-load kernel (one warp per vector, persistent grid: n = 40000
    gives every warp several vectors; dim 1100 exceeds its 8 chunks per lane), other dims the
    scalar kernel."""
    rng = np.random.default_rng(dim * 10 + bits)
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


@pytest.mark.parametrize("n,dim", [(5001, 77), (70001, 768), (1, 4), (2048, 130), (4099, 256)])
def test_column_mean(lv, n, dim):
    """FP64 column sums in row chunks of 2048 (float4 loads when dim % 4 == 0), rounded to fp32:
    equal to NumPy's FP64 mean rounded to fp32 up to the last bit, and the same on a second call."""
    rng = np.random.default_rng(n + dim)
    X = (rng.standard_normal((n, dim)) + 0.5).astype(np.float32)
    got = lv.leanvec_column_mean(t(X)).cpu().numpy()
    ref = X.astype(np.float64).mean(axis=0)
    assert np.all(np.abs(got - ref) <= np.abs(ref) * 2.0 ** -23 + 1e-30)
    np.testing.assert_array_equal(got, lv.leanvec_column_mean(t(X)).cpu().numpy())


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
