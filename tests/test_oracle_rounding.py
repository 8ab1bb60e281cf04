"""Pins for the oracle's operand rounding of the reduced-precision projections (bfloat16 and
per-row scaled e4m3): hand-worked values from the format definitions, brute force over the
enumerated e4m3 value set, and the conversions of PyTorch's CPU library where it has them."""
import numpy as np
import pytest
import torch

from oracle import rounding


def test_bf16_hand_values():
    u = 2.0 ** -7  # bfloat16 spacing in [1, 2)
    cases = [
        (1.0, 1.0),
        (1.0 + u / 2, 1.0),                      # halfway, ties to the even mantissa (0)
        (1.0 + 3 * u / 2, 1.0 + 2 * u),          # halfway between mantissas 1 and 2 -> 2
        (1.0 + u / 2 + 2.0 ** -20, 1.0 + u),     # just above halfway -> up
        (1.0 + u / 2 - 2.0 ** -20, 1.0),         # just below halfway -> down
        (-(1.0 + 3 * u / 2), -(1.0 + 2 * u)),    # sign-symmetric
        (2.0 ** -130, 2.0 ** -130),              # float32 subnormal with 7 significant bits: exact
    ]
    x = np.array([c[0] for c in cases], np.float32)
    want = np.array([c[1] for c in cases], np.float64)
    np.testing.assert_array_equal(rounding.bf16_round(x).astype(np.float64), want)
    # a large value: the result keeps 8 significant bits and is within half a unit of the input
    big = np.float32(3.0e38)
    r = float(rounding.bf16_round(np.array([big]))[0])
    ulp = 2.0 ** (np.floor(np.log2(float(big))) - 7)
    assert abs(r - float(big)) <= ulp / 2
    assert float(np.float32(r)) == r and (np.float32(r).view(np.uint32) & 0xFFFF) == 0


def test_bf16_matches_torch_cpu():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(200_000) * np.exp(rng.uniform(-30, 30, 200_000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(rounding.bf16_round(x), ref)


def test_e4m3_value_set():
    v = rounding.e4m3_values()
    assert v.shape == (127,) and np.all(np.diff(v) > 0)
    assert v[0] == 0.0 and v[1] == 2.0 ** -9 and v[8] == 2.0 ** -6 and v[-1] == 448.0
    assert v[56] == 1.0  # code 0x38: exponent 7 (unbiased 0), mantissa 0


def test_e4m3_hand_values():
    cases = [(448.0, 448.0), (500.0, 448.0), (-1e4, -448.0), (460.0, 448.0),
             (2.0 ** -10, 0.0),            # halfway between codes 0 and 1 -> code 0 (even)
             (3 * 2.0 ** -10, 2.0 ** -8),  # halfway between codes 1 and 2 -> code 2
             (17.0, 16.0), (19.0, 20.0),   # spacing 2 in [16, 32): 8.5 -> 8, 9.5 -> 10
             (1.0625, 1.0), (1.1875, 1.25), (0.0, 0.0), (-0.3, -0.3125)]
    x = np.array([c[0] for c in cases], np.float32)
    np.testing.assert_array_equal(rounding.e4m3_round(x), np.array([c[1] for c in cases]))


def _nearest_in_set(v: np.ndarray) -> np.ndarray:
    """Brute force: the nearest enumerated e4m3 value (ties to the even code), saturating."""
    vals = rounding.e4m3_values()
    a = np.minimum(np.abs(v.astype(np.float64)), 448.0)
    dist = np.abs(a[:, None] - vals[None, :])
    best = dist.min(axis=1, keepdims=True)
    tied = dist == best
    codes = np.arange(vals.shape[0])[None, :]
    # among tied codes prefer the even one
    pick = np.where(tied & (codes % 2 == 0), codes, 10_000).min(axis=1)
    pick = np.where(pick == 10_000, np.argmax(tied, axis=1), pick)
    return np.copysign(vals[pick], v)


def test_e4m3_brute_force():
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.uniform(-470, 470, 20_000), rng.standard_normal(20_000) * 2.0 ** -6,
                        rng.uniform(-1, 1, 20_000) * 2.0 ** rng.integers(-12, 9, 20_000)]).astype(np.float32)
    # exact halfway points of every binade
    vals = rounding.e4m3_values()
    mids = ((vals[1:] + vals[:-1]) / 2).astype(np.float32)
    v = np.concatenate([v, mids, -mids])
    np.testing.assert_array_equal(rounding.e4m3_round(v), _nearest_in_set(v))


@pytest.mark.skipif(not hasattr(torch, "float8_e4m3fn"), reason="torch without float8_e4m3fn")
def test_e4m3_matches_torch_cpu_in_range():
    rng = np.random.default_rng(3)
    v = (rng.uniform(-448, 448, 50_000) * 2.0 ** rng.integers(-16, 1, 50_000)).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float32).numpy().astype(np.float64)
    np.testing.assert_array_equal(rounding.e4m3_round(v), ref)


def test_e4m3_rows_scaling():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((64, 200)).astype(np.float32)
    X[3] = 0.0
    q, s = rounding.e4m3_rows(X)
    assert s.dtype == np.float32 and s[3] == 1.0 and not q[3].any()
    amax = np.abs(X).max(axis=1)
    np.testing.assert_array_equal(s[np.arange(64) != 3], (amax / np.float32(448))[np.arange(64) != 3])
    assert np.all(np.abs(q) <= 448.0)
    assert np.all(np.abs(q[np.arange(64) != 3]).max(axis=1) == 448.0)  # the largest element maps to 448
    # each element: within half an e4m3 spacing (relative 2^-4) of x / s, or below 2^-6 (subnormal range)
    rel = np.abs(q - X.astype(np.float64) / s[:, None].astype(np.float64))
    assert np.all(rel <= np.maximum(2.0 ** -4 * np.abs(q), 2.0 ** -10) * (1 + 1e-6))


def test_project_bounds():
    """The projections from rounded operands stay within the rounding's bounds of the FP64
    product: bf16 keeps 8 significant bits (2^-8 of ||q|| ||a||), e4m3 4 bits (2^-3)."""
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((300, 128)).astype(np.float32)
    A = rng.standard_normal((32, 128)).astype(np.float32)
    exact = Q.astype(np.float64) @ A.astype(np.float64).T
    scale = np.linalg.norm(Q, axis=1)[:, None] * np.linalg.norm(A, axis=1)[None, :]
    np.testing.assert_array_equal(rounding.project(Q, A, "fp32"), exact)
    eb = np.abs(rounding.project(Q, A, "bf16") - exact) / scale
    assert eb.max() <= 2.0 ** -8 and eb.max() > 0
    e8 = np.abs(rounding.project(Q, A, "e4m3") - exact) / scale
    assert e8.max() <= 2.0 ** -3 and e8.mean() <= 2e-2 and e8.max() > eb.max()
    with pytest.raises(ValueError):
        rounding.project(Q, A, "fp16")
