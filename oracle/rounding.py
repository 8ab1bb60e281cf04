"""Operand rounding of the reduced-precision query projections -- TEST INFRASTRUCTURE ONLY.

The precision form projects the queries, q -> A q (Sec. 2, "Search"), on tensor cores
with operands rounded to bfloat16 or to FP8 e4m3 (with one scale per row) and products
summed in float32.  The rounding of the operands is a defined, data-independent input
transform; the oracle applies it itself to the float32 inputs and then computes the
projection in FP64, so that a search over reduced-precision projections can be held to
the same id tolerance as the float32 path.  Nothing here reads a GPU result.

Formats, from their public definitions:
* bfloat16: the upper 16 bits of an IEEE binary32 (8 exponent bits, 7 stored mantissa
  bits); float32 -> bfloat16 rounds to nearest, ties to the even stored mantissa.
* e4m3 ("E4M3FN" of the OCP 8-bit floating point specification): 1 sign, 4 exponent
  bits with bias 7, 3 mantissa bits; normal values 2^(e-7) (1 + m/8) for e = 1..15
  (e = 15, m = 7 is NaN, so the largest finite value is 448), subnormal values
  2^-6 m/8; no infinities.  float32 -> e4m3 with saturation rounds to nearest, ties to
  even, and clamps finite magnitudes above 448 to 448.
* Per-row scaling: a row x gets s = max_j |x_j| / 448 (float32 division; 1 for a zero
  row), its elements x_j * (1 / s) (float32 reciprocal and product) are rounded to e4m3,
  and a product of two rows is rescaled by s_x s_p.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16, round to nearest, ties to even; returned as float32 values."""
    x = np.ascontiguousarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    down = u & 0xFFFF0000
    up = down + 0x10000
    rest = u & 0xFFFF                       # the 16 discarded bits
    half = 0x8000
    keep_lsb = (down >> 16) & 1             # stored mantissa LSB of the truncated value
    take_up = (rest > half) | ((rest == half) & (keep_lsb == 1))
    out = np.where(take_up, up, down).astype(np.uint32)
    return out.view(np.float32).reshape(x.shape)


def e4m3_values() -> np.ndarray:
    """The finite non-negative e4m3 values by code 0..126 (code 127 = NaN), from the format's
    definition; ascending."""
    vals = []
    for code in range(127):
        e, m = code >> 3, code & 7
        vals.append(2.0 ** -6 * m / 8 if e == 0 else 2.0 ** (e - 7) * (1 + m / 8))
    return np.array(vals, np.float64)


def e4m3_round(v: np.ndarray) -> np.ndarray:
    """Round float32 values to e4m3 (nearest, ties to even, saturating at +-448); FP64 result."""
    v = np.asarray(v, np.float64)
    a = np.abs(v)
    # quantum of the binade that holds a: 2^-9 below 2^-6 (subnormals), else 2^(E-3) for
    # a in [2^E, 2^(E+1))
    _, ex = np.frexp(np.where(a > 0, a, 1.0))  # a = f 2^ex, f in [0.5, 1)
    quantum = np.where(a < 2.0 ** -6, 2.0 ** -9, np.ldexp(1.0, ex - 1 - 3))
    r = np.rint(a / quantum) * quantum        # np.rint: halves to even; a / quantum is exact
    r = np.minimum(r, E4M3_MAX)
    return np.copysign(r, v)


def e4m3_rows(X: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per-row scaled e4m3 operand of the rows of X: (rounded values in FP64, float32 scales)."""
    X = np.ascontiguousarray(X, np.float32)
    amax = np.abs(X).max(axis=1) if X.shape[1] else np.zeros(X.shape[0], np.float32)
    s = np.where(amax > 0, amax / np.float32(E4M3_MAX), np.float32(1.0)).astype(np.float32)
    inv = (np.float32(1.0) / s).astype(np.float32)
    scaled = (X * inv[:, None]).astype(np.float32)
    return e4m3_round(scaled), s


def project(Q: np.ndarray, A: np.ndarray, precision: str) -> np.ndarray:
    """q' = A q for the rows of Q in FP64 from the operands the precision form multiplies:
    'fp32' (the float32 inputs as they are), 'bf16' (both operands rounded to bfloat16) or
    'e4m3' (both operands per-row scaled and rounded to e4m3, the product rescaled)."""
    if precision == "fp32":
        return np.asarray(Q, np.float32).astype(np.float64) @ np.asarray(A, np.float32).astype(np.float64).T
    if precision == "bf16":
        return bf16_round(Q).astype(np.float64) @ bf16_round(A).astype(np.float64).T
    if precision == "e4m3":
        q8, sq = e4m3_rows(Q)
        a8, sa = e4m3_rows(A)
        return (q8 @ a8.T) * sq.astype(np.float64)[:, None] * sa.astype(np.float64)[None, :]
    raise ValueError(f"unknown precision {precision!r}")
