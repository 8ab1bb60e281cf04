"""The BF16 / e4m3 tcgen05 GEMMs (projection q -> A q / x -> B x and second moments K = X^T X)
against FP64 references.

Tolerances.  Against the unrounded FP64 product: bf16 keeps 8 significant bits, so each operand
carries a relative error <= 2^-9 and a dot product of two rounded vectors is off by at most about
2 * 2^-9 * sum|x_i p_i| <= 2^-8 * ||x|| * ||p|| (the tests use 2^-7); e4m3 keeps 4 (per-row scaled),
and the tests hold it to the 2e-2 * ||x|| * ||p|| of the reduced-precision paths.  Against the
oracle's product of the same rounded operands (``oracle.rounding``, FP64): only the float32
accumulation differs, within 1e-5 * ||x|| * ||p||.  Searches over a reduced-precision projection
are compared with the oracle's search over the projection of the same rounded operands, and held
to the float32 path's bar (>= 99 % of ids position by position)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import gpu_index, small_problem, t
from oracle import fit, rounding

pytestmark = pytest.mark.gpu
TOL = 2.0 ** -7


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


@pytest.mark.parametrize("n,D,d,ldy", [(300, 128, 32, 32), (1000, 768, 160, 160), (77, 200, 64, 80),
                                       (5000, 512, 128, 128), (129, 64, 16, 16), (1, 768, 160, 176),
                                       (50, 100, 16, 16), (333, 77, 8, 8), (100000, 256, 64, 72),
                                       (40000, 132, 256, 256), (3000, 64, 1, 4)])
def test_projection_bf16(lv, n, D, d, ldy):
    """D % 4 == 0: X is converted to bf16 inside the persistent GEMM (n = 100000 and 40000 give
    every CTA several 128-row tiles, so both tensor-memory accumulators and the stage ring wrap;
    D = 132 leaves a ragged K block, d = 1 and 256 the extreme widths); D = 77 takes the cast into
    a bf16 copy first."""
    rng = np.random.default_rng(n + D + d)
    X = rng.standard_normal((n, D)).astype(np.float32)
    P = rng.standard_normal((d, D)).astype(np.float32)
    Y = lv.leanvec_project(t(X), t(P), ldy=ldy, precision=lv.PREC_BF16).cpu().numpy()
    ref = X.astype(np.float64) @ P.T.astype(np.float64)
    norms = np.linalg.norm(X, axis=1)[:, None] * np.linalg.norm(P, axis=1)[None, :]
    assert np.all(np.abs(Y[:, :d] - ref) <= TOL * norms)
    assert not Y[:, d:].any()
    # and not merely within tolerance by luck: the error is of the bf16 size, not zero
    assert np.abs(Y[:, :d] - ref).max() > 0
    # the same rounded operands in FP64: only the float32 accumulation differs
    assert np.all(np.abs(Y[:, :d] - rounding.project(X, P, "bf16")) <= 1e-5 * norms)


@pytest.mark.parametrize("n,D", [(1000, 64), (20000, 768), (3001, 200), (3001, 100), (517, 77)])
def test_second_moment_bf16(lv, n, D):
    """Against the FP64 second moment of the unrounded rows (D = 77 takes the transposed bf16 copy of
    X and the general GEMM, the others the float32-input kernel)."""
    rng = np.random.default_rng(n * 7 + D)
    X = rng.standard_normal((n, D)).astype(np.float32)
    K = lv.leanvec_second_moment(t(X), precision=lv.PREC_BF16).cpu().numpy().astype(np.float64)
    ref = fit.second_moment(X)
    norms = np.linalg.norm(X, axis=0)
    assert np.all(np.abs(K - ref) <= TOL * np.outer(norms, norms))
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-3 * norms.max() ** 2)


@pytest.mark.parametrize("n,D", [(1000, 64), (20000, 768), (3001, 200), (5, 8), (129, 260), (100, 1024),
                                 (70001, 256), (4000, 516)])
def test_second_moment_bf16_float32_input(lv, n, D):
    """D % 4 == 0: the rows are rounded to bf16 inside the GEMM (upper-triangle 256 x 256 tiles, two
    TMEM halves, split over row ranges): against the FP64 product of the same rounded rows only the
    float32 accumulation differs; K is exactly symmetric.  Ragged shapes: fewer rows than one 64-row
    block (n = 5), a column block with 4 valid columns (D = 260, 516), ten tiles (D = 1024), more
    rows than one range (n = 70001)."""
    rng = np.random.default_rng(n * 13 + D)
    X = rng.standard_normal((n, D)).astype(np.float32)
    K = lv.leanvec_second_moment(t(X), precision=lv.PREC_BF16).cpu().numpy()
    assert np.array_equal(K, K.T)
    K = K.astype(np.float64)
    Xb = rounding.bf16_round(X).astype(np.float64)
    ref = Xb.T @ Xb
    nb = np.linalg.norm(Xb, axis=0)
    tol = (2e-7 * np.sqrt(n) + 1e-6) * np.outer(nb, nb)
    assert np.all(np.abs(K - ref) <= tol), float(np.max(np.abs(K - ref) / np.outer(nb, nb)))
    norms = np.linalg.norm(X, axis=0)
    assert np.all(np.abs(K - fit.second_moment(X)) <= TOL * np.outer(norms, norms))


@pytest.mark.parametrize("prec", ["bf16", "e4m3"])
def test_search_with_reduced_precision_projection(lv, prec):
    """bf16 / e4m3 query projection against the oracle's search over the projection of the same
    rounded operands: ids >= 99 % identical position by position and recall@10 within 0.002 of it;
    primary scores within 1e-4 ||q'|| ||y|| of the oracle's decoded scores from the rounded
    projection and within 2e-2 of the unrounded FP64 ones; the rerank restores FP32-accurate final
    scores."""
    precision = {"bf16": lv.PREC_BF16, "e4m3": lv.PREC_FP8}[prec]
    # D = 128: per-row scaled e4m3 keeps every primary score of this problem within 1.5e-2 (at
    # D = 64 a few pairs reach 2.1e-2: fewer coordinates average out less of the rounding)
    pb = small_problem(oracle, n=3000, D=128, d=32, m=300)
    idx = gpu_index(lv, pb)
    Qd, Pd = t(pb["Q"]), t(pb["P"])
    ids, sc = idx.search(Qd, Pd, k=10, L=48, rerank=48, projection=precision)
    idx.sync_status()
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    qp = rounding.project(pb["Q"], pb["P"], prec)
    qs = pb["Q"].astype(np.float64)
    ref = oracle.search(pb["graph"], pb["entry"], qp, k=10, L=48, rerank=48, prim=pb["prim"], sec=pb["sec"], qs=qs)
    truth, _ = oracle.bruteforce(pb["X"], pb["Q"], 10)
    assert (ids == ref["ids"]).mean() >= 0.99
    assert abs(oracle.recall(ids, truth, 10) - oracle.recall(ref["ids"], truth, 10)) <= 0.002
    dec = pb["sec"].decode()
    for j in range(ids.shape[0]):
        exact = dec[ids[j]] @ qs[j]
        assert np.all(np.abs(sc[j] - exact) <= 1e-4 * np.linalg.norm(qs[j]) * np.linalg.norm(dec[ids[j]], axis=1))
    # primary scores of the whole beam (no rerank): per pair against both FP64 references
    ids_p, sc_p = idx.search(Qd, Pd, k=48, L=48, rerank=0, projection=precision)
    ids_p, sc_p = ids_p.cpu().numpy(), sc_p.cpu().numpy()
    pdec = pb["prim"].decode()
    q64 = qs @ pb["P"].T.astype(np.float64)
    for j in range(ids_p.shape[0]):
        u = ids_p[j][ids_p[j] >= 0]
        yn = np.linalg.norm(pdec[u], axis=1)
        assert np.all(np.abs(sc_p[j][:len(u)] - pdec[u] @ qp[j]) <= 1e-4 * np.linalg.norm(qp[j]) * yn)
        assert np.all(np.abs(sc_p[j][:len(u)] - pdec[u] @ q64[j]) <= 2e-2 * np.linalg.norm(q64[j]) * yn)


def test_encode_with_bf16_projection(lv):
    pb = small_problem(oracle, n=2000, D=128, d=32, m=10)
    idx = lv.Index(0).encode(t(pb["X"]), t(pb["P"]), 8, 8, precision=lv.PREC_BF16)
    idx.sync_status()
    rec = idx.primary_records().cpu().numpy()
    from gpu_util import unpack_records
    codes, delta, lower, _, _, _, _ = unpack_records(rec, 32, 8)
    mean = idx.primary_mean().cpu().numpy().astype(np.float64)
    dec = mean[None, :] + lower[:, None].astype(np.float64) + delta[:, None].astype(np.float64) * codes
    Y = pb["X"].astype(np.float64) @ pb["P"].T.astype(np.float64)
    err = np.abs(dec - Y).max(axis=1)
    bound = delta / 2 + TOL * np.linalg.norm(pb["X"], axis=1) * np.linalg.norm(pb["P"], axis=1).max()
    assert np.all(err <= bound)


@pytest.mark.parametrize("n,D,d", [(300, 128, 32), (1000, 768, 160), (77, 200, 64), (4097, 768, 160)])
def test_projection_fp8_per_row_scaled(lv, n, D, d):
    """e4m3 operands (3 mantissa bits, per-row scales max|row|/448) on the tcgen05 f8f6f4 path:
    within 2e-2 ||x|| ||p|| of the unrounded FP64 product (the reduced-precision paths' bound; the
    worst case of the rounding alone is 2^-3, reached only by adversarial rows), and within
    1e-5 ||x|| ||p|| of the oracle's FP64 product of the same per-row scaled e4m3 operands."""
    rng = np.random.default_rng(n + 2 * D + d)
    X = rng.standard_normal((n, D)).astype(np.float32)
    P = rng.standard_normal((d, D)).astype(np.float32)
    Y = lv.leanvec_project(t(X), t(P), precision=lv.PREC_FP8).cpu().numpy()
    ref = X.astype(np.float64) @ P.T.astype(np.float64)
    scale = np.linalg.norm(X, axis=1)[:, None] * np.linalg.norm(P, axis=1)[None, :]
    err = np.abs(Y[:, :d] - ref) / scale
    assert err.max() <= 2e-2
    assert err.mean() <= 5e-3
    assert np.all(np.abs(Y[:, :d] - rounding.project(X, P, "e4m3")) <= 1e-5 * scale)


def test_scratch_pool_reuse_and_trim(lv):
    """Repeated offline calls reuse the library's scratch pool (results unchanged) and
    leanvec_trim_scratch returns its unused blocks without disturbing later calls."""
    rng = np.random.default_rng(5)
    X = t(rng.standard_normal((3000, 256)).astype(np.float32))
    K1 = lv.leanvec_second_moment(X, precision=lv.PREC_BF16)
    K2 = lv.leanvec_second_moment(X, precision=lv.PREC_BF16)
    torch.testing.assert_close(K1, K2, rtol=0, atol=0)
    torch.cuda.synchronize()
    lv.leanvec_trim_scratch(0)
    K3 = lv.leanvec_second_moment(X, precision=lv.PREC_BF16)
    torch.testing.assert_close(K1, K3, rtol=0, atol=0)


@pytest.mark.parametrize("n,D,d,ldy", [(300, 128, 32, 32), (1000, 768, 160, 160), (77, 200, 64, 80),
                                       (100000, 256, 64, 72), (40000, 132, 256, 256), (3000, 64, 1, 4),
                                       (1, 768, 160, 176)])
def test_projection_tf32x3(lv, n, D, d, ldy):
    """float32-accurate projection on the tensor cores (tf32 hi / lo splits, three products): the
    FP32 bound 1e-5 ||x|| ||p|| of the CUDA-core path holds, and the error is far below bf16's.
    n = 100000 / 40000 wrap both TMEM accumulators and the stage rings; d = 256 takes one
    operand stage (shared memory); D = 132 leaves a ragged K block."""
    rng = np.random.default_rng(n + 3 * D + d)
    X = rng.standard_normal((n, D)).astype(np.float32)
    P = rng.standard_normal((d, D)).astype(np.float32)
    Y = lv.leanvec_project(t(X), t(P), ldy=ldy, precision=lv.PREC_TF32X3).cpu().numpy()
    ref = X.astype(np.float64) @ P.T.astype(np.float64)
    scale = np.linalg.norm(X, axis=1)[:, None] * np.linalg.norm(P, axis=1)[None, :]
    err = np.abs(Y[:, :d] - ref) / scale
    assert err.max() <= 1e-5
    assert err.max() <= 2.0 ** -14
    assert not Y[:, d:].any()


def test_search_and_encode_with_tf32x3_projection(lv):
    """Search with the tf32x3 query projection agrees with the FP64-projected oracle like the
    float32 path (>= 99 % of ids); encode with it decodes within delta / 2 + 1e-5 ||x|| ||p||."""
    pb = small_problem(oracle, n=3000, D=64, d=16, m=300, seed=8)
    idx = gpu_index(lv, pb)
    ids, _ = idx.search(t(pb["Q"]), t(pb["P"]), k=10, L=48, rerank=48, projection=lv.PREC_TF32X3)
    ref = oracle.search(pb["graph"], pb["entry"], pb["Q"].astype(np.float64) @ pb["P"].T.astype(np.float64),
                        k=10, L=48, rerank=48, prim=pb["prim"], sec=pb["sec"], qs=pb["Q"].astype(np.float64))
    assert (ids.cpu().numpy() == ref["ids"]).mean() >= 0.99
    idx2 = lv.Index(0).encode(t(pb["X"]), t(pb["P"]), 8, 8, precision=lv.PREC_TF32X3)
    idx2.sync_status()
    from gpu_util import unpack_records
    codes, delta, lower, _, _, _, _ = unpack_records(idx2.primary_records().cpu().numpy(), 16, 8)
    mean = idx2.primary_mean().cpu().numpy().astype(np.float64)
    dec = mean[None, :] + lower[:, None].astype(np.float64) + delta[:, None].astype(np.float64) * codes
    Yr = pb["X"].astype(np.float64) @ pb["P"].T.astype(np.float64)
    bound = delta / 2 + 1e-5 * np.linalg.norm(pb["X"], axis=1) * np.linalg.norm(pb["P"], axis=1).max()
    assert np.all(np.abs(dec - Yr).max(axis=1) <= bound * (1 + 1e-6))
