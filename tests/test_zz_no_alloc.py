"""leanvec_search_noalloc, the search entry point for callers that cannot let the
library allocate device memory (hosts that own all device memory through their own
pool, or serving loops that cannot afford an allocation's implicit synchronisation
mid-request): through the C ABI it must return what leanvec_search returns, call
after call, although every call reuses the same static scratch array.

Collected last on purpose (file name), so that a run stopping at the first failure
has already run every other test."""
import pytest
import torch

import oracle
from gpu_util import gpu_index, small_problem, t

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lv():
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    return lv


def _agree(ids, sc, ref_ids, ref_sc):
    """The tolerance of the search parity tests: >= 99 % identical ids position by
    position, scores of identical ids within 1e-4 of the norm product (unit-norm data)."""
    same = ids == ref_ids
    assert same.float().mean().item() >= 0.99
    assert torch.all((sc - ref_sc).abs()[same] <= 1e-4)


def test_noalloc_matches_search_on_consecutive_calls(lv):
    pb = small_problem(oracle, n=3000, D=64, d=16, m=300)
    idx = gpu_index(lv, pb)
    Q, P = t(pb["Q"]), t(pb["P"])
    ref_ids, ref_sc = idx.search(Q, P, k=10, L=40, rerank=40)
    for _ in range(2):  # the second call finds the first call's scratch contents
        ids, sc = idx.search_noalloc(Q, P, k=10, L=40, rerank=40)
        torch.cuda.synchronize()
        _agree(ids, sc, ref_ids, ref_sc)
    # a different batch size and beam on the next call
    ref2 = idx.search(Q[:77], P, k=5, L=24, rerank=16)
    got2 = idx.search_noalloc(Q[:77], P, k=5, L=24, rerank=16)
    _agree(got2[0], got2[1], ref2[0], ref2[1])
    idx.sync_status()


def test_noalloc_bf16_projection_matches_search(lv):
    """The bf16 projection (queries converted inside the tensor-core GEMM, the bf16 copy of A in
    the static scratch) gives the same results as leanvec_search with the same projection, bit
    for bit; a projection that would need a converted copy of Q is refused."""
    pb = small_problem(oracle, n=3000, D=64, d=16, m=300, seed=4)
    idx = gpu_index(lv, pb)
    Q, P = t(pb["Q"]), t(pb["P"])
    ref = idx.search(Q, P, k=10, L=40, rerank=40, width=2, projection=lv.PREC_BF16)
    got = idx.search_noalloc(Q, P, k=10, L=40, rerank=40, width=2, projection=lv.PREC_BF16)
    torch.testing.assert_close(got[0], ref[0], rtol=0, atol=0)
    torch.testing.assert_close(got[1], ref[1], rtol=0, atol=0)
    with pytest.raises(lv.LeanVecError):
        idx.search_noalloc(Q, P, k=10, L=40, rerank=40, projection=lv.PREC_FP8)


def test_noalloc_rejects_batches_beyond_the_static_scratch(lv):
    pb = small_problem(oracle, n=500, D=64, d=16, m=10, seed=2)
    idx = gpu_index(lv, pb)
    # 16 MiB / (4 * 16 + 16) bytes per query: 300,000 queries do not fit
    Q = torch.zeros((300_000, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(lv.LeanVecError) as e:
        idx.search_noalloc(Q, t(pb["P"]), k=5, L=16, rerank=16)
    assert e.value.code == -4 and "16 MiB" in str(e.value)


def test_noalloc_float32_index_and_descriptors(lv):
    """A float32 (full-dimensional) index, whose padded queries go to the static scratch, and an
    uneven batch of per-query descriptors: the same results as leanvec_search; a float32 index
    ignores the projection, as leanvec_search does."""
    import numpy as np
    pb = small_problem(oracle, n=3000, D=64, d=16, m=300, seed=6)
    Q, P = t(pb["Q"]), t(pb["P"])
    base = lv.Index(0).encode_fp32(t(pb["X"])).set_graph(t(pb["graph"]), pb["entry"])
    ref = base.search(Q, None, k=10, L=40, width=2)
    for prec in (lv.PREC_FP32, lv.PREC_BF16):
        got = base.search_noalloc(Q, None, k=10, L=40, width=2, projection=prec)
        torch.testing.assert_close(got[0], ref[0], rtol=0, atol=0)
        torch.testing.assert_close(got[1], ref[1], rtol=0, atol=0)
    idx = gpu_index(lv, pb)
    rng = np.random.default_rng(3)
    m = Q.shape[0]
    k = rng.choice([1, 5, 10], m)
    L = np.maximum(rng.integers(10, 64, m), k)
    r = np.minimum(L, rng.integers(0, 48, m))
    desc = t(np.stack([k, L, r, np.zeros(m, int)], 1).astype(np.int32))
    ref = idx.search(Q, P, k=10, L=64, rerank=64, desc=desc, ldo=10, width=2)
    for _ in range(2):
        got = idx.search_noalloc(Q, P, k=10, L=64, rerank=64, desc=desc, ldo=10, width=2)
        torch.testing.assert_close(got[0], ref[0], rtol=0, atol=0)
        torch.testing.assert_close(got[1], ref[1], rtol=0, atol=0)
    idx.sync_status()


def test_noalloc_allocates_no_device_memory(lv):
    """The entry point's promise: after a first call (which loads the kernels and looks up the
    scratch array's address), calls with more queries and a wider beam leave the device's free
    memory unchanged (the outputs are preallocated by the caller)."""
    pb = small_problem(oracle, n=3000, D=64, d=16, m=300, seed=7)
    idx = gpu_index(lv, pb)
    Q, P = t(pb["Q"]), t(pb["P"])
    ids = torch.empty((300, 10), dtype=torch.int32, device="cuda")
    sc = torch.empty((300, 10), dtype=torch.float32, device="cuda")
    idx.search_noalloc(Q[:50], P, k=10, L=24, rerank=24, width=2, out=(ids[:50], sc[:50]))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for m, L in ((300, 64), (300, 128), (120, 96)):
        idx.search_noalloc(Q[:m], P, k=10, L=L, rerank=L, width=2, out=(ids[:m], sc[:m]))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    idx.sync_status()
