"""GPU graph construction against the oracle's batch-synchronous Vamana: the
adjacency and the entry point are bit-exact (same order within every row)."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import t

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lv():
    import paper_2312_16335_gb300 as lv
    return lv


def _prims(n, d, bits, seed):
    rng = np.random.default_rng(seed)
    means = rng.standard_normal((20, d))
    Y = workloads.unit_rows(means[rng.integers(0, 20, n)] + 0.4 * rng.standard_normal((n, d)))
    mu = oracle.mean_fp32(Y)
    return Y, mu, oracle.lvq_encode(Y, mu, bits)


@pytest.mark.parametrize("n,d,bits,R,Lb,alpha,batch,rule", [
    (600, 16, 8, 8, 16, 0.95, 1, 0),
    (600, 16, 8, 8, 16, 1.0, 64, 0),
    (1000, 24, 4, 12, 24, 0.95, 100, 0),
    (1500, 32, 8, 16, 40, 1.0, 1500, 0),
    (777, 40, 8, 32, 64, 1.2, 128, 0),   # ragged sizes, R > 32
    (900, 24, 8, 16, 32, 1.2, 64, 1),    # unit-L2 rule
    (700, 16, 4, 12, 24, 1.3, 50, 1),
    (500, 256, 8, 16, 32, 1.0, 64, 0),   # long records: a whole warp per record (17 chunks)
    (400, 400, 4, 12, 24, 1.02, 50, 1),  # long LVQ-4 records (13 chunks)
])
def test_build_bit_exact(lv, n, d, bits, R, Lb, alpha, batch, rule):
    Y, mu, q = _prims(n, d, bits, seed=n + d)
    g_ref, e_ref = oracle.vamana_build(q, R=R, L_build=Lb, alpha=alpha, passes=2, batch=batch, seed=42, rule=rule)
    idx = lv.Index(0)
    idx.set_primary(t(Y), t(mu), bits, d)
    idx.build_graph(R=R, L_build=Lb, alpha=alpha, passes=2, batch=batch, seed=42, rule=rule)
    idx.sync_status()
    g, e = idx.get_graph()
    assert e == e_ref
    np.testing.assert_array_equal(g.cpu().numpy(), g_ref)


def test_build_id_small_config(lv):
    """The 10k x 128 ID workload: PCA d = 32, LVQ-8, R = 32, L_build = 64, alpha = 0.95."""
    from oracle import fit
    w = workloads.workload_id_small()
    P = fit.fit_id(fit.second_moment(w.X), 32).astype(np.float32)
    Y = (w.X.astype(np.float64) @ P.T.astype(np.float64)).astype(np.float32)
    mu = oracle.mean_fp32(Y)
    q = oracle.lvq_encode(Y, mu, 8)
    g_ref, e_ref = oracle.vamana_build(q, R=32, L_build=64, alpha=0.95, passes=2, batch=1024, seed=5001)
    idx = lv.Index(0)
    idx.set_primary(t(Y), t(mu), 8, 128).build_graph(R=32, L_build=64, alpha=0.95, passes=2, batch=1024, seed=5001)
    g, e = idx.get_graph()
    assert e == e_ref
    np.testing.assert_array_equal(g.cpu().numpy(), g_ref)
