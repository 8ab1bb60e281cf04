"""Helpers shared by the GPU tests: record unpacking (from the documented layout in
include/leanvec.h) and seeded fixtures built with the oracle."""
import numpy as np
import torch


def dev():
    return torch.device("cuda", 0)


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def code_area(dim, bits):
    cb = dim if bits == 8 else (dim + 1) // 2
    return (cb + 15) // 16 * 16


def unpack_records(rec: np.ndarray, dim: int, bits: int):
    """codes (n x dim), delta, lower, G, H and the padding bytes of LVQ records."""
    co = code_area(dim, bits)
    raw = rec[:, :co]
    if bits == 8:
        codes = raw[:, :dim]
    else:
        lo = raw & 0x0F
        hi = raw >> 4
        codes = np.empty((rec.shape[0], 2 * co), np.uint8)
        codes[:, 0::2] = lo
        codes[:, 1::2] = hi
        codes = codes[:, :dim]
    consts = np.ascontiguousarray(rec[:, co:co + 16]).view(np.float32)
    pad_codes = raw[:, dim:] if bits == 8 else None
    tail = rec[:, co + 16:]
    return codes, consts[:, 0], consts[:, 1], consts[:, 2], consts[:, 3], pad_codes, tail


def small_problem(oracle, n=3000, D=64, d=16, m=200, comps=30, seed=0, bits=8, R=16, Lb=32, alpha=1.0,
                  batch=256, ood=False):
    """Seeded mixture, ID PCA projection, oracle-encoded stores and an oracle-built graph."""
    import workloads
    from oracle import fit
    w = workloads.make_workload("isotropic", n, m, D, comps, cfg=100 + seed, sigma=0.3, ood=ood, m_learn=0)
    X, Q = w.X, w.Q
    P = fit.fit_id(fit.second_moment(X), d).astype(np.float32)
    Y = (X.astype(np.float64) @ P.T.astype(np.float64)).astype(np.float32)
    mu_p, mu_s = oracle.mean_fp32(Y), oracle.mean_fp32(X)
    prim = oracle.lvq_encode(Y, mu_p, bits)
    sec = oracle.lvq_encode(X, mu_s, 8)
    graph, entry = oracle.vamana_build(prim, R=R, L_build=Lb, alpha=alpha, passes=2, batch=batch, seed=5000 + seed)
    return dict(X=X, Q=Q, P=P, Y=Y, mu_p=mu_p, mu_s=mu_s, prim=prim, sec=sec, graph=graph, entry=entry, d=d, D=D,
                bits=bits)


def gpu_index(lv, pb):
    idx = lv.Index(0)
    idx.set_primary(t(pb["Y"]), t(pb["mu_p"]), pb["bits"], pb["D"])
    idx.set_secondary(t(pb["X"]), t(pb["mu_s"]))
    idx.set_graph(t(pb["graph"]), pb["entry"])
    return idx


def encode_parallel(oracle, Y, mu, bits, parts=16):
    """oracle.lvq_encode over row blocks on threads (the oracle's C call releases the GIL): the
    same codes and constants as one call, for the full-size stores."""
    from concurrent.futures import ThreadPoolExecutor
    n, dim = Y.shape
    codes = np.empty((n, dim), np.uint8)
    delta = np.empty(n, np.float32)
    lower = np.empty(n, np.float32)
    bounds = np.linspace(0, n, parts + 1).astype(np.int64)

    def one(i):
        a, b = bounds[i], bounds[i + 1]
        e = oracle.lvq_encode(Y[a:b], mu, bits)
        codes[a:b], delta[a:b], lower[a:b] = e.codes, e.delta, e.lower

    with ThreadPoolExecutor(parts) as ex:
        list(ex.map(one, range(parts)))
    return oracle.LVQ(codes, delta, lower, np.ascontiguousarray(mu, np.float32), bits)
