"""CPU oracle for the LeanVec search path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It shares no code with the CUDA library: the C part
(``leanvec_oracle.c``) is compiled here with gcc into ``_build/liboracle.so`` and
loaded with ctypes; the projection-learning part (``fit.py``) is FP64 NumPy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "leanvec_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain C, OpenMP over queries, no FMA contraction)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Store(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dim", ctypes.c_int),
                ("codes", ctypes.c_void_p), ("delta", ctypes.c_void_p),
                ("lower", ctypes.c_void_p), ("mean", ctypes.c_void_p),
                ("vecs", ctypes.c_void_p), ("metric", ctypes.c_int), ("sqnorm", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OUT)
        i64, i32, u64, vp, f32 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_float
        L.orc_lvq_encode.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp]
        L.orc_lvq_decode.argtypes = [vp, vp, vp, vp, i64, i32, vp]
        L.orc_lvq_decode.restype = None
        L.orc_build_prepare.argtypes = [vp, vp, vp, vp, i64, i32, vp, vp, vp, vp]
        L.orc_build_score.argtypes = [vp, vp, vp, vp, vp, vp, f32, i32, i64, i64]
        L.orc_build_score.restype = f32
        L.orc_search.argtypes = [vp, vp, vp, vp, i64, vp, i64, i32, ctypes.c_int32, vp, i32, vp, vp,
                                 i32, vp, vp, vp, vp, i32, i32]
        L.orc_bruteforce.argtypes = [vp, i64, vp, i64, i32, i32, vp, vp, i32, i32]
        L.orc_splitmix.argtypes = [u64, u64, u64]
        L.orc_splitmix.restype = u64
        L.orc_random_graph.argtypes = [i64, i32, u64, vp]
        L.orc_random_graph.restype = None
        L.orc_permutation.argtypes = [i64, u64, vp]
        L.orc_permutation.restype = None
        L.orc_robust_prune.argtypes = [vp, vp, vp, vp, vp, vp, f32, i32, ctypes.c_int32, vp, i32, f32, f32, i32,
                                       vp]
        L.orc_entry_point.argtypes = [vp, vp, i64]
        L.orc_entry_point.restype = ctypes.c_int32
        L.orc_vamana_build.argtypes = [vp, vp, vp, vp, vp, vp, f32, i32, i64, i32, i32, f32, i32, i32, u64, i32,
                                       vp, vp, i32]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# LVQ
# --------------------------------------------------------------------------
class LVQ:
    """Result of LVQ encoding: one code per byte (unpacked), per-vector delta/lower."""

    def __init__(self, codes, delta, lower, mean, bits):
        self.codes, self.delta, self.lower, self.mean, self.bits = codes, delta, lower, mean, bits

    @property
    def dim(self):
        return self.codes.shape[1]

    def decode(self) -> np.ndarray:
        n, dim = self.codes.shape
        out = np.empty((n, dim), np.float64)
        lib().orc_lvq_decode(_p(self.codes), _p(self.delta), _p(self.lower), _p(self.mean), n, dim, _p(out))
        return out


def lvq_encode(Y: np.ndarray, mean: np.ndarray, bits: int) -> LVQ:
    Y = _c(Y, np.float32)
    mean = _c(mean, np.float32)
    n, dim = Y.shape
    codes = np.empty((n, dim), np.uint8)
    delta = np.empty(n, np.float32)
    lower = np.empty(n, np.float32)
    rc = lib().orc_lvq_encode(_p(Y), n, dim, _p(mean), bits, _p(codes), _p(delta), _p(lower))
    if rc != 0:
        raise ValueError(f"orc_lvq_encode failed ({rc})")
    return LVQ(codes, delta, lower, mean, bits)


def mean_fp32(Y: np.ndarray) -> np.ndarray:
    """Dataset mean accumulated in FP64 and rounded to fp32."""
    return np.asarray(Y, np.float64).mean(axis=0).astype(np.float32)


def sqnorms_fp32(X: np.ndarray) -> np.ndarray:
    """||x_i||^2 of the original vectors for the L2 metric: squares exact in FP64, summed in FP64,
    rounded to fp32."""
    X = np.asarray(X, np.float64)
    return np.einsum("ij,ij->i", X, X).astype(np.float32)


# --------------------------------------------------------------------------
# Build-score store (bit-exact FP32 formula over integer sums)
# --------------------------------------------------------------------------
class BuildStore:
    """metric 0: the build score is <y_a, y_b>; metric 1 (L2): -||y_a - y_b||^2 =
    2 <y_a, y_b> - (N_a + N_b), N_i = <y_i, y_i>, all in the same fixed FP32 arithmetic."""

    def __init__(self, lvq: LVQ, metric: int = 0):
        self.lvq = lvq
        n, dim = lvq.codes.shape
        self.G = np.empty(n, np.float32)
        self.H = np.empty(n, np.float32)
        self.N = np.empty(n, np.float32) if metric else None
        mu2 = ctypes.c_float(0.0)
        rc = lib().orc_build_prepare(_p(lvq.codes), _p(lvq.delta), _p(lvq.lower), _p(lvq.mean), n, dim,
                                     _p(self.G), _p(self.H), _p(self.N) if metric else None, ctypes.byref(mu2))
        if rc != 0:
            raise ValueError(f"orc_build_prepare failed ({rc})")
        self.mu2 = np.float32(mu2.value)

    def _args(self):
        l = self.lvq
        return (_p(l.codes), _p(l.delta), _p(l.lower), _p(self.G), _p(self.H),
                _p(self.N) if self.N is not None else None, float(self.mu2), l.dim)

    def score(self, a: int, b: int) -> np.float32:
        return np.float32(lib().orc_build_score(*self._args(), int(a), int(b)))

    def entry(self) -> int:
        return int(lib().orc_entry_point(_p(self.G), _p(self.N) if self.N is not None else None,
                                         self.G.shape[0]))

    def robust_prune(self, p: int, pool, alpha: float, R: int, shift: float = 0.0) -> np.ndarray:
        pool = _c(pool, np.int32)
        out = np.empty(R, np.int32)
        k = lib().orc_robust_prune(*self._args(), int(p), _p(pool), len(pool), float(alpha), float(shift), R,
                                   _p(out))
        return out[:k].copy()


def vamana_build(lvq: LVQ, R: int, L_build: int, alpha: float, passes: int, batch: int, seed: int,
                 nthreads: int = 0, rule: int = 0, metric: int = 0):
    """rule 0: drop p' when alpha s(p*,p') >= s(p,p'); rule 1: when alpha s(p*,p') >= s(p,p') + alpha - 1.
    metric 1: the L2 build score s = -||y_a - y_b||^2 (rule 0 is then Vamana's alpha d(p*,p') <= d(p,p')
    on squared distances)."""
    bs = BuildStore(lvq, metric)
    n = lvq.codes.shape[0]
    graph = np.empty((n, R), np.int32)
    entry = ctypes.c_int32(0)
    rc = lib().orc_vamana_build(*bs._args(), n, R, L_build, float(alpha), passes, batch, seed, rule,
                                _p(graph), ctypes.byref(entry), nthreads)
    if rc != 0:
        raise RuntimeError(f"orc_vamana_build failed ({rc})")
    return graph, int(entry.value)


def random_graph(n: int, R: int, seed: int) -> np.ndarray:
    g = np.empty((n, R), np.int32)
    lib().orc_random_graph(n, R, seed, _p(g))
    return g


def permutation(n: int, seed: int) -> np.ndarray:
    p = np.empty(n, np.int32)
    lib().orc_permutation(n, seed, _p(p))
    return p


def splitmix(seed: int, a: int, b: int) -> int:
    return int(lib().orc_splitmix(seed, a, b))


# --------------------------------------------------------------------------
# Search
# --------------------------------------------------------------------------
def _store(kind, dim, lvq: LVQ | None = None, vecs=None, metric: int = 0, sqnorm=None):
    s = _Store()
    s.kind, s.dim, s.metric = kind, dim, metric
    keep = []
    if sqnorm is not None:
        sqnorm = _c(sqnorm, np.float32)
        s.sqnorm = _p(sqnorm)
        keep.append(sqnorm)
    if lvq is not None:
        s.codes, s.delta, s.lower, s.mean = _p(lvq.codes), _p(lvq.delta), _p(lvq.lower), _p(lvq.mean)
        keep.append(lvq)
    if vecs is not None:
        s.vecs = _p(vecs)
        keep.append(vecs)
    return s, keep


def search(graph: np.ndarray, entry: int, qp: np.ndarray, k: int, L: int, rerank: int = 0,
           prim: LVQ | None = None, prim_vecs: np.ndarray | None = None,
           sec: LVQ | None = None, qs: np.ndarray | None = None, max_hops: int = 0,
           desc: np.ndarray | None = None, want_beam: bool = False, nthreads: int = 0, width: int = 1,
           sec_vecs: np.ndarray | None = None, metric: int = 0, sqnorm: np.ndarray | None = None,
           sec_sqnorm: np.ndarray | None = None) -> dict:
    """Beam search + rerank for all queries (search width `width`: parents expanded
    per round).  qp: m x d_primary (already projected, FP64).  prim: LVQ primary store, or prim_vecs: raw fp32 vectors.  sec/qs: the
    secondary store and the unreduced queries for the rerank; sec_vecs instead of sec: raw
    secondary vectors (e.g. x rounded to IEEE half, given as their exact float32 values), scored
    as plain FP64 inner products.  desc (m x 4 int32: k, L, r, max_hops) overrides the uniform
    parameters.  metric 1 (L2): scores are 2 <q, x> - ||x||^2 with ||x||^2 = sqnorm (the original
    vectors' squared norms) for the primaries and LVQ secondaries; raw-vector secondaries use
    sec_sqnorm, by default their own norms (raw primaries without sqnorm likewise)."""
    graph = _c(graph, np.int32)
    n, R = graph.shape
    qp = _c(qp, np.float64)
    m = qp.shape[0]
    if prim is not None:
        ps, keep1 = _store(0, prim.dim, lvq=prim, metric=metric, sqnorm=sqnorm)
    else:
        pv = _c(prim_vecs, np.float32)
        ps, keep1 = _store(1, pv.shape[1], vecs=pv, metric=metric, sqnorm=sqnorm)
    ss, keep2 = (None, [])
    qsp = None
    if sec is not None and rerank != 0:
        ss, keep2 = _store(0, sec.dim, lvq=sec, metric=metric, sqnorm=sqnorm)
        qs = _c(qs, np.float64)
        qsp = _p(qs)
    elif sec_vecs is not None and rerank != 0:
        sv = _c(sec_vecs, np.float32)
        ss, keep2 = _store(1, sv.shape[1], vecs=sv, metric=metric, sqnorm=sec_sqnorm)
        qs = _c(qs, np.float64)
        qsp = _p(qs)
    if desc is None:
        desc = np.tile(np.array([k, L, rerank, max_hops], np.int32), (m, 1))
    desc = _c(desc, np.int32)
    kmax = int(desc[:, 0].max()) if m else k
    Lmax = int(desc[:, 1].max()) if m else L
    ids = np.full((m, kmax), -1, np.int32)
    scores = np.full((m, kmax), -np.inf, np.float64)
    bids = np.full((m, Lmax), -1, np.int32) if want_beam else None
    bsc = np.full((m, Lmax), -np.inf, np.float64) if want_beam else None
    hops = np.zeros(m, np.int64)
    scored = np.zeros(m, np.int64)
    rc = lib().orc_search(ctypes.byref(ps), ctypes.byref(ss) if ss is not None else None, _p(qp), qsp,
                          m, _p(graph), n, R, int(entry), _p(desc), kmax, _p(ids), _p(scores),
                          Lmax if want_beam else 0, _p(bids) if want_beam else None,
                          _p(bsc) if want_beam else None, _p(hops), _p(scored), width, nthreads)
    del keep1, keep2
    if rc != 0:
        raise RuntimeError(f"orc_search failed ({rc})")
    out = {"ids": ids, "scores": scores, "hops": hops, "scored": scored}
    if want_beam:
        out["beam_ids"], out["beam_scores"] = bids, bsc
    return out


def bruteforce(X: np.ndarray, Q: np.ndarray, k: int, nthreads: int = 0, metric: int = 0):
    """Exact top-k by <q, x> (metric 0) or by -||q - x||^2 (metric 1; the scores returned are
    2 <q, x> - ||x||^2), FP64, ties -> smaller id."""
    X = _c(X, np.float32)
    Q = _c(Q, np.float32)
    n, D = X.shape
    m = Q.shape[0]
    ids = np.empty((m, k), np.int32)
    sc = np.empty((m, k), np.float64)
    rc = lib().orc_bruteforce(_p(X), n, _p(Q), m, D, k, _p(ids), _p(sc), metric, nthreads)
    if rc != 0:
        raise RuntimeError("orc_bruteforce failed")
    return ids, sc


def recall(found: np.ndarray, truth: np.ndarray, k: int) -> float:
    """k-recall@k = |S ∩ G| / k averaged over queries (App. D.3)."""
    tot = 0
    for a, b in zip(found[:, :k], truth[:, :k]):
        tot += len(set(int(x) for x in a if x >= 0) & set(int(x) for x in b))
    return tot / (k * found.shape[0])
