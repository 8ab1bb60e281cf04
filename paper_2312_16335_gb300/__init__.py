"""LeanVec search on GB300: Python binding of the C ABI in include/leanvec.h.

Every function here only marshals arguments (torch CUDA tensors -> device
pointers, the current CUDA stream) and calls the same-named C entry point; all
arithmetic runs in the library's CUDA kernels.  The functions mirror the paper's
pipeline (LeanVec, arXiv 2312.16335, Sec. 2): learn A, B; encode primary
(LVQ(B x)) and secondary (LVQ(x)) vectors; build a graph on the primaries; search
with A q and rerank with the secondaries.
"""
from __future__ import annotations

import ctypes
import os

import torch

from ._native import (LVFitOpts, LVFitReport, LVIndexInfo, LVQueryDesc, LVSearchParams, LeanVecError, check, lib)

__all__ = ["Index", "LeanVecError", "leanvec_record_stride", "leanvec_column_mean", "leanvec_lvq_encode", "leanvec_eigh_top",
           "leanvec_project", "leanvec_second_moment", "leanvec_eigh", "leanvec_fit_id", "leanvec_fit_ood",
           "leanvec_ood_loss_fwd", "leanvec_ood_loss_bwd", "leanvec_spectral_clip", "OODLoss", "fit_ood_gradient",
           "autotune", "autotune_target_d", "autotune_uneven", "SearchGraph", "UnevenGraph", "leanvec_trim_scratch", "leanvec_index_file_check", "PREC_FP32", "PREC_BF16", "PREC_FP8", "PREC_TF32X3", "FIT_FW", "FIT_ES", "FIT_ES_FW"]

PREC_FP32, PREC_BF16, PREC_FP8, PREC_TF32X3 = 0, 1, 2, 3
PRUNE_SCALED, PRUNE_UNIT_L2 = 0, 1
METRIC_IP, METRIC_L2 = 0, 1


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t: torch.Tensor | None):
    """Pointer to a contiguous host (CPU) tensor."""
    if t is None:
        return None
    if t.is_cuda:
        raise ValueError("expected a host (CPU) tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _f32(t: torch.Tensor) -> torch.Tensor:
    if t.dtype != torch.float32:
        raise TypeError("expected float32")
    return t.contiguous()


def leanvec_index_file_check(path: str) -> dict:
    """Validate an index file (magic, version, header, strides, size, checksum, graph ids) without a
    device; returns its header as leanvec_index_info's fields (LeanVecError LV_ERR_CORRUPT if not)."""
    inf = LVIndexInfo()
    check(lib().leanvec_index_file_check(os.fsencode(path), ctypes.byref(inf)))
    return {f: getattr(inf, f) for f, _ in LVIndexInfo._fields_}


def leanvec_trim_scratch(device: int | torch.device | None = None) -> None:
    """Return the unused blocks of the library's scratch pool on `device` to the driver."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device("cuda", device) \
        if isinstance(device, int) else device
    check(lib().leanvec_trim_scratch(dev.index))


def leanvec_record_stride(dim: int, bits: int) -> int:
    return check(lib().leanvec_record_stride(dim, bits))


def leanvec_column_mean(X: torch.Tensor) -> torch.Tensor:
    X = _f32(X)
    out = torch.empty(X.shape[1], dtype=torch.float32, device=X.device)
    check(lib().leanvec_column_mean(_ptr(X), X.shape[0], X.shape[1], _ptr(out), _stream(X.device)))
    return out


def leanvec_lvq_encode(V: torch.Tensor, mean: torch.Tensor, bits: int) -> torch.Tensor:
    V = _f32(V)
    mean = _f32(mean)
    n, dim = V.shape
    rec = torch.empty((n, leanvec_record_stride(dim, bits)), dtype=torch.uint8, device=V.device)
    check(lib().leanvec_lvq_encode(_ptr(V), n, dim, _ptr(mean), bits, _ptr(rec), _stream(V.device)))
    return rec


def leanvec_project(X: torch.Tensor, P: torch.Tensor, ldy: int | None = None, precision: int = PREC_FP32) -> torch.Tensor:
    X = _f32(X)
    P = _f32(P)
    n, D = X.shape
    d = P.shape[0]
    ldy = d if ldy is None else ldy
    Y = torch.empty((n, ldy), dtype=torch.float32, device=X.device)
    check(lib().leanvec_project(_ptr(X), n, D, _ptr(P), d, _ptr(Y), ldy, precision, _stream(X.device)))
    return Y


def leanvec_second_moment(X: torch.Tensor, precision: int = PREC_FP32) -> torch.Tensor:
    X = _f32(X)
    K = torch.empty((X.shape[1], X.shape[1]), dtype=torch.float32, device=X.device)
    check(lib().leanvec_second_moment(_ptr(X), X.shape[0], X.shape[1], _ptr(K), precision, _stream(X.device)))
    return K


def leanvec_eigh(K: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    if K.dtype != torch.float64:
        raise TypeError("expected float64")
    K = K.contiguous()
    D = K.shape[0]
    w = torch.empty(D, dtype=torch.float64, device=K.device)
    V = torch.empty((D, D), dtype=torch.float64, device=K.device)
    check(lib().leanvec_eigh(_ptr(K), D, _ptr(w), _ptr(V), _stream(K.device)))
    return w, V


def leanvec_eigh_top(K: torch.Tensor, nout: int) -> tuple[torch.Tensor, torch.Tensor]:
    """The nout leading eigenpairs of symmetric FP64 K (tridiagonal reduction, bisection,
    inverse iteration): eigenvalues descending, eigenvectors as rows."""
    if K.dtype != torch.float64:
        raise TypeError("expected float64")
    K = K.contiguous()
    D = K.shape[0]
    w = torch.empty(nout, dtype=torch.float64, device=K.device)
    V = torch.empty((nout, D), dtype=torch.float64, device=K.device)
    check(lib().leanvec_eigh_top(_ptr(K), D, nout, _ptr(w), _ptr(V), _stream(K.device)))
    return w, V


def leanvec_fit_id(X: torch.Tensor, d: int, precision: int = PREC_FP32) -> torch.Tensor:
    """A = B (d x D) for LeanVec-ID."""
    X = _f32(X)
    A = torch.empty((d, X.shape[1]), dtype=torch.float32, device=X.device)
    check(lib().leanvec_fit_id(_ptr(X), X.shape[0], X.shape[1], d, _ptr(A), None, precision, _stream(X.device)))
    return A


FIT_FW, FIT_ES, FIT_ES_FW = 0, 1, 2


def leanvec_fit_ood(X: torch.Tensor, Q: torch.Tensor, d: int, method: int = FIT_FW, alpha: float = 0.5,
                    tol: float = 1e-3, max_iter: int = 500, line_search: bool = False, precision: int = PREC_FP32,
                    es_xatol: float = 1e-5):
    """LeanVec-OOD: returns (A, B, report) learned from database rows X and learning queries Q."""
    X, Q = _f32(X), _f32(Q)
    D = X.shape[1]
    A = torch.empty((d, D), dtype=torch.float32, device=X.device)
    B = torch.empty((d, D), dtype=torch.float32, device=X.device)
    trace = (ctypes.c_double * (max_iter + 2))()
    rep = LVFitReport(0, 0, 0.0, 0.0, 0.0, trace, max_iter + 2)
    opts = LVFitOpts(method, alpha, tol, max_iter, int(line_search), precision, es_xatol)
    check(lib().leanvec_fit_ood(_ptr(X), X.shape[0], _ptr(Q), Q.shape[0], D, d, ctypes.byref(opts), _ptr(A), _ptr(B),
                                ctypes.byref(rep), _stream(X.device)))
    out = {"iterations": rep.iterations, "evaluations": rep.evaluations, "beta": rep.beta, "loss0": rep.loss0,
           "loss": rep.loss, "loss_trace": [trace[i] for i in range(min(rep.iterations + 1, max_iter + 2))]}
    return A, B, out


def leanvec_ood_loss_fwd(A: torch.Tensor, B: torch.Tensor, Q: torch.Tensor, X: torch.Tensor) -> float:
    A, B, Q, X = _f32(A), _f32(B), _f32(Q), _f32(X)
    out = ctypes.c_double()
    check(lib().leanvec_ood_loss_fwd(_ptr(A), _ptr(B), _ptr(Q), Q.shape[0], _ptr(X), X.shape[0], X.shape[1],
                                     A.shape[0], ctypes.byref(out), _stream(A.device)))
    return out.value


def leanvec_ood_loss_bwd(A, B, Q, X, scale: float = 1.0):
    A, B, Q, X = _f32(A), _f32(B), _f32(Q), _f32(X)
    gA, gB = torch.empty_like(A), torch.empty_like(B)
    check(lib().leanvec_ood_loss_bwd(_ptr(A), _ptr(B), _ptr(Q), Q.shape[0], _ptr(X), X.shape[0], X.shape[1],
                                     A.shape[0], float(scale), _ptr(gA), _ptr(gB), _stream(A.device)))
    return gA, gB


def leanvec_spectral_clip(A: torch.Tensor) -> torch.Tensor:
    """In place: project A onto {||A||_op <= 1}."""
    if not A.is_contiguous() or A.dtype != torch.float32:
        raise ValueError("expected a contiguous float32 tensor")
    check(lib().leanvec_spectral_clip(_ptr(A), A.shape[0], A.shape[1], _stream(A.device)))
    return A


class OODLoss(torch.autograd.Function):
    """L(A, B) = sum_ij (q_j^T x_i - (A q_j)^T (B x_i))^2 / (n m) over the sample pairs of
    Q (m x D) and X (n x D), with the hand-written CUDA forward and backward (tf32x3 tensor
    cores when D % 4 == 0: the forward sums the squares of the residual tiles without storing
    them, the backward keeps the residual matrix per chunk of database rows; float32 CUDA-core
    pair tiles otherwise).  Gradients flow to A and B only."""

    @staticmethod
    def forward(ctx, A, B, Q, X):
        ctx.save_for_backward(A, B, Q, X)
        return torch.tensor(leanvec_ood_loss_fwd(A.detach(), B.detach(), Q, X), dtype=torch.float32,
                            device=A.device)

    @staticmethod
    def backward(ctx, grad_out):
        A, B, Q, X = ctx.saved_tensors
        gA, gB = leanvec_ood_loss_bwd(A.detach(), B.detach(), Q, X, float(grad_out))
        return gA, gB, None, None


def fit_ood_gradient(X: torch.Tensor, Q: torch.Tensor, d: int, steps: int = 100, lr: float = 1e-2,
                     A0: torch.Tensor | None = None, B0: torch.Tensor | None = None, log=None):
    """A gradient optimiser for LeanVec-OOD beside Frank-Wolfe: Adam on the pair loss
    (OODLoss, hand-written fwd/bwd) with a projection onto the spectral-norm ball after
    every step (the relaxed problem "leanvec").  Starts from LeanVec-ID unless A0/B0 given.
    Returns the iterate with the lowest loss seen (Adam's steps do not decrease the loss
    monotonically once the projection is active), and the loss of every iterate."""
    if A0 is None:
        A0 = leanvec_fit_id(X, d)
    A = torch.nn.Parameter(A0.clone().contiguous())
    B = torch.nn.Parameter((A0 if B0 is None else B0).clone().contiguous())
    opt = torch.optim.Adam([A, B], lr=lr)
    trace = []
    best = (float("inf"), None, None)
    for _ in range(steps + 1):
        opt.zero_grad()
        loss = OODLoss.apply(A, B, Q, X)
        cur = float(loss.detach())
        trace.append(cur)
        if log:
            log(cur)
        if cur < best[0]:
            best = (cur, A.detach().clone(), B.detach().clone())
        if len(trace) > steps:  # the last entry is the loss of the final iterate
            break
        loss.backward()
        opt.step()
        with torch.no_grad():
            leanvec_spectral_clip(A.data)
            leanvec_spectral_clip(B.data)
    return best[1], best[2], trace


class Index:
    """Owns an ``lv_index*`` (stores + graph on one CUDA device)."""

    def __init__(self, device: int | torch.device | None = None, metric: int = METRIC_IP):
        """metric: METRIC_IP (inner product) or METRIC_L2 (squared Euclidean distance, scores
        2 <q, x> - ||x||^2); see leanvec_set_metric."""
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device if isinstance(device, int) else device.index or 0)
        h = ctypes.c_void_p()
        check(lib().leanvec_index_create(ctypes.byref(h), self.device.index))
        self._h = h
        if metric:
            check(lib().leanvec_set_metric(self._h, int(metric)))

    def close(self):
        if getattr(self, "_h", None):
            lib().leanvec_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = LVIndexInfo()
        check(lib().leanvec_index_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in LVIndexInfo._fields_}

    def save(self, path: str) -> "Index":
        """leanvec_index_save: write the stores, graph and entry point to `path`."""
        check(lib().leanvec_index_save(self._h, os.fsencode(path), _stream(self.device)))
        return self

    def load(self, path: str) -> "Index":
        """leanvec_index_load: replace this index's stores (and metric) with those of `path`,
        after validating the whole file."""
        check(lib().leanvec_index_load(self._h, os.fsencode(path), _stream(self.device)))
        return self

    def buffers(self) -> dict:
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        check(lib().leanvec_index_buffers(self._h, *[ctypes.byref(p) for p in ptrs]))
        return dict(zip(["primary", "primary_mean", "secondary", "secondary_mean", "graph"], [p.value for p in ptrs]))

    def _view(self, ptr: int, shape, dtype) -> torch.Tensor:
        """Copy a device buffer owned by the index into a new tensor (inspection, tests)."""
        typestr = {torch.uint8: "|u1", torch.float32: "<f4", torch.int32: "<i4"}[dtype]

        class _Buf:
            __cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                        "data": (int(ptr), False), "version": 2, "strides": None}

        torch.cuda.current_stream(self.device).synchronize()
        return torch.as_tensor(_Buf(), device=self.device).clone()

    def primary_records(self) -> torch.Tensor:
        inf = self.info()
        return self._view(self.buffers()["primary"], (inf["n"], inf["primary_stride"]), torch.uint8)

    def secondary_records(self) -> torch.Tensor:
        inf = self.info()
        return self._view(self.buffers()["secondary"], (inf["n"], inf["secondary_stride"]), torch.uint8)

    def primary_mean(self) -> torch.Tensor:
        return self._view(self.buffers()["primary_mean"], (self.info()["d"],), torch.float32)

    # -- encoding ------------------------------------------------------------
    def encode(self, X: torch.Tensor, B: torch.Tensor, primary_bits: int = 8, secondary_bits: int = 8,
               precision: int = PREC_FP32) -> "Index":
        X, B = _f32(X), _f32(B)
        check(lib().leanvec_encode(self._h, _ptr(X), X.shape[0], X.shape[1], _ptr(B), B.shape[0], primary_bits,
                                   secondary_bits, precision, _stream(self.device)))
        return self

    def set_primary(self, Y: torch.Tensor, mean: torch.Tensor | None, bits: int, D: int) -> "Index":
        Y = _f32(Y)
        m = _f32(mean) if mean is not None else None
        check(lib().leanvec_set_primary(self._h, _ptr(Y), Y.shape[0], Y.shape[1], _ptr(m), bits, D,
                                        _stream(self.device)))
        return self

    def set_secondary(self, X: torch.Tensor, mean: torch.Tensor | None = None) -> "Index":
        X = _f32(X)
        m = _f32(mean) if mean is not None else None
        check(lib().leanvec_set_secondary(self._h, _ptr(X), X.shape[0], X.shape[1], _ptr(m), _stream(self.device)))
        return self

    def encode_fp32(self, X: torch.Tensor) -> "Index":
        X = _f32(X)
        check(lib().leanvec_encode_fp32(self._h, _ptr(X), X.shape[0], X.shape[1], _stream(self.device)))
        return self

    # -- graph ----------------------------------------------------------------
    def set_graph(self, adj: torch.Tensor, entry: int = -1) -> "Index":
        adj = adj.to(device=self.device, dtype=torch.int32).contiguous()
        check(lib().leanvec_set_graph(self._h, _ptr(adj), adj.shape[1], entry, _stream(self.device)))
        return self

    def get_graph(self) -> tuple[torch.Tensor, int]:
        inf = self.info()
        adj = torch.empty((inf["n"], inf["R"]), dtype=torch.int32, device=self.device)
        e = ctypes.c_int32()
        check(lib().leanvec_get_graph(self._h, _ptr(adj), ctypes.byref(e), _stream(self.device)))
        torch.cuda.current_stream(self.device).synchronize()
        return adj, int(e.value)

    def build_graph(self, R: int, L_build: int, alpha: float, passes: int = 2, batch: int = 4096,
                    seed: int = 5000, rule: int = 0) -> "Index":
        """rule 0 (PRUNE_SCALED): drop p' when alpha s(p*,p') >= s(p,p'); rule 1 (PRUNE_UNIT_L2):
        when alpha s(p*,p') >= s(p,p') + alpha - 1."""
        check(lib().leanvec_build_graph(self._h, R, L_build, float(alpha), passes, batch, seed, rule,
                                        _stream(self.device)))
        return self

    # -- search ----------------------------------------------------------------
    def search(self, Q: torch.Tensor, A: torch.Tensor | None, k: int, L: int, rerank: int = 0, max_hops: int = 0,
               desc: torch.Tensor | None = None, ldo: int | None = None, stats: bool = False,
               projection: int = PREC_FP32, hash_slots: int = 0, warps_per_block: int = 0,
               out: tuple[torch.Tensor, torch.Tensor] | None = None, events=None, width: int = 1,
               warps_per_query: int = 0, queries_per_warp: int = 0, visited_bits: int = 0):
        """Search m queries. desc: optional (m, 4) int32 CUDA tensor of per-query
        (k, L, rerank, max_hops); then k/L are the upper bounds used for capacity.
        events: optional pair of torch.cuda.Event recorded around the search kernels.
        width: beam members expanded per round (1 = classic best-first).
        warps_per_query: warps sharing one query (1, 2, 4; divides width; 0 = 1);
        queries_per_warp: 1, or 2 (one query per 16 lanes; LVQ primaries, width <= 2,
        width * R <= 128), 0 = 1.  visited_bits: slot width of the visited cache, 32 (ids; 0 =
        32) or 16 (tags, twice the default slots in the same bytes; n <= 65535 * slots / 8).  The
        results depend on none of these."""
        Q = _f32(Q)
        m = Q.shape[0]
        ldo = k if ldo is None else ldo
        if out is None:
            ids = torch.empty((m, ldo), dtype=torch.int32, device=self.device)
            sc = torch.empty((m, ldo), dtype=torch.float32, device=self.device)
        else:
            ids, sc = out
        st = torch.empty((m, 2), dtype=torch.int32, device=self.device) if stats else None
        ev0, ev1 = (None, None) if events is None else (events[0].cuda_event, events[1].cuda_event)
        prm = LVSearchParams(LVQueryDesc(k, L, rerank, max_hops), projection, hash_slots, warps_per_block, width,
                             warps_per_query, ev0, ev1, queries_per_warp, visited_bits)
        if desc is not None:
            desc = desc.to(device=self.device, dtype=torch.int32).contiguous()
        Ac = _f32(A) if A is not None else None
        check(lib().leanvec_search(self._h, _ptr(Q), m, _ptr(Ac), ctypes.byref(prm), _ptr(desc), _ptr(ids), _ptr(sc),
                                   ldo, _ptr(st), _stream(self.device)))
        return (ids, sc, st) if stats else (ids, sc)

    def search_host(self, Qh: torch.Tensor, A: torch.Tensor | None, k: int, L: int, rerank: int = 0,
                    max_hops: int = 0, desc: torch.Tensor | None = None, ldo: int | None = None,
                    out: tuple[torch.Tensor, torch.Tensor] | None = None, batch: int = 0,
                    projection: int = PREC_FP32, hash_slots: int = 0, warps_per_block: int = 0, width: int = 1,
                    warps_per_query: int = 0, queries_per_warp: int = 0, visited_bits: int = 0):
        """leanvec_search_host: queries Qh (m x D float32) and the results in host memory (use
        pinned tensors, ``.pin_memory()``, for the copies to overlap the searches); searched in
        batches of `batch` rows (0 = one batch), each exactly as ``search`` over those rows.
        desc: optional (m, 4) int32 host tensor of per-query (k, L, rerank, max_hops).  The
        results are complete once the current stream has completed."""
        Qh = _f32(Qh)
        m = Qh.shape[0]
        ldo = k if ldo is None else ldo
        if out is None:
            ids = torch.empty((m, ldo), dtype=torch.int32).pin_memory()
            sc = torch.empty((m, ldo), dtype=torch.float32).pin_memory()
        else:
            ids, sc = out
        prm = LVSearchParams(LVQueryDesc(k, L, rerank, max_hops), projection, hash_slots, warps_per_block, width,
                             warps_per_query, None, None, queries_per_warp, visited_bits)
        if desc is not None:
            desc = desc.to(dtype=torch.int32).contiguous()
        Ac = _f32(A) if A is not None else None
        check(lib().leanvec_search_host(self._h, _hptr(Qh), m, _ptr(Ac), ctypes.byref(prm), _hptr(desc), _hptr(ids),
                                        _hptr(sc), ldo, batch, _stream(self.device)))
        return ids, sc

    def search_noalloc(self, Q: torch.Tensor, A: torch.Tensor | None, k: int, L: int, rerank: int = 0,
                       max_hops: int = 0, ldo: int | None = None,
                       out: tuple[torch.Tensor, torch.Tensor] | None = None, projection: int = PREC_FP32,
                       width: int = 1, desc: torch.Tensor | None = None, queries_per_warp: int = 0):
        """leanvec_search_noalloc: the same search for callers that cannot let the
        library allocate device memory; its scratch is a static 16 MiB device array
        shared by all calls on a device (serialise overlapping calls).  The output
        tensors are the caller's (pass `out` to reuse preallocated ones).  projection:
        PREC_FP32 or PREC_BF16 (queries converted inside the tensor-core GEMM).  desc:
        optional (m, 4) int32 CUDA tensor of per-query (k, L, rerank, max_hops)."""
        Q = _f32(Q)
        m = Q.shape[0]
        ldo = k if ldo is None else ldo
        if out is None:
            ids = torch.empty((m, ldo), dtype=torch.int32, device=self.device)
            sc = torch.empty((m, ldo), dtype=torch.float32, device=self.device)
        else:
            ids, sc = out
        prm = LVSearchParams(LVQueryDesc(k, L, rerank, max_hops), projection, 0, 0, width, 0, None, None,
                             queries_per_warp)
        if desc is not None:
            desc = desc.to(device=self.device, dtype=torch.int32).contiguous()
        Ac = _f32(A) if A is not None else None
        check(lib().leanvec_search_noalloc(self._h, _ptr(Q), m, _ptr(Ac), ctypes.byref(prm), _ptr(desc), _ptr(ids),
                                           _ptr(sc), ldo, None, _stream(self.device)))
        return ids, sc

    def sync_status(self) -> int:
        return check(lib().leanvec_sync_status(self._h, _stream(self.device)))


# warps per block tried for two queries per warp (20 warps, 40 queries per SM at 96 registers)
HALF_WARPS = (5, 10)


def autotune(index: "Index", Q: torch.Tensor, A: torch.Tensor | None, k: int, L: int, rerank: int = 0,
             desc: torch.Tensor | None = None, width: int = 1, projection: int = PREC_FP32,
             warps=(4, 8), hash_slots=(512, 1024, 2048, 4096), queries_per_warp=(1, 2), reps: int = 3) -> dict:
    """Pick the launch shape (queries per warp, warps per block, i.e. queries per CTA) and the
    visited-cache size for this batch by timing each candidate with CUDA events (two queries per
    warp with the block sizes of HALF_WARPS, where the index and width allow it).  None of the
    knobs changes the result (the visited cache is exact-preserving), only occupancy versus
    re-scoring."""
    best = None
    table = []
    ldo = k
    ids = torch.empty((Q.shape[0], ldo), dtype=torch.int32, device=index.device)
    sc = torch.empty((Q.shape[0], ldo), dtype=torch.float32, device=index.device)
    for qpw in queries_per_warp:
        for w in (HALF_WARPS if qpw == 2 else warps):
            for h in hash_slots:
                if h < 2 * ((L + 31) // 32 * 32):
                    continue
                try:
                    run = lambda: index.search(Q, A, k=k, L=L, rerank=rerank, desc=desc, ldo=ldo, out=(ids, sc),
                                               width=width, projection=projection, hash_slots=h, warps_per_block=w,
                                               queries_per_warp=qpw)
                    run()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        run()
                    e1.record()
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / reps
                except LeanVecError:
                    continue
                table.append({"queries_per_warp": qpw, "warps_per_block": w, "hash_slots": h, "ms": ms})
                if best is None or ms < best["ms"]:
                    best = table[-1]
    return {"best": best, "table": table}


def autotune_uneven(index: "Index", Q: torch.Tensor, A: torch.Tensor | None, desc: torch.Tensor, ldo: int,
                    width: int = 2, projection: int = PREC_FP32, bounds=(64, 128, 192, 256, 320),
                    teams=(1, 2), hash_slots=(0, 512, 1024, 2048), warps=(4, 8), queries_per_warp=(1, 2),
                    reps: int = 3) -> dict:
    """The batching form's autotuner for an uneven batch (per-query k, L, rerank in `desc`).
    Three plans, each a reordering of the batch (done once) followed by one or more launches of
    contiguous slices, all captured in one CUDA graph by UnevenGraph:
      "one"      -- the batch in the caller's order, one launch;
      "longest"  -- the batch sorted by L, largest first, one launch: the persistent kernel takes
                    the longest searches first and fills the end of the launch with short ones;
      "classes"  -- beam-width classes L in (b_{c-1}, b_c] (`bounds`; the last class takes every
                    larger L), one launch per class, each with its own beam capacity (its largest
                    L rounded up to 32, which sizes a query's shared memory and so the queries
                    resident per SM).
    For every launch of every plan the fastest warps per query (`teams`, dividing `width`), queries
    per warp (two with one warp per query, where the index allows it, with the block sizes of
    HALF_WARPS), visited-cache slots (0 = the library's default) and warps per block are picked by
    timing the launch alone with CUDA events; the plan with the smallest total wins.  None of the knobs or
    plans changes a query's result.  Returns {"plan": name, "order": the permutation (device,
    int64) of the winning plan, "classes": its launches [{slice, L range, queries, k / L / rerank
    maxima, capacity, the chosen knobs, ms, qps}], "plans": {name: total ms}, "table": every timed
    candidate}; UnevenGraph runs it."""
    dev = index.device
    desc = desc.to(device=dev, dtype=torch.int32)
    Lq = desc[:, 1].to(torch.int64)
    m = Q.shape[0]
    ids = torch.empty((m, ldo), dtype=torch.int32, device=dev)
    sc = torch.empty((m, ldo), dtype=torch.float32, device=dev)
    table = []

    def tune(name, c, Qs, ds, sl, lo, hi):
        dc = ds[sl]
        kmax, Lmax, rmax = (int(dc[:, j].max()) for j in range(3))
        best = None
        shapes = [(T, 1) for T in teams] + [(1, 2)] * (2 in queries_per_warp)
        for T, qpw in shapes:
            if width % T or (qpw == 1 and 1 not in queries_per_warp):
                continue
            for h in hash_slots:
                if h and h < 2 * ((Lmax + 31) // 32 * 32):
                    continue
                for w in (HALF_WARPS if qpw == 2 else warps):
                    if w % T:
                        continue
                    kw = dict(k=kmax, L=Lmax, rerank=rmax, desc=dc, ldo=ldo, out=(ids[sl], sc[sl]), width=width,
                              projection=projection, hash_slots=h, warps_per_block=w, warps_per_query=T,
                              queries_per_warp=qpw)
                    try:
                        index.search(Qs[sl], A, **kw)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        for _ in range(reps):
                            index.search(Qs[sl], A, **kw)
                        e1.record()
                        torch.cuda.synchronize(dev)
                        ms = e0.elapsed_time(e1) / reps
                    except LeanVecError:
                        continue
                    row = {"plan": name, "launch": c, "warps_per_query": T, "queries_per_warp": qpw,
                           "hash_slots": h, "warps_per_block": w, "ms": ms}
                    table.append(row)
                    if best is None or ms < best["ms"]:
                        best = row
        n_c = sl.stop - sl.start
        return {"slice": (sl.start, sl.stop), "L_range": (lo, hi), "queries": n_c, "k_max": kmax, "L_max": Lmax,
                "rerank_max": rmax, "beam_capacity": (Lmax + 31) // 32 * 32,
                "warps_per_query": best["warps_per_query"], "queries_per_warp": best["queries_per_warp"],
                "hash_slots": best["hash_slots"], "warps_per_block": best["warps_per_block"], "ms": best["ms"],
                "qps": n_c / (best["ms"] / 1e3)}

    b = torch.tensor(list(bounds), dtype=torch.int64, device=dev)
    cls = torch.clamp(torch.bucketize(Lq, b, right=False), max=len(bounds) - 1)
    orders = {"one": torch.arange(m, device=dev), "longest": torch.argsort(-Lq, stable=True),
              "classes": torch.argsort(cls, stable=True)}
    plans = {}
    for name, order in orders.items():
        Qs = Q.index_select(0, order).contiguous()
        ds = desc.index_select(0, order).contiguous()
        launches = []
        if name == "classes":
            counts = torch.bincount(cls, minlength=len(bounds)).tolist()
            a0 = 0
            for c, cnt in enumerate(counts):
                if cnt == 0:
                    continue
                lo = 1 if c == 0 else bounds[c - 1] + 1
                launches.append(tune(name, c, Qs, ds, slice(a0, a0 + cnt), lo,
                                     None if c == len(bounds) - 1 else bounds[c]))
                a0 += cnt
        else:
            launches.append(tune(name, 0, Qs, ds, slice(0, m), int(Lq.min()), int(Lq.max())))
        plans[name] = {"order": order, "classes": launches, "ms": sum(x["ms"] for x in launches)}
    win = min(plans, key=lambda k: plans[k]["ms"])
    return {"plan": win, "order": plans[win]["order"], "classes": plans[win]["classes"],
            "plans": {k: v["ms"] for k, v in plans.items()},
            "plan_launches": {k: v["classes"] for k, v in plans.items()},
            "plan_orders": {k: v["order"] for k, v in plans.items()}, "table": table}


class UnevenGraph:
    """An uneven batch served by the plan of autotune_uneven: the batch sorted by class once
    (outside the graph), then every class searched with its own capacity and launch shape, all
    captured in one CUDA graph and replayed per batch.  Q and desc are the caller's (unsorted)
    batch; the graph reads sorted copies (update them with ``load`` to serve a new batch of the
    same classes).  ``replay`` returns ids / scores in sorted order, ``unsorted`` maps rows
    back to the caller's order."""

    def __init__(self, index: "Index", Q: torch.Tensor, A: torch.Tensor | None, desc: torch.Tensor, plan: dict,
                 ldo: int, width: int = 2, projection: int = PREC_FP32):
        dev = index.device
        self.index, self.A, self.plan, self.ldo = index, A, plan, ldo
        self.order = plan["order"]
        self.Qs = Q.index_select(0, self.order).contiguous()
        self.ds = desc.to(device=dev, dtype=torch.int32).index_select(0, self.order).contiguous()
        self.ids = torch.empty((Q.shape[0], ldo), dtype=torch.int32, device=dev)
        self.scores = torch.empty((Q.shape[0], ldo), dtype=torch.float32, device=dev)
        self.calls = []
        for c in plan["classes"]:
            sl = slice(*c["slice"])
            self.calls.append((sl, dict(k=c["k_max"], L=c["L_max"], rerank=c["rerank_max"], desc=self.ds[sl], ldo=ldo,
                                        out=(self.ids[sl], self.scores[sl]), width=width, projection=projection,
                                        hash_slots=c["hash_slots"], warps_per_block=c["warps_per_block"],
                                        warps_per_query=c["warps_per_query"],
                                        queries_per_warp=c.get("queries_per_warp", 1))))
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            self._run()  # warm-up: sizes the index's workspaces for every class outside the capture
        torch.cuda.current_stream(dev).wait_stream(s)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            self._run()

    def _run(self):
        for sl, kw in self.calls:
            self.index.search(self.Qs[sl], self.A, **kw)

    def load(self, Q: torch.Tensor):
        """Copy a new batch (same size and classes, caller's order) into the graph's sorted input."""
        torch.index_select(Q, 0, self.order, out=self.Qs)

    def replay(self):
        self.graph.replay()
        return self.ids, self.scores

    def unsorted(self, t: torch.Tensor) -> torch.Tensor:
        """Rows of a sorted result back in the caller's order."""
        out = torch.empty_like(t)
        out.index_copy_(0, self.order, t)
        return out


def _recall(ids: torch.Tensor, truth: torch.Tensor, k: int) -> float:
    a = ids[:, :k].long()
    hit = (a.unsqueeze(2) == truth[:, :k].long().unsqueeze(1)).any(dim=2) & (a >= 0)
    return float(hit.float().sum().item()) / (k * ids.shape[0])


def autotune_target_d(X: torch.Tensor, Q: torch.Tensor, truth: torch.Tensor, graph: torch.Tensor, entry: int,
                      ds=(64, 96, 128, 160, 192, 224, 256), k: int = 10, target: float = 0.90,
                      L_grid=(16, 24, 32, 48, 64, 80, 96, 112, 128, 144, 160, 192, 224, 256, 320, 384, 448, 512),
                      fit=None, primary_bits: int = 8, secondary_bits: int = 8, width: int = 2,
                      projection: int = PREC_BF16, hop_factor: float = 0.0, reps: int = 5) -> dict:
    """Target dimensionality d (the paper picks, per dataset, the d of highest QPS at the target
    accuracy on a fixed graph, App. D.2): for each d of `ds`, learn the projection with `fit(X, d)`
    (default: LeanVec-ID on X), encode X, search the validation queries Q on the given graph for
    the smallest L of `L_grid` whose recall@k against `truth` (m x k ids of the exact neighbours,
    computed by the caller) reaches `target`, with max_hops = ceil(hop_factor L) (0: none), and
    time that search with CUDA events.  Returns {"best": entry of the fastest d, "table": [...]};
    an entry holds d, L, max_hops, recall, qps and the projection A (for LeanVec-ID A = B)."""
    import math
    fit = fit or (lambda X_, d_: (lambda P: (P, P))(leanvec_fit_id(X_, d_, precision=PREC_BF16)))
    dev = X.device
    m = Q.shape[0]
    table, best = [], None
    for d in ds:
        if d > X.shape[1]:
            continue
        A, B = fit(X, d)
        idx = Index(dev).encode(X, B, primary_bits, secondary_bits, precision=PREC_BF16).set_graph(graph, entry)
        chosen = None
        for L in L_grid:
            if L < k:
                continue
            mh = int(math.ceil(hop_factor * L - 1e-9)) if hop_factor else 0
            r = _recall(idx.search(Q, A, k=k, L=L, rerank=L, max_hops=mh, width=width, projection=projection)[0],
                        truth, k)
            if r >= target:
                chosen = (L, mh, r)
                break
        row = {"d": d, "L": None, "max_hops": None, "recall": None, "qps": None}
        if chosen:
            L, mh, r = chosen
            run = lambda: idx.search(Q, A, k=k, L=L, rerank=L, max_hops=mh, width=width, projection=projection)
            run()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                run()
            e1.record()
            torch.cuda.synchronize()
            row.update(L=L, max_hops=mh, recall=r, qps=m * reps / (e0.elapsed_time(e1) / 1e3), A=A)
            if best is None or row["qps"] > best["qps"]:
                best = row
        table.append(row)
        idx.close()
    return {"best": best, "table": table}


class SearchGraph:
    """The whole search (projection, per-query prologue, persistent beam kernel with
    rerank) captured once in a CUDA graph for fixed query / output buffers, replayed per
    batch: a batch of uneven queries (per-query k, L, rerank in `desc`) is one graph launch.
    The first (uncaptured) call sizes the index's workspace before the capture."""

    def __init__(self, index: "Index", Q: torch.Tensor, A: torch.Tensor | None, k: int, L: int, rerank: int = 0,
                 desc: torch.Tensor | None = None, ldo: int | None = None, **kw):
        self.index, self.Q, self.A, self.desc = index, Q, A, desc
        self.ldo = k if ldo is None else ldo
        self.ids = torch.empty((Q.shape[0], self.ldo), dtype=torch.int32, device=index.device)
        self.scores = torch.empty((Q.shape[0], self.ldo), dtype=torch.float32, device=index.device)
        self.args = dict(k=k, L=L, rerank=rerank, desc=desc, ldo=self.ldo, out=(self.ids, self.scores), **kw)
        s = torch.cuda.Stream(device=index.device)
        s.wait_stream(torch.cuda.current_stream(index.device))
        with torch.cuda.stream(s):
            index.search(Q, A, **self.args)  # warm-up: sizes the workspace outside the capture
        torch.cuda.current_stream(index.device).wait_stream(s)
        torch.cuda.synchronize(index.device)
        self.graph = torch.cuda.CUDAGraph()
        # relaxed: the launch path queries occupancy and sets kernel attributes (no stream work)
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            index.search(Q, A, **self.args)

    def replay(self):
        self.graph.replay()
        return self.ids, self.scores