"""ctypes loader for ``_build/libleanvec.so`` (the C ABI of include/leanvec.h).

There is no fallback: if the library is missing or cannot be loaded, every call
raises.  Build it with ``__graft_entry__.build()`` or ``python -m
paper_2312_16335_gb300.build_lib``.
"""
from __future__ import annotations

import ctypes
import os

from . import build_lib

_lib = None

c_i32, c_i64, c_u64, c_f32, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float, ctypes.c_void_p


class LVQueryDesc(ctypes.Structure):
    _fields_ = [("k", c_i32), ("L", c_i32), ("rerank", c_i32), ("max_hops", c_i32)]


class LVSearchParams(ctypes.Structure):
    _fields_ = [("uniform", LVQueryDesc), ("projection", c_i32), ("hash_slots", c_i32),
                ("warps_per_block", c_i32), ("width", c_i32), ("warps_per_query", c_i32), ("event_begin", c_vp),
                ("event_end", c_vp), ("queries_per_warp", c_i32),
                ("visited_bits", c_i32)]


class LVIndexInfo(ctypes.Structure):
    _fields_ = [("n", c_i64), ("D", c_i32), ("d", c_i32), ("primary_bits", c_i32),
                ("secondary_bits", c_i32), ("primary_stride", c_i64), ("secondary_stride", c_i64),
                ("R", c_i32), ("entry", c_i32), ("mu2", c_f32), ("last_search_kernels", c_i32)]


class LVFitOpts(ctypes.Structure):
    _fields_ = [("method", c_i32), ("alpha", c_f32), ("tol", c_f32), ("max_iter", c_i32), ("line_search", c_i32),
                ("precision", c_i32), ("es_xatol", ctypes.c_double)]


class LVFitReport(ctypes.Structure):
    _fields_ = [("iterations", c_i32), ("evaluations", c_i32), ("beta", ctypes.c_double), ("loss0", ctypes.c_double),
                ("loss", ctypes.c_double), ("loss_trace", ctypes.POINTER(ctypes.c_double)),
                ("trace_capacity", c_i32)]


# (name, restype, argtypes) for every symbol of include/leanvec.h
SIGNATURES = {
    "leanvec_last_error": (ctypes.c_char_p, []),
    "leanvec_trim_scratch": (ctypes.c_int, [ctypes.c_int]),
    "leanvec_record_stride": (c_i64, [c_i32, c_i32]),
    "leanvec_column_mean": (c_i32, [c_vp, c_i64, c_i32, c_vp, c_vp]),
    "leanvec_lvq_encode": (c_i32, [c_vp, c_i64, c_i32, c_vp, c_i32, c_vp, c_vp]),
    "leanvec_project": (c_i32, [c_vp, c_i64, c_i32, c_vp, c_i32, c_vp, c_i32, c_i32, c_vp]),
    "leanvec_index_create": (c_i32, [ctypes.POINTER(c_vp), c_i32]),
    "leanvec_index_free": (c_i32, [c_vp]),
    "leanvec_index_info": (c_i32, [c_vp, ctypes.POINTER(LVIndexInfo)]),
    "leanvec_index_save": (c_i32, [c_vp, ctypes.c_char_p, c_vp]),
    "leanvec_index_load": (c_i32, [c_vp, ctypes.c_char_p, c_vp]),
    "leanvec_index_file_check": (c_i32, [ctypes.c_char_p, ctypes.POINTER(LVIndexInfo)]),
    "leanvec_set_metric": (c_i32, [c_vp, c_i32]),
    "leanvec_index_buffers": (c_i32, [c_vp] + [ctypes.POINTER(c_vp)] * 5),
    "leanvec_encode": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp, c_i32, c_i32, c_i32, c_i32, c_vp]),
    "leanvec_set_primary": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp, c_i32, c_i32, c_vp]),
    "leanvec_set_secondary": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp, c_vp]),
    "leanvec_encode_fp32": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp]),
    "leanvec_set_graph": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_vp]),
    "leanvec_get_graph": (c_i32, [c_vp, c_vp, ctypes.POINTER(c_i32), c_vp]),
    "leanvec_build_graph": (c_i32, [c_vp, c_i32, c_i32, c_f32, c_i32, c_i32, c_u64, c_i32, c_vp]),
    "leanvec_search": (c_i32, [c_vp, c_vp, c_i64, c_vp, ctypes.POINTER(LVSearchParams), c_vp, c_vp, c_vp,
                               c_i32, c_vp, c_vp]),
    "leanvec_sync_status": (c_i32, [c_vp, c_vp]),
    "leanvec_search_host": (c_i32, [c_vp, c_vp, c_i64, c_vp, ctypes.POINTER(LVSearchParams), c_vp, c_vp, c_vp,
                                    c_i32, c_i64, c_vp]),
    "leanvec_search_noalloc": (c_i32, [c_vp, c_vp, c_i64, c_vp, ctypes.POINTER(LVSearchParams), c_vp, c_vp, c_vp,
                                       c_i32, c_vp, c_vp]),
    "leanvec_second_moment": (c_i32, [c_vp, c_i64, c_i32, c_vp, c_i32, c_vp]),
    "leanvec_eigh": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "leanvec_eigh_top": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp, c_vp]),
    "leanvec_fit_id": (c_i32, [c_vp, c_i64, c_i32, c_i32, c_vp, c_vp, c_i32, c_vp]),
    "leanvec_ood_loss_fwd": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, c_i64, c_i32, c_i32,
                                     ctypes.POINTER(ctypes.c_double), c_vp]),
    "leanvec_ood_loss_bwd": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, c_i64, c_i32, c_i32, c_f32, c_vp, c_vp, c_vp]),
    "leanvec_spectral_clip": (c_i32, [c_vp, c_i32, c_i32, c_vp]),
    "leanvec_fit_ood": (c_i32, [c_vp, c_i64, c_vp, c_i64, c_i32, c_i32, ctypes.POINTER(LVFitOpts), c_vp, c_vp,
                                ctypes.POINTER(LVFitReport), c_vp]),
}


class LeanVecError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"leanvec error {code}: {msg}")
        self.code = code


def lib():
    global _lib
    if _lib is None:
        path = build_lib.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first (__graft_entry__.build())")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> int:
    if rc < 0:
        raise LeanVecError(rc, lib().leanvec_last_error().decode())
    return rc
