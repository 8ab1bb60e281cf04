"""The C ABI library loads and exports every function include/leanvec.h declares;
host-only entry points behave as documented without a GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT, cuda_available


@pytest.fixture(scope="module")
def native():
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    from paper_2312_16335_gb300 import _native
    return _native


def _declared():
    src = open(os.path.join(ROOT, "include", "leanvec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(leanvec_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(native):
    lib = native.lib()
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(native.SIGNATURES), "binding and header disagree"


def test_record_stride(native):
    lib = native.lib()
    assert lib.leanvec_record_stride(160, 8) == 192    # 160 codes + 16 B constants -> 176 -> 192
    assert lib.leanvec_record_stride(32, 8) == 64
    assert lib.leanvec_record_stride(160, 4) == 96     # 80 B codes + 16 -> 96
    assert lib.leanvec_record_stride(768, 8) == 800    # 768 + 16 = 784 -> 800
    assert lib.leanvec_record_stride(200, 8) == 224    # codes padded to 208, + 16 = 224
    assert lib.leanvec_record_stride(768, 32) == 3072
    assert lib.leanvec_record_stride(0, 8) < 0
    assert lib.leanvec_record_stride(16, 5) < 0
    assert b"bits" in lib.leanvec_last_error()


def test_argument_errors_need_no_gpu(native):
    lib = native.lib()
    assert lib.leanvec_column_mean(None, 0, 4, None, None) == -1
    assert lib.leanvec_lvq_encode(None, 4, 8, None, 8, None, None) == -1
    assert lib.leanvec_search(None, None, 1, None, None, None, None, None, 10, None, None) == -1
    assert lib.leanvec_search_host(None, None, 1, None, None, None, None, None, 10, 0, None) == -1
    assert b"search_host" in lib.leanvec_last_error()
    assert lib.leanvec_search_noalloc(None, None, 1, None, None, None, None, None, 10, None, None) == -1
    assert lib.leanvec_index_free(None) == 0
    # the scratch pool: a negative ordinal is an argument error; a device without a pool is a no-op
    assert lib.leanvec_trim_scratch(-1) == -1
    assert lib.leanvec_trim_scratch(63) == 0


@pytest.mark.skipif(cuda_available(), reason="checks the no-GPU failure path")
def test_index_create_fails_cleanly_without_gpu(native):
    lib = native.lib()
    h = ctypes.c_void_p()
    rc = lib.leanvec_index_create(ctypes.byref(h), 0)
    assert rc < 0 and not h.value


def _header_structs():
    """{typedef name: [field names]} of the plain structs include/leanvec.h declares."""
    src = open(os.path.join(ROOT, "include", "leanvec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        out[name] = [re.findall(r"(\w+)\s*(?:\[\w*\])?$", f.strip())[0] for f in body.split(";") if f.strip()]
    return out


def test_binding_structs_mirror_the_header(native):
    """The ctypes structures have the header's fields in the header's order (a field added to
    one side only would shift every later field)."""
    hs = _header_structs()
    pairs = {"lv_query_desc": native.LVQueryDesc, "lv_search_params": native.LVSearchParams,
             "lv_index_info": native.LVIndexInfo, "lv_fit_opts": native.LVFitOpts,
             "lv_fit_report": native.LVFitReport}
    for cname, py in pairs.items():
        assert cname in hs, cname
        assert hs[cname] == [f[0] for f in py._fields_], cname
