"""Index files without a GPU: files written here by an independent writer that follows the layout
documented in include/leanvec.h are accepted by leanvec_index_file_check, and every kind of damage
(a flipped byte, truncation, a wrong magic or version, a stride that does not match the record
geometry, a graph id out of range, an entry out of range) is rejected as LV_ERR_CORRUPT."""
import struct

import numpy as np
import pytest

LV_ERR_CORRUPT = -7
MASK = (1 << 64) - 1


@pytest.fixture(scope="module")
def lv():
    from paper_2312_16335_gb300 import build_lib
    build_lib.build()
    import paper_2312_16335_gb300 as lv
    return lv


def checksum(data: bytes) -> int:
    """64-bit FNV-1a over little-endian 64-bit words, the last one zero-padded."""
    if len(data) % 8:
        data = data + bytes(8 - len(data) % 8)
    h = 0xCBF29CE484222325
    for (w,) in struct.iter_unpack("<Q", data):
        h = ((h ^ w) * 0x100000001B3) & MASK
    return h


def _up(x, a):
    return (x + a - 1) // a * a


def stride(dim, bits, metric=0):
    """Record stride of the documented geometry: LVQ codes padded to 16 bytes + 16 (IP) or 32 (L2)
    bytes of constants, FP16 / float32 vectors, each rounded up to 32 bytes."""
    if bits in (4, 8):
        cb = dim if bits == 8 else (dim + 1) // 2
        return _up(_up(cb, 16) + (32 if metric else 16), 32)
    return _up(dim * bits // 8, 32)


def make_file(n=7, D=12, d=5, pbits=8, sbits=8, R=3, metric=0, entry=2, seed=0, **over):
    rng = np.random.default_rng(seed)
    ps, ss = stride(d, pbits, metric), (stride(D, sbits, metric) if sbits else 0)
    f = dict(metric=metric, D=D, d=d, pbits=pbits, sbits=sbits, R=R, entry=entry, n=n, ps=ps, ss=ss, version=1,
             magic=b"LEANVEC\0")
    f.update(over)
    head = (f["magic"] + struct.pack("<II", f["version"], 96)
            + struct.pack("<7i", f["metric"], f["D"], f["d"], f["pbits"], f["sbits"], f["R"], f["entry"])
            + struct.pack("<f", 0.25) + struct.pack("<3q", f["n"], f["ps"], f["ss"]) + bytes(24))
    assert len(head) == 96
    body = rng.integers(0, 256, n * ps, dtype=np.uint8).tobytes()
    if pbits != 32:
        body += rng.standard_normal(d).astype("<f4").tobytes()
    if sbits:
        body += rng.integers(0, 256, n * ss, dtype=np.uint8).tobytes()
    if sbits == 8:
        body += rng.standard_normal(D).astype("<f4").tobytes()
    g = rng.integers(-1, n, (n, R)).astype("<i4")
    if "graph" in over:
        g = np.asarray(over["graph"], "<i4")
    body += g.tobytes()
    return head + body, f


def write(tmp_path, name, head_body, raw_checksum=None):
    data = head_body
    cs = checksum(data) if raw_checksum is None else raw_checksum
    p = tmp_path / name
    p.write_bytes(data + struct.pack("<Q", cs))
    return str(p)


def corrupt_code(lv, path):
    with pytest.raises(lv.LeanVecError) as e:
        lv.leanvec_index_file_check(path)
    return e.value.code


@pytest.mark.parametrize("kw", [dict(), dict(pbits=4), dict(sbits=16), dict(sbits=0), dict(metric=1),
                                dict(R=0, entry=-1), dict(pbits=32, d=12, sbits=0)])
def test_valid_files_are_accepted(lv, tmp_path, kw):
    data, f = make_file(**kw)
    info = lv.leanvec_index_file_check(write(tmp_path, "ok.lvi", data))
    assert (info["n"], info["D"], info["d"]) == (f["n"], f["D"], f["d"])
    assert (info["primary_bits"], info["secondary_bits"], info["R"], info["entry"]) == (
        f["pbits"], f["sbits"], f["R"], f["entry"])
    assert (info["primary_stride"], info["secondary_stride"]) == (f["ps"], f["ss"])
    assert info["mu2"] == 0.25


def test_damage_is_rejected(lv, tmp_path):
    data, _ = make_file()
    good = write(tmp_path, "good.lvi", data)
    raw = open(good, "rb").read()
    for pos in (0, 20, 96, len(raw) // 2, len(raw) - 9, len(raw) - 1):  # header, records, graph, checksum
        b = bytearray(raw)
        b[pos] ^= 0x40
        p = tmp_path / f"flip{pos}.lvi"
        p.write_bytes(bytes(b))
        assert corrupt_code(lv, str(p)) == LV_ERR_CORRUPT
    short = tmp_path / "short.lvi"
    short.write_bytes(raw[:-12])
    assert corrupt_code(lv, str(short)) == LV_ERR_CORRUPT
    tiny = tmp_path / "tiny.lvi"
    tiny.write_bytes(raw[:50])
    assert corrupt_code(lv, str(tiny)) == LV_ERR_CORRUPT


@pytest.mark.parametrize("over", [dict(magic=b"LEANVEX\0"), dict(version=2), dict(ps=64), dict(ss=64),
                                  dict(entry=7), dict(entry=-1), dict(pbits=5), dict(d=13),
                                  dict(graph=[[0, 1, 7]] + [[0, 1, 2]] * 6),
                                  dict(graph=[[0, 1, -2]] + [[0, 1, 2]] * 6)])
def test_inconsistent_files_are_rejected(lv, tmp_path, over):
    """Valid checksums over inconsistent contents: each is caught by the validation itself."""
    data, _ = make_file(**over)
    assert corrupt_code(lv, write(tmp_path, "bad.lvi", data)) == LV_ERR_CORRUPT


def test_missing_file_is_an_argument_error(lv, tmp_path):
    with pytest.raises(lv.LeanVecError) as e:
        lv.leanvec_index_file_check(str(tmp_path / "absent.lvi"))
    assert e.value.code == -1
