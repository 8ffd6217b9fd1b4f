"""CPU-side checks of the boundary: the library builds for sm_103a, loads, and exports every
function include/ace.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1706_06664_gb300 import ace, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ace.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ace_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(ace.LIB_PATH)


def test_header_declares_expected_entry_points():
    names = _declared()
    assert "ace_create" in names and "ace_insert_score" in names
    assert sorted(ace.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_declares_and_reports_version():
    lib = ace.load_library()
    assert b"sm_103a" in lib.ace_version()
    assert lib.ace_last_error() == b""


def test_errors_without_device_work():
    lib = ace.load_library()
    h = ctypes.c_void_p()
    # invalid shapes are rejected before any CUDA call
    assert lib.ace_create(0, 4, 4, 1, ctypes.byref(h)) == ace.ACE_ERR_ARG
    assert b"invalid shape" in lib.ace_last_error()
    assert lib.ace_create(4, 25, 4, 1, ctypes.byref(h)) == ace.ACE_ERR_ARG
    assert lib.ace_set_precision(None, 0) == ace.ACE_ERR_ARG
    assert lib.ace_insert(None, None, 0, 0, None) == ace.ACE_ERR_ARG
    # every entry point checks its arguments before any CUDA call (ace.h's error contract)
    E = ace.ACE_ERR_ARG
    t = ctypes.c_uint64()
    st = ctypes.c_uint32()
    nbytes = ctypes.c_size_t()
    one = ctypes.c_int64(1)
    assert lib.ace_host_wait(None) == E
    assert lib.ace_window_enable(None, 10) == E
    assert lib.ace_set_privacy(None, ctypes.c_float(1.0), 1) == E
    assert lib.ace_save_size(None, ctypes.byref(nbytes)) == E
    assert lib.ace_save(None, None, 0, None) == E
    assert lib.ace_batch_insert_score(None, 1, None, None, 0, 1.0, None, None, None, None) == E
    assert lib.ace_server_create(None, 1, 1 << 20, ctypes.byref(t)) == E
    assert lib.ace_server_submit(None, 0, 1, None, 1, 0, 1.0, None, None, None, ctypes.byref(t)) == E
    assert lib.ace_server_wait(None, 1, None) == E
    assert lib.ace_server_drain(None) == E
    assert lib.ace_server_info(None, None, None) == E
    assert lib.ace_server_destroy(None) == ace.ACE_OK  # destroying nothing is a no-op
    assert lib.ace_exact_score(None, -1, None, 0, 4, 0, 4, None, None) == E
    assert lib.ace_exact_score(ctypes.byref(one), 1, None, 0, 4, 0, 65, ctypes.byref(one), None) == E
    assert b"K <= 64" in lib.ace_last_error()
    assert lib.ace_exact_score(ctypes.byref(one), 1, None, 0, 4, 7, 4, ctypes.byref(one), None) == E
    assert lib.ace_wait_probe(2, 1000000, ctypes.byref(st), None) == E
    assert lib.ace_wait_probe(0, 10, ctypes.byref(st), None) == E
    assert lib.ace_wait_probe(0, 1000000, None, None) == E


def _fnv1a64(b: bytes) -> int:
    h = 0xCBF29CE484222325
    for c in b:
        h = ((h ^ c) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def _blob(d=3, K=2, L=2, version=2, hdr_patch=None, extra=b"", payload=None):
    """A checkpoint laid out as ace_save writes it: magic, header words (version, d, K, L, ...;
    version 2 adds the privacy words 16-19), W (d x KL binary32), the L x 2^K counts (zeros,
    or `payload` in their place), and the FNV-1a 64 checksum of everything before it."""
    words = 16 if version == 1 else 20
    hdr = [0] * words
    hdr[0], hdr[1], hdr[2], hdr[3] = version, d, K, L
    for k, v in (hdr_patch or {}).items():
        hdr[k] = v
    body = b"ACEDET01" + b"".join(int(v).to_bytes(8, "little") for v in hdr)
    body += (b"\0" * (d * K * L * 4 + (1 << K) * L * 4) if payload is None else payload) + extra
    return body + _fnv1a64(body).to_bytes(8, "little")


def test_checkpoint_loader_rejects_malformed_blobs_before_device_work():
    lib = ace.load_library()
    h = ctypes.c_void_p()

    def load(b):
        buf = ctypes.create_string_buffer(b, len(b))
        return lib.ace_load(buf, len(b), ctypes.byref(h)), lib.ace_last_error().decode()

    assert lib.ace_load(None, 0, ctypes.byref(h)) == ace.ACE_ERR_ARG
    good = _blob()
    cases = [
        (good[:100], "not an ACE checkpoint"),
        (b"ACEDET02" + good[8:], "not an ACE checkpoint"),
        (_blob(version=3), "version 3 is not supported"),
        (_blob(K=25, payload=b""), "shape"),
        (_blob(d=0, payload=b""), "shape"),
        (_blob(K=16, L=4097, payload=b""), "shape"),
        (_blob(extra=b"\0"), "needs"),
        (_blob(hdr_patch={16: 0x7FC00000}), "privacy sigma"),  # sigma = NaN
        (_blob(hdr_patch={16: 1 << 32}), "privacy sigma"),
        (good[:-1] + bytes([good[-1] ^ 1]), "checksum"),
        (good[:40] + bytes([good[40] ^ 1]) + good[41:], "checksum"),
        (_blob(version=1)[:-1] + b"\0", "checksum"),  # the earlier layout, without privacy words
    ]
    # (the checksum is the last check: a blob that only fails it passed all the others)
    for b, msg in cases:
        rc, err = load(b)
        assert rc == ace.ACE_ERR_ARG and msg in err, (msg, rc, err)
