"""The C-ABI library builds, loads without a GPU and exports every declared call."""
from __future__ import annotations

import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "emb.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(emb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_01251_gb300 import build as B
    if not os.path.exists(B.LIB) and shutil.which(B.NVCC) is None and not os.path.exists(B.NVCC):
        pytest.skip("nvcc not available and libemb.so not built")
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_path():
    names = _declared()
    for n in ["emb_bin", "emb_voxelize", "emb_refine_flags", "emb_cutlinks", "emb_cutlinks_backward",
              "emb_mex_force", "emb_mex_force_backward", "emb_mesh_create", "emb_forest_root", "emb_forest_refine"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2512_01251_gb300._lib import SIGNATURES
    assert set(SIGNATURES) == set(_declared())


def test_direction_table_matches_the_oracle(lib, orc):
    buf = (ctypes.c_int32 * 81)()
    assert lib.emb_directions(buf) == 0
    got = np.array(list(buf), dtype=np.int64).reshape(27, 3)
    np.testing.assert_array_equal(got, orc.directions())
    # opposite pairs are adjacent
    for i in range(1, 27, 2):
        np.testing.assert_array_equal(got[i], -got[i + 1])


def test_status_strings(lib):
    lib.emb_status_string.restype = ctypes.c_char_p
    assert lib.emb_status_string(0) == b"EMB_OK"
    assert lib.emb_status_string(-3) == b"EMB_ERR_CAPACITY"


def test_package_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2512_01251_gb300._lib as L
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(ImportError):
        L.load()


def test_argument_errors_are_reported_before_any_device_work(lib):
    """Host-side validation of the boundary: each call below returns its documented error
    from the argument checks alone (no handle, no device buffer is touched)."""
    from paper_2512_01251_gb300._lib import SIGNATURES
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    BAD, RANGE = -1, -6
    fake = ctypes.c_void_p(16)  # never dereferenced: every case fails a check first
    out = ctypes.c_void_p()
    # meshes: an empty triangle list, too few vertices, R out of range, a frame that overflows
    assert lib.emb_mesh_create(fake, fake, 3, 0, 4, 0, None, ctypes.byref(out)) == BAD
    assert lib.emb_mesh_create(fake, fake, 2, 1, 4, 0, None, ctypes.byref(out)) == BAD
    assert lib.emb_mesh_create(fake, fake, 3, 1, 0, 0, None, ctypes.byref(out)) == BAD
    assert lib.emb_mesh_create(fake, fake, 3, 1, 1 << 18, 0, None, ctypes.byref(out)) == RANGE
    assert lib.emb_mesh_create(fake, fake, 3, 1, 33, 0, None, ctypes.byref(out)) == RANGE  # 33 * 2^20 >= 2^25
    assert lib.emb_mesh_create(None, fake, 3, 1, 4, 0, None, ctypes.byref(out)) == BAD
    assert out.value is None
    # forests: R and level count out of range
    assert lib.emb_forest_root(0, 2, None, ctypes.byref(out)) == BAD
    assert lib.emb_forest_root(4, 16, None, ctypes.byref(out)) == BAD
    assert lib.emb_forest_root(4, -1, None, ctypes.byref(out)) == BAD
    # every stage rejects missing handles
    assert lib.emb_bin(None, None, 0, 19, None, ctypes.byref(out)) == BAD
    assert lib.emb_bin_ex(fake, fake, 0, 21, 0, None, ctypes.byref(out)) == BAD  # no such lattice
    assert lib.emb_bin_ex(fake, fake, 0, 19, 7, None, ctypes.byref(out)) == BAD  # no such binning mode
    assert lib.emb_voxelize(None, None, 0, None, None) == BAD
    assert lib.emb_voxelize_guard(None, None, None, None, None) == BAD
    assert lib.emb_refine_flags(None, None, 0, 2, None, None) == BAD
    assert lib.emb_refine_flags(fake, fake, 0, 0, None, None) == BAD  # band below 1
    assert lib.emb_refine_flags_paper(fake, 0, -1.0, None, None) == BAD
    n = ctypes.c_int64(0)
    assert lib.emb_cutlinks_count(fake, 20, ctypes.byref(n), None) == BAD
    assert lib.emb_cutlinks_prepare(fake, 20, None) == BAD
    assert lib.emb_cutlinks_prepare(None, 19, None) == BAD
    assert lib.emb_cutlinks(None, None, 19, None, None, None, None, 0, None, None) == BAD
    assert lib.emb_lbm_step(fake, 19, None, None, None, 0, 2.5, fake, fake, fake, 64, 7, None) == BAD  # omega
    assert lib.emb_lbm_step(fake, 19, None, None, None, 0, 1.0, fake, fake, fake, 64, 8, None) == BAD  # phases
    assert lib.emb_batch_create(None, None, None, None, 1, None, ctypes.byref(out)) == BAD
    arr = (ctypes.c_void_p * 1)(16)
    lv = (ctypes.c_int32 * 1)(2)
    assert lib.emb_batch_create(arr, lv, lv, lv, 0, None, ctypes.byref(out)) == BAD  # empty batch
