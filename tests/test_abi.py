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
