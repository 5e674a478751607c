"""ctypes loader for libemb.so (the C ABI declared in include/emb.h).

Loading fails loudly when the in-tree library has not been built: there is no
CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# EMB_LIBRARY=check selects the bounds-mode build (lib/libemb_check.so, see build.py)
LIB_PATH = os.path.join(HERE, "lib", "libemb_check.so" if os.environ.get("EMB_LIBRARY") == "check" else "libemb.so")

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
PI64 = ctypes.POINTER(ctypes.c_int64)
PI32 = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes); mirrors include/emb.h
SIGNATURES = {
    "emb_status_string": (ctypes.c_char_p, [I32]),
    "emb_status_get": (I32, [P, PI32]),
    "emb_directions": (I32, [PI32]),
    "emb_launch_count": (I32, [PI64]),
    "emb_probe_predicates": (I32, [I32, P, I64, P, P, P]),
    "emb_mesh_create": (I32, [P, P, I64, I64, I32, I32, P, ctypes.POINTER(P)]),
    "emb_mesh_destroy": (None, [P]),
    "emb_mesh_update": (I32, [P, P, I64, P]),
    "emb_forest_root": (I32, [I32, I32, P, ctypes.POINTER(P)]),
    "emb_forest_destroy": (None, [P]),
    "emb_forest_root_window": (I32, [I32, I32, I32, I32, I32, I32, P, ctypes.POINTER(P)]),
    "emb_mesh_subset": (I32, [P, I64, I64, I64, I64, P, I64, P, ctypes.POINTER(P), PI64]),
    "emb_splice": (I32, [P, P, I32, I32, I32, I32, P, P, P, P, I64, P, P, P, P, I64, P, P, P, P, P, I64, PI64, P]),
    "emb_forest_refine": (I32, [P, I32, P, P]),
    "emb_forest_num_blocks": (I32, [P, I32, PI64]),
    "emb_forest_blocks": (I32, [P, I32, P, P]),
    "emb_forest_neighbors": (I32, [P, I32, P, P]),
    "emb_forest_masks": (I32, [P, I32, P, P]),
    "emb_bin": (I32, [P, P, I32, I32, P, ctypes.POINTER(P)]),
    "emb_bin_ex": (I32, [P, P, I32, I32, I32, P, ctypes.POINTER(P)]),
    "emb_bins_destroy": (None, [P]),
    "emb_bins_stats": (I32, [P, PI64, PI64]),
    "emb_bins_copy": (I32, [P, P, P, P, P]),
    "emb_voxelize": (I32, [P, P, I32, P, P]),
    "emb_voxelize_guard": (I32, [P, P, P, P, P]),
    "emb_refine_flags": (I32, [P, P, I32, I32, P, P]),
    "emb_refine_flags_paper": (I32, [P, I32, ctypes.c_double, P, P]),
    "emb_cutlinks_count": (I32, [P, I32, PI64, P]),
    "emb_cutlinks_prepare": (I32, [P, I32, P]),
    "emb_cutlinks": (I32, [P, P, I32, P, P, P, P, I64, P, P]),
    "emb_mex_force": (I32, [P, I32, P, P, P, I64, P, I64, P, P]),
    "emb_mex_force_backward": (I32, [P, I32, P, P, P, I64, P, I64, P, P, P]),
    "emb_mex_force_noalloc": (I32, [P, I32, P, P, P, I64, P, I64, P, P]),
    "emb_cutlinks_backward": (I32, [P, P, P, P, P, P, I64, P, P, P]),
    "emb_lbm_step": (I32, [P, I32, P, P, P, I64, ctypes.c_float, P, P, P, I64, I32, P]),
    "emb_batch_create": (I32, [P, P, P, P, I32, P, ctypes.POINTER(P)]),
    "emb_batch_run": (I32, [P, P]),
    "emb_batch_capture": (I32, [P, P]),
    "emb_batch_launch": (I32, [P, P]),
    "emb_batch_autotune": (I32, [P, P, P]),
    "emb_batch_autotune_ex": (I32, [P, P, I32, P]),
    "emb_batch_create_ex": (I32, [P, P, P, P, I32, I32, P, ctypes.POINTER(P)]),
    "emb_batch_counts": (I32, [P, I32, P, P, P]),
    "emb_batch_configure": (I32, [P, P]),
    "emb_batch_info": (I32, [P, I32, P, PI64]),
    "emb_batch_results": (I32, [P, I32, I32, P, P, P, P, P, P, P]),
    "emb_batch_destroy": (None, [P]),
}

_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2512_01251_gb300.build` "
                "(or __graft_entry__.build()); this package has no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
