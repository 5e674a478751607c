"""The bounds-mode build (-DEMB_CHECK, lib/libemb_check.so): every index a kernel
derives from data (block ids from the level index and the neighbour table, link work
items, bin triangle ids, voxelizer accumulators) is checked before use, and one out of
range would set EMB_ERR_BOUNDS in the device status instead of faulting.  The parity
cases and the ~112K-triangle workload run through that build in a child process: the
status must stay EMB_OK and every output must equal the oracle's."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch
import paper_2512_01251_gb300 as P
from paper_2512_01251_gb300 import _lib
assert _lib.LIB_PATH.endswith("libemb_check.so"), _lib.LIB_PATH
from oracle import oracle as O
from gpu_common import compare_full, gpu_embed
from synth import workload
import corner_case as K
cases = [(workload(n).build_mesh(), workload(n), lat) for n, lat in
         [("icosphere_320", 19), ("star_4k_r3", 27), ("star_112k", 27)]]
for (v, t), w, lat in cases:
    _, g = gpu_embed(v, t, w.R, w.levels, w.band, lat)
    assert P.emb_status_get() == P.EMB_OK
    compare_full(g, O.embed_lines(v, t, w.R, w.levels, w.band, lat), w.levels)
v, t = K.mesh()
_, g = gpu_embed(v, t, K.R, K.LEVELS, K.BAND, K.LATTICE)
assert P.emb_status_get() == P.EMB_OK
compare_full(g, O.embed_lines(v, t, K.R, K.LEVELS, K.BAND, K.LATTICE), K.LEVELS)
print("bounds mode ok")
'''


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_bounds_mode_build_runs_clean():
    from paper_2512_01251_gb300 import build as B
    B.build(check=True)
    env = dict(os.environ, EMB_LIBRARY="check")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "bounds mode ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
