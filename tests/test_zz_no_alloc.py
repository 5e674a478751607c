"""The allocation-free force entry point against the regular one.

emb_mex_force_noalloc serves callers that cannot call cudaMalloc mid-run: a
solver loop that reserved all device memory through its own pool, or a time
step that must not pay a driver allocation.  It keeps its partial sums in a
fixed array inside the library.  This test calls it through the C ABI twice in
a row (the second call reuses the array left by the first) and compares both
results with emb_mex_force under the tolerance of the force parity test.  This
file is collected last on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from synth import populations, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _call_noalloc(lib, E, L, pop, out, n=None, stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return lib.emb_mex_force_noalloc(E.forest.h, 19, ctypes.c_void_p(L["cell"].data_ptr()),
                                     ctypes.c_void_p(L["dir"].data_ptr()), ctypes.c_void_p(L["q"].data_ptr()),
                                     L["q"].numel() if n is None else n, ctypes.c_void_p(pop.data_ptr()), pop.shape[1],
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))


@pytest.mark.parametrize("name", ["icosphere_320", "star_1k"])
def test_noalloc_force_matches_regular_entry_point_twice(name):
    import torch

    import paper_2512_01251_gb300 as P
    from paper_2512_01251_gb300._lib import load
    lib = load()
    w = workload(name)
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), w.R, w.levels, w.band, 19)  # builds the neighbour table
    L = E.links
    nblk = P.emb_forest_num_blocks(E.forest, w.levels)
    pop = torch.from_numpy(populations(nblk * 64, seed=31)).cuda()
    ref = P.emb_mex_force(E.forest, 19, L["cell"], L["dir"], L["q"], pop).cpu().numpy().astype(np.float64)
    for rep in range(2):
        out = torch.full((3,), float("nan"), dtype=torch.float32, device="cuda")
        assert _call_noalloc(lib, E, L, pop, out) == P.EMB_OK
        got = out.cpu().numpy().astype(np.float64)
        # same tolerance as the force parity test against the FP64 oracle
        assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref) + 1e-9 * (L["q"].numel() + 1)), (rep, got, ref)
    assert P.emb_status_get() == P.EMB_OK


def test_noalloc_force_rejects_too_many_links():
    import torch

    import paper_2512_01251_gb300 as P
    from paper_2512_01251_gb300._lib import load
    lib = load()
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), w.R, w.levels, w.band, 19)
    L = E.links
    nblk = P.emb_forest_num_blocks(E.forest, w.levels)
    pop = torch.from_numpy(populations(nblk * 64, seed=32)).cuda()
    out = torch.zeros(3, dtype=torch.float32, device="cuda")
    # beyond the 2,097,152-link limit the call is refused before any work is enqueued
    assert _call_noalloc(lib, E, L, pop, out, n=2_097_153) == P.EMB_ERR_CAPACITY
    assert _call_noalloc(lib, E, L, pop, out, n=L["q"].numel()) == P.EMB_OK
