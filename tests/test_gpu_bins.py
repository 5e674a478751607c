"""The binning step's outputs on the GPU (emb_bin, read back with emb_bins_copy) against
the oracle, element by element: the filtered triangle ids of every level (ascending,
exact) and, at the finest level, each block's bin as a set (the CUDA bins are unordered
within a bin; the oracle's are ascending)."""
from __future__ import annotations

import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name", ["icosphere_320", "star_4k_r3"])
def test_bins_match_the_oracle(orc, name):
    import torch

    import paper_2512_01251_gb300 as P
    w = workload(name)
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), w.R, w.levels, w.band, 19, keep_bins=True)
    tri9 = orc.tri_coords(orc.int_coords(v, w.R), t)
    blocks = [b.cpu().numpy().astype(np.int64) for b in E.fetch_blocks()]
    for L in range(w.levels + 1):
        c = P.emb_bins_copy(E.bins[L], E.forest if L == w.levels else None)
        np.testing.assert_array_equal(c["filtered"].cpu().numpy().astype(np.int64), orc.xfilter(tri9, w.R, L),
                                      err_msg=f"filtered ids L={L}")
    off = c["off"].cpu().numpy().astype(np.int64)
    ent = c["ent"].cpu().numpy().astype(np.int64)
    ob = orc.finest_bins(tri9, w.R, w.levels, blocks[w.levels])
    assert len(off) == len(ob) + 1 and off[0] == 0 and off[-1] == len(ent)
    assert len(ent) == sum(len(x) for x in ob)
    for i, want in enumerate(ob):
        np.testing.assert_array_equal(np.sort(ent[off[i]:off[i + 1]]), want, err_msg=f"bin of block {i}")
    assert P.emb_status_get() == P.EMB_OK
