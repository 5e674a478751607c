"""The binning ablation (the paper's variants 'n', 'r' and 'rc' of Sec. 4): the x-line
filter is exact, so running the voxelizer on every triangle, or on the filter's flags
without compaction, gives the same forest, masks, flags and link table as the
default filtered and compacted list."""
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


@pytest.mark.parametrize("name", ["star_1k", "star_20k", "star_4k_r3"])
def test_filter_modes_give_identical_embeddings(name):
    import torch

    import paper_2512_01251_gb300 as P
    w = workload(name)
    v, t = w.build_mesh()
    lat = max(w.lattices)
    res = {}
    for mode in (P.EMB_BIN_FILTER_COMPACT, P.EMB_BIN_FILTER_ONLY, P.EMB_BIN_NO_FILTER):
        E = P.embed(torch.from_numpy(v), torch.from_numpy(t), w.R, w.levels, w.band, lat, bin_mode=mode)
        res[mode] = dict(blocks=[b.cpu().numpy() for b in E.fetch_blocks()], masks=[m.cpu().numpy() for m in E.masks],
                         flags=[f.cpu().numpy() for f in E.flags],
                         links={k: E.links[k].cpu().numpy() for k in ("cell", "dir", "q", "tri")})
    a = res[P.EMB_BIN_FILTER_COMPACT]
    for mode in (P.EMB_BIN_FILTER_ONLY, P.EMB_BIN_NO_FILTER):
        b = res[mode]
        for L in range(w.levels + 1):
            np.testing.assert_array_equal(a["blocks"][L], b["blocks"][L], err_msg=f"mode {mode} blocks L={L}")
            np.testing.assert_array_equal(a["masks"][L], b["masks"][L], err_msg=f"mode {mode} masks L={L}")
        for L in range(w.levels):
            np.testing.assert_array_equal(a["flags"][L], b["flags"][L], err_msg=f"mode {mode} flags L={L}")
        for k in ("cell", "dir", "tri"):
            np.testing.assert_array_equal(a["links"][k], b["links"][k], err_msg=f"mode {mode} links {k}")
        np.testing.assert_array_equal(a["links"]["q"].view(np.uint32), b["links"]["q"].view(np.uint32))


def test_filter_counts_and_bad_mode():
    import torch

    import paper_2512_01251_gb300 as P
    w = workload("star_20k")
    v, t = w.build_mesh()
    m = P.emb_mesh_create(torch.from_numpy(v), torch.from_numpy(t), w.R)
    f = P.emb_forest_root(w.R, w.levels)
    b0 = P.emb_bin(m, f, 0, 27)
    b2 = P.emb_bin(m, f, 0, 27, mode=P.EMB_BIN_NO_FILTER)
    nf0, _ = P.emb_bins_stats(b0)
    nf2, _ = P.emb_bins_stats(b2)
    assert nf2 == len(t) and 0 < nf0 < len(t)  # the filter drops triangles that no root-level x-line crosses
    with pytest.raises(P.EmbError):
        P.emb_bin(m, f, 0, 27, mode=7)
