"""The paper's block-layer refinement rules on the GPU (emb_refine_flags_paper and the
voxelizer's handling of surface inside unrefined regions) against the oracle, element
by element: forest, masks of every level, flags, and the cut-link table (neighbours
in missing blocks count as fluid)."""
from __future__ import annotations

import numpy as np
import pytest

from synth import workload
from synth.meshes import axis_box, icosphere, snap

pytestmark = pytest.mark.gpu

Q_TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _compare(orc, v, t, R, levels, lattice, d_spec):
    import torch

    import paper_2512_01251_gb300 as P
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), R, levels, 2, lattice, d_spec=d_spec)
    o = orc.embed(v, t, R, levels, 2, lattice, d_spec=d_spec)
    blocks = [b.cpu().numpy().astype(np.int64) for b in E.fetch_blocks()]
    for L in range(levels + 1):
        np.testing.assert_array_equal(blocks[L], o["blocks"][L], err_msg=f"blocks L={L}")
        np.testing.assert_array_equal(E.masks[L].cpu().numpy().view(np.uint64), o["masks"][L], err_msg=f"masks L={L}")
        if L < levels:
            np.testing.assert_array_equal(E.flags[L].cpu().numpy(), o["flags"][L], err_msg=f"flags L={L}")
    lk = E.links
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(lk[k].cpu().numpy().astype(np.int64), o["links"][k], err_msg=f"links {k}")
    dq = np.abs(lk["q"].cpu().numpy().astype(np.float64) - o["links"]["q"])
    assert dq.max(initial=0) <= Q_TOL
    assert P.emb_status_get() == P.EMB_OK
    return E, o


def test_icosphere_paper_rules(orc):
    v, t = icosphere(2, radius=0.3, centre=(0.5, 0.5, 0.5))
    _compare(orc, v, t, 2, 2, 19, 0.2)


def test_icosphere_partially_refined_root(orc):
    v, t = icosphere(3, radius=0.2, centre=(0.5, 0.5, 0.5))
    E, o = _compare(orc, v, t, 8, 2, 19, 0.1)
    assert len(o["blocks"][1]) < 8 * 8 ** 3  # not every root block is refined


def test_star_paper_rules(orc):
    w = workload("star_4k_r3")
    v, t = w.build_mesh()
    _compare(orc, v, t, w.R, w.levels, max(w.lattices), 0.15)


def test_surface_in_unrefined_regions(orc):
    # a box, and beside it a slab thin in y (0.595..0.605) and long in x (0.3..0.9): no
    # root cell centre lies in it, so the root level does not see it and refines only
    # around the box (x, y, z below 0.75).  At level 1 the slab is solid where blocks
    # exist, and each x-line through it crosses its far face at x = 0.9, inside root
    # blocks that were not refined: that one crossing must still flip every cell of the
    # row to its left, or the slab's cells between 0.3 and 0.75 come out fluid.
    g = 1 << 20
    bv, bt = axis_box([g // 4] * 3, [g // 2] * 3)
    sv, st = axis_box([int(0.3 * g), int(0.595 * g), int(0.3 * g)], [int(0.9 * g), int(0.605 * g), int(0.45 * g)])
    v = np.concatenate([bv, sv]).astype(np.float32)
    t = np.concatenate([bt, st + len(bv)]).astype(np.int32)
    E, o = _compare(orc, v, t, 8, 2, 19, 0.1)
    b1, m1 = o["blocks"][1], o["masks"][1]
    rows = (b1[:, 1] == 9) & (b1[:, 2] >= 4) & (b1[:, 2] <= 7)  # level-1 blocks holding the slab's lines
    assert b1[rows][:, 0].max() < 12  # the refined region stops at x = 0.75 ...
    assert np.any(m1[rows] != 0)  # ... and the slab is solid inside it
    assert orc.balanced_2to1(o["blocks"], 8)
