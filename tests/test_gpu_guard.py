"""The paper's guard-cell voxelizer on the GPU (emb_voxelize_guard) against the oracle,
bit for bit: solid and guard words of every finest block.  Cases: a box with an
unrefined interior (runs that start at solid holes), a box whose faces lie on planes
of cell centres (distances of exactly zero, lines along face edges), the apex of an
octahedron on a centre line (equal distances, lowest face id), a generic sphere, and
a star mesh with R = 3 (cell centres that binary32 rounds)."""
from __future__ import annotations

import numpy as np
import pytest

from synth import workload
from synth.meshes import axis_box, icosphere, octahedron

pytestmark = pytest.mark.gpu

GRID = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _compare(orc, v, t, R, levels, band=2):
    import torch

    import paper_2512_01251_gb300 as P
    v = np.ascontiguousarray(v, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.int32)
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), R, levels, band, 19, keep_bins=True)
    solid, guard = P.emb_voxelize_guard(E.forest, E.bins[-1])
    tri9 = orc.tri_coords(orc.int_coords(v, R), t)
    blocks, _ = orc.build_forest(tri9, R, levels, band)
    masks = [orc.masks(tri9, R, L, blocks[L]) for L in range(levels + 1)]
    gb = E.fetch_blocks()[levels].cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(gb, blocks[levels])
    o_solid, o_guard = orc.guard_voxelize(v, t, R, levels, blocks, masks)
    np.testing.assert_array_equal(solid.cpu().numpy().view(np.uint64), o_solid, err_msg="solid words")
    np.testing.assert_array_equal(guard.cpu().numpy().view(np.uint64), o_guard, err_msg="guard words")
    assert P.emb_status_get() == P.EMB_OK
    # the forest's own (exact) masks are left as they were
    np.testing.assert_array_equal(E.masks[levels].cpu().numpy().view(np.uint64), masks[levels])
    return o_solid, masks[levels]


def test_box_with_unrefined_interior_matches(orc):
    lo, hi = int(0.1 * GRID) + 5, int(0.85 * GRID) + 11
    v, t = axis_box([lo] * 3, [hi] * 3)
    s, m = _compare(orc, v, t, 4, 2)
    np.testing.assert_array_equal(s, m)


def test_box_on_centre_planes(orc):
    n = 16  # cells per axis at R = 4, level 0
    lo, hi = 7 * GRID // (2 * n), 23 * GRID // (2 * n)
    v, t = axis_box([lo] * 3, [hi] * 3)
    s, m = _compare(orc, v, t, 4, 0)
    assert np.count_nonzero(s != m) > 0  # the two voxelizers differ on the faces' planes


def test_octahedron_apex_on_a_centre_line(orc):
    g = GRID // 32
    v, t = octahedron([16 * g, 17 * g, 16 * g], [8 * g, 8 * g, 9 * g])
    _compare(orc, v, t, 4, 1)


def test_generic_sphere(orc):
    v, t = icosphere(3, radius=0.31, centre=(0.503, 0.497, 0.51), seed=5)
    s, m = _compare(orc, v, t, 4, 2)
    np.testing.assert_array_equal(s, m)


@pytest.mark.parametrize("name", ["icosphere_320", "star_4k_r3"])
def test_workloads(orc, name):
    w = workload(name)
    v, t = w.build_mesh()
    _compare(orc, v, t, w.R, w.levels, w.band)


def test_guard_rejects_bins_of_another_level():
    import torch

    import paper_2512_01251_gb300 as P
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), w.R, w.levels, w.band, 19, keep_bins=True)
    with pytest.raises(P.EmbError) as e:
        P.emb_voxelize_guard(E.forest, E.bins[0])  # the root's bins: only the finest level has block bins
    assert e.value.code == P.EMB_ERR_STATE
    s, g = P.emb_voxelize_guard(E.forest, E.bins[-1])
    assert s.numel() == g.numel() == E.masks[-1].numel()
    assert P.emb_status_get() == P.EMB_OK
