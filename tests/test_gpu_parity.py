"""Element-by-element parity of the CUDA path (through the C ABI) with the oracle.

Forest blocks, solid masks, refine flags, the cut-link set and each link's
triangle must be identical; q must agree within 2e-6.  Cases span several
blocks per level, non-power-of-two roots, both lattices, and degenerate
geometry (faces through cell centres, vertices on lattice lines, several
crossings per link, an embedding without links).
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import compare_full, gpu_embed
from synth import axis_box, octahedron, tetrahedron, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name,lattice", [("icosphere_320", 19), ("star_1k", 19), ("star_1k", 27),
                                          ("star_4k_r3", 27)])
def test_workload_full_parity(orc, name, lattice):
    w = workload(name)
    v, t = w.build_mesh()
    o = orc.embed(v, t, w.R, w.levels, w.band, lattice)
    _, g = gpu_embed(v, t, w.R, w.levels, w.band, lattice)
    compare_full(g, o, w.levels)
    assert len(g["links"]["q"]) > 100


def _box_on_centres(R, L):
    r_o, k = 1, 0
    while R % (2 ** (k + 1)) == 0:
        k += 1
    half = 1 << (17 - k - L)
    lo = (2 * 9 + 1) * half
    hi = (2 * 37 + 1) * half
    return axis_box([lo, lo, lo + 2 * half], [hi, hi - 4 * half, hi])


def test_degenerate_box_faces_on_cell_centres(orc):
    R, levels = 2, 3
    v, t = _box_on_centres(R, levels)
    o = orc.embed(v, t, R, levels, 2, 27)
    _, g = gpu_embed(v, t, R, levels, 2, 27)
    compare_full(g, o, levels)


def test_degenerate_vertices_on_lattice_lines(orc):
    R, levels = 2, 2
    h = 1 << (18 - 1 - levels)
    half = h // 2
    # octahedron with vertices and edges on cell centre lines, tetrahedron with faces through centres
    for v, t in [octahedron([16 * h + half, 15 * h + half, 17 * h + half], [7 * h, 9 * h, 6 * h]),
                 tetrahedron(np.array([[5 * h + half, 6 * h + half, 7 * h + half], [26 * h + half, 6 * h + half, 7 * h + half],
                                       [5 * h + half, 27 * h + half, 7 * h + half], [5 * h + half, 6 * h + half, 25 * h + half]]))]:
        o = orc.embed(v, t, R, levels, 2, 27)
        _, g = gpu_embed(v, t, R, levels, 2, 27)
        compare_full(g, o, levels)


def test_two_slabs_three_crossings(orc):
    R, levels = 2, 2
    h = 1 << (18 - 1 - levels)
    px = (2 * 12 + 1) * (h // 2)
    a = px + h // 8
    v1, t1 = axis_box([a, 6 * h, 6 * h], [a + h // 8, 26 * h, 26 * h])
    v2, t2 = axis_box([a + h // 4, 6 * h, 6 * h], [px + 2 * h, 26 * h, 26 * h])
    v = np.concatenate([v1, v2])
    t = np.concatenate([t1, t2 + len(v1)]).astype(np.int32)
    o = orc.embed(v, t, R, levels, 2, 19)
    assert (o["links"]["ncross"] == 3).sum() > 0
    _, g = gpu_embed(v, t, R, levels, 2, 19)
    compare_full(g, o, levels)


def test_tiny_solid_without_links(orc):
    """A tetrahedron that holds no cell centre: empty masks, no links, a short forest."""
    R, levels = 2, 2
    h = 1 << (18 - 1 - levels)
    base = 12 * h + 3
    v, t = tetrahedron(np.array([[base, base, base], [base + h // 4, base, base], [base, base + h // 4, base],
                                 [base, base, base + h // 4]]))
    o = orc.embed(v, t, R, levels, 2, 19)
    assert len(o["links"]["cell"]) == 0
    _, g = gpu_embed(v, t, R, levels, 2, 19)
    compare_full(g, o, levels)


def test_deterministic_repeat():
    w = workload("star_1k")
    v, t = w.build_mesh()
    _, a = gpu_embed(v, t, w.R, w.levels, w.band, 27)
    _, b = gpu_embed(v, t, w.R, w.levels, w.band, 27)
    for L in range(w.levels + 1):
        np.testing.assert_array_equal(a["masks"][L], b["masks"][L])
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(a["links"][k], b["links"][k])
    np.testing.assert_array_equal(a["links"]["q"].view(np.uint32), b["links"]["q"].view(np.uint32))


# --------------------------------------------------------------------------- #
# error paths (all detected on the host or by bounded device checks)
# --------------------------------------------------------------------------- #
def test_rejects_unsnapped_vertices():
    import torch

    import paper_2512_01251_gb300 as P
    v, t = workload("icosphere_320").build_mesh()
    v = v.copy()
    v[3, 1] = np.float32(v[3, 1] + np.float32(3e-8))
    with pytest.raises(P.EmbError) as e:
        P.emb_mesh_create(torch.from_numpy(v), torch.from_numpy(t), 2)
    assert e.value.code == P.EMB_ERR_BAD_INPUT


def test_rejects_open_and_flipped_meshes():
    import torch

    import paper_2512_01251_gb300 as P
    v, t = workload("icosphere_320").build_mesh()
    with pytest.raises(P.EmbError) as e:
        P.emb_mesh_create(torch.from_numpy(v), torch.from_numpy(t[:-1].copy()), 2)
    assert e.value.code == P.EMB_ERR_NOT_WATERTIGHT
    f = t.copy()
    f[5] = f[5][::-1]
    with pytest.raises(P.EmbError) as e:
        P.emb_mesh_create(torch.from_numpy(v), torch.from_numpy(f), 2)
    assert e.value.code == P.EMB_ERR_NOT_WATERTIGHT
    bad = t.copy()
    bad[0, 0] = len(v) + 5
    with pytest.raises(P.EmbError) as e:
        P.emb_mesh_create(torch.from_numpy(v), torch.from_numpy(bad), 2, check_watertight=False)
    assert e.value.code == P.EMB_ERR_BAD_INPUT


def test_capacity_and_state_errors():
    import torch

    import paper_2512_01251_gb300 as P
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), w.R, w.levels, w.band, 19, keep_bins=True)
    n = E.links["q"].numel()
    fin = E.bins[-1]
    with pytest.raises(P.EmbError) as e:
        P.emb_cutlinks(E.forest, fin, 19, capacity=n - 1)
    assert e.value.code == P.EMB_ERR_CAPACITY
    assert P.emb_status_get() == P.EMB_ERR_CAPACITY
    assert P.emb_status_get() == P.EMB_OK  # cleared by the read
    out = P.emb_cutlinks(E.forest, fin, 19, capacity=n)
    assert int(out["count"].item()) == n
    with pytest.raises(P.EmbError) as e:
        P.emb_voxelize(E.forest, E.bins[0], 1)  # bins of another level
    assert e.value.code == P.EMB_ERR_STATE
    with pytest.raises(P.EmbError) as e:
        P.emb_forest_root(1 << 10, 9)  # k + level beyond the integer frame
    assert e.value.code == P.EMB_ERR_RANGE


def test_deep_forest_looked_up_through_the_hash(orc):
    # R = 32 with 6 levels: the finest level has 2048^3 block positions, more than the
    # rank bitmap covers (2^32), so its blocks are found through the level hash (the
    # coarser levels use bitmaps); a small body keeps the refined region small
    from synth.meshes import icosphere
    v, t = icosphere(1, radius=0.004, centre=(0.5013, 0.4987, 0.5021))
    o = orc.embed(v, t, 32, 6, 2, 19)
    _, g = gpu_embed(v, t, 32, 6, 2, 19)
    compare_full(g, o, 6)
    assert len(g["links"]["q"]) > 1000


def test_corner_faces_beyond_int32(orc):
    """Faces perpendicular to the four D3Q27 corner lines with every vertex within
    2^14 of a finest cell centre, where c . n = 9 a^2 exceeds 2^31: the link kernel's
    narrow 32-bit path must still find each crossing (q = 1/8 at the face centroid)."""
    import corner_case as K
    v, t = K.mesh()
    o = orc.embed(v, t, K.R, K.LEVELS, K.BAND, K.LATTICE)
    _, g = gpu_embed(v, t, K.R, K.LEVELS, K.BAND, K.LATTICE)
    compare_full(g, o, K.LEVELS)
    P = orc.cell_centres(K.R, K.LEVELS, g["blocks"][-1])
    for i in range(4):
        cell = int(np.nonzero((P == K.centres()[i][None, :]).all(axis=1))[0][0])
        sel = (g["links"]["cell"] == cell) & (g["links"]["dir"] == K.direction_index(K.SIGNS[i]))
        assert sel.sum() == 1 and abs(float(g["links"]["q"][sel][0]) - 0.125) <= 2e-6
