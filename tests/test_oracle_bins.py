"""Pins of the oracle's binning outputs (Sec. 3.3): the x-line filter of step 1 and the
per-block bins of the finest level (Alg. 2), against facts that do not restate them:

- an axis-aligned box: the four triangles of its x faces are kept, the eight faces
  parallel to x never are;
- a line through the edge (or the vertex) shared by flat triangles crosses exactly
  one of them, so exactly one is kept;
- a triangle is kept iff deleting it from the mesh changes the solid state of some
  cell of the level (the parity test of ``solid`` decides, cell by cell);
- every solid mask is the same computed from the kept triangles only;
- the bins reach exactly half a cell beyond the block: a face that far away is in,
  one unit further is out, on both sides;
- a triangle whose bounding box overlaps the dilated block but which passes a corner
  at a distance is out (a true overlap test, not a box test), and in when it touches;
- degenerate triangles are in no bin;
- every cut link's triangle is in the bin of the link's block.
"""
from __future__ import annotations

import numpy as np

from synth.meshes import axis_box, icosphere

GRID = 1 << 20


def _tri9(orc, v, t, R):
    return orc.tri_coords(orc.int_coords(v, R), t)


def test_box_keeps_exactly_its_x_faces(orc):
    R = 4
    v, t = axis_box([int(0.3 * GRID)] * 3, [int(0.7 * GRID)] * 3)
    tri9 = _tri9(orc, v, t, R)
    for L in (0, 1, 2):
        np.testing.assert_array_equal(orc.xfilter(tri9, R, L), [0, 1, 2, 3])  # -x and +x quads come first


def _flat(x0, pts):
    return np.array([[x0, y, z] for y, z in pts], dtype=np.int64).reshape(-1)


def test_line_through_a_shared_edge_or_vertex_crosses_one_triangle(orc):
    R, L = 4, 1
    h = orc.h_units(R, L)
    half = h // 2
    j, k = 11, 7
    yc, zc = (2 * j + 1) * half, (2 * k + 1) * half
    a = half // 2  # no other centre line within reach
    x0 = 300001
    # two triangles sharing the diagonal edge through the centre, oriented alike
    pair = np.stack([_flat(x0, [(yc - a, zc - a), (yc + a, zc - a), (yc + a, zc + a)]),
                     _flat(x0, [(yc + a, zc + a), (yc - a, zc + a), (yc - a, zc - a)])])
    assert len(orc.xfilter(pair, R, L)) == 1
    # four triangles of a square fanned around a vertex on the centre line
    c = (yc, zc)
    sq = [(yc - a, zc - a), (yc + a, zc - a), (yc + a, zc + a), (yc - a, zc + a)]
    fan = np.stack([_flat(x0, [c, sq[i], sq[(i + 1) % 4]]) for i in range(4)])
    assert len(orc.xfilter(fan, R, L)) == 1
    # the same square moved a quarter cell off the line: no line crosses it
    off = fan.copy()
    off[:, 1::3] += a + 1
    assert len(orc.xfilter(off, R, L)) == 0


def test_kept_iff_deleting_the_triangle_changes_some_cell(orc):
    R, L = 4, 0
    v, t = icosphere(1, radius=0.3, centre=(0.5, 0.5, 0.5))
    tri9 = _tri9(orc, v, t, R)
    kept = set(orc.xfilter(tri9, R, L).tolist())
    h = orc.h_units(R, L)
    half = h // 2
    n = orc.cells_per_axis(R, L)
    xs = (2 * np.arange(n) + 1) * half
    for i in range(len(tri9)):
        ys, zs = tri9[i, 1::3], tri9[i, 2::3]
        jr = range(max(0, -(-(ys.min() - half) // h)), min(n - 1, (ys.max() - half) // h) + 1)
        kr = range(max(0, -(-(zs.min() - half) // h)), min(n - 1, (zs.max() - half) // h) + 1)
        pts = np.array([[x, (2 * j + 1) * half, (2 * k + 1) * half] for j in jr for k in kr for x in xs],
                       dtype=np.int64).reshape(-1, 3)
        changed = False
        if len(pts):
            rest = np.delete(tri9, i, axis=0)
            changed = bool(np.any(orc.solid(tri9, pts) != orc.solid(rest, pts)))
        assert changed == (i in kept), i
    assert 0 < len(kept) < len(tri9)


def test_masks_are_unchanged_by_the_filter(orc):
    R, levels = 4, 2
    v, t = icosphere(2, radius=0.27, centre=(0.49, 0.52, 0.5))
    tri9 = _tri9(orc, v, t, R)
    blocks, _ = orc.build_forest(tri9, R, levels, 2)
    for L in range(levels + 1):
        keep = orc.xfilter(tri9, R, L)
        assert len(keep) < len(tri9)
        np.testing.assert_array_equal(orc.masks(tri9[keep], R, L, blocks[L]), orc.masks(tri9, R, L, blocks[L]))


def _single(pts):
    return np.array(pts, dtype=np.int64).reshape(1, 9)


def test_bins_reach_exactly_half_a_cell(orc):
    R, L = 4, 2
    h = orc.h_units(R, L)
    W = 4 * h
    b = np.array([[5, 6, 7]], dtype=np.int64)
    lo, hi = b[0] * W, (b[0] + 1) * W
    y0, y1, z0, z1 = lo[1] + 10, hi[1] - 10, lo[2] + 10, hi[2] - 10
    for x, inside in ((hi[0] + h // 2, True), (hi[0] + h // 2 + 1, False),
                      (lo[0] - h // 2, True), (lo[0] - h // 2 - 1, False)):
        tri = _single([x, y0, z0, x, y1, z0, x, y0, z1])
        got = orc.finest_bins(tri, R, L, b)[0]
        assert (len(got) == 1) == inside, (x, inside)


def test_bins_use_a_true_overlap_test_at_a_corner(orc):
    R, L = 4, 2
    h = orc.h_units(R, L)
    W = 4 * h
    b = np.array([[5, 6, 7]], dtype=np.int64)
    hx, hy = (b[0, 0] + 1) * W + h // 2, (b[0, 1] + 1) * W + h // 2  # corner of the dilated box in x-y
    zm = b[0, 2] * W + 2 * h
    for gap, inside in ((0, True), (10, False)):
        # every point satisfies x + y >= hx + hy + gap; the bounding box reaches 10 units into the block
        tri = _single([hx + 10 + gap, hy - 10, zm, hx - 10, hy + 10 + gap, zm, hx + 20 + gap, hy + 20 + gap, zm])
        assert (len(orc.finest_bins(tri, R, L, b)[0]) == 1) == inside, gap


def test_degenerate_triangles_are_never_binned(orc):
    R, L = 4, 2
    W = 4 * orc.h_units(R, L)
    b = np.array([[5, 6, 7]], dtype=np.int64)
    c = (b[0] * W + W // 2).tolist()
    tri = _single(c + [c[0] + 100, c[1] + 50, c[2] + 30] + [c[0] + 200, c[1] + 100, c[2] + 60])  # collinear
    assert orc.degenerate(tri)[0]
    assert len(orc.finest_bins(tri, R, L, b)[0]) == 0


def test_every_cut_link_triangle_is_in_its_blocks_bin(orc):
    R, levels = 4, 2
    v, t = icosphere(2, radius=0.27, centre=(0.49, 0.52, 0.5))
    tri9 = _tri9(orc, v, t, R)
    blocks, _ = orc.build_forest(tri9, R, levels, 2)
    bf = blocks[levels]
    m = orc.masks(tri9, R, levels, bf)
    lk = orc.cut_links(tri9, R, levels, bf, m, 27)
    bins = orc.finest_bins(tri9, R, levels, bf)
    assert len(lk["tri"]) > 0
    for c, tr in zip(lk["cell"], lk["tri"]):
        assert tr in bins[c // 64]
    # and the bins hold more than the links need (a triangle can overlap without a link)
    assert sum(len(x) for x in bins) > len(set(zip((lk["cell"] // 64).tolist(), lk["tri"].tolist())))
