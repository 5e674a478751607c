"""Pins of the oracle's paper refinement rules (Sec. 3.4, "Refinement Flagging and
Propagation", Eq. N_prop), against closed forms and invariants rather than against a
second copy of the rules:

- Eq. N_prop evaluated by hand;
- a box whose faces lie on root-block boundaries: the solid blocks are exactly the
  blocks inside, so the marked root blocks are those inside within three layers of
  the surface (the solid boundary plus two layers inward) and those outside within
  1 + N_prop layers (Chebyshev distance in blocks);
- the finer levels of the resulting forest stay 2:1 balanced;
- cut links with neighbours restricted to existing blocks: on a single-level forest
  (every block exists) they equal the full definition.
"""
from __future__ import annotations

import numpy as np

from synth.meshes import axis_box, icosphere

GRID = 1 << 20


def test_n_prop_by_hand(orc):
    # 1 + floor(d R / sqrt 2): 0.1 * 16 / 1.41421 = 1.131, 0.2 * 16 / 1.41421 = 2.263
    assert orc.n_prop(0.1, 16) == 2
    assert orc.n_prop(0.2, 16) == 3
    assert orc.n_prop(0.05, 16) == 1
    assert orc.n_prop(0.0, 8) == 1


def _box_case(orc, lo_blk, hi_blk, R, levels, d_spec):
    # faces on root-block boundaries: block b spans [b, b + 1) / R of the unit cube
    lo = [lo_blk * GRID // R] * 3
    hi = [hi_blk * GRID // R] * 3
    v, t = axis_box(lo, hi)
    X = orc.int_coords(v, R)
    tri9 = orc.tri_coords(X, t)
    return orc.build_forest_paper(tri9, R, levels, d_spec)


def test_block_aligned_box_marks_closed_form(orc):
    R, lo_b, hi_b = 16, 2, 10  # eight blocks wide: inside depths 1..4
    blocks, flags, masks = _box_case(orc, lo_b, hi_b, R, 1, 0.1)
    nprop = orc.n_prop(0.1, R)
    assert nprop == 2
    b = blocks[0]
    inside = np.all((b >= lo_b) & (b < hi_b), axis=1)
    # the solid blocks are exactly the inside ones, and they are completely solid
    assert np.array_equal(masks[0] != 0, inside)
    assert np.all(masks[0][inside] == np.uint64(0xFFFFFFFFFFFFFFFF))
    depth = np.min(np.minimum(b - lo_b + 1, hi_b - b), axis=1)  # 1 on the inside shell
    dist = np.max(np.maximum(np.maximum(lo_b - b, b - (hi_b - 1)), 0), axis=1)  # Chebyshev, 0 inside
    expect = np.where(inside, depth <= 3, dist <= 1 + nprop)
    np.testing.assert_array_equal(flags[0].astype(bool), expect)
    assert not np.all(expect[inside])  # the depth-4 core stays unrefined
    assert orc.balanced_2to1(blocks, R)


def test_paper_forest_is_balanced_on_a_sphere(orc):
    v, t = icosphere(3, radius=0.23, centre=(0.5, 0.5, 0.5))
    R = 4
    X = orc.int_coords(v, R)
    tri9 = orc.tri_coords(X, t)
    blocks, flags, masks = orc.build_forest_paper(tri9, R, 3, 0.15)
    assert all(len(b) > 0 for b in blocks)
    assert len(blocks[3]) < (R << 3) ** 3 // 2  # refinement stays local
    assert orc.balanced_2to1(blocks, R)
    # masks are the point predicate whatever the forest: a block present in two forests has one mask
    b0, f0 = orc.build_forest(tri9, R, 1, 2)
    m_def = orc.masks(tri9, R, 1, b0[1])
    common = {tuple(x): i for i, x in enumerate(b0[1].tolist())}
    for i, x in enumerate(blocks[1].tolist()):
        if tuple(x) in common:
            assert masks[1][i] == m_def[common[tuple(x)]]


def test_existing_only_links_equal_full_definition_on_one_level(orc):
    v, t = icosphere(2, radius=0.3, centre=(0.5, 0.5, 0.5))
    R = 4
    X = orc.int_coords(v, R)
    tri9 = orc.tri_coords(X, t)
    blocks = orc.root_blocks(R)
    m = orc.masks(tri9, R, 0, blocks)
    a = orc.cut_links(tri9, R, 0, blocks, m, 19)
    b = orc.cut_links(tri9, R, 0, blocks, m, 19, existing_only=True)
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(a["q"], b["q"])
    assert len(a["q"]) > 0


def test_blocks_on_the_refinement_interface_are_never_marked(orc):
    # level 1 of a forest with R = 4 (8 blocks per axis) whose parent (3, 3, 3) was not
    # refined: its 2 x 2 x 2 children are missing.  Blocks with x <= 2 are solid, the
    # rest fully fluid; with many propagation rounds every block would be marked, but
    # the blocks next to the hole are on the refinement interface and must stay unmarked.
    nb = 8
    g = np.stack(np.meshgrid(np.arange(nb), np.arange(nb), np.arange(nb), indexing="ij"), -1).reshape(-1, 3)
    hole = np.all(g >= 6, axis=1)
    full = orc.sort_blocks(g)
    holed = orc.sort_blocks(g[~hole])
    full_mask = np.where(full[:, 0] <= 2, np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0))
    holed_mask = np.where(holed[:, 0] <= 2, np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0))
    assert np.all(orc.paper_flags(full, full_mask, nb, 1, 8) == 1)
    f = orc.paper_flags(holed, holed_mask, nb, 1, 8).astype(bool)
    next_to_hole = np.all((holed >= 5) & (holed <= 7), axis=1)
    np.testing.assert_array_equal(f, ~next_to_hole)
