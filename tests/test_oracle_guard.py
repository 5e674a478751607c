"""Pins of the oracle's guard-cell voxelizer (Sec. 3.4, "Partial Surface Voxelization"
with Alg. 3 and "External Cell Flag Propagation"), the paper's single-precision method
built as an ablation of the exact parity voxelizer.  Closed forms:

- an axis-aligned box whose faces lie between cell centres: the solid cells are exactly
  those with the centre inside, on a single-level forest (every block present, one
  +x sweep) and on a two-level forest whose interior was not refined (runs of blocks
  that start at a hole left by a solid coarse block start from the solid);
- a box whose faces lie on planes of cell centres: a centre on an x face is at distance
  0 from it (n_x d = 0: guard, then fluid), a centre on a y or z face is hit by the
  x faces' edges and lies behind them (solid): the solid set is open in x and closed in
  y and z;
- the cells of a row (a block's x-line of four cells) share one line and one bin, so
  a row is hit everywhere or nowhere; the blocks between a box's x faces are reached
  only by the external propagation (without it their cells stay fluid);
- the internal propagation rules on hand-seeded rows (a guard arriving with a solid
  in the same round wins), and the external ones on hand-made runs of blocks (a run
  next to a solid hole starts from the solid, in either direction; the -x sweep
  fills what only a solid status from the right reaches);
- equal distances go to the lowest face id (the order of the paper's sorted bins): an
  x-line through the apex of an octahedron touches its four upper faces at one point,
  and the first of them, whose normal points to +x, makes the cells before the apex
  solid and those after it guards;
- a generic sphere: the result equals the exact parity voxelizer's.
"""
from __future__ import annotations

import numpy as np

from synth.meshes import axis_box, icosphere, octahedron

GRID = 1 << 20


def _forest(orc, v, t, R, levels):
    tri9 = orc.tri_coords(orc.int_coords(v, R), t)
    blocks, _ = orc.build_forest(tri9, R, levels, 2)
    masks = [orc.masks(tri9, R, L, blocks[L]) for L in range(levels + 1)]
    return tri9, blocks, masks


def _centres_unit(orc, R, L, blocks):
    n = orc.cells_per_axis(R, L)
    t = np.arange(64)
    loc = np.stack([t % 4, (t // 4) % 4, t // 16], axis=1)
    g = 4 * blocks[:, None, :] + loc[None]
    return (2 * g + 1).reshape(-1, 3), 2 * n  # centre = num / den, exactly


def test_box_between_centres_single_level(orc):
    R = 8
    lo, hi = int(0.2 * GRID) + 7, int(0.7 * GRID) + 3  # no centre plane
    v, t = axis_box([lo] * 3, [hi] * 3)
    tri9, blocks, masks = _forest(orc, v, t, R, 0)
    solid, guard = orc.guard_voxelize(v, t, R, 0, blocks, masks)
    np.testing.assert_array_equal(solid, masks[0])
    num, den = _centres_unit(orc, R, 0, blocks[0])
    inside = np.all((num * GRID > lo * den) & (num * GRID < hi * den), axis=1)
    np.testing.assert_array_equal(orc.unpack_masks(solid).reshape(-1).astype(bool), inside)
    assert not np.any(orc.unpack_masks(solid) & orc.unpack_masks(guard))


def test_box_between_centres_with_unrefined_interior(orc):
    R, levels = 4, 2
    lo, hi = int(0.1 * GRID) + 5, int(0.85 * GRID) + 11
    v, t = axis_box([lo] * 3, [hi] * 3)
    tri9, blocks, masks = _forest(orc, v, t, R, levels)
    L = levels
    # the interior of the finest level has holes: root blocks deep inside were not refined
    assert len(blocks[L]) < (R << L) ** 3
    solid, _ = orc.guard_voxelize(v, t, R, L, blocks, masks)
    np.testing.assert_array_equal(solid, masks[L])
    assert np.count_nonzero(solid) > 0


def test_box_on_centre_planes(orc):
    R, L = 4, 0
    n = orc.cells_per_axis(R, L)  # 16 cells per axis
    # faces at the centres of cells 3 and 11 (centre of cell i: (2 i + 1) / 32)
    lo, hi = 7 * GRID // (2 * n), 23 * GRID // (2 * n)
    v, t = axis_box([lo] * 3, [hi] * 3)
    tri9, blocks, masks = _forest(orc, v, t, R, 0)
    solid, _ = orc.guard_voxelize(v, t, R, 0, blocks, masks)
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    want = np.zeros((len(blocks[0]), 64), dtype=bool)
    idx = orc._block_index(blocks[0])
    for x, y, z in g.tolist():
        ins = 3 < x < 11 and 3 <= y <= 11 and 3 <= z <= 11
        want[idx[(x // 4, y // 4, z // 4)], (x % 4) + 4 * (y % 4) + 16 * (z % 4)] = ins
    np.testing.assert_array_equal(orc.unpack_masks(solid).astype(bool), want)
    # the exact voxelizer differs exactly on the faces' planes (its perturbed centres decide)
    assert np.count_nonzero(solid != masks[0]) > 0


def test_without_propagation_the_interior_is_empty(orc):
    R = 8
    lo, hi = int(0.2 * GRID) + 7, int(0.7 * GRID) + 3
    v, t = axis_box([lo] * 3, [hi] * 3)
    tri9, blocks, masks = _forest(orc, v, t, R, 0)
    st = orc.guard_surface(v, t, R, 0, blocks[0])
    n_surface = np.count_nonzero(st == orc.SOLID)
    n_full = np.count_nonzero(orc.unpack_masks(masks[0]))
    assert 0 < n_surface < n_full  # the hits alone cover only the blocks near the x faces
    # the cells of a row share one x-line and one bin: a row is hit everywhere or nowhere,
    # so the internal propagation has nothing left to fill
    inner = orc.guard_internal(st)
    np.testing.assert_array_equal(inner, st)
    full = orc.guard_external(inner, R, 0, blocks, masks)
    assert np.count_nonzero(full == orc.SOLID) == n_full


def test_internal_propagation_fills_a_row_from_its_hits(orc):
    # rows seeded by hand: guard wins over solid when both arrive in the same round
    st = np.zeros((1, 64), dtype=np.uint8)
    st[0, 0] = orc.SOLID  # row (y 0, z 0): S . . .
    st[0, 4 + 1] = orc.GUARD  # row (y 1, z 0): . G . .
    st[0, 8 + 0], st[0, 8 + 2] = orc.SOLID, orc.GUARD  # row (y 2, z 0): S . G .
    out = orc.guard_internal(st).reshape(4, 4, 4)
    S, G = orc.SOLID, orc.GUARD
    np.testing.assert_array_equal(out[0, 0], [S, S, S, S])
    np.testing.assert_array_equal(out[0, 1], [G, G, G, G])
    np.testing.assert_array_equal(out[0, 2], [S, G, G, G])
    assert np.all(out[1:] == orc.FLUID)


def test_external_propagation_on_hand_made_runs(orc):
    R, L = 2, 1  # 4 blocks per axis at level 1, 2 at the root
    S, G, F = orc.SOLID, orc.GUARD, orc.FLUID
    root = orc.root_blocks(R)
    solid_roots = {(1, 0, 0), (0, 0, 1)}
    root_masks = np.array([np.uint64(1) if tuple(b) in solid_roots else np.uint64(0) for b in root.tolist()],
                          dtype=np.uint64)
    runs = {"A": [(0, 0, 0), (1, 0, 0), (2, 0, 0)],  # right end borders (3,0,0), inside solid root (1,0,0)
            "B": [(1, 2, 0), (2, 2, 0)],  # both ends border fluid roots
            "C": [(2, 1, 2), (3, 1, 2)]}  # left end borders (1,1,2), inside solid root (0,0,1)
    blocks = orc.sort_blocks(np.array([b for r in runs.values() for b in r]))
    idx = orc._block_index(blocks)
    st = np.full((len(blocks), 4, 4, 4), F, dtype=np.uint8)  # (block, z, y, x)
    st[idx[(0, 0, 0)], 0, 0] = G  # an outside row at the start of run A
    st[idx[(2, 2, 0)], 0, 1] = S  # a solid row at the right end of run B
    out = orc.guard_external(st.reshape(-1, 64), R, L, [root, blocks], [root_masks, None]).reshape(-1, 4, 4, 4)
    a0, a1, a2 = (out[idx[b]] for b in runs["A"])
    assert np.all(a2 == S) and np.all(a1 == S)  # -x sweep from the solid hole
    assert np.all(a0[0, 0] == G) and np.count_nonzero(a0 == S) == 60  # the outside row keeps its guards
    b0, b1 = (out[idx[b]] for b in runs["B"])
    assert np.all(b0[0, 1] == S) and np.count_nonzero(b0 == S) == 4  # only the -x sweep reaches it
    assert np.count_nonzero(b1 == S) == 4
    c0, c1 = (out[idx[b]] for b in runs["C"])
    assert np.all(c0 == S) and np.all(c1 == S)  # +x sweep from the solid hole


def test_equal_distances_go_to_the_lowest_face_id(orc):
    R, L = 4, 0  # 16 cells per axis, centre of cell i at (2 i + 1) / 32
    g = GRID // 32
    # apex (16, 17, 25) / 32: between cells 7 and 8 in x, on the centre line of cells y 8, z 12
    v, t = octahedron([16 * g, 17 * g, 16 * g], [8 * g, 8 * g, 9 * g])
    assert set(t[0]) == {0, 2, 4}  # face 0 joins +x, +y and the apex +z: its normal points to +x
    blocks = orc.sort_blocks(np.array([[1, 2, 3], [2, 2, 3]]))
    st = orc.guard_surface(v, t, R, L, blocks).reshape(-1, 4, 4, 4)
    idx = orc._block_index(blocks)
    S, G = orc.SOLID, orc.GUARD
    np.testing.assert_array_equal(st[idx[(1, 2, 3)], 0, 0], [S, S, S, S])  # cells 4..7, before the apex
    np.testing.assert_array_equal(st[idx[(2, 2, 3)], 0, 0], [G, G, G, G])  # cells 8..11, after it


def test_generic_sphere_equals_the_exact_voxelizer(orc):
    R, levels = 4, 2
    v, t = icosphere(3, radius=0.31, centre=(0.503, 0.497, 0.51), seed=5)
    tri9, blocks, masks = _forest(orc, v, t, R, levels)
    solid, guard = orc.guard_voxelize(v, t, R, levels, blocks, masks)
    np.testing.assert_array_equal(solid, masks[levels])
    assert np.count_nonzero(guard) > 0
