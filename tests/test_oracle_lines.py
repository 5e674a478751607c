"""The sorted-line oracle tier against the brute-force tier, output by output.

Both tiers evaluate the same exact definitions (oracle/emb_oracle.c by brute force
over every triangle per query; oracle/emb_oracle_lines.c triangle-major along sorted
lattice lines).  On every case here they must agree on every block, refine flag,
mask word and cut link, including q bit for bit and the number of faces each link
crosses.  The cases cover both lattices, non-power-of-two roots, faces and vertices
on cell-centre lines and planes, links crossing three faces, an embedding without
links, faces far beyond the 32-bit range of c . n, and a batch mesh.
"""
from __future__ import annotations

import numpy as np
import pytest

from synth import axis_box, batch_meshes, octahedron, tetrahedron, workload


def _same(a, b, levels):
    for L in range(levels + 1):
        np.testing.assert_array_equal(a["blocks"][L], b["blocks"][L], err_msg=f"blocks L={L}")
        np.testing.assert_array_equal(a["masks"][L], b["masks"][L], err_msg=f"masks L={L}")
        if L < levels:
            np.testing.assert_array_equal(a["flags"][L], b["flags"][L], err_msg=f"flags L={L}")
    for k in ("cell", "dir", "tri", "ncross"):
        np.testing.assert_array_equal(a["links"][k], b["links"][k], err_msg=f"links {k}")
    np.testing.assert_array_equal(a["links"]["q"], b["links"]["q"], err_msg="links q")


@pytest.mark.parametrize("name,lattice", [("icosphere_320", 19), ("star_1k", 27), ("star_4k_r3", 27)])
def test_workloads(orc, name, lattice):
    w = workload(name)
    v, t = w.build_mesh()
    a = orc.embed(v, t, w.R, w.levels, w.band, lattice)
    b = orc.embed_lines(v, t, w.R, w.levels, w.band, lattice)
    assert len(b["links"]["q"]) > 1000
    _same(a, b, w.levels)


def test_rotated_batch_mesh_with_odd_root(orc):
    """A randomly rotated batch mesh on a root of 5^3 blocks (odd part 5 in the frame)."""
    c = batch_meshes(3, t_max=3e3)[2]
    a = orc.embed(c["verts"], c["tris"], 5, 2, 2, 19)
    b = orc.embed_lines(c["verts"], c["tris"], 5, 2, 2, 19)
    assert len(b["links"]["q"]) > 1000
    _same(a, b, 2)


def _degenerate_cases():
    cases = []
    # box with faces through cell centres (R = 2, levels 0..3)
    half = 1 << (17 - 1 - 3)
    lo, hi = (2 * 9 + 1) * half, (2 * 37 + 1) * half
    cases.append((axis_box([lo, lo, lo + 2 * half], [hi, hi - 4 * half, hi]), 2, 3, 27))
    # octahedron and tetrahedron with vertices, edges and faces on centre lines (R = 2, levels 0..2)
    h = 1 << (18 - 1 - 2)
    hf = h // 2
    cases.append((octahedron([16 * h + hf, 15 * h + hf, 17 * h + hf], [7 * h, 9 * h, 6 * h]), 2, 2, 27))
    cases.append((tetrahedron(np.array([[5 * h + hf, 6 * h + hf, 7 * h + hf], [26 * h + hf, 6 * h + hf, 7 * h + hf],
                                        [5 * h + hf, 27 * h + hf, 7 * h + hf], [5 * h + hf, 6 * h + hf, 25 * h + hf]])),
                  2, 2, 27))
    # two slabs: links crossing three faces
    px = (2 * 12 + 1) * hf
    a = px + h // 8
    v1, t1 = axis_box([a, 6 * h, 6 * h], [a + h // 8, 26 * h, 26 * h])
    v2, t2 = axis_box([a + h // 4, 6 * h, 6 * h], [px + 2 * h, 26 * h, 26 * h])
    cases.append(((np.concatenate([v1, v2]), np.concatenate([t1, t2 + len(v1)]).astype(np.int32)), 2, 2, 19))
    # a solid holding no cell centre
    base = 12 * h + 3
    cases.append((tetrahedron(np.array([[base, base, base], [base + h // 4, base, base], [base, base + h // 4, base],
                                        [base, base, base + h // 4]])), 2, 2, 19))
    return cases


@pytest.mark.parametrize("case", range(5))
def test_degenerate_geometry(orc, case):
    (v, t), R, levels, lattice = _degenerate_cases()[case]
    a = orc.embed(v, t, R, levels, 2, lattice)
    b = orc.embed_lines(v, t, R, levels, 2, lattice)
    _same(a, b, levels)


def test_corner_faces(orc):
    import corner_case as K
    v, t = K.mesh()
    a = orc.embed(v, t, K.R, K.LEVELS, K.BAND, K.LATTICE)
    b = orc.embed_lines(v, t, K.R, K.LEVELS, K.BAND, K.LATTICE)
    _same(a, b, K.LEVELS)


def test_every_link_crosses_a_face_on_a_large_mesh(orc):
    """On a closed mesh every fluid-to-solid link crosses the surface an odd number of
    times (the two end states differ), so no link of the sorted-line tier is left
    without a triangle; checked on the ~112K-triangle mesh with both lattices."""
    w = workload("star_112k")
    v, t = w.build_mesh()
    for lattice in (19, 27):
        b = orc.embed_lines(v, t, w.R, w.levels, w.band, lattice)
        assert np.all(b["links"]["tri"] >= 0)
        assert np.all(b["links"]["ncross"] % 2 == 1)
        assert np.all((b["links"]["q"] >= 0) & (b["links"]["q"] <= 1))
