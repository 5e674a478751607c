"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each check uses an independent route to the same answer: closed forms of simple
solids, the half-space representation of convex bodies (a different predicate
from ray parity), Cyrus-Beck clipping for link lengths, Sutherland-Hodgman
clipping in exact rationals for triangle/box overlap, hand counts, invariants
(ray direction, translation), volume bounds and finite differences.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

from synth import axis_box, icosphere, octahedron, radial_star, signed_volume, tetrahedron, workload

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------- #
# helpers written independently of the oracle
# --------------------------------------------------------------------------- #
def _halfspace_inside(tri9, P):
    """Inside test for a CONVEX closed mesh from its face planes, with the query
    point pushed by (e, e^2, e^3): inside iff n_f . (P' - A_f) < 0 for every face."""
    for t in tri9:
        A, B, C = [tuple(int(x) for x in t[3 * k:3 * k + 3]) for k in range(3)]
        u = [B[d] - A[d] for d in range(3)]
        v = [C[d] - A[d] for d in range(3)]
        n = (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
        if n == (0, 0, 0):
            continue
        s = sum(n[d] * (int(P[d]) - A[d]) for d in range(3))
        if s == 0:
            s = next(x for x in n if x != 0)  # n . e for e -> 0+
        if s > 0:
            return False
    return True


def _grid_points(R, L, lo_cell, hi_cell):
    from oracle.oracle import frame
    _, k = frame(R)
    half = 1 << (17 - k - L)
    g = np.stack(np.meshgrid(*[np.arange(lo_cell, hi_cell)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return (2 * g + 1) * half


def _clip_nonempty(tri, lo, hi):
    """Sutherland-Hodgman clipping of a triangle against the closed box, in exact rationals."""
    poly = [tuple(Fraction(int(x)) for x in tri[3 * k:3 * k + 3]) for k in range(3)]
    for d in range(3):
        for side, bound in ((1, lo[d]), (-1, hi[d])):
            def inside(p):
                return side * (p[d] - bound) >= 0

            out = []
            for i in range(len(poly)):
                S, E = poly[i - 1], poly[i]
                if inside(E):
                    if not inside(S):
                        tt = (bound - S[d]) / (E[d] - S[d])
                        out.append(tuple(S[j] + tt * (E[j] - S[j]) for j in range(3)))
                    out.append(E)
                elif inside(S):
                    tt = (bound - S[d]) / (E[d] - S[d])
                    out.append(tuple(S[j] + tt * (E[j] - S[j]) for j in range(3)))
            poly = out
            if not poly:
                return False
    return True


# --------------------------------------------------------------------------- #
# solid mask
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("R", [2, 3])
def test_cube_faces_on_centres(orc, R):
    """Axis box whose faces pass through cell centres: solid iff lo <= P < hi per axis."""
    r_o, k = orc.frame(R)
    L = 2
    half = 1 << (17 - k - L)
    ncell = 4 * R * (1 << L)
    # pick centre indices whose coordinate is a multiple of r_o in 2^-20 units
    idx = [i for i in range(ncell) if ((2 * i + 1) * half) % r_o == 0]
    i_lo, i_hi = idx[1], idx[-2]
    lo = (2 * i_lo + 1) * half // r_o
    hi = (2 * i_hi + 1) * half // r_o
    v, t = axis_box([lo, lo + 0, lo], [hi, hi, hi])
    X = orc.int_coords(v, R)
    tri9 = orc.tri_coords(X, t)
    P = _grid_points(R, L, max(0, i_lo - 2), min(ncell, i_hi + 3))
    lo_u, hi_u = lo * r_o, hi * r_o
    expect = np.all((P >= lo_u) & (P < hi_u), axis=1).astype(np.uint8)
    assert expect.sum() > 0 and (1 - expect).sum() > 0
    for d in range(1, 7):
        np.testing.assert_array_equal(orc.solid(tri9, P, d), expect, err_msg=f"ray dir {d}")


def test_convex_halfspace_agreement(orc):
    """Random tetrahedra/octahedra on a coarse lattice (faces through many centres)."""
    rng = np.random.default_rng(7)
    R, L = 2, 1
    _, k = orc.frame(R)
    half = 1 << (17 - k - L)
    P = _grid_points(R, L, 0, 16)
    for trial in range(12):
        if trial % 2 == 0:
            pts = rng.integers(2, 30, size=(4, 3)) * half  # on centres and cell faces
            v, t = tetrahedron(pts)
        else:
            c = rng.integers(10, 22, size=3) * half
            r = rng.integers(3, 9, size=3) * half
            v, t = octahedron(c, r)
        X = orc.int_coords(v, R)
        tri9 = orc.tri_coords(X, t)
        if abs(signed_volume(v, t)) == 0:
            continue
        expect = np.array([_halfspace_inside(tri9, p) for p in P], dtype=np.uint8)
        for d in (1, 2, 3, 4, 5, 6):
            got = orc.solid(tri9, P, d)
            np.testing.assert_array_equal(got, expect, err_msg=f"trial {trial} dir {d}")


def test_hand_counted_tetrahedra(orc):
    lines = [ln for ln in open(os.path.join(HERE, "golden", "tetra_cells.txt")) if not ln.startswith("#")]
    gold = {ln.split(":")[0]: sorted(int(x) for x in ln.split(":")[1].split()) for ln in lines if ":" in ln}
    R, L = 2, 2
    h = orc.h_units(R, L)
    corner = np.array([4 * h * 3, 4 * h * 2, 4 * h * 4])  # block (3, 2, 4) at level 2
    cases = {
        "corner": [corner, corner + [4 * h, 0, 0], corner + [0, 4 * h, 0], corner + [0, 0, 4 * h]],
        "centred": [corner + h // 2, corner + h // 2 + [3 * h, 0, 0], corner + h // 2 + [0, 3 * h, 0],
                    corner + h // 2 + [0, 0, 3 * h]],
    }
    blocks = np.array([[3, 2, 4]])
    for name, pts in cases.items():
        v, t = tetrahedron(np.array(pts))
        tri9 = orc.tri_coords(orc.int_coords(v, R), t)
        bits = orc.unpack_masks(orc.masks(tri9, R, L, blocks))[0]
        assert sorted(np.nonzero(bits)[0].tolist()) == gold[name], name


@pytest.mark.parametrize("name", ["icosphere_320", "star_1k"])
def test_parity_all_directions_agree(orc, name):
    w = workload(name)
    v, t = w.build_mesh()
    X = orc.int_coords(v, w.R)
    tri9 = orc.tri_coords(X, t)
    rng = np.random.default_rng(3)
    L = 3
    ncell = 4 * w.R * 8
    _, k = orc.frame(w.R)
    g = rng.integers(0, ncell, size=(3000, 3))
    P = (2 * g + 1) * (1 << (17 - k - L))
    ref = orc.solid(tri9, P, 1)
    assert 0 < ref.sum() < len(ref)
    for d in range(2, 7):
        np.testing.assert_array_equal(orc.solid(tri9, P, d), ref, err_msg=f"dir {d}")


def test_translation_by_whole_cells(orc):
    R, L = 2, 2
    h = orc.h_units(R, L)
    v, t = icosphere(2, 0.25, seed=11)
    X = orc.int_coords(v, R)
    shift = np.array([3 * h, -2 * h, 5 * h])
    tri_a = orc.tri_coords(X, t)
    tri_b = orc.tri_coords(X + shift, t)
    P = _grid_points(R, L, 2, 30)
    np.testing.assert_array_equal(orc.solid(tri_a, P), orc.solid(tri_b, P + shift))


def test_volume_bound_and_convergence(orc):
    """|sum(solid) h^3 - V_poly| <= sqrt(3) h * area, and the error shrinks with h."""
    v, t = icosphere(3, 0.3, seed=5)
    R = 2
    X = orc.int_coords(v, R)
    tri9 = orc.tri_coords(X, t)
    vw = v.astype(np.float64)
    area = 0.5 * np.linalg.norm(np.cross(vw[t[:, 1]] - vw[t[:, 0]], vw[t[:, 2]] - vw[t[:, 0]]), axis=1).sum()
    vol = signed_volume(v, t)
    errs = []
    for L in (1, 2, 3):
        n = 4 * R * (1 << L)
        hw = 1.0 / n
        P = _grid_points(R, L, 0, n)
        s = orc.solid(tri9, P)
        err = abs(s.sum() * hw ** 3 - vol)
        assert err <= math.sqrt(3) * hw * area, (L, err)
        errs.append(err)
    assert errs[2] < errs[0]
    # the polyhedral volume itself is below the sphere's and close to it
    assert vol < 4 / 3 * math.pi * 0.3 ** 3 and vol > 0.97 * 4 / 3 * math.pi * 0.3 ** 3


# --------------------------------------------------------------------------- #
# triangle / box overlap and refine flags
# --------------------------------------------------------------------------- #
def test_sat_matches_exact_clipping(orc):
    rng = np.random.default_rng(1)
    n_overlap = n_sep = 0
    for i in range(2500):
        tri = rng.integers(0, 13, size=9)
        if i % 5 == 0:  # degenerate: collinear or repeated vertices
            tri[6:9] = tri[0:3] + (tri[3:6] - tri[0:3]) * rng.integers(-1, 3)
        lo = rng.integers(2, 8, size=3)
        hi = lo + rng.integers(0, 5, size=3)
        a = orc.sat(tri, lo, hi)
        b = _clip_nonempty(tri, lo, hi)
        assert a == b, (tri.tolist(), lo.tolist(), hi.tolist())
        n_overlap += a
        n_sep += not a
    assert n_overlap > 300 and n_sep > 300


@pytest.mark.parametrize("L", [0, 1, 2])
def test_refine_flags_cube_closed_form(orc, L):
    """For a box-shaped solid, flag(b) iff the dilated block box touches the box surface."""
    R, levels, band = 2, 3, 2
    hf = orc.h_units(R, 2)
    a, b = 7 * hf + hf // 3, 25 * hf - 5  # arbitrary integer faces
    v, t = axis_box([a, a, a], [b, b, b])
    h = orc.h_units(R, L)
    tri9 = orc.tri_coords(orc.int_coords(v, R), t)
    nb = R << L
    blocks = orc.sort_blocks(np.stack(np.meshgrid(*[np.arange(nb)] * 3, indexing="ij"), -1).reshape(-1, 3))
    got = orc.refine_flags(tri9, R, L, levels, band, blocks)
    W, D = 4 * h, orc.dilation(R, L, levels, band)
    lo, hi = blocks * W - D, (blocks + 1) * W + D
    meets = np.all((lo <= b) & (hi >= a), axis=1)
    inside_open = np.all((lo > a) & (hi < b), axis=1)
    np.testing.assert_array_equal(got, (meets & ~inside_open).astype(np.uint8))
    assert 0 < got.sum() and (L < 2 or got.sum() < len(got))


def test_rho_schedule_values(orc):
    rho = orc.rho_schedule(4, 2)
    assert rho == [Fraction(37, 8), Fraction(17, 4), Fraction(7, 2), Fraction(2)]


def test_forest_balance_and_surface_free_gaps(orc):
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    R = 3
    levels = 3
    tri9 = orc.tri_coords(orc.int_coords(v, R), t)
    blocks, flags = orc.build_forest(tri9, R, levels, 2)
    for L in range(levels):
        W = 4 * orc.h_units(R, L)
        unflag = blocks[L][flags[L] == 0]
        # unrefined blocks hold no surface
        assert not orc.boxes_any(tri9, unflag * W, (unflag + 1) * W).any()
        if L == 0:
            continue
        present = {tuple(x) for x in blocks[L].tolist()}
        nmax = R << L
        for bb in blocks[L][flags[L] == 1]:
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        nb = (bb[0] + dx, bb[1] + dy, bb[2] + dz)
                        if all(0 <= c < nmax for c in nb):
                            assert nb in present, (L, bb, nb)


# --------------------------------------------------------------------------- #
# link lengths
# --------------------------------------------------------------------------- #
def _cyrus_beck_entry(tri9, P, c, h):
    """Entry parameter of the segment P -> P + h c into a convex body (exact Fraction)."""
    t_in = Fraction(-10 ** 9)
    c = [int(x) for x in c]
    h = int(h)
    for tr in tri9:
        A, B, C = [tuple(int(x) for x in tr[3 * k:3 * k + 3]) for k in range(3)]
        u = [B[d] - A[d] for d in range(3)]
        v = [C[d] - A[d] for d in range(3)]
        n = (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
        nc = sum(n[d] * c[d] for d in range(3))
        if nc < 0:
            t_in = max(t_in, Fraction(sum(n[d] * (A[d] - int(P[d])) for d in range(3)), h * nc))
    return t_in


def test_link_lengths_convex_cyrus_beck(orc):
    rng = np.random.default_rng(5)
    R, L = 2, 2
    h = orc.h_units(R, L)
    C = orc.directions()
    solids = [axis_box([9 * h + 17, 8 * h, 10 * h + h // 2], [20 * h + 3, 23 * h + 11, 21 * h + h // 2])]
    for _ in range(3):
        solids.append(tetrahedron(rng.integers(4, 28, size=(4, 3)) * h + rng.integers(0, h, size=(4, 3))))
    solids.append(octahedron([16 * h, 16 * h, 16 * h], [9 * h + 5, 7 * h, 8 * h + h // 2]))
    checked = 0
    for v, t in solids:
        tri9 = orc.tri_coords(orc.int_coords(v, R), t)
        if abs(signed_volume(v, t)) < 1e-6:
            continue
        blocks = orc.sort_blocks(np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3))
        m = orc.masks(tri9, R, L, blocks)
        lk = orc.cut_links(tri9, R, L, blocks, m, 27)
        assert len(lk["cell"]) > 0
        assert np.all(lk["ncross"] == 1)  # a convex body is entered exactly once
        P = orc.cell_centres(R, L, blocks)
        sel = rng.choice(len(lk["cell"]), size=min(400, len(lk["cell"])), replace=False)
        for i in sel:
            p = P[lk["cell"][i]]
            c = C[lk["dir"][i]]
            assert _halfspace_inside(tri9, p) is False and _halfspace_inside(tri9, p + h * c) is True
            t_in = _cyrus_beck_entry(tri9, p, c, h)
            assert 0 <= t_in <= 1
            assert abs(lk["q"][i] - float(t_in)) <= 1e-15
            checked += 1
    assert checked > 1000


def test_link_set_is_fluid_to_solid(orc):
    """Each emitted link joins a fluid centre to a solid one; every such pair is emitted."""
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    r = orc.embed(v, t, w.R, w.levels, w.band, 19)
    lk = r["links"]
    P = orc.cell_centres(w.R, w.levels, r["blocks"][-1])
    h = orc.h_units(w.R, w.levels)
    C = orc.directions()
    assert np.all(orc.solid(r["tri9"], P[lk["cell"]]) == 0)
    assert np.all(orc.solid(r["tri9"], P[lk["cell"]] + h * C[lk["dir"]]) == 1)
    assert np.all((lk["q"] >= 0) & (lk["q"] <= 1))
    key = lk["cell"] * 32 + lk["dir"]
    assert np.all(np.diff(key) > 0)  # sorted by (cell, dir), unique


# --------------------------------------------------------------------------- #
# derivatives and the force
# --------------------------------------------------------------------------- #
def test_dq_dverts_finite_differences(orc):
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    r = orc.embed(v, t, w.R, w.levels, w.band, 19)
    lk = r["links"]
    rng = np.random.default_rng(9)
    sel = rng.choice(len(lk["cell"]), size=60, replace=False)
    sub = {k: lk[k][sel] for k in ("cell", "dir", "q", "tri")}
    scale = float(orc.domain_units(w.R))
    h = orc.h_units(w.R, w.levels) / scale
    C = orc.directions().astype(np.float64)
    P = orc.cell_centres(w.R, w.levels, r["blocks"][-1]).astype(np.float64) / scale
    Xw = r["X"].astype(np.float64) / scale
    for j, i in enumerate(sel):
        gq = np.zeros(len(sel))
        gq[j] = 1.0
        g = orc.grad_verts_from_gq(sub, gq, r["X"], t, w.R, w.levels, r["blocks"][-1], len(v))
        tri = t[lk["tri"][i]]
        p, c = P[lk["cell"][i]], C[lk["dir"][i]]

        def q_of(Y):
            A, B, Cc = Y[tri[0]], Y[tri[1]], Y[tri[2]]
            n = np.cross(B - A, Cc - A)
            return np.dot(n, A - p) / (h * np.dot(n, c))

        assert abs(q_of(Xw) - lk["q"][i]) < 1e-12
        for vid in tri:
            for d in range(3):
                eps = 1e-7 * h
                Yp, Ym = Xw.copy(), Xw.copy()
                Yp[vid, d] += eps
                Ym[vid, d] -= eps
                fd = (q_of(Yp) - q_of(Ym)) / (2 * eps)
                assert abs(fd - g[vid, d]) <= 1e-5 * max(1.0, abs(fd)), (i, vid, d, fd, g[vid, d])


def test_dq_dverts_slab_closed_form(orc):
    """Links through the +x face of a box: moving that face by dx changes q by dx / (h c_x)."""
    R, L = 2, 2
    h = orc.h_units(R, L)
    v, t = axis_box([8 * h + 100, 8 * h, 8 * h], [22 * h + 77, 24 * h, 24 * h])
    X = orc.int_coords(v, R)
    tri9 = orc.tri_coords(X, t)
    blocks = orc.sort_blocks(np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3))
    m = orc.masks(tri9, R, L, blocks)
    lk = orc.cut_links(tri9, R, L, blocks, m, 19)
    C = orc.directions()
    face = np.nonzero(v[:, 0] == v[:, 0].max())[0]
    hw = h / float(orc.domain_units(R))
    n = 0
    for i in range(len(lk["cell"])):
        c = C[lk["dir"][i]]
        if c[0] >= 0:
            continue
        tri = t[lk["tri"][i]]
        if not set(tri.tolist()) <= set(face.tolist()):
            continue
        sub = {k: lk[k][i:i + 1] for k in ("cell", "dir", "q", "tri")}
        g = orc.grad_verts_from_gq(sub, np.ones(1), X, t, R, L, blocks, len(v))
        assert abs(g[face, 0].sum() - 1.0 / (hw * c[0])) <= 1e-9 / hw
        n += 1
    assert n > 20


def test_bouzidi_continuity_and_rest_state(orc):
    f_i, f_p, f_o = 0.11, 0.07, 0.13
    a = orc.bouzidi_incoming(np.array([0.5 - 1e-12]), f_i, f_p, f_o, np.array([True]))
    b = orc.bouzidi_incoming(np.array([0.5]), f_i, f_p, f_o, np.array([True]))
    assert abs(a[0] - b[0]) < 1e-10
    # uniform populations: the wall returns the outgoing population unchanged, for any q
    q = np.linspace(0.0, 1.0, 11)
    inc = orc.bouzidi_incoming(q, 0.2, 0.2, 0.2, np.ones_like(q, dtype=bool))
    np.testing.assert_allclose(inc, 0.2, rtol=0, atol=1e-15)


def test_force_sign_and_symmetry(orc):
    """Uniform flow in +x pushes a box in +x; at rest a centred box feels no force."""
    from synth import D3Q19_WEIGHTS, D3Q27_DIRS
    R, L = 2, 2
    h = orc.h_units(R, L)
    v, t = axis_box([10 * h, 10 * h, 10 * h], [22 * h, 22 * h, 22 * h])
    X = orc.int_coords(v, R)
    tri9 = orc.tri_coords(X, t)
    blocks = orc.sort_blocks(np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3))
    m = orc.masks(tri9, R, L, blocks)
    lk = orc.cut_links(tri9, R, L, blocks, m, 19)
    partner = orc.partner_cells(R, L, blocks, m, lk["cell"], lk["dir"])
    ncell = len(blocks) * 64
    c = D3Q27_DIRS[:19].astype(np.float64)
    rest = np.repeat(D3Q19_WEIGHTS[:, None], ncell, axis=1)
    F0 = orc.mex_force(lk, rest, partner)
    np.testing.assert_allclose(F0, 0.0, atol=1e-12)
    u = np.array([0.05, 0.0, 0.0])
    cu = c @ u
    feq = D3Q19_WEIGHTS * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * u @ u)
    F = orc.mex_force(lk, np.repeat(feq[:, None], ncell, axis=1), partner)
    assert F[0] > 0 and abs(F[1]) < 1e-12 and abs(F[2]) < 1e-12


def test_force_dq_finite_differences(orc):
    from synth import populations
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    r = orc.embed(v, t, w.R, w.levels, w.band, 19)
    lk = r["links"]
    bf, mf = r["blocks"][-1], r["masks"][-1]
    partner = orc.partner_cells(w.R, w.levels, bf, mf, lk["cell"], lk["dir"])
    pop = populations(len(bf) * 64, seed=4)
    g = orc.mex_force_dq(lk, pop, partner)
    rng = np.random.default_rng(2)
    for i in rng.choice(len(lk["q"]), size=40, replace=False):
        q0 = lk["q"][i]
        eps = 1e-6
        if abs(q0 - 0.5) < 2 * eps or q0 < 2 * eps:
            continue
        lp = dict(lk)
        lm = dict(lk)
        lp["q"] = lk["q"].copy()
        lm["q"] = lk["q"].copy()
        lp["q"][i] += eps
        lm["q"][i] -= eps
        fd = (orc.mex_force(lp, pop, partner) - orc.mex_force(lm, pop, partner)) / (2 * eps)
        np.testing.assert_allclose(fd, g[i], rtol=1e-5, atol=1e-8)


def test_watertight_check(orc):
    v, t = icosphere(1, 0.3)
    assert orc.watertight(t)
    assert not orc.watertight(t[:-1])
    flipped = t.copy()
    flipped[0] = flipped[0][::-1]
    assert not orc.watertight(flipped)


def test_int_coords_rejects_unsnapped(orc):
    v, _ = icosphere(1, 0.3)
    bad = v.copy()
    bad[0, 0] = np.float32(0.3) + np.float32(1e-7)
    with pytest.raises(ValueError):
        orc.int_coords(bad, 2)
    with pytest.raises(ValueError):
        orc.int_coords(np.array([[0.0, 0.5, 0.5]], dtype=np.float32), 2)


def test_link_takes_nearest_of_several_crossings(orc):
    """Two thin slabs inside one link: the segment crosses three faces, q is the first."""
    from synth.meshes import snap
    R, L = 2, 2
    h = orc.h_units(R, L)
    px = (2 * 12 + 1) * (h // 2)          # centre x of cell column 12
    a = px + h // 8                        # first slab [a, a + h/8]
    b1 = a + h // 8
    a2 = a + h // 4                        # second slab [a2, px + 2h]
    b2 = px + 2 * h
    lo_yz, hi_yz = 6 * h, 26 * h
    v1, t1 = axis_box([a, lo_yz, lo_yz], [b1, hi_yz, hi_yz])
    v2, t2 = axis_box([a2, lo_yz, lo_yz], [b2, hi_yz, hi_yz])
    v = np.concatenate([v1, v2])
    t = np.concatenate([t1, t2 + len(v1)])
    assert orc.watertight(t)
    tri9 = orc.tri_coords(orc.int_coords(v, R), t)
    blocks = orc.sort_blocks(np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3))
    m = orc.masks(tri9, R, L, blocks)
    lk = orc.cut_links(tri9, R, L, blocks, m, 19)
    P = orc.cell_centres(R, L, blocks)
    sel = (lk["dir"] == 1) & (P[lk["cell"], 0] == px)
    assert sel.sum() > 50
    assert np.all(lk["ncross"][sel] == 3)
    np.testing.assert_allclose(lk["q"][sel], 0.125, rtol=0, atol=1e-15)
