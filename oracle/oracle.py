"""CPU oracle for the mesh-embedding hot path of arXiv 2512.01251.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product package never imports
it, and it never imports the product package.  It is plain and slow on
purpose: every result is the definition evaluated by brute force over all
triangles (C core in ``emb_oracle.c``), driven by numpy.

Parity status of each function (see also the module functions' docstrings):
  * ``build_forest``, ``masks``, ``refine_flags``, ``cut_links`` — pinned by
    closed forms, half-space representations, clipping and invariants
    (tests/test_oracle_pins.py).
  * ``lbm_step`` (one step on the finest level with Bouzidi bounce-back from the
    link table) — pinned by the rest state, a pulse streaming one cell, a pulse
    bounced by a halfway wall, and mass conservation in a cavity with halfway walls
    (tests/test_oracle_lbm.py).  The D3Q19/D3Q27 weights and BGK are the textbook
    ones (the paper cites its LBM and prints neither).
  * ``xfilter`` and ``finest_bins`` (the binning step's two outputs) — pinned by
    the closed form of an axis-aligned box, the single crossing of a line through
    an edge shared by two triangles, the invariance of every solid mask under the
    filter, the exact reach of the half-cell dilation, a corner that only a true
    overlap test rejects, and the coverage of every cut link
    (tests/test_oracle_bins.py).
  * ``guard_voxelize`` (the paper's single-precision guard-cell voxelizer, built as
    an ablation of the exact one) — pinned by closed forms: a box whose faces lie
    between cell centres gives exactly its inside, with every block present and
    with the interior left unrefined (holes entered from the solid side); a box
    whose faces lie on centre planes gives the half-open set the nearest-face rule
    implies (tests/test_oracle_guard.py).  The box half-width of the point-in-face
    test (the binary32 epsilon) is a reading with no closed form to pin it.
  * ``paper_flags``, ``build_forest_paper``, ``n_prop`` (the paper's block-layer
    refinement rules) — pinned by the closed form of a block-aligned box and the
    2:1 invariant (tests/test_oracle_paper_policy.py).
  * ``mex_force``/``mex_force_dq``/``dq_dverts`` — the derivative formulas are
    pinned by finite differences and a closed form; the Bouzidi branch rule for
    a missing interpolation partner and the momentum-exchange sign convention
    are readings of the paper (it prints neither formula): parity unpinned for
    that branch rule.

Integer frame.  With R = r_o 2^k root blocks per axis (r_o odd), a vertex
coordinate v (a multiple of 2^-20 in (0,1)) maps to X = v 2^20 r_o.  At level L
the cell size is h_L = 2^(18-k-L) units and cell i has its centre at
(2 i + 1) 2^(17-k-L), so every query point is an integer.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "emb_oracle.c")
_SRC_LINES = os.path.join(_HERE, "emb_oracle_lines.c")


def build(force: bool = False) -> str:
    """Compile the C core (brute force and sorted-line tiers) with gcc (OpenMP) into
    oracle/liboracle.so."""
    srcs = [_SRC, _SRC_LINES]
    if force or not os.path.exists(_LIB_PATH) or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(x) for x in srcs):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-o", tmp,
                               *srcs, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.orc_solid.argtypes = [P, i64, P, i64, ctypes.c_int, P]
        L.orc_links.argtypes = [P, i64, P, P, i64, i64, P, P, P]
        L.orc_boxes_any.argtypes = [P, i64, P, P, i64, P]
        L.orc_box_pairs.argtypes = [P, i64, P, P, i64, P]
        L.orc_guard_surface.argtypes = [P, P, P, i64, P, P, i64, P]
        L.orc_sat.argtypes = [P, P, P]
        L.orc_sat.restype = ctypes.c_int
        L.orc_segment_hit.argtypes = [P, P, ctypes.c_int, i64, P]
        L.orc_segment_hit.restype = ctypes.c_int
        L.orc_line_hits.argtypes = [P, P, ctypes.c_int]
        L.orc_line_hits.restype = ctypes.c_int
        L.orc_directions.argtypes = [P]
        L.orc_each_line.argtypes = [P, P, P, i64, P]
        L.orc_each_segment.argtypes = [P, P, P, P, i64, P, P]
        L.orc_each_box.argtypes = [P, P, P, i64, P]
        L.orc_lines_flags.argtypes = [P, i64, P, i64, i64, i64, i64, P]
        L.orc_lines_masks.argtypes = [P, i64, P, i64, i64, i64, P]
        L.orc_lines_links.argtypes = [P, i64, P, i64, P, i64, i64, ctypes.c_int]
        L.orc_lines_links.restype = i64
        L.orc_lines_links_take.argtypes = [P, P, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


# --------------------------------------------------------------------------- #
# frame
# --------------------------------------------------------------------------- #
def frame(R: int):
    """(r_o, k) with R = r_o 2^k, r_o odd."""
    if R < 1:
        raise ValueError("R must be positive")
    k = 0
    while R % 2 == 0:
        R //= 2
        k += 1
    return R, k


def h_units(R: int, L: int) -> int:
    _, k = frame(R)
    if k + L > 17:
        raise ValueError("level too fine for the integer frame")
    return 1 << (18 - k - L)


def domain_units(R: int) -> int:
    return (1 << 20) * frame(R)[0]


def int_coords(verts: np.ndarray, R: int) -> np.ndarray:
    """Vertex coordinates in frame units (int64); raises on unsnapped input."""
    m = np.asarray(verts, dtype=np.float64) * float(1 << 20)
    if not np.all(m == np.round(m)):
        raise ValueError("vertices are not on the 2^-20 grid")
    if not (np.all(m > 0) and np.all(m < (1 << 20))):
        raise ValueError("vertices must lie strictly inside (0, 1)")
    return m.astype(np.int64) * frame(R)[0]


def tri_coords(X: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """(T, 9) int64 records A, B, C."""
    t = np.asarray(tris, dtype=np.int64)
    return _c64(np.concatenate([X[t[:, 0]], X[t[:, 1]], X[t[:, 2]]], axis=1))


def directions() -> np.ndarray:
    out = np.zeros((27, 3), dtype=np.int32)
    lib().orc_directions(_p(out))
    return out.astype(np.int64)


def opposite(i: int) -> int:
    """Index of -c_i (pairs (1,2), (3,4), ... , (25,26))."""
    return i + 1 if i % 2 == 1 else i - 1


def watertight(tris: np.ndarray) -> bool:
    """Every directed edge appears exactly once and its reverse exactly once."""
    t = np.asarray(tris, dtype=np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    if np.any(e[:, 0] == e[:, 1]):
        return False
    key = e[:, 0] * (1 << 32) + e[:, 1]
    rkey = e[:, 1] * (1 << 32) + e[:, 0]
    u, cnt = np.unique(key, return_counts=True)
    if np.any(cnt != 1):
        return False
    return bool(np.all(np.isin(rkey, u)))


# --------------------------------------------------------------------------- #
# primitive queries (brute force over all triangles, C core)
# --------------------------------------------------------------------------- #
def solid(tri9: np.ndarray, pts: np.ndarray, dir: int = 1) -> np.ndarray:
    """Parity of crossings of the perturbed ray from each point along DIR[dir]."""
    tri9, pts = _c64(tri9), _c64(pts).reshape(-1, 3)
    out = np.zeros(len(pts), dtype=np.uint8)
    if len(pts):
        lib().orc_solid(_p(tri9), len(tri9), _p(pts), len(pts), int(dir), _p(out))
    return out


def links(tri9: np.ndarray, pts: np.ndarray, dirs: np.ndarray, h: int):
    """Nearest crossing of each segment P -> P + h c: (q float64, argmin tri, number of crossings)."""
    tri9, pts = _c64(tri9), _c64(pts).reshape(-1, 3)
    d = np.ascontiguousarray(dirs, dtype=np.int32)
    q = np.zeros(len(pts), dtype=np.float64)
    arg = np.zeros(len(pts), dtype=np.int64)
    nc = np.zeros(len(pts), dtype=np.int32)
    if len(pts):
        lib().orc_links(_p(tri9), len(tri9), _p(pts), _p(d), len(pts), int(h), _p(q), _p(arg), _p(nc))
    return q, arg, nc


def boxes_any(tri9: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    tri9 = _c64(tri9)
    lo, hi = _c64(lo).reshape(-1, 3), _c64(hi).reshape(-1, 3)
    out = np.zeros(len(lo), dtype=np.uint8)
    if len(lo):
        lib().orc_boxes_any(_p(tri9), len(tri9), _p(lo), _p(hi), len(lo), _p(out))
    return out


def sat(tri9_one, lo, hi) -> bool:
    return bool(lib().orc_sat(_p(_c64(tri9_one)), _p(_c64(lo)), _p(_c64(hi))))


def each_line(tri9, pts, dirs) -> np.ndarray:
    """One query per triangle: the perturbed line through pts[i] along DIR[dirs[i]] crosses tri9[i]."""
    tri9, pts = _c64(tri9).reshape(-1, 9), _c64(pts).reshape(-1, 3)
    d = np.ascontiguousarray(dirs, dtype=np.int32)
    out = np.zeros(len(tri9), dtype=np.uint8)
    if len(tri9):
        lib().orc_each_line(_p(tri9), _p(pts), _p(d), len(tri9), _p(out))
    return out


def each_segment(tri9, pts, dirs, h):
    """One query per triangle: (hit, t in FP64) of the perturbed segment pts[i] -> pts[i] + h[i] c."""
    tri9, pts = _c64(tri9).reshape(-1, 9), _c64(pts).reshape(-1, 3)
    d = np.ascontiguousarray(dirs, dtype=np.int32)
    hh = _c64(np.broadcast_to(np.asarray(h, dtype=np.int64), (len(tri9),)))
    hit = np.zeros(len(tri9), dtype=np.uint8)
    t = np.zeros(len(tri9), dtype=np.float64)
    if len(tri9):
        lib().orc_each_segment(_p(tri9), _p(pts), _p(d), _p(hh), len(tri9), _p(hit), _p(t))
    return hit, t


def each_box(tri9, lo, hi) -> np.ndarray:
    """One query per triangle: tri9[i] overlaps the closed box [lo[i], hi[i]]."""
    tri9 = _c64(tri9).reshape(-1, 9)
    lo, hi = _c64(lo).reshape(-1, 3), _c64(hi).reshape(-1, 3)
    out = np.zeros(len(tri9), dtype=np.uint8)
    if len(tri9):
        lib().orc_each_box(_p(tri9), _p(lo), _p(hi), len(tri9), _p(out))
    return out


def cells_per_axis(R: int, L: int) -> int:
    return 4 * R << L


def xfilter(tri9: np.ndarray, R: int, L: int) -> np.ndarray:
    """Sec. 3.3, step 1 (the 1-D ray indicator of Alg. 1): the ids, ascending, of the
    triangles that the +x line through the centre of some level-L cell crosses.  The
    line is the perturbed one of ``solid``, so a triangle the filter drops takes part
    in no crossing parity of the level.  Brute force over the centre lines inside the
    triangle's y-z bounding box (no other line can meet it)."""
    tri9 = _c64(tri9)
    h = h_units(R, L)
    half = h // 2
    n = cells_per_axis(R, L)
    keep = []
    for t in range(len(tri9)):
        ys, zs = tri9[t, 1::3], tri9[t, 2::3]
        j0, j1 = max(0, -(-(int(ys.min()) - half) // h)), min(n - 1, (int(ys.max()) - half) // h)
        k0, k1 = max(0, -(-(int(zs.min()) - half) // h)), min(n - 1, (int(zs.max()) - half) // h)
        hit = False
        for k in range(k0, k1 + 1):
            for j in range(j0, j1 + 1):
                P = np.array([half, (2 * j + 1) * half, (2 * k + 1) * half], dtype=np.int64)
                if lib().orc_line_hits(_p(tri9[t]), _p(P), 1):
                    hit = True
                    break
            if hit:
                break
        if hit:
            keep.append(t)
    return np.array(keep, dtype=np.int64)


def degenerate(tri9: np.ndarray) -> np.ndarray:
    """True for triangles with a zero normal (collinear vertices)."""
    t = _c64(tri9).astype(object)
    u, v = t[:, 3:6] - t[:, 0:3], t[:, 6:9] - t[:, 0:3]
    n = np.stack([u[:, 1] * v[:, 2] - u[:, 2] * v[:, 1], u[:, 2] * v[:, 0] - u[:, 0] * v[:, 2],
                  u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]], axis=1)
    return np.all(n == 0, axis=1).astype(bool)


def finest_bins(tri9: np.ndarray, R: int, L: int, blocks: np.ndarray) -> list:
    """Alg. 2 at the finest level: per block, the ids (ascending) of the non-degenerate
    triangles that overlap the closed block box dilated by half a cell.  A link starts
    at a cell centre, half a cell inside its block, and reaches one cell further, so
    it stays inside that box (Alg. 2 dilates by a whole cell; half suffices)."""
    tri9 = _c64(tri9)
    h = h_units(R, L)
    W = 4 * h
    blocks = _c64(blocks).reshape(-1, 3)
    lo = _c64(blocks * W - h // 2)
    hi = _c64((blocks + 1) * W + h // 2)
    T = len(tri9)
    inc = np.zeros((len(blocks), T), dtype=np.uint8)
    if len(blocks) and T:
        lib().orc_box_pairs(_p(tri9), T, _p(lo), _p(hi), len(blocks), _p(inc))
    ok = ~degenerate(tri9) if T else np.zeros(0, dtype=bool)
    return [np.nonzero(inc[i].astype(bool) & ok)[0].astype(np.int64) for i in range(len(blocks))]


# --------------------------------------------------------------------------- #
# forest, refinement, masks, links
# --------------------------------------------------------------------------- #
def rho_schedule(levels: int, band: int):
    """Near-wall distance rho_L (in level-L cells) for L = 0 .. levels-1.

    rho at the level below the finest equals ``band``; coarser levels use
    rho_L = max(band, rho_{L+1}/2 + 5/2), which makes every neighbour of a
    refined block exist (2:1 balance, Sec. 3.2) and every unrefined block's
    closed box free of the surface.
    """
    rho = [Fraction(0)] * levels
    for L in range(levels - 1, -1, -1):
        rho[L] = Fraction(band) if L == levels - 1 else max(Fraction(band), rho[L + 1] / 2 + Fraction(5, 2))
    return rho


def dilation(R: int, L: int, levels: int, band: int) -> int:
    """(rho_L - 1/2) h_L in frame units: the box dilation of the refine test at level L."""
    d = (rho_schedule(levels, band)[L] - Fraction(1, 2)) * h_units(R, L)
    if d.denominator != 1:
        raise ValueError("dilation is not an integer in this frame")
    return int(d)


def sort_blocks(b: np.ndarray) -> np.ndarray:
    b = np.asarray(b, dtype=np.int64).reshape(-1, 3)
    order = np.lexsort((b[:, 0], b[:, 1], b[:, 2]))
    return b[order]


def root_blocks(R: int) -> np.ndarray:
    g = np.stack(np.meshgrid(np.arange(R), np.arange(R), np.arange(R), indexing="ij"), -1).reshape(-1, 3)
    return sort_blocks(g)


def refine_flags(tri9, R, L, levels, band, blocks) -> np.ndarray:
    """flag(b) = some triangle overlaps the closed block box dilated by (rho_L - 1/2) h_L."""
    W = 4 * h_units(R, L)
    D = dilation(R, L, levels, band)
    lo = blocks * W - D
    hi = (blocks + 1) * W + D
    return boxes_any(tri9, lo, hi)


def children(blocks: np.ndarray, flags: np.ndarray) -> np.ndarray:
    p = blocks[flags.astype(bool)]
    off = np.array([[dx, dy, dz] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)], dtype=np.int64)
    ch = (2 * p[:, None, :] + off[None, :, :]).reshape(-1, 3)
    return sort_blocks(ch)


def build_forest(tri9, R: int, levels: int, band: int):
    """Top-down forest: blocks per level (sorted by z, y, x) and flags for levels < finest."""
    blocks = [root_blocks(R)]
    flags = []
    for L in range(levels):
        f = refine_flags(tri9, R, L, levels, band, blocks[L])
        flags.append(f)
        blocks.append(children(blocks[L], f))
    return blocks, flags


# --------------------------------------------------------------------------- #
# The paper's refinement policy (Sec. 3.4, "Refinement Flagging and Propagation")
# --------------------------------------------------------------------------- #
def n_prop(d_spec: float, R: int) -> int:
    """Eq. N_prop: 1 + floor((1/2^L) d_spec / (sqrt(2) Dx_{b,L})) with Dx_{b,L} = 4 Dx_L the
    block length.  With Dx_L = Dx_0 / 2^L the 2^L factors cancel, so the count is the
    same on every level: 1 + floor(d_spec R / sqrt(2)) for d_spec in units of the unit
    domain (Dx_{b,0} = 1 / R)."""
    return 1 + int(np.floor((float(d_spec) * R) / np.sqrt(2.0)))


def _nbr_offsets() -> np.ndarray:
    return np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                     if (dx, dy, dz) != (0, 0, 0)], dtype=np.int64)


def paper_flags(blocks: np.ndarray, mask_words: np.ndarray, nb: int, L: int, nprop: int) -> np.ndarray:
    """Refinement flags of one level under the paper's block-layer rules, step by step:

    - a block is solid if one of its cells is solid and fully fluid otherwise;
    - solid-boundary: a solid block with a fully fluid neighbour (among the blocks of
      the level, 26-neighbourhood); marked;
    - every block next to a solid-boundary block is marked (the fluid ones are the
      solid-adjacent blocks);
    - nprop rounds of propagation, each reading the marks of the previous round
      (ping-pong): an unmarked block next to a marked one is marked if it is fully
      fluid, or solid and this is the first round;
    - a block on the refinement interface (an in-domain neighbour position without a
      block of this level, L > 0) is never marked: refining it would break 2:1.
    Returns a uint8 flag per block (blocks sorted by z, y, x)."""
    blocks = np.asarray(blocks, dtype=np.int64)
    n = len(blocks)
    idx = {tuple(b): i for i, b in enumerate(blocks.tolist())}
    solid = np.asarray(mask_words, dtype=np.uint64) != 0
    off = _nbr_offsets()
    nbr = np.full((n, 26), -1, dtype=np.int64)
    eligible = np.ones(n, dtype=bool)
    for i, b in enumerate(blocks.tolist()):
        for d, o in enumerate(off.tolist()):
            q = (b[0] + o[0], b[1] + o[1], b[2] + o[2])
            if all(0 <= c < nb for c in q):
                j = idx.get(q, -1)
                nbr[i, d] = j
                if j < 0 and L > 0:
                    eligible[i] = False

    def any_nbr(sel: np.ndarray) -> np.ndarray:
        out = np.zeros(n, dtype=bool)
        for d in range(26):
            j = nbr[:, d]
            ok = j >= 0
            out[ok] |= sel[j[ok]]
        return out

    fluid_b = ~solid
    sb = solid & any_nbr(fluid_b)
    marked = sb & eligible
    marked = marked | (any_nbr(sb) & eligible)
    for r in range(nprop):
        scope = fluid_b | (solid if r == 0 else np.zeros(n, dtype=bool))
        marked = marked | (any_nbr(marked) & scope & eligible)
    return marked.astype(np.uint8)


def build_forest_paper(tri9, R: int, levels: int, d_spec: float):
    """Top-down forest under the paper's rules: per level the exact masks, then
    paper_flags.  Returns blocks per level, flags per level (< finest), masks per level."""
    blocks = [root_blocks(R)]
    flags, m = [], []
    np_ = n_prop(d_spec, R)
    for L in range(levels + 1):
        m.append(masks(tri9, R, L, blocks[L]))
        if L == levels:
            break
        f = paper_flags(blocks[L], m[L], R << L, L, np_)
        flags.append(f)
        blocks.append(children(blocks[L], f))
    return blocks, flags, m


def balanced_2to1(blocks_by_level, R: int) -> bool:
    """2:1 balance: the 26 neighbour positions of every block of level L+1 are covered by
    blocks of level L+1 or by their parent positions at level L (inside the domain)."""
    off = _nbr_offsets()
    for L in range(1, len(blocks_by_level)):
        fine = {tuple(b) for b in blocks_by_level[L].tolist()}
        coarse = {tuple(b) for b in blocks_by_level[L - 1].tolist()}
        nb = R << L
        for b in blocks_by_level[L].tolist():
            for o in off.tolist():
                q = (b[0] + o[0], b[1] + o[1], b[2] + o[2])
                if not all(0 <= c < nb for c in q):
                    continue
                if q not in fine and (q[0] // 2, q[1] // 2, q[2] // 2) not in coarse:
                    return False
    return True


# --------------------------------------------------------------------------- #
# The paper's guard-cell voxelizer (Sec. 3.4, "Partial Surface Voxelization" with
# Alg. 3, and "External Cell Flag Propagation"), on the finest level of a forest
# --------------------------------------------------------------------------- #
FLUID, SOLID, GUARD = 0, 1, 2


def guard_surface(verts, tris, R: int, L: int, blocks: np.ndarray) -> np.ndarray:
    """(n, 64) cell states before propagation: each cell takes the nearest face of its
    block's bin crossed by its x-line (binary32, C core ``orc_guard_surface``):
    SOLID if the centre is behind that face (n_x d > 0), GUARD if in front, FLUID if no
    face of the bin is hit."""
    v = np.ascontiguousarray(np.asarray(verts, dtype=np.float32))
    t = np.ascontiguousarray(np.asarray(tris, dtype=np.int32))
    tri9 = tri_coords(int_coords(v, R), t)
    blocks = _c64(blocks).reshape(-1, 3)
    bins = finest_bins(tri9, R, L, blocks)
    off = _c64(np.concatenate([[0], np.cumsum([len(b) for b in bins])]).astype(np.int64))
    ent = _c64(np.concatenate(bins).astype(np.int64) if len(bins) else np.zeros(0, np.int64))
    state = np.zeros((len(blocks), 64), dtype=np.uint8)
    if len(blocks):
        lib().orc_guard_surface(_p(v), _p(t), _p(blocks), len(blocks), _p(off), _p(ent), cells_per_axis(R, L),
                                _p(state))
    return state


def guard_internal(state: np.ndarray) -> np.ndarray:
    """Internal propagation along x inside each block: three rounds in which every cell
    looks at its two x-neighbours of the previous round; a FLUID cell next to a GUARD
    becomes GUARD, then a cell that is not GUARD next to a SOLID becomes SOLID.  Three
    rounds carry a flag across a row of four cells."""
    H = state.reshape(-1, 4, 4, 4).copy()  # (block, z, y, x)
    for _ in range(3):
        left = np.full_like(H, FLUID)
        right = np.full_like(H, FLUID)
        left[..., 1:] = H[..., :-1]
        right[..., :-1] = H[..., 1:]
        new = H.copy()
        new[(H == FLUID) & ((left == GUARD) | (right == GUARD))] = GUARD
        new[(new != GUARD) & ((left == SOLID) | (right == SOLID))] = SOLID
        H = new
    return H.reshape(-1, 64)


def guard_external(state: np.ndarray, R: int, L: int, blocks_by_level, masks_by_level) -> np.ndarray:
    """External propagation along +x, then (levels L > 0) along -x.  Each maximal run of
    consecutive blocks along the direction is walked from its first block, row by row:
    the status is the row's cell on the face ahead; a run whose first block borders a
    hole left by a coarser block with a solid cell starts from the solid (the row's
    non-guard cells turn SOLID unless the status is GUARD); in each following block a
    SOLID status turns the row's non-guard cells SOLID, and the status is read again."""
    H = state.reshape(-1, 4, 4, 4).copy()
    blocks = _c64(blocks_by_level[L]).reshape(-1, 3)
    index = {tuple(b): i for i, b in enumerate(blocks.tolist())}
    coarse = [{tuple(b): i for i, b in enumerate(_c64(blocks_by_level[l]).reshape(-1, 3).tolist())} for l in range(L)]
    nb = R << L

    def hole_is_solid(p):
        for l in range(L - 1, -1, -1):
            q = tuple(c >> (L - l) for c in p)
            j = coarse[l].get(q)
            if j is not None:
                return bool(np.asarray(masks_by_level[l], dtype=np.uint64)[j] != 0)
        return False

    for step in ([1, -1] if L > 0 else [1]):
        face = 3 if step > 0 else 0
        for i, b in enumerate(blocks.tolist()):
            before = (b[0] - step, b[1], b[2])
            if before in index:
                continue  # not the first block of its run
            special = 0 <= before[0] < nb and hole_is_solid(before)
            run = [i]
            nxt = (b[0] + step, b[1], b[2])
            while nxt in index:
                run.append(index[nxt])
                nxt = (nxt[0] + step, nxt[1], nxt[2])
            for z in range(4):
                for y in range(4):
                    status = H[i, z, y, face]
                    if special and status != GUARD:
                        row = H[i, z, y]
                        row[row != GUARD] = SOLID
                        status = SOLID
                    for j in run[1:]:
                        if status == SOLID:
                            row = H[j, z, y]
                            row[row != GUARD] = SOLID
                        status = H[j, z, y, face]
    return H.reshape(-1, 64)


def guard_voxelize(verts, tris, R: int, L: int, blocks_by_level, masks_by_level):
    """The guard-cell voxelizer on level L of a forest: (solid words, guard words) per
    block after both propagations; the paper then turns the guards back into fluid, so
    the solid words are its cell masks.  masks_by_level[l] for l < L decide the holes."""
    st = guard_surface(verts, tris, R, L, blocks_by_level[L])
    st = guard_external(guard_internal(st), R, L, blocks_by_level, masks_by_level)
    return pack_masks(st == SOLID), pack_masks(st == GUARD)


def cell_centres(R: int, L: int, blocks: np.ndarray) -> np.ndarray:
    """(n*64, 3) integer centres; cell t = x + 4 y + 16 z inside each block."""
    _, k = frame(R)
    half = 1 << (17 - k - L)
    t = np.arange(64)
    loc = np.stack([t % 4, (t // 4) % 4, t // 16], axis=1)
    g = 4 * blocks[:, None, :] + loc[None, :, :]
    return ((2 * g + 1) * half).reshape(-1, 3)


def pack_masks(bits: np.ndarray) -> np.ndarray:
    b = bits.reshape(-1, 64).astype(np.uint64)
    return (b << np.arange(64, dtype=np.uint64)[None, :]).sum(axis=1, dtype=np.uint64)


def unpack_masks(words: np.ndarray) -> np.ndarray:
    w = np.asarray(words, dtype=np.uint64)
    return ((w[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.uint8)


def masks(tri9, R, L, blocks, dir: int = 1) -> np.ndarray:
    """Solid mask word per block: bit t set iff the centre of cell t is inside."""
    return pack_masks(solid(tri9, cell_centres(R, L, blocks), dir))


def cut_links(tri9, R, levels, blocks_f, mask_f, lattice: int, existing_only: bool = False):
    """Flat cut-link table at the finest level, sorted by (cell, dir).

    For every fluid cell P and every lattice direction i != 0 whose neighbour
    P + h c_i is solid (decided by the same point predicate; a neighbour outside
    the domain is fluid): q = min over crossed triangles of the crossing
    parameter t in [0, 1].  With existing_only, a neighbour cell whose block is
    not in the finest level counts as fluid (the paper identifies boundary cells
    from the masks of neighbouring blocks of the level).  Returns dict(cell, dir,
    q, tri, ncross).
    """
    h = h_units(R, levels)
    dom = domain_units(R)
    C = directions()
    P = cell_centres(R, levels, blocks_f)
    fluid = unpack_masks(mask_f).reshape(-1) == 0
    cells = np.nonzero(fluid)[0]
    dirs = np.arange(1, lattice)
    cand_cell = np.repeat(cells, len(dirs))
    cand_dir = np.tile(dirs, len(cells))
    Q = P[cand_cell] + h * C[cand_dir]
    inside = np.all((Q > 0) & (Q < dom), axis=1)
    if existing_only:
        present = {tuple(b) for b in np.asarray(blocks_f, dtype=np.int64).tolist()}
        qb = (Q // (4 * h)).astype(np.int64)
        inside &= np.array([tuple(x) in present for x in qb.tolist()], dtype=bool)
    s = np.zeros(len(Q), dtype=np.uint8)
    if np.any(inside):
        uq, inv = np.unique(Q[inside], axis=0, return_inverse=True)
        s[inside] = solid(tri9, uq)[inv.reshape(-1)]
    keep = s.astype(bool)
    cell = cand_cell[keep]
    d = cand_dir[keep]
    q, arg, ncross = links(tri9, P[cell], d, h)
    return dict(cell=cell.astype(np.int64), dir=d.astype(np.int64), q=q, tri=arg, ncross=ncross)


def embed(verts, tris, R: int, levels: int, band: int = 2, lattice: int = 19, d_spec: float | None = None):
    """Whole path: forest, masks per level, refine flags, cut links.  With d_spec (a
    near-wall distance in units of the unit domain) the forest follows the paper's
    block-layer refinement rules instead of the exact distance rule of `band`."""
    X = int_coords(verts, R)
    tri9 = tri_coords(X, tris)
    if d_spec is None:
        blocks, flags = build_forest(tri9, R, levels, band)
        m = [masks(tri9, R, L, blocks[L]) for L in range(levels + 1)]
        lk = cut_links(tri9, R, levels, blocks[levels], m[levels], lattice)
    else:
        blocks, flags, m = build_forest_paper(tri9, R, levels, d_spec)
        lk = cut_links(tri9, R, levels, blocks[levels], m[levels], lattice, existing_only=True)
    return dict(X=X, tri9=tri9, blocks=blocks, flags=flags, masks=m, links=lk)


# --------------------------------------------------------------------------- #
# Tier B: the same definitions along sorted lattice lines (emb_oracle_lines.c)
# --------------------------------------------------------------------------- #
def _block_keys(blocks: np.ndarray, nb: int) -> np.ndarray:
    b = _c64(blocks).reshape(-1, 3)
    return _c64((b[:, 2] * nb + b[:, 1]) * nb + b[:, 0])


def lines_flags(tri9, R, L, levels, band, blocks) -> np.ndarray:
    """refine_flags, triangle-major: each triangle visits the blocks of the level whose
    dilated box can meet its bounding box."""
    tri9 = _c64(tri9)
    blocks = _c64(blocks).reshape(-1, 3)
    nb = R << L
    out = np.zeros(len(blocks), dtype=np.uint8)
    if len(blocks):
        lib().orc_lines_flags(_p(tri9), len(tri9), _p(_block_keys(blocks, nb)), len(blocks), nb,
                              4 * h_units(R, L), dilation(R, L, levels, band), _p(out))
    return out


def lines_masks(tri9, R, L, blocks) -> np.ndarray:
    """masks, from the sorted crossings of the level's +x centre lines."""
    tri9 = _c64(tri9)
    blocks = _c64(blocks).reshape(-1, 3)
    out = np.zeros(len(blocks), dtype=np.uint64)
    if len(blocks):
        lib().orc_lines_masks(_p(tri9), len(tri9), _p(blocks), len(blocks), h_units(R, L) // 2, cells_per_axis(R, L),
                              _p(out))
    return out


def lines_links(tri9, R, levels, blocks_f, mask_f, lattice: int) -> dict:
    """cut_links, with the crossings found triangle-major (one direction per thread)."""
    tri9 = _c64(tri9)
    blocks_f = _c64(blocks_f).reshape(-1, 3)
    m = np.ascontiguousarray(mask_f, dtype=np.uint64)
    n = lib().orc_lines_links(_p(tri9), len(tri9), _p(blocks_f), len(blocks_f), _p(m), h_units(R, levels) // 2,
                              cells_per_axis(R, levels), int(lattice))
    cell = np.zeros(n, dtype=np.int64)
    d = np.zeros(n, dtype=np.int32)
    q = np.zeros(n, dtype=np.float64)
    tri = np.zeros(n, dtype=np.int64)
    nc = np.zeros(n, dtype=np.int32)
    lib().orc_lines_links_take(_p(cell), _p(d), _p(q), _p(tri), _p(nc))
    return dict(cell=cell, dir=d.astype(np.int64), q=q, tri=tri, ncross=nc)


def embed_lines(verts, tris, R: int, levels: int, band: int = 2, lattice: int = 19):
    """The whole path (forest, masks per level, refine flags, cut links) by the
    sorted-line tier; same results as ``embed`` (checked against it wherever both run),
    fast enough for meshes of millions of triangles."""
    X = int_coords(verts, R)
    out = embed_lines_tri9(tri_coords(X, tris), R, levels, band, lattice)
    out["X"] = X
    return out


def embed_lines_tri9(tri9, R: int, levels: int, band: int = 2, lattice: int = 19):
    """embed_lines from triangle records in frame units ((T, 9) int64)."""
    tri9 = _c64(tri9)
    blocks = [root_blocks(R)]
    flags = []
    for L in range(levels):
        f = lines_flags(tri9, R, L, levels, band, blocks[L])
        flags.append(f)
        blocks.append(children(blocks[L], f))
    m = [lines_masks(tri9, R, L, blocks[L]) for L in range(levels + 1)]
    lk = lines_links(tri9, R, levels, blocks[levels], m[levels], lattice)
    return dict(tri9=tri9, blocks=blocks, flags=flags, masks=m, links=lk)


# --------------------------------------------------------------------------- #
# Bouzidi interpolated bounce-back, momentum exchange, and their derivatives
# --------------------------------------------------------------------------- #
def _block_index(blocks: np.ndarray):
    return {tuple(b): i for i, b in enumerate(blocks.tolist())}


def partner_cells(R, levels, blocks_f, mask_f, cell, dir):
    """Cell id of x_f - c_i at the finest level, or -1 if that cell is absent or solid."""
    C = directions()
    idx = _block_index(blocks_f)
    b = cell // 64
    t = cell % 64
    loc = np.stack([t % 4, (t // 4) % 4, t // 16], axis=1)
    g = 4 * blocks_f[b] + loc - C[dir]
    bb = np.floor_divide(g, 4)
    ll = g - 4 * bb
    bits = unpack_masks(mask_f)
    out = np.full(len(cell), -1, dtype=np.int64)
    for k in range(len(cell)):
        j = idx.get(tuple(bb[k].tolist()))
        if j is None:
            continue
        tt = int(ll[k, 0] + 4 * ll[k, 1] + 16 * ll[k, 2])
        if bits[j, tt] == 0:
            out[k] = j * 64 + tt
    return out


def bouzidi_incoming(q, f_i, f_i_partner, f_opp, has_partner):
    """Interpolated population entering x_f along -c_i (linear Bouzidi rule).

    q < 1/2 with a fluid partner x_f - c_i:  2q f_i(x_f) + (1-2q) f_i(x_f - c_i)
    q >= 1/2:                                f_i(x_f)/(2q) + (2q-1)/(2q) f_-i(x_f)
    q < 1/2 without a fluid partner:         f_i(x_f)   (simple bounce-back)
    """
    q = np.asarray(q, dtype=np.float64)
    lo = q < 0.5
    qs = np.where(lo, 1.0, q)
    hi_val = f_i / (2 * qs) + (2 * qs - 1) / (2 * qs) * f_opp
    lo_val = np.where(has_partner, 2 * q * f_i + (1 - 2 * q) * f_i_partner, f_i)
    return np.where(lo, lo_val, hi_val)


def _link_pops(links_, pop, partner):
    C = directions()
    d = links_["dir"]
    opp = np.array([opposite(int(i)) for i in d], dtype=np.int64)
    cell = links_["cell"]
    f_i = pop[d, cell].astype(np.float64)
    f_opp = pop[opp, cell].astype(np.float64)
    has = partner >= 0
    f_p = np.where(has, pop[d, np.where(has, partner, 0)].astype(np.float64), 0.0)
    return C[d].astype(np.float64), f_i, f_opp, f_p, has


def mex_force(links_, pop, partner) -> np.ndarray:
    """Momentum-exchange force on the body: sum over links of c_i (f_i(x_f) + f~_-i(x_f))."""
    c, f_i, f_opp, f_p, has = _link_pops(links_, pop, partner)
    inc = bouzidi_incoming(links_["q"], f_i, f_p, f_opp, has)
    return (c * (f_i + inc)[:, None]).sum(axis=0)


def mex_force_dq(links_, pop, partner) -> np.ndarray:
    """dF/dq_k (n_links, 3): c_i 2(f_i - f_i(partner)) for q < 1/2 with a partner,
    0 for the bounce-back fallback, c_i (f_-i - f_i) / (2 q^2) for q >= 1/2."""
    c, f_i, f_opp, f_p, has = _link_pops(links_, pop, partner)
    q = links_["q"]
    lo = q < 0.5
    qs = np.where(lo, 1.0, q)
    g = np.where(lo, np.where(has, 2 * (f_i - f_p), 0.0), (f_opp - f_i) / (2 * qs * qs))
    return c * g[:, None]


def dq_dverts(links_, X, tris, R, levels):
    """Per link: the three vertex ids of the nearest crossed triangle and dq/dV (n, 3, 3).

    Moving vertex j of the crossed triangle by dV moves the hit point's plane
    by lambda_j (n . dV)/|n|, with lambda the barycentric coordinates of the
    hit; along the link (length h, direction c) this changes q by
    lambda_j n . dV / (h n . c).  World units: coordinates are X / (2^20 r_o).
    """
    scale = float(domain_units(R))
    h = h_units(R, levels) / scale
    C = directions().astype(np.float64)
    Xw = X.astype(np.float64) / scale
    t = np.asarray(tris, dtype=np.int64)[links_["tri"]]
    A, B, Cc = Xw[t[:, 0]], Xw[t[:, 1]], Xw[t[:, 2]]
    cell = links_["cell"]
    c = C[links_["dir"]]
    n = np.cross(B - A, Cc - A)
    nn = np.einsum("ij,ij->i", n, n)
    return t, n, nn, A, B, Cc, c, h


def grad_verts_from_gq(links_, gq, X, tris, R, levels, blocks_f, n_verts):
    """sum_k gq_k dq_k/dV  (float64, (V, 3))."""
    t, n, nn, A, B, Cc, c, h = dq_dverts(links_, X, tris, R, levels)
    scale = float(domain_units(R))
    P = cell_centres(R, levels, blocks_f)[links_["cell"]].astype(np.float64) / scale
    Xh = P + (links_["q"] * h)[:, None] * c
    lamA = np.einsum("ij,ij->i", n, np.cross(B - Xh, Cc - Xh)) / nn
    lamB = np.einsum("ij,ij->i", n, np.cross(Cc - Xh, A - Xh)) / nn
    lamC = np.einsum("ij,ij->i", n, np.cross(A - Xh, B - Xh)) / nn
    base = n / (h * np.einsum("ij,ij->i", n, c))[:, None]
    g = np.zeros((n_verts, 3), dtype=np.float64)
    for j, lam in enumerate((lamA, lamB, lamC)):
        np.add.at(g, t[:, j], (gq * lam)[:, None] * base)
    return g


# --------------------------------------------------------------------------- #
# One lattice-Boltzmann step on the finest level: the table's consumer
# --------------------------------------------------------------------------- #
def lattice_weights(lattice: int) -> np.ndarray:
    """D3Q19 / D3Q27 weights in the direction order of directions() (rest, axes, edges,
    corners): 1/3, 1/18, 1/36 and 8/27, 2/27, 1/54, 1/216."""
    C = directions()[:lattice]
    kind = np.abs(C).sum(axis=1)
    table = {0: 1 / 3, 1: 1 / 18, 2: 1 / 36} if lattice == 19 else {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}
    return np.array([table[int(k)] for k in kind], dtype=np.float64)


def equilibrium(rho: np.ndarray, u: np.ndarray, lattice: int) -> np.ndarray:
    """(Q, n) second-order equilibrium w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)."""
    C = directions()[:lattice].astype(np.float64)
    w = lattice_weights(lattice)
    cu = u @ C.T
    usq = (u * u).sum(axis=1)
    return (w[None, :] * rho[:, None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq[:, None])).T


def lbm_sources(R, levels, blocks_f, mask_f, lattice):
    """For every finest cell x and direction i: the cell x - c_i if it is a fluid cell of
    the level, -1 if it is solid, -2 if its block is missing (edge of the level)."""
    C = directions()[:lattice]
    idx = _block_index(blocks_f)
    bits = unpack_masks(mask_f)
    n = len(blocks_f) * 64
    t = np.arange(64)
    loc = np.stack([t % 4, (t // 4) % 4, t // 16], axis=1)
    src = np.full((lattice, n), -2, dtype=np.int64)
    for b, blk in enumerate(np.asarray(blocks_f, dtype=np.int64).tolist()):
        g = 4 * np.array(blk)[None, :] + loc
        for i in range(lattice):
            s_ = g - C[i]
            bb = np.floor_divide(s_, 4)
            ll = s_ - 4 * bb
            for c in range(64):
                j = idx.get(tuple(bb[c].tolist()))
                if j is None:
                    continue
                tt = int(ll[c, 0] + 4 * ll[c, 1] + 16 * ll[c, 2])
                src[i, b * 64 + c] = -1 if bits[j, tt] else j * 64 + tt
    return src


def lbm_step(R, levels, blocks_f, mask_f, links_, pop, omega: float, lattice: int) -> np.ndarray:
    """One step from post-collision populations pop (Q, n_cells) at t to those at t + 1:
    1. pull streaming: f_i(x) = f*_i(x - c_i) when x - c_i is a fluid cell of the level,
       f*_i(x) when its block is missing (zero gradient at the edge of the level; the
       coupling to coarser levels is out of scope);
    2. at every cut link (x, d, q), the population entering x against c_d, where
       x - c_{-d} = x + c_d is solid: the linear Bouzidi rule (bouzidi_incoming) on f*;
    3. BGK collision f* = f - omega (f - f_eq(rho, u)) at fluid cells; solid cells are 0.
    """
    pop = np.asarray(pop, dtype=np.float64)
    n = pop.shape[1]
    src = lbm_sources(R, levels, blocks_f, mask_f, lattice)
    fluid = unpack_masks(mask_f).reshape(-1) == 0
    pre = np.zeros_like(pop)
    for i in range(lattice):
        ok = src[i] >= 0
        pre[i, ok] = pop[i, src[i, ok]]
        edge = src[i] == -2
        pre[i, edge] = pop[i, edge]
    partner = partner_cells(R, levels, blocks_f, mask_f, links_["cell"], links_["dir"])
    _, f_i, f_opp, f_p, has = _link_pops(links_, pop, partner)
    inc = bouzidi_incoming(links_["q"], f_i, f_p, f_opp, has)
    opp = np.array([opposite(int(d)) for d in links_["dir"]], dtype=np.int64)
    pre[opp, links_["cell"]] = inc
    C = directions()[:lattice].astype(np.float64)
    rho = pre.sum(axis=0)
    rs = np.where(rho != 0, rho, 1.0)
    u = (C.T @ pre).T / rs[:, None]
    out = pre - omega * (pre - equilibrium(rho, u, lattice))
    out[:, ~fluid] = 0.0
    return out