"""Seeded adversarial queries for the single-decision predicate tests.

Each generator returns queries in the 15-int64 layout of emb_probe_predicates: a
triangle in frame units, then the query (a line, a segment or a box).  They mix
degenerate geometry on the cell lattice (vertices on lines, edges through cell
centres, faces through both ends of a link, boxes touching a triangle at a point)
with the magnitudes at which the integer arithmetic changes width: vertex offsets at
and around 2^14 from the query point, corner-direction faces whose c . n passes 2^31,
and coordinates near 0 and 2^25."""
from __future__ import annotations

import numpy as np

TOP = 1 << 25
GATE = 1 << 14
CORNERS = np.array([[1, 1, 1], [1, 1, -1], [1, -1, 1], [-1, 1, 1]], dtype=np.int64)


def _clip(v):
    return np.clip(v, 0, TOP - 1)


def _offsets(rng, n, half):
    """Vertex offsets (n, 3, 3) from a query point, by regime; half: (n,) half cell sizes."""
    half = np.broadcast_to(np.asarray(half, dtype=np.int64), (n,))
    kind = rng.integers(0, 6, n)
    hh = half[:, None, None]
    lattice = rng.integers(-3, 4, (n, 3, 3)) * hh  # vertices and edges through centres and link ends
    gate = rng.choice([-GATE - 1, -GATE, -GATE + 1, GATE - 1, GATE, GATE + 1, 0], (n, 3, 3))
    gate = np.where(rng.random((n, 3, 3)) < 0.15, hh, gate)  # around the 32-bit gate of the link kernel
    # a face perpendicular to a corner direction, |c . n| = 9 a^2 > 2^31
    c = CORNERS[rng.integers(0, 4, n)] * rng.choice([-1, 1], (n, 1))
    a = rng.integers(15_500, GATE, n)[:, None, None]
    dmax = np.minimum(half, GATE - 1 - a[:, 0, 0])  # every vertex stays within the gate
    d = np.floor(rng.random(n) * (2 * dmax + 1)).astype(np.int64) - dmax
    u = np.array([[1, -1, 0], [0, 1, -1], [-1, 0, 1]], dtype=np.int64)[None, :, :] * c[:, None, :]
    corner = d[:, None, None] * c[:, None, :] + a * u
    inside = rng.integers(-GATE + 1, GATE, (n, 3, 3))  # random within the gate
    large = rng.integers(-(1 << 24), 1 << 24, (n, 3, 3))  # large faces
    small = np.floor((rng.random((n, 3, 3)) * 2 - 1) * 2 * hh).astype(np.int64)  # small faces near the link
    opts = np.stack([lattice, gate, corner, inside, large, small])
    return opts[kind, np.arange(n)]


def segment_queries(seed: int, n: int):
    """(queries (n, 15), tri9 (n, 9), P (n, 3), dirs (n,), h (n,)) for segment tests."""
    rng = np.random.default_rng(seed)
    h = (1 << rng.integers(8, 19, n)).astype(np.int64)
    half = h // 2
    ncell = TOP // h
    g = np.floor(rng.random((n, 3)) * ncell[:, None]).astype(np.int64)
    edge = rng.random(n) < 0.1  # near the ends of the frame
    ends = np.stack([np.zeros(n, np.int64), np.ones(n, np.int64), ncell - 2, ncell - 1], axis=1)
    g = np.where(edge[:, None], np.take_along_axis(ends, rng.integers(0, 4, (n, 3)), axis=1), g)
    P = (2 * g + 1) * half[:, None]
    tri = _clip(P[:, None, :] + _offsets(rng, n, half)).reshape(n, 9)
    dirs = rng.integers(1, 27, n).astype(np.int64)
    q = np.zeros((n, 15), dtype=np.int64)
    q[:, 0:9] = tri
    q[:, 9:12] = P
    q[:, 12] = dirs
    q[:, 13] = h
    return q, tri, P, dirs, h


def xline_queries(seed: int, n: int):
    """(queries, tri9, P) for +x line tests (P = (0, y, z) of the line)."""
    rng = np.random.default_rng(seed)
    half = (1 << rng.integers(3, 18, n)).astype(np.int64)
    ncell = TOP // (2 * half)
    g = np.floor(rng.random((n, 3)) * ncell[:, None]).astype(np.int64)
    edge = rng.random(n) < 0.1
    ends = np.stack([np.zeros(n, np.int64), ncell - 1], axis=1)
    g = np.where(edge[:, None], np.take_along_axis(ends, rng.integers(0, 2, (n, 3)), axis=1), g)
    c = (2 * g + 1) * half[:, None]
    tri = _clip(c[:, None, :] + _offsets(rng, n, half)).reshape(n, 9)
    P = c.copy()
    P[:, 0] = 0
    q = np.zeros((n, 15), dtype=np.int64)
    q[:, 0:9] = tri
    q[:, 10] = P[:, 1]
    q[:, 11] = P[:, 2]
    return q, tri, P


def box_queries(seed: int, n: int):
    """(queries, tri9, lo, hi) for closed-box overlap tests."""
    rng = np.random.default_rng(seed)
    W = (1 << rng.integers(4, 21, n)).astype(np.int64)
    b = np.floor(rng.random((n, 3)) * (TOP // W)[:, None]).astype(np.int64)
    dil = np.choose(rng.integers(0, 4, n), [np.zeros(n, np.int64), W // 8, W // 2, W])
    lo = b * W[:, None] - dil[:, None]
    hi = (b + 1) * W[:, None] + dil[:, None]
    Wc = W[:, None, None]
    # vertices on the box's lattice: touching faces, edges and corners
    k0 = lo[:, None, :] + rng.integers(-2, 3, (n, 3, 3)) * (W // 2 + dil)[:, None, None]
    # a corner just outside, a triangle across an edge
    k1 = np.stack([lo - rng.integers(0, 3, (n, 3)), hi + rng.integers(0, 3, (n, 3)),
                   lo + np.floor((rng.random((n, 3)) * 3 - 1) * W[:, None]).astype(np.int64)], axis=1)
    k2 = lo[:, None, :] + np.floor((rng.random((n, 3, 3)) * 5 - 2) * Wc).astype(np.int64)
    k3 = rng.integers(0, TOP, (n, 3, 3))  # large triangles
    pts = np.stack([k0, k1, k2, k3])[rng.integers(0, 4, n), np.arange(n)]
    tri = _clip(pts).reshape(n, 9)
    q = np.zeros((n, 15), dtype=np.int64)
    q[:, 0:9] = tri
    q[:, 9:12] = lo
    q[:, 12:15] = hi
    return q, tri, lo, hi
