"""Closed, outward-oriented triangle meshes in the unit cube, snapped to 2^-20.

Every generator returns ``(verts, tris)``: ``verts`` float32 (V, 3) whose
coordinates are exact multiples of 2^-20 strictly inside (0, 1), and ``tris``
int32 (T, 3) listing vertex ids counter-clockwise as seen from outside (the
geometry orientation convention of Sec. 3.1, Fig. "orientation").
"""
from __future__ import annotations

import math

import numpy as np

GRID_BITS = 20
_GRID = float(1 << GRID_BITS)


def snap(v: np.ndarray) -> np.ndarray:
    """Round float64 coordinates to the 2^-20 grid (round-half-even), as float32."""
    v = np.asarray(v, dtype=np.float64)
    s = np.round(v * _GRID) / _GRID
    if not (np.all(s > 0.0) and np.all(s < 1.0)):
        raise ValueError("snapped vertices must lie strictly inside the unit cube")
    return s.astype(np.float32)


def signed_volume(verts: np.ndarray, tris: np.ndarray) -> float:
    """Volume enclosed by a closed oriented mesh (divergence theorem), float64."""
    v = np.asarray(verts, dtype=np.float64)
    a, b, c = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


# --------------------------------------------------------------------------- #
# icosphere
# --------------------------------------------------------------------------- #
def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
         [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
         [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # make every face outward (the solid is convex and centred at the origin)
    for i, (a, b, c) in enumerate(f):
        n = np.cross(v[b] - v[a], v[c] - v[a])
        if np.dot(n, v[a] + v[b] + v[c]) < 0:
            f[i] = [a, c, b]
    return v, f


def icosphere(subdiv: int = 2, radius: float = 0.3, centre=(0.5, 0.5, 0.5), seed: int | None = None,
              jitter: float = 0.01):
    """Icosahedron with ``subdiv`` midpoint subdivisions projected to the sphere.

    ``subdiv=2`` gives 320 triangles and 162 vertices.  With ``seed`` set, the
    centre is moved by U(-jitter, jitter) per axis (PCG64).
    """
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = (np.asarray(verts[a]) + np.asarray(verts[b])) / 2.0
                m /= np.linalg.norm(m)
                verts.append(tuple(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [ab, b, bc], [ca, bc, c], [ab, bc, ca]]
        f = np.array(nf, dtype=np.int64)
    c = np.asarray(centre, dtype=np.float64)
    if seed is not None:
        rng = np.random.default_rng(seed)
        c = c + rng.uniform(-jitter, jitter, size=3)
    pts = np.asarray(verts) * radius + c
    return snap(pts), f.astype(np.int32)


# --------------------------------------------------------------------------- #
# radial "star" surfaces on a latitude-longitude grid
# --------------------------------------------------------------------------- #
def _real_sh_theta_parts(lmax: int, theta: np.ndarray) -> np.ndarray:
    """Fully normalised associated Legendre values P(l, m, cos theta).

    Returns array (lmax+1, lmax+1, len(theta)) with entry [l, m] for m <= l,
    normalised so that the real harmonics built from them are orthonormal on
    the unit sphere.  Standard three-term recurrences.
    """
    x = np.cos(theta)
    s = np.sin(theta)
    P = np.zeros((lmax + 1, lmax + 1, theta.size))
    P[0, 0] = 1.0 / math.sqrt(4.0 * math.pi)
    for m in range(1, lmax + 1):
        P[m, m] = -math.sqrt((2 * m + 1) / (2.0 * m)) * s * P[m - 1, m - 1]
    for m in range(0, lmax):
        P[m + 1, m] = math.sqrt(2 * m + 3) * x * P[m, m]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1) ** 2 - m * m) / (4.0 * (l - 1) ** 2 - 1.0))
            P[l, m] = a * (x * P[l - 1, m] - b * P[l - 2, m])
    return P


def _radius_field(theta: np.ndarray, phi: np.ndarray, coeffs: dict[tuple[int, int], float], lmax: int):
    """sum_{l,m} a_lm Y_lm(theta, phi) on the outer product grid (theta x phi)."""
    P = _real_sh_theta_parts(lmax, theta)
    # G[:, col] holds sum_l a_lm P_lm(theta) for each signed m; trig[col] the phi factor
    cols_g, cols_t = [], []
    for m in range(-lmax, lmax + 1):
        am = abs(m)
        g = np.zeros(theta.size)
        for l in range(max(am, 1), lmax + 1):
            a = coeffs.get((l, m), 0.0)
            if a:
                g += a * P[l, am]
        if m == 0:
            t = np.ones(phi.size)
        elif m > 0:
            g = g * math.sqrt(2.0)
            t = np.cos(m * phi)
        else:
            g = g * math.sqrt(2.0)
            t = np.sin(am * phi)
        cols_g.append(g)
        cols_t.append(t)
    G = np.stack(cols_g, axis=1)
    Tr = np.stack(cols_t, axis=0)
    return G @ Tr


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a uniform unit quaternion (Shoemake)."""
    u1, u2, u3 = rng.uniform(0.0, 1.0, size=3)
    q = np.array([
        math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
        math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
        math.sqrt(u1) * math.sin(2 * math.pi * u3),
        math.sqrt(u1) * math.cos(2 * math.pi * u3),
    ])
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def radial_star(n_theta: int, n_phi: int, lmax: int, sigma, seed: int, base_radius: float = 0.3,
                scale=(1.0, 1.0, 1.0), centre=(0.5, 0.5, 0.5), jitter: float = 0.0,
                rotate: bool = False):
    """Closed star-shaped surface r(theta, phi) = base (1 + sum a_lm Y_lm).

    ``n_theta`` latitude bands and ``n_phi`` longitude segments: two poles,
    ``n_theta - 1`` rings of ``n_phi`` vertices, pole fans, and two triangles
    per quad, i.e. ``2 n_phi (n_theta - 1)`` triangles sharing seam vertices.
    ``sigma(l)`` is the standard deviation of every a_lm of degree l (PCG64,
    drawn in (l, m) order).  Anisotropic ``scale`` is applied about the centre,
    then an optional uniform random rotation, then the centre offset.
    """
    rng = np.random.default_rng(seed)
    coeffs = {}
    for l in range(1, lmax + 1):
        sd = float(sigma(l))
        for m in range(-l, l + 1):
            coeffs[(l, m)] = float(rng.normal(0.0, sd))
    c = np.asarray(centre, dtype=np.float64)
    if jitter:
        c = c + rng.uniform(-jitter, jitter, size=3)
    Rm = _random_rotation(rng) if rotate else np.eye(3)

    theta_r = np.arange(1, n_theta) * (math.pi / n_theta)
    phi = np.arange(n_phi) * (2.0 * math.pi / n_phi)
    rad = base_radius * (1.0 + _radius_field(theta_r, phi, coeffs, lmax))
    pole = base_radius * (1.0 + _radius_field(np.array([0.0, math.pi]), np.array([0.0]), coeffs, lmax))[:, 0]
    if np.any(rad <= 0) or np.any(pole <= 0):
        raise ValueError("radial field is not positive")
    st, ct = np.sin(theta_r)[:, None], np.cos(theta_r)[:, None]
    ring = np.stack([rad * st * np.cos(phi)[None, :], rad * st * np.sin(phi)[None, :], rad * ct], axis=-1)
    pts = np.concatenate([
        np.array([[0.0, 0.0, pole[0]]]),
        ring.reshape(-1, 3),
        np.array([[0.0, 0.0, -pole[1]]]),
    ])
    pts = pts * np.asarray(scale, dtype=np.float64)
    pts = pts @ Rm.T
    pts = pts + c

    nr = n_theta - 1
    north, south = 0, 1 + nr * n_phi
    j = np.arange(n_phi)
    jn = (j + 1) % n_phi
    ringid = lambda k, jj: 1 + k * n_phi + jj  # noqa: E731
    tris = [np.stack([np.full(n_phi, north), ringid(0, j), ringid(0, jn)], axis=1)]
    for k in range(nr - 1):
        a, b = ringid(k, j), ringid(k, jn)
        cc, d = ringid(k + 1, j), ringid(k + 1, jn)
        tris.append(np.stack([a, cc, b], axis=1))
        tris.append(np.stack([b, cc, d], axis=1))
    tris.append(np.stack([np.full(n_phi, south), ringid(nr - 1, jn), ringid(nr - 1, j)], axis=1))
    t = np.concatenate(tris).astype(np.int32)
    return snap(pts), t


# --------------------------------------------------------------------------- #
# small exact solids for closed-form checks
# --------------------------------------------------------------------------- #
def axis_box(lo, hi):
    """Axis-aligned box [lo, hi] as 12 outward triangles; corners given in 2^-20 units (ints)."""
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    corners = np.array([[(hi if (i >> d) & 1 else lo)[d] for d in range(3)] for i in range(8)], dtype=np.float64)
    quads = [  # each quad listed counter-clockwise seen from outside
        (0, 4, 6, 2),  # -x
        (1, 3, 7, 5),  # +x
        (0, 1, 5, 4),  # -y
        (2, 6, 7, 3),  # +y
        (0, 2, 3, 1),  # -z
        (4, 5, 7, 6),  # +z
    ]
    tris = []
    for a, b, c, d in quads:
        tris += [[a, b, c], [a, c, d]]
    return snap(corners / _GRID), np.array(tris, dtype=np.int32)


def tetrahedron(pts):
    """Tetrahedron from 4 integer points (2^-20 units), oriented outward."""
    p = np.asarray(pts, dtype=np.float64)
    f = [[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]]
    cen = p.mean(axis=0)
    out = []
    for a, b, c in f:
        n = np.cross(p[b] - p[a], p[c] - p[a])
        out.append([a, b, c] if np.dot(n, p[a] - cen) > 0 else [a, c, b])
    return snap(p / _GRID), np.array(out, dtype=np.int32)


def octahedron(centre, radii):
    """Octahedron |x/rx| + |y/ry| + |z/rz| <= 1 with integer centre and radii (2^-20 units)."""
    c = np.asarray(centre, dtype=np.int64)
    r = np.asarray(radii, dtype=np.int64)
    p = np.array([c + [r[0], 0, 0], c - [r[0], 0, 0], c + [0, r[1], 0], c - [0, r[1], 0],
                  c + [0, 0, r[2]], c - [0, 0, r[2]]], dtype=np.float64)
    tris = []
    for xs in (0, 1):
        for ys in (2, 3):
            for zs in (4, 5):
                a, b, cc = xs, ys, zs
                n = np.cross(p[b] - p[a], p[cc] - p[a])
                tris.append([a, b, cc] if np.dot(n, p[a] - c) > 0 else [a, cc, b])
    return snap(p / _GRID), np.array(tris, dtype=np.int32)


def corner_face_tetrahedra(centres, signs, a: int, delta: int, depth: int):
    """Tetrahedra whose large face is perpendicular to a corner direction c = signs[i].

    For each integer point P = centres[i] (2^-20 units) the face has its centroid at
    G = P + delta c and its vertices at G + a u_k, with u_k = c * (1,-1,0), c * (0,1,-1),
    c * (-1,0,1) (componentwise), so every vertex lies within a + |delta| of P on each
    axis while the face normal is 3 a^2 c.  The fourth vertex is G + depth c.  The
    segment from P along c meets the face at its centroid, at parameter delta / h for a
    link of length h.  Returns one mesh (verts, tris) holding all the tetrahedra.
    """
    vs, ts = [], []
    for P, c in zip(np.asarray(centres, dtype=np.int64), np.asarray(signs, dtype=np.int64)):
        G = P + delta * c
        u = np.array([[1, -1, 0], [0, 1, -1], [-1, 0, 1]], dtype=np.int64) * c[None, :]
        pts = np.concatenate([G[None, :] + a * u, (G + depth * c)[None, :]])
        v, t = tetrahedron(pts)
        ts.append(t + 4 * len(vs))
        vs.append(v)
    return np.concatenate(vs).astype(np.float32), np.concatenate(ts).astype(np.int32)


def bump(verts: np.ndarray, axis, cos_min: float, push_units: int, centre=(0.5, 0.5, 0.5)):
    """A local deformation of a star-shaped mesh: every vertex whose direction from
    `centre` lies within the cone cos(angle to `axis`) >= cos_min moves outward along
    that direction by about push_units grid units (2^-20), rounded to the grid per axis.
    Returns (new verts float32, ids of the moved vertices)."""
    v = np.asarray(verts, dtype=np.float64)
    d = v - np.asarray(centre, dtype=np.float64)[None, :]
    u = d / np.linalg.norm(d, axis=1, keepdims=True)
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    sel = np.nonzero(u @ a >= cos_min)[0]
    out = (np.round(v * _GRID)).astype(np.int64)
    out[sel] += np.round(u[sel] * push_units).astype(np.int64)
    return snap(out / _GRID), sel
