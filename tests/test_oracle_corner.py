"""CPU pins for the corner-face case: each tetrahedron's big face is met by the
link from its cell centre P along the corner direction c at the face's centroid,
so q = delta / h exactly (1/8), and the face is the argmin triangle.  The case is
built so that c . n leaves the 32-bit range while every vertex offset from P stays
below 2^14 (checked here in exact integers)."""
from __future__ import annotations

import numpy as np

import corner_case as K


def test_corner_case_leaves_the_int32_range():
    v, t = K.mesh()
    X = (v.astype(np.float64) * (1 << 20)).astype(np.int64)
    P = K.centres()
    for i in range(4):
        tet = t[4 * i:4 * i + 4]
        assert np.all(np.abs(X[tet.reshape(-1)] - P[i][None, :]) < (1 << 14)), "every vertex within 2^14 of P"
        face = [f for f in tet if 4 * i + 3 not in f]  # the face without the apex
        assert len(face) == 1
        a, b, c = (X[j] - P[i] for j in face[0])
        n = np.cross(b - a, c - a)
        nc = int(np.dot(n, K.SIGNS[i]))
        assert abs(nc) == 9 * K.A * K.A and abs(nc) >= 2 ** 31
        assert np.all(np.abs(n) < 2 ** 31)


def test_oracle_corner_links_closed_form(orc):
    v, t = K.mesh()
    o = orc.embed(v, t, K.R, K.LEVELS, K.BAND, K.LATTICE)
    blocks = o["blocks"][-1]
    lk = o["links"]
    P = orc.cell_centres(K.R, K.LEVELS, blocks)
    for i in range(4):
        d = K.direction_index(K.SIGNS[i])
        cell = int(np.nonzero((P == K.centres()[i][None, :]).all(axis=1))[0][0])
        sel = np.nonzero((lk["cell"] == cell) & (lk["dir"] == d))[0]
        assert len(sel) == 1, "the link from P along c is a cut link"
        k = sel[0]
        assert lk["q"][k] == K.DELTA / K.H
        assert 4 * i + 3 not in t[lk["tri"][k]], "the big face is the argmin"
