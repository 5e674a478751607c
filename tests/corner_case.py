"""The corner-face mesh shared by the CPU pin and the GPU regression test: four
tetrahedra whose large faces are perpendicular to the four corner lines of D3Q27,
each face centred a sixteenth of a cell beyond a finest cell centre P of a 16^3
root with levels 0..3 (cell size 2048 frame units), with every vertex within
16,256 units of P.  Its face normal is 3 a^2 c with a = 16,000, so c . n = 9 a^2 =
2.304e9 exceeds the 32-bit range while each vertex offset stays below 2^14."""
from __future__ import annotations

import numpy as np

from synth import corner_face_tetrahedra

R, LEVELS, BAND, LATTICE = 16, 3, 2, 27
H = 1 << (18 - 4 - LEVELS)  # 2048
HALF = H // 2
A, DELTA, DEPTH = 16_000, H // 8, 5 * H
CELLS = np.array([[150, 150, 150], [150, 350, 350], [350, 150, 350], [350, 350, 150]], dtype=np.int64)
SIGNS = np.array([[1, 1, 1], [1, 1, -1], [1, -1, 1], [-1, 1, 1]], dtype=np.int64)


def centres():
    return (2 * CELLS + 1) * HALF


def mesh():
    return corner_face_tetrahedra(centres(), SIGNS, A, DELTA, DEPTH)


def direction_index(c) -> int:
    from oracle import oracle as O
    C = O.directions()
    return int(np.nonzero((C == np.asarray(c)[None, :]).all(axis=1))[0][0])
