"""The oracle's bulk single-decision entry points (one triangle per query) agree with
its single-query functions on the adversarial cases of predicate_cases.py, and the
cases reach what they are meant to reach (both sides of the 2^14 gate, c . n beyond
2^31, crossings at both ends of a link, touching boxes)."""
from __future__ import annotations

import numpy as np

import predicate_cases as PC


def test_each_segment_matches_single_queries(orc):
    q, tri, P, dirs, h = PC.segment_queries(5, 400)
    hit, t = orc.each_segment(tri, P, dirs, h)
    for i in range(len(q)):
        out = np.zeros(1)
        one = orc.lib().orc_segment_hit(orc._p(np.ascontiguousarray(tri[i])), orc._p(np.ascontiguousarray(P[i])),
                                        int(dirs[i]), int(h[i]), orc._p(out))
        assert one == hit[i] and (not one or out[0] == t[i])
    assert 20 < hit.sum() < len(q)
    off = np.abs(tri.reshape(-1, 3, 3) - P[:, None, :]).max(axis=(1, 2))
    assert (off < PC.GATE).sum() > 50 and (off >= PC.GATE).sum() > 50
    n = np.cross(tri[:, 3:6] - tri[:, 0:3], tri[:, 6:9] - tri[:, 0:3])
    assert (np.abs(n @ PC.CORNERS.T).max(axis=1) >= 2 ** 31)[off < PC.GATE].sum() > 10


def test_each_line_and_box_match_single_queries(orc):
    q, tri, P = PC.xline_queries(6, 300)
    hit = orc.each_line(tri, P, np.ones(len(q), dtype=np.int32))
    for i in range(len(q)):
        assert orc.lib().orc_line_hits(orc._p(np.ascontiguousarray(tri[i])), orc._p(np.ascontiguousarray(P[i])), 1) == hit[i]
    assert 10 < hit.sum() < len(q)
    q, tri, lo, hi = PC.box_queries(7, 300)
    hit = orc.each_box(tri, lo, hi)
    for i in range(len(q)):
        assert orc.sat(tri[i], lo[i], hi[i]) == bool(hit[i])
    assert 30 < hit.sum() < len(q) - 30
