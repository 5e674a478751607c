"""The library's exact device predicates, one decision at a time, against the oracle's
host evaluation on seeded adversarial queries (predicate_cases.py): the +x line test of
the filter and the voxelizer, the link kernel's exact per-direction segment test and its
per-pair path (32-bit moments within 2^14 of the link start, 64-bit beyond), and the
closed-box overlap test of the binning and the refine flags.  Decisions must be
identical; q within 2e-6 of the FP64 parameter."""
from __future__ import annotations

import numpy as np
import pytest

import predicate_cases as PC

pytestmark = pytest.mark.gpu

N = 200_000


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _probe(kind, q):
    import torch

    import paper_2512_01251_gb300 as P
    hit, qq = P.emb_probe_predicates(kind, torch.from_numpy(q))
    torch.cuda.synchronize()
    return hit.cpu().numpy(), qq.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("kind", ["segment", "pair"])
def test_segment_decisions(orc, kind):
    import paper_2512_01251_gb300 as P
    q, tri, Pt, dirs, h = PC.segment_queries(101, N)
    hit, t = orc.each_segment(tri, Pt, dirs, h)
    g_hit, g_q = _probe(P.EMB_PROBE_SEGMENT if kind == "segment" else P.EMB_PROBE_PAIR, q)
    bad = np.nonzero(g_hit != hit)[0]
    assert len(bad) == 0, (len(bad), q[bad[:3]].tolist())
    sel = hit == 1
    assert np.abs(g_q[sel] - t[sel]).max() <= 2e-6
    assert np.all(g_q[~sel] == -1)


def test_xline_decisions(orc):
    import paper_2512_01251_gb300 as P
    q, tri, Pt = PC.xline_queries(102, N)
    hit = orc.each_line(tri, Pt, np.ones(len(q), dtype=np.int32))
    g_hit, _ = _probe(P.EMB_PROBE_XLINE, q)
    assert np.array_equal(g_hit, hit.astype(np.int32))


def test_box_decisions(orc):
    import paper_2512_01251_gb300 as P
    q, tri, lo, hi = PC.box_queries(103, N)
    hit = orc.each_box(tri, lo, hi)
    g_hit, _ = _probe(P.EMB_PROBE_BOX, q)
    assert np.array_equal(g_hit, hit.astype(np.int32))


def test_probe_rejects_bad_queries():
    import torch

    import paper_2512_01251_gb300 as P
    q = np.zeros((2, 15), dtype=np.int64)
    q[:, 13] = 256
    q[0, 12] = 0
    q[1, 12] = 27
    hit, _ = _probe(P.EMB_PROBE_SEGMENT, q)
    assert np.all(hit == -1)
    with pytest.raises(P.EmbError):
        P.emb_probe_predicates(7, torch.from_numpy(q))
