"""Incremental re-embedding (reembed_window: a window forest, a triangle subset and
emb_splice) after local deformations of a closed mesh, several steps in a row: every
block, mask word and cut link must equal the oracle's embedding of the deformed mesh."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import Q_TOL, compare_full
from synth import bump, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def changed_extent(v_old, v_new, tris, moved, R):
    """y-z extent, in root blocks (half-open), of the triangles touching moved vertices,
    at their old and new positions."""
    hit = np.isin(tris, moved).any(axis=1)
    pts = np.concatenate([v_old[tris[hit]].reshape(-1, 3), v_new[tris[hit]].reshape(-1, 3)])
    lo = np.floor(pts.min(axis=0) * R).astype(int)
    hi = np.floor(pts.max(axis=0) * R).astype(int) + 1
    return int(lo[1]), int(hi[1]), int(lo[2]), int(hi[2])


def _state(E):
    return dict(blocks=[b.cpu().numpy().astype(np.int64) for b in E.fetch_blocks()],
                masks=[m.cpu().numpy().view(np.uint64) for m in E.masks],
                flags=[], links={k: E.links[k].cpu().numpy().astype(np.int64 if k != "q" else np.float32)
                                 for k in ("cell", "dir", "q", "tri")})


@pytest.mark.parametrize("lattice,axis", [(19, (0.2, 1.0, 0.3)), (27, (-0.4, -0.3, 1.0))])
def test_local_deformation_steps(orc, lattice, axis):
    import torch

    import paper_2512_01251_gb300 as P
    w = workload("star_112k")
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), w.R, w.levels, w.band, lattice)
    for step in range(3):
        v_new, moved = bump(v, axis, 0.97, 900 * (step + 1) if step % 2 == 0 else -700)
        ext = changed_extent(v, v_new, t, moved, w.R)
        assert ext[1] - ext[0] < w.R and ext[3] - ext[2] < w.R  # a local change
        P.reembed_window(E, torch.from_numpy(v_new).cuda(), ext, w.band)
        assert P.emb_status_get() == P.EMB_OK
        o = orc.embed_lines(v_new, t, w.R, w.levels, w.band, lattice)
        g = _state(E)
        for L in range(w.levels + 1):
            np.testing.assert_array_equal(g["blocks"][L], o["blocks"][L], err_msg=f"step {step} blocks L={L}")
            np.testing.assert_array_equal(g["masks"][L], o["masks"][L], err_msg=f"step {step} masks L={L}")
        for k in ("cell", "dir", "tri"):
            np.testing.assert_array_equal(g["links"][k], o["links"][k], err_msg=f"step {step} links {k}")
        assert np.abs(g["links"]["q"].astype(np.float64) - o["links"]["q"]).max() <= Q_TOL
        v = v_new


def test_local_deformation_on_the_bench_workload(orc):
    """The same on the ~7.2M-triangle mesh (D3Q27): a cap of about 5,000 vertices pushed
    out, then back in; the spliced embedding equals the oracle's after each step."""
    import torch

    import paper_2512_01251_gb300 as P
    w = workload("star_7m")
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), w.R, w.levels, w.band, 27)
    for step, push in enumerate((300, -300)):
        v_new, moved = bump(v, (0.2, 1.0, 0.3), 0.995, push)
        ext = changed_extent(v, v_new, t, moved, w.R)
        P.reembed_window(E, torch.from_numpy(v_new).cuda(), ext, w.band)
        assert P.emb_status_get() == P.EMB_OK
        o = orc.embed_lines(v_new, t, w.R, w.levels, w.band, 27)
        g = _state(E)
        for L in range(w.levels + 1):
            np.testing.assert_array_equal(g["blocks"][L], o["blocks"][L], err_msg=f"step {step} blocks L={L}")
            np.testing.assert_array_equal(g["masks"][L], o["masks"][L], err_msg=f"step {step} masks L={L}")
        for k in ("cell", "dir", "tri"):
            np.testing.assert_array_equal(g["links"][k], o["links"][k], err_msg=f"step {step} links {k}")
        assert np.abs(g["links"]["q"].astype(np.float64) - o["links"]["q"]).max() <= Q_TOL
        v = v_new
