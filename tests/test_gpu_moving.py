"""Moving geometry: emb_mesh_update rewrites a mesh's records for new vertex
positions (same triangles), and a planned batch replay re-embeds the moved mesh.

- the update to the same positions changes nothing;
- an updated mesh embeds exactly like a mesh created from the new positions, and
  like the oracle on them;
- a translation by one root block keeps every count of the plan (the embedding is
  equivariant under whole-block shifts of the integer frame), so the replay is
  exact without re-planning;
- a scaling changes the counts: the replay reports EMB_ERR_STATE on the device,
  stays in bounds, and a re-planned batch is exact again.
"""
from __future__ import annotations

import numpy as np
import pytest

from synth.meshes import icosphere, snap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _result(P, E):
    return dict(blocks=[b.cpu().numpy() for b in E.fetch_blocks()],
                masks=[m.cpu().numpy() for m in E.masks],
                links={k: E.links[k].cpu().numpy() for k in ("cell", "dir", "q", "tri")})


def _batch_result(P, B, j):
    r = P.emb_batch_results(B, j)
    return dict(blocks=[b.cpu().numpy() for b in r["blocks"]], masks=[m.cpu().numpy() for m in r["masks"]],
                links={k: r["links"][k].cpu().numpy() for k in ("cell", "dir", "q", "tri")})


def _same(a, b, what):
    assert len(a["blocks"]) == len(b["blocks"]), what
    for L in range(len(a["blocks"])):
        np.testing.assert_array_equal(a["blocks"][L], b["blocks"][L], err_msg=f"{what}: blocks L={L}")
        np.testing.assert_array_equal(a["masks"][L], b["masks"][L], err_msg=f"{what}: masks L={L}")
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(a["links"][k], b["links"][k], err_msg=f"{what}: links {k}")
    np.testing.assert_array_equal(a["links"]["q"].view(np.uint32), b["links"]["q"].view(np.uint32), err_msg=what)


def _embed(P, v, t, R, levels, lattice, mesh=None):
    import torch
    return P.embed(torch.from_numpy(v), torch.from_numpy(t), R, levels, 2, lattice, mesh=mesh)


def test_update_to_same_positions_changes_nothing():
    import torch

    import paper_2512_01251_gb300 as P
    v, t = icosphere(3, radius=0.2, centre=(0.5, 0.5, 0.5))
    m = P.emb_mesh_create(torch.from_numpy(v), torch.from_numpy(t), 4)
    a = _result(P, _embed(P, v, t, 4, 3, 19, mesh=m))
    P.emb_mesh_update(m, torch.from_numpy(v))
    b = _result(P, _embed(P, v, t, 4, 3, 19, mesh=m))
    assert P.emb_status_get() == P.EMB_OK
    _same(a, b, "same positions")


def test_updated_mesh_embeds_like_a_new_mesh_and_the_oracle(orc):
    import torch

    import paper_2512_01251_gb300 as P
    v0, t = icosphere(2, radius=0.2, centre=(0.5, 0.5, 0.5))
    # move and stretch the body: a new shape on the same triangles, snapped to the 2^-20 grid
    v1 = snap((v0 - 0.5) * np.array([1.1, 0.9, 1.25]) + np.array([0.53, 0.47, 0.51]))
    m = P.emb_mesh_create(torch.from_numpy(v0), torch.from_numpy(t), 2)
    P.emb_mesh_update(m, torch.from_numpy(v1))
    moved = _result(P, _embed(P, v1, t, 2, 2, 19, mesh=m))
    fresh = _result(P, _embed(P, v1, t, 2, 2, 19))
    assert P.emb_status_get() == P.EMB_OK
    _same(moved, fresh, "updated vs new mesh")
    o = orc.embed(v1, t, 2, 2, 2, 19)
    for L in range(3):
        np.testing.assert_array_equal(moved["blocks"][L].astype(np.int64), o["blocks"][L])
        np.testing.assert_array_equal(moved["masks"][L].view(np.uint64), o["masks"][L])
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(moved["links"][k].astype(np.int64), o["links"][k])
    assert np.abs(moved["links"]["q"].astype(np.float64) - o["links"]["q"]).max(initial=0) <= 2e-6


def test_update_rejects_off_grid_vertices():
    import torch

    import paper_2512_01251_gb300 as P
    v, t = icosphere(2, radius=0.2, centre=(0.5, 0.5, 0.5))
    m = P.emb_mesh_create(torch.from_numpy(v), torch.from_numpy(t), 2)
    bad = v.copy()
    bad[0, 0] += np.float32(2.0 ** -22)  # off the 2^-20 grid
    P.emb_mesh_update(m, torch.from_numpy(bad))
    assert P.emb_status_get() == P.EMB_ERR_BAD_INPUT
    with pytest.raises(P.EmbError):
        P.emb_mesh_update(m, torch.from_numpy(v[:-1]))  # vertex count differs


def _moving_batch(P):
    import torch
    # R = 8 (a power of two): a shift by one root block, 1/8, is a whole number of 2^-20 steps
    specs = [(icosphere(3, radius=0.15, centre=(0.5, 0.5, 0.5)), 8, 3), (icosphere(2, radius=0.25, centre=(0.5, 0.5, 0.5)), 4, 2),
             (icosphere(3, radius=0.2, centre=(0.48, 0.52, 0.5)), 12, 2)]
    meshes = [P.emb_mesh_create(torch.from_numpy(v), torch.from_numpy(t), R) for (v, t), R, _ in specs]
    B = P.emb_batch_create(meshes, [lv for _, _, lv in specs], [2] * 3, [19] * 3)
    return specs, meshes, B


def test_batch_replay_follows_a_whole_block_translation():
    import torch

    import paper_2512_01251_gb300 as P
    specs, meshes, B = _moving_batch(P)
    (v0, t0), R0, lv0 = specs[0]
    v1 = snap(v0 + np.array([0.125, 0.0, -0.125], dtype=np.float64))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        P.emb_batch_run(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
        P.emb_mesh_update(meshes[0], torch.from_numpy(v1), s)
        P.emb_batch_capture(B, s)
        P.emb_batch_launch(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
        got = _batch_result(P, B, 0)
    ref = _result(P, _embed(P, v1, t0, R0, lv0, 19))
    _same(got, ref, "translated mesh")
    for j in (1, 2):  # the other meshes did not move
        (v, t), R, lv = specs[j]
        _same(_batch_result(P, B, j), _result(P, _embed(P, v, t, R, lv, 19)), f"mesh {j}")


def test_batch_replay_reports_changed_counts_and_replans():
    import torch

    import paper_2512_01251_gb300 as P
    specs, meshes, B = _moving_batch(P)
    (v0, t0), R0, lv0 = specs[0]
    v1 = snap((v0 - 0.5) * 1.3 + 0.5)  # a larger body: more blocks, more links
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        P.emb_batch_run(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
        P.emb_mesh_update(meshes[0], torch.from_numpy(v1), s)
        P.emb_batch_run(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_ERR_STATE
        # the context is intact and a new plan is exact
        B2 = P.emb_batch_create(meshes, [lv for _, _, lv in specs], [2] * 3, [19] * 3, stream=s)
        P.emb_batch_run(B2, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
        got = _batch_result(P, B2, 0)
    _same(got, _result(P, _embed(P, v1, t0, R0, lv0, 19)), "re-planned mesh")


def test_headroom_replay_follows_changed_counts_without_replanning():
    """A batch planned with headroom replays a body that grows, shrinks and moves: its
    block, bin and link counts change, the replay (also as one captured graph, launched
    after each move) stays exact against the per-call path, and a body that outgrows the
    capacities is reported as EMB_ERR_CAPACITY on the device, in bounds."""
    import torch

    import paper_2512_01251_gb300 as P
    specs = [(icosphere(3, radius=0.15, centre=(0.5, 0.5, 0.5)), 8, 3),
             (icosphere(3, radius=0.2, centre=(0.48, 0.52, 0.5)), 12, 2)]
    meshes = [P.emb_mesh_create(torch.from_numpy(v), torch.from_numpy(t), R) for (v, t), R, _ in specs]
    B = P.emb_batch_create(meshes, [lv for _, _, lv in specs], [2] * 2, [19] * 2, headroom=60)
    planned = P.emb_batch_info(B, 0)
    (v0, t0), R0, lv0 = specs[0]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        P.emb_batch_capture(B, s)
        seen = set()
        for k, f in enumerate((1.0, 1.12, 0.9, 1.05)):
            v1 = snap((v0 - 0.5) * f + 0.5 + np.array([0.01 * k, 0.0, -0.01 * k]))
            P.emb_mesh_update(meshes[0], torch.from_numpy(v1), s)
            if k % 2:
                P.emb_batch_launch(B, s)  # the same graph for every count
            else:
                P.emb_batch_run(B, s)
            s.synchronize()
            assert P.emb_status_get(s) == P.EMB_OK, f
            ref = _result(P, _embed(P, v1, t0, R0, lv0, 19))
            _same(_batch_result(P, B, 0), ref, f"scale {f}")
            blocks, links = P.emb_batch_counts(B, 0, s)
            assert blocks == [len(b) for b in ref["blocks"]] and links == len(ref["links"]["q"])
            seen.add((tuple(blocks), links))
        assert len(seen) > 1  # the counts did change
        (v, t), R, lv = specs[1]  # the other mesh did not move
        _same(_batch_result(P, B, 1), _result(P, _embed(P, v, t, R, lv, 19)), "mesh 1")
        # far beyond the capacities: reported, not faulted, and the context stays usable
        v2 = snap((v0 - 0.5) * 2.2 + 0.5)
        P.emb_mesh_update(meshes[0], torch.from_numpy(v2), s)
        P.emb_batch_launch(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_ERR_CAPACITY
        P.emb_mesh_update(meshes[0], torch.from_numpy(snap(v0)), s)
        P.emb_batch_run(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
    assert P.emb_batch_info(B, 0) == planned
    _same(_batch_result(P, B, 0), _result(P, _embed(P, snap(v0), t0, R0, lv0, 19)), "back to the start")
