"""The batched path (planned replay, CUDA graph, autotuned launch shape) against the
per-call path, mesh by mesh, and one batch mesh against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

from synth import batch_meshes, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    cases = []
    for name, lat in [("icosphere_320", 19), ("star_1k", 27), ("star_4k_r3", 27)]:
        w = workload(name)
        v, t = w.build_mesh()
        cases.append(dict(verts=v, tris=t, R=w.R, levels=w.levels, band=w.band, lattice=lat))
    cases += batch_meshes(5, t_max=2e4)
    return cases


def _plain(P, c, mesh):
    import torch
    E = P.embed(torch.from_numpy(c["verts"]), torch.from_numpy(c["tris"]), c["R"], c["levels"], c["band"], c["lattice"],
                mesh=mesh)
    return dict(blocks=[b.cpu().numpy() for b in E.fetch_blocks()],
                masks=[m.cpu().numpy() for m in E.masks],
                links={k: E.links[k].cpu().numpy() for k in ("cell", "dir", "q", "tri")})


def _batch_result(P, B, j):
    r = P.emb_batch_results(B, j)
    return dict(blocks=[b.cpu().numpy() for b in r["blocks"]], masks=[m.cpu().numpy() for m in r["masks"]],
                links={k: r["links"][k].cpu().numpy() for k in ("cell", "dir", "q", "tri")})


def _same(a, b, j):
    assert len(a["blocks"]) == len(b["blocks"])
    for L in range(len(a["blocks"])):
        np.testing.assert_array_equal(a["blocks"][L], b["blocks"][L], err_msg=f"mesh {j} blocks L={L}")
        np.testing.assert_array_equal(a["masks"][L], b["masks"][L], err_msg=f"mesh {j} masks L={L}")
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(a["links"][k], b["links"][k], err_msg=f"mesh {j} links {k}")
    np.testing.assert_array_equal(a["links"]["q"].view(np.uint32), b["links"]["q"].view(np.uint32))


def test_batch_replay_graph_and_autotune_match_per_call_path():
    import torch

    import paper_2512_01251_gb300 as P
    cases = _cases()
    meshes = [P.emb_mesh_create(torch.from_numpy(c["verts"]), torch.from_numpy(c["tris"]), c["R"]) for c in cases]
    plain = [_plain(P, c, m) for c, m in zip(cases, meshes)]
    B = P.emb_batch_create(meshes, [c["levels"] for c in cases], [c["band"] for c in cases],
                           [c["lattice"] for c in cases])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        P.emb_batch_run(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
        for j in range(len(cases)):
            _same(plain[j], _batch_result(P, B, j), j)
        # the captured graph, launched twice
        P.emb_batch_capture(B, s)
        for _ in range(2):
            P.emb_batch_launch(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
        for j in range(len(cases)):
            _same(plain[j], _batch_result(P, B, j), j)
        choice = P.emb_batch_autotune(B, s)
        assert choice[0] >= 1 and choice[1] in (128, 256, 512) and choice[3] in (0, 1, 2)
        P.emb_batch_run(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
        for j in range(len(cases)):
            _same(plain[j], _batch_result(P, B, j), j)
        # both link placements, each replayed and captured
        for shape in ((3, 128, 0, 0), (5, 512, 1, 1), (16, 256, 0, 1), (7, 256, 2, 2), (16, 128, 0, 2)):
            P.emb_batch_configure(B, *shape)
            P.emb_batch_run(B, s)
            s.synchronize()
            assert P.emb_status_get(s) == P.EMB_OK
            for j in range(len(cases)):
                _same(plain[j], _batch_result(P, B, j), j)
            P.emb_batch_capture(B, s)
            P.emb_batch_launch(B, s)
            s.synchronize()
            assert P.emb_status_get(s) == P.EMB_OK
            for j in range(len(cases)):
                _same(plain[j], _batch_result(P, B, j), j)
        with pytest.raises(P.EmbError):
            P.emb_batch_configure(B, 0, 256, 0, 1)
        with pytest.raises(P.EmbError):
            P.emb_batch_configure(B, 4, 96, 0, 1)
        with pytest.raises(P.EmbError):
            P.emb_batch_configure(B, 4, 256, 0, 3)


def test_batch_mesh_matches_oracle(orc):
    import torch

    import paper_2512_01251_gb300 as P
    c = batch_meshes(3, t_max=3e3)[2]
    o = orc.embed(c["verts"], c["tris"], c["R"], c["levels"], c["band"], c["lattice"])
    m = P.emb_mesh_create(torch.from_numpy(c["verts"]), torch.from_numpy(c["tris"]), c["R"])
    B = P.emb_batch_create([m], [c["levels"]], [c["band"]], [c["lattice"]])
    P.emb_batch_run(B)
    torch.cuda.synchronize()
    assert P.emb_status_get() == P.EMB_OK
    r = _batch_result(P, B, 0)
    # the refine flags are not kept by the batch; they are implied by the next level's blocks
    for L in range(c["levels"] + 1):
        np.testing.assert_array_equal(r["blocks"][L].astype(np.int64), o["blocks"][L], err_msg=f"blocks L={L}")
        np.testing.assert_array_equal(r["masks"][L].view(np.uint64), o["masks"][L], err_msg=f"masks L={L}")
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(r["links"][k].astype(np.int64), o["links"][k], err_msg=f"links {k}")
    assert np.abs(r["links"]["q"].astype(np.float64) - o["links"]["q"]).max(initial=0) <= 2e-6


def test_autotune_cache_reuses_and_persists_the_shape(tmp_path, monkeypatch):
    """A timed shape is cached under (SM count, triangle and mesh-count buckets, lattice):
    the next call with the same kind of batch takes it without timing, and the cache file
    named by EMB_TUNE_CACHE holds it as a line of 8 integers."""
    import torch

    import paper_2512_01251_gb300 as P
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("EMB_TUNE_CACHE", str(path))
    cases = batch_meshes(3, t_max=5e3)
    meshes = [P.emb_mesh_create(torch.from_numpy(c["verts"]), torch.from_numpy(c["tris"]), c["R"]) for c in cases]
    B = P.emb_batch_create(meshes, [c["levels"] for c in cases], [c["band"] for c in cases],
                           [c["lattice"] for c in cases])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        timed, cached = P.emb_batch_autotune_ex(B, s, force=True)
        assert not cached
        again, cached = P.emb_batch_autotune_ex(B, s)
        assert cached and again == timed
        assert P.emb_batch_autotune(B, s) == timed
        P.emb_batch_run(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
    rows = [tuple(int(x) for x in ln.split()) for ln in path.read_text().splitlines() if ln.strip()]
    assert any(len(r) == 8 and r[4:] == tuple(timed) for r in rows)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert all(r[0] == sm for r in rows)
