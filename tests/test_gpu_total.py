"""Every output of the full-size workloads against the sorted-line oracle tier.

The sorted-line tier (oracle/emb_oracle_lines.c) evaluates the same exact
definitions as the brute force, triangle-major along sorted lattice lines, and is
checked against the brute force on every case both can run
(tests/test_oracle_lines.py).  Here it covers the full workloads in the launch
configurations the bench times: every block, mask word, refine flag and cut link
(cell, direction and triangle identical, |q - q_oracle| <= 2e-6) of
  - the ~112K-triangle mesh (root 16^3, levels 0..3) with D3Q19 and D3Q27,
  - the ~7.2M-triangle mesh (root 32^3, levels 0..4, D3Q27), per-call path,
  - all 48 meshes of the batch, through the autotuned, captured batch graph,
and, on the differentiation workload, the force gradient and the gradient of
L = sum_k w_k q_k against the oracle's FP64 analytic gradients evaluated on the
oracle's own link table (its q, triangles and interpolation partners).
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import Q_TOL, compare_full, gpu_embed
from synth import batch_meshes, link_weights, populations, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name,lattice", [("star_112k", 19), ("star_112k", 27), ("star_7m", 27)])
def test_full_size_every_output(orc, name, lattice):
    w = workload(name)
    v, t = w.build_mesh()
    _, g = gpu_embed(v, t, w.R, w.levels, w.band, lattice)
    o = orc.embed_lines(v, t, w.R, w.levels, w.band, lattice)
    assert np.all(o["links"]["tri"] >= 0), "every oracle cut link crosses a face"
    compare_full(g, o, w.levels)


def test_batch_of_48_every_output(orc):
    import torch

    import paper_2512_01251_gb300 as P
    cases = batch_meshes(48)
    meshes = [P.emb_mesh_create(torch.from_numpy(c["verts"]), torch.from_numpy(c["tris"]), c["R"]) for c in cases]
    B = P.emb_batch_create(meshes, [c["levels"] for c in cases], [c["band"] for c in cases],
                           [c["lattice"] for c in cases])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        P.emb_batch_autotune(B, s)
        P.emb_batch_capture(B, s)
        P.emb_batch_launch(B, s)
        s.synchronize()
        assert P.emb_status_get(s) == P.EMB_OK
    for j, c in enumerate(cases):
        r = P.emb_batch_results(B, j)
        o = orc.embed_lines(c["verts"], c["tris"], c["R"], c["levels"], c["band"], c["lattice"])
        assert len(r["blocks"]) == c["levels"] + 1
        # the batch keeps no refine flags; they are implied by the next level's blocks
        for L in range(c["levels"] + 1):
            np.testing.assert_array_equal(r["blocks"][L].cpu().numpy().astype(np.int64), o["blocks"][L],
                                          err_msg=f"mesh {j} blocks L={L}")
            np.testing.assert_array_equal(r["masks"][L].cpu().numpy().view(np.uint64), o["masks"][L],
                                          err_msg=f"mesh {j} masks L={L}")
        for k in ("cell", "dir", "tri"):
            np.testing.assert_array_equal(r["links"][k].cpu().numpy().astype(np.int64), o["links"][k],
                                          err_msg=f"mesh {j} links {k}")
        dq = np.abs(r["links"]["q"].cpu().numpy().astype(np.float64) - o["links"]["q"])
        assert dq.max(initial=0.0) <= Q_TOL, (j, dq.max())


def test_diff_112k_gradients_against_the_oracle_table(orc):
    import torch

    from paper_2512_01251_gb300 import emb_cutlinks_backward
    from paper_2512_01251_gb300.autograd import embed_q, mex_force
    w = workload("diff_112k")
    v, t = w.build_mesh()
    o = orc.embed_lines(v, t, w.R, w.levels, w.band, 19)
    ol = o["links"]
    verts = torch.from_numpy(v).cuda().requires_grad_(True)
    E, q = embed_q(verts, torch.from_numpy(t), w.R, w.levels, w.band, 19)
    # the link set first: same cells, directions and triangles, q within 2e-6
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(E.links[k].cpu().numpy().astype(np.int64), ol[k], err_msg=k)
    assert np.abs(E.links["q"].cpu().numpy().astype(np.float64) - ol["q"]).max() <= Q_TOL
    blocks_f, mask_f = o["blocks"][-1], o["masks"][-1]
    pop_np = populations(len(blocks_f) * 64, seed=w.extra["pop_seed"])
    partner = orc.partner_cells(w.R, w.levels, blocks_f, mask_f, ol["cell"], ol["dir"])
    X = orc.int_coords(v, w.R)

    # dF_x / dverts through the autograd chain, against the FP64 oracle on its own table
    F = mex_force(q, E, torch.from_numpy(pop_np).cuda())
    F[0].backward()
    g = verts.grad.cpu().numpy().astype(np.float64)
    ref = orc.grad_verts_from_gq(ol, orc.mex_force_dq(ol, pop_np, partner)[:, 0], X, t, w.R, w.levels, blocks_f, len(v))
    assert np.linalg.norm(g - ref) <= 1e-4 * np.linalg.norm(ref)
    assert np.abs(g - ref).max() <= 1e-4 * np.abs(ref).max()

    # dL / dverts for L = sum_k w_k q_k
    wk = link_weights(len(ol["q"]), seed=w.extra["w_seed"])
    L = E.links
    gl = emb_cutlinks_backward(E.mesh, E.forest, L["cell"], L["dir"], L["q"], L["tri"],
                               torch.from_numpy(wk).cuda()).cpu().numpy().astype(np.float64)
    refl = orc.grad_verts_from_gq(ol, wk.astype(np.float64), X, t, w.R, w.levels, blocks_f, len(v))
    assert np.linalg.norm(gl - refl) <= 1e-4 * np.linalg.norm(refl)
    assert np.abs(gl - refl).max() <= 1e-4 * np.abs(refl).max()
