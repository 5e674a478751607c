"""The neighbour table of every level (Sec. 3.2: neighbour links over the full halo)
against its plain definition: entry [b, d-1] is the id of the block at offset c_d from
block b at the same level, or -1.  The ids come from the forest's own block list, so
the check needs no other part of the path: bitmap levels, a hashed level and the
edges of the domain are covered."""
from __future__ import annotations

import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _expected(blocks: np.ndarray, nb: int, dirs) -> np.ndarray:
    """Neighbour ids by a dictionary of block positions."""
    pos = {tuple(p): i for i, p in enumerate(blocks.tolist())}
    out = np.full((len(blocks), 26), -1, dtype=np.int32)
    for i, (x, y, z) in enumerate(blocks.tolist()):
        for d in range(1, 27):
            cx, cy, cz = dirs[d]
            q = (x + cx, y + cy, z + cz)
            if all(0 <= c < nb for c in q):
                out[i, d - 1] = pos.get(q, -1)
    return out


def _check_forest(P, E, R, levels):
    dirs = P.emb_directions()
    for L in range(levels + 1):
        blocks = P.emb_forest_blocks(E.forest, L).cpu().numpy()
        got = P.emb_forest_neighbors(E.forest, L).cpu().numpy()
        want = _expected(blocks, R << L, dirs)
        np.testing.assert_array_equal(got, want, err_msg=f"level {L}")


@pytest.mark.parametrize("name", ["icosphere_320", "star_4k_r3"])
def test_neighbor_table_matches_block_positions(name):
    import torch

    import paper_2512_01251_gb300 as P
    w = workload(name)
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), w.R, w.levels, w.band, 19)
    _check_forest(P, E, w.R, w.levels)


def test_neighbor_table_on_a_hashed_level():
    # R = 32 with 6 levels: the finest level has more block positions than the rank
    # bitmap covers, so its neighbours are found through the level hash
    import torch

    import paper_2512_01251_gb300 as P
    from synth.meshes import icosphere
    v, t = icosphere(1, radius=0.004, centre=(0.5013, 0.4987, 0.5021))
    E = P.embed(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), 32, 6, 2, 19)
    dirs = P.emb_directions()
    L = 6
    blocks = P.emb_forest_blocks(E.forest, L).cpu().numpy()
    got = P.emb_forest_neighbors(E.forest, L).cpu().numpy()
    np.testing.assert_array_equal(got, _expected(blocks, 32 << L, dirs))
    assert (got >= 0).sum() > 0


def test_neighbor_table_at_the_domain_edge():
    # the root level of a small forest: every block on the boundary of the domain has
    # neighbour positions outside it, which must read -1
    import torch

    import paper_2512_01251_gb300 as P
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), w.R, w.levels, w.band, 19)
    blocks = P.emb_forest_blocks(E.forest, 0).cpu().numpy()
    got = P.emb_forest_neighbors(E.forest, 0).cpu().numpy()
    assert len(blocks) == w.R ** 3
    np.testing.assert_array_equal(got, _expected(blocks, w.R, P.emb_directions()))
    assert (got < 0).sum() > 0
