"""Full-size workloads (the ~112K- and ~7.2M-triangle meshes) in the launch
configuration the bench times: the oracle checks sampled outputs one by one, and
properties that hold at any size are checked on every output."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import Q_TOL, gpu_embed
from synth import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _lookup(blocks):
    key = (blocks[:, 2] << 42) | (blocks[:, 1] << 21) | blocks[:, 0]
    return key


def _find(key_sorted, b):
    k = (b[:, 2] << 42) | (b[:, 1] << 21) | b[:, 0]
    i = np.searchsorted(key_sorted, k)
    i = np.minimum(i, len(key_sorted) - 1)
    ok = (key_sorted[i] == k) & np.all(b >= 0, axis=1)
    return np.where(ok, i, -1)


def _mask_bit(masks, ids, t):
    w = masks[np.maximum(ids, 0)]
    return np.where(ids >= 0, (w >> t.astype(np.uint64)) & np.uint64(1), 0).astype(np.uint8)


@pytest.mark.parametrize("name,lattice,n_blk,n_cellblk,n_link", [
    ("star_112k", 19, 96, 48, 600),
    ("star_112k", 27, 32, 16, 300),
    ("star_7m", 27, 24, 8, 160),
])
def test_fullsize_sampled(orc, name, lattice, n_blk, n_cellblk, n_link):
    w = workload(name)
    v, t = w.build_mesh()
    _, g = gpu_embed(v, t, w.R, w.levels, w.band, lattice)
    X = orc.int_coords(v, w.R)
    tri9 = orc.tri_coords(X, t)
    rng = np.random.default_rng(20251220)
    C = orc.directions()
    levels = w.levels

    # -- forest structure: children of flagged blocks, sorted; 2:1 neighbourhood present
    for L in range(levels):
        np.testing.assert_array_equal(g["blocks"][L + 1], orc.children(g["blocks"][L], g["flags"][L]))
    for L in range(1, levels):
        key = _lookup(g["blocks"][L])
        fl = g["blocks"][L][g["flags"][L] == 1]
        nmax = w.R << L
        for d in range(1, 27):
            nb = fl + C[d]
            inside = np.all((nb >= 0) & (nb < nmax), axis=1)
            assert np.all(_find(key, nb[inside]) >= 0), f"2:1 violated at level {L}"

    # -- sampled refine flags against the brute-force overlap test
    for L in range(levels):
        B = g["blocks"][L]
        f = g["flags"][L]
        on, off = np.nonzero(f)[0], np.nonzero(f == 0)[0]
        sel = np.concatenate([rng.choice(on, min(n_blk // 2, len(on)), replace=False),
                              rng.choice(off, min(n_blk // 2, len(off)), replace=False)])
        W = 4 * orc.h_units(w.R, L)
        D = orc.dilation(w.R, L, levels, w.band)
        exp = orc.boxes_any(tri9, B[sel] * W - D, (B[sel] + 1) * W + D)
        np.testing.assert_array_equal(f[sel], exp, err_msg=f"flags L={L}")

    # -- sampled solid masks (blocks mixing solid and fluid first, then uniform ones)
    for L in range(levels + 1):
        B = g["blocks"][L]
        m = g["masks"][L]
        mixed = np.nonzero((m != 0) & (m != np.uint64(0xFFFFFFFFFFFFFFFF)))[0]
        uni = np.nonzero((m == 0) | (m == np.uint64(0xFFFFFFFFFFFFFFFF)))[0]
        sel = np.concatenate([rng.choice(mixed, min(n_cellblk, len(mixed)), replace=False),
                              rng.choice(uni, min(n_cellblk // 4, len(uni)), replace=False)])
        exp = orc.masks(tri9, w.R, L, B[sel])
        np.testing.assert_array_equal(m[sel], exp, err_msg=f"masks L={L}")

    # -- whole table: sorted, fluid -> solid according to the masks, q in [0, 1]
    lk = g["links"]
    Bf, mf = g["blocks"][levels], g["masks"][levels]
    keyf = _lookup(Bf)
    assert np.all(np.diff(lk["cell"] * 32 + lk["dir"]) > 0)
    assert np.all((lk["q"] >= 0) & (lk["q"] <= 1))
    b, tt = lk["cell"] // 64, lk["cell"] % 64
    assert np.all(_mask_bit(mf, b, tt) == 0)
    loc = np.stack([tt % 4, (tt // 4) % 4, tt // 16], axis=1) + C[lk["dir"]]
    nb = Bf[b] + np.floor_divide(loc, 4)
    nid = _find(keyf, nb)
    assert np.all(_mask_bit(mf, nid, (loc % 4) @ np.array([1, 4, 16])) == 1)
    # completeness on sampled blocks: every fluid cell with a solid neighbour has its link
    sb = rng.choice(len(Bf), min(3000, len(Bf)), replace=False)
    cells = (sb[:, None] * 64 + np.arange(64)[None, :]).reshape(-1)
    cb, ct = cells // 64, cells % 64
    have = set((lk["cell"] * 32 + lk["dir"]).tolist())
    fluid = _mask_bit(mf, cb, ct) == 0
    for d in range(1, lattice):
        l2 = np.stack([ct % 4, (ct // 4) % 4, ct // 16], axis=1) + C[d]
        nid = _find(keyf, Bf[cb] + np.floor_divide(l2, 4))
        solid_nb = _mask_bit(mf, nid, (l2 % 4) @ np.array([1, 4, 16])) == 1
        want = cells[fluid & solid_nb] * 32 + d
        assert all(x in have for x in want.tolist()), f"missing links in direction {d}"

    # -- sampled links: the nearest crossed triangle and q against the brute force
    sel = rng.choice(len(lk["q"]), min(n_link, len(lk["q"])), replace=False)
    half = orc.h_units(w.R, levels) // 2
    ts = lk["cell"][sel] % 64
    gcell = 4 * Bf[lk["cell"][sel] // 64] + np.stack([ts % 4, (ts // 4) % 4, ts // 16], axis=1)
    P = (2 * gcell + 1) * half
    q, arg, nc = orc.links(tri9, P, lk["dir"][sel], orc.h_units(w.R, levels))
    np.testing.assert_array_equal(lk["tri"][sel], arg)
    assert np.max(np.abs(lk["q"][sel].astype(np.float64) - q)) <= Q_TOL
    # and the sampled link endpoints agree with the point predicate
    s0 = orc.solid(tri9, P)
    s1 = orc.solid(tri9, P + orc.h_units(w.R, levels) * C[lk["dir"][sel]])
    assert np.all(s0 == 0) and np.all(s1 == 1)
