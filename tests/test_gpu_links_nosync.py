"""The cut-link table without a count read-back: emb_cutlinks_prepare enqueues the
candidate cells without waiting for the GPU, emb_cutlinks with a caller capacity keeps
the count on the device; the tables equal the counted path bit for bit, and a short
capacity writes the table's prefix, reports the full count and sets EMB_ERR_CAPACITY."""
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


def _to_finest(P, torch, w, lattice):
    """The stages up to the finest level's bins and mask, with no link work done."""
    v, t = w.build_mesh()
    m = P.emb_mesh_create(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), w.R)
    f = P.emb_forest_root(w.R, w.levels)
    for L in range(w.levels + 1):
        b = P.emb_bin(m, f, L, lattice)
        P.emb_voxelize(f, b, L)
        if L == w.levels:
            return m, f, b
        fl = P.emb_refine_flags(f, b, L, w.band)
        P.emb_forest_refine(f, L, fl)
        b.close()


def _host(links, n):
    return {k: links[k][:n].cpu().numpy() for k in ("cell", "dir", "q", "tri")}


def _assert_same(a, b):
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    np.testing.assert_array_equal(a["q"].view(np.uint32), b["q"].view(np.uint32))


@pytest.mark.parametrize("name,lattice", [("star_4k_r3", 27), ("icosphere_320", 19)])
def test_prepare_and_device_count_equal_counted_path(name, lattice):
    import torch

    import paper_2512_01251_gb300 as P
    w = workload(name)
    v, t = w.build_mesh()
    ref = P.embed(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), w.R, w.levels, w.band, lattice)
    n = ref.links["q"].numel()
    want = _host(ref.links, n)

    # emb_cutlinks with a capacity on a forest whose candidates are not built yet
    m, f, b = _to_finest(P, torch, w, lattice)
    got = P.emb_cutlinks(f, b, lattice, capacity=n + 100)
    assert got["q"].numel() == n and int(got["count"].item()) == n
    _assert_same(_host(got, n), want)
    assert P.emb_cutlinks_count(f, lattice) == n  # reads the count the call left on the device

    # emb_cutlinks_prepare, then an unsynchronised call that returns the whole buffers
    m, f, b = _to_finest(P, torch, w, lattice)
    P.emb_cutlinks_prepare(f, lattice)
    P.emb_cutlinks_prepare(f, lattice)  # a second call reuses the candidates
    raw = P.emb_cutlinks(f, b, lattice, capacity=n, sync=False)
    assert raw["q"].numel() == max(n, 1)
    torch.cuda.synchronize()
    assert int(raw["count"].item()) == n
    _assert_same(_host(raw, n), want)
    assert P.emb_status_get() == P.EMB_OK


def test_short_capacity_writes_the_prefix_and_reports_the_count():
    import torch

    import paper_2512_01251_gb300 as P
    w = workload("icosphere_320")
    lattice = 19
    v, t = w.build_mesh()
    ref = P.embed(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), w.R, w.levels, w.band, lattice)
    n = ref.links["q"].numel()
    assert n > 40
    want = _host(ref.links, n)

    cap = n - 37
    m, f, b = _to_finest(P, torch, w, lattice)
    out = dict(cell=torch.full((cap,), -7, dtype=torch.int32, device="cuda"),
               dir=torch.full((cap,), 99, dtype=torch.uint8, device="cuda"),
               q=torch.full((cap,), -1.0, dtype=torch.float32, device="cuda"),
               tri=torch.full((cap,), -7, dtype=torch.int32, device="cuda"),
               count=torch.zeros(1, dtype=torch.int64, device="cuda"))
    with pytest.raises(P.EmbError) as ei:
        P.emb_cutlinks(f, b, lattice, capacity=cap, out=out)
    assert ei.value.code == P.EMB_ERR_CAPACITY
    assert int(out["count"].item()) == n
    assert P.emb_status_get() == P.EMB_ERR_CAPACITY
    assert P.emb_status_get() == P.EMB_OK
    _assert_same(_host(out, cap), {k: a[:cap] for k, a in want.items()})
    # the count is now known on the host: a second short call is refused before the launch
    with pytest.raises(P.EmbError) as ei:
        P.emb_cutlinks(f, b, lattice, capacity=cap, out=out)
    assert ei.value.code == P.EMB_ERR_CAPACITY
    P.emb_status_get()

    # room for none on a forest whose count is still on the device
    m, f, b = _to_finest(P, torch, w, lattice)
    with pytest.raises(P.EmbError) as ei:
        P.emb_cutlinks(f, b, lattice, capacity=0)
    assert ei.value.code == P.EMB_ERR_CAPACITY
    assert P.emb_status_get() == P.EMB_ERR_CAPACITY


def test_embed_into_short_host_buffers_is_refused_with_the_prefix_written():
    import torch

    import paper_2512_01251_gb300 as P
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    dv, dt = torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()
    ref = P.embed(dv, dt, w.R, w.levels, w.band, 19)
    n = ref.links["q"].numel()
    cap = n // 2
    out = dict(cell=torch.empty(cap, dtype=torch.int32).pin_memory(), dir=torch.empty(cap, dtype=torch.uint8).pin_memory(),
               q=torch.empty(cap, dtype=torch.float32).pin_memory(), tri=torch.empty(cap, dtype=torch.int32).pin_memory(),
               count=torch.zeros(1, dtype=torch.int64).pin_memory())
    with pytest.raises(P.EmbError) as ei:
        P.embed(dv, dt, w.R, w.levels, w.band, 19, links_out=out)
    assert ei.value.code == P.EMB_ERR_CAPACITY
    assert int(out["count"][0]) == n
    _assert_same({k: out[k].numpy() for k in ("cell", "dir", "q", "tri")},
                 {k: a[:cap] for k, a in _host(ref.links, n).items()})
    assert P.emb_status_get() == P.EMB_OK  # embed read the status of the short table
