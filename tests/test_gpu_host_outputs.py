"""Outputs in host memory: emb_cutlinks and emb_voxelize accept page-locked host buffers,
which the library fills over the host link (the link kernel stores straight into them),
and refuse pageable host memory before anything is enqueued."""
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


@pytest.mark.parametrize("name,lattice", [("star_4k_r3", 27), ("icosphere_320", 19)])
def test_pinned_host_outputs_equal_device_outputs(name, lattice):
    import torch

    import paper_2512_01251_gb300 as P
    w = workload(name)
    v, t = w.build_mesh()
    dv, dt = torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()
    ref = P.embed(dv, dt, w.R, w.levels, w.band, lattice)
    n, nm = ref.links["q"].numel(), ref.masks[-1].numel()
    out = dict(cell=torch.full((n + 5,), -7, dtype=torch.int32).pin_memory(),
               dir=torch.full((n + 5,), 99, dtype=torch.uint8).pin_memory(),
               q=torch.full((n + 5,), -1.0, dtype=torch.float32).pin_memory(),
               tri=torch.full((n + 5,), -7, dtype=torch.int32).pin_memory(),
               count=torch.zeros(1, dtype=torch.int64).pin_memory())
    mask = torch.zeros(nm + 3, dtype=torch.int64).pin_memory()
    E = P.embed(dv, dt, w.R, w.levels, w.band, lattice, links_out=out, finest_mask_out=mask)
    torch.cuda.synchronize()
    assert int(out["count"][0]) == n
    for k in ("cell", "dir", "tri"):
        np.testing.assert_array_equal(out[k][:n].numpy(), ref.links[k].cpu().numpy(), err_msg=k)
    np.testing.assert_array_equal(out["q"][:n].numpy().view(np.uint32), ref.links["q"].cpu().numpy().view(np.uint32))
    np.testing.assert_array_equal(mask[:nm].numpy(), ref.masks[-1].cpu().numpy())
    # nothing written past the table
    assert (out["cell"][n:].numpy() == -7).all() and (out["dir"][n:].numpy() == 99).all()
    assert E.links["q"].numel() == n and E.masks[-1].numel() == nm


def test_pageable_host_outputs_are_refused():
    import torch

    import paper_2512_01251_gb300 as P
    w = workload("icosphere_320")
    v, t = w.build_mesh()
    dv, dt = torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()
    ref = P.embed(dv, dt, w.R, w.levels, w.band, 19)
    n = ref.links["q"].numel()
    pageable = dict(cell=torch.empty(n, dtype=torch.int32), dir=torch.empty(n, dtype=torch.uint8),
                    q=torch.empty(n, dtype=torch.float32), tri=torch.empty(n, dtype=torch.int32),
                    count=torch.zeros(1, dtype=torch.int64))
    with pytest.raises(P.EmbError) as ei:
        P.embed(dv, dt, w.R, w.levels, w.band, 19, links_out=pageable)
    assert ei.value.code == P.EMB_ERR_BAD_INPUT
    with pytest.raises(P.EmbError) as ei:
        P.embed(dv, dt, w.R, w.levels, w.band, 19, finest_mask_out=torch.empty(10 ** 6, dtype=torch.int64))
    assert ei.value.code == P.EMB_ERR_BAD_INPUT
    assert P.emb_status_get() == P.EMB_OK  # refused before anything was enqueued
