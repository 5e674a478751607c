"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and
compare it with the oracle element by element."""
from __future__ import annotations

import numpy as np

Q_TOL = 2e-6  # |q_gpu - q_oracle| bound (FP32 table against the FP64 oracle)


def gpu_embed(v, t, R, levels, band=2, lattice=19, **kw):
    import torch

    import paper_2512_01251_gb300 as P
    Em = P.embed(torch.from_numpy(np.ascontiguousarray(v)), torch.from_numpy(np.ascontiguousarray(t)), R, levels, band,
                 lattice, **kw)
    out = dict(
        blocks=[b.cpu().numpy().astype(np.int64) for b in Em.fetch_blocks()],
        masks=[m.cpu().numpy().view(np.uint64) for m in Em.masks],
        flags=[f.cpu().numpy() for f in Em.flags],
        links=dict(cell=Em.links["cell"].cpu().numpy().astype(np.int64),
                   dir=Em.links["dir"].cpu().numpy().astype(np.int64),
                   q=Em.links["q"].cpu().numpy(),
                   tri=Em.links["tri"].cpu().numpy().astype(np.int64)),
    )
    return Em, out


def compare_full(g, o, levels):
    for L in range(levels + 1):
        np.testing.assert_array_equal(g["blocks"][L], o["blocks"][L], err_msg=f"blocks L={L}")
        np.testing.assert_array_equal(g["masks"][L], o["masks"][L], err_msg=f"masks L={L}")
        if L < levels:
            np.testing.assert_array_equal(g["flags"][L], o["flags"][L], err_msg=f"flags L={L}")
    gl, ol = g["links"], o["links"]
    np.testing.assert_array_equal(gl["cell"], ol["cell"], err_msg="link cells")
    np.testing.assert_array_equal(gl["dir"], ol["dir"], err_msg="link dirs")
    np.testing.assert_array_equal(gl["tri"], ol["tri"], err_msg="link triangles")
    err = np.abs(gl["q"].astype(np.float64) - ol["q"])
    assert err.max(initial=0.0) <= Q_TOL, f"max |dq| = {err.max()}"
