"""One lattice-Boltzmann step on the finest level (emb_lbm_step) against the oracle's
step, element by element on the same seeded populations: pull streaming, Bouzidi
bounce-back from the cut-link table, BGK collision; and, on the GPU alone, mass
conservation over many steps in a cavity closed by halfway walls."""
from __future__ import annotations

import numpy as np
import pytest

from synth import populations, workload
from synth.meshes import axis_box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _fluid_pops(P, E, lattice, seed):
    import torch
    nblk = P.emb_forest_num_blocks(E.forest, E.levels)
    pop = populations(nblk * 64, seed=seed, u=(0.04, -0.02, 0.01), noise=0.05, lattice=lattice)
    fluid = ((E.masks[-1].cpu().numpy().view(np.uint64)[:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)) == 0
    pop = np.where(fluid.reshape(1, -1), pop, np.float32(0))
    return torch.from_numpy(pop).cuda(), pop


@pytest.mark.parametrize("name,lattice,omega", [("icosphere_320", 19, 1.3), ("star_1k", 27, 0.8), ("star_4k_r3", 27, 1.7)])
def test_lbm_step_matches_oracle(orc, name, lattice, omega):
    import torch

    import paper_2512_01251_gb300 as P
    w = workload(name)
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), w.R, w.levels, w.band, lattice)
    o = orc.embed(v, t, w.R, w.levels, w.band, lattice)
    pop_d, pop = _fluid_pops(P, E, lattice, seed=11)
    out = P.emb_lbm_step(E.forest, lattice, E.links, omega, pop_d)
    got = out.cpu().numpy().astype(np.float64)
    ref = orc.lbm_step(w.R, w.levels, o["blocks"][-1], o["masks"][-1], o["links"], pop.astype(np.float64), omega, lattice)
    assert P.emb_status_get() == P.EMB_OK
    err = np.abs(got - ref)
    assert np.all(err <= 1e-6 + 2e-5 * np.abs(ref)), (err.max(), np.unravel_index(err.argmax(), err.shape))
    # the boundary pass did something: the populations entering link cells differ from plain streaming
    pre_only = P.emb_lbm_step(E.forest, lattice, E.links, omega, pop_d, phases=1 | 4).cpu().numpy()
    assert np.any(pre_only != got)


def test_cavity_mass_over_many_steps():
    import torch

    import paper_2512_01251_gb300 as P
    g = 1 << 20
    ov, ot = axis_box([8 * g // 32] * 3, [24 * g // 32] * 3)
    iv, it = axis_box([12 * g // 32] * 3, [20 * g // 32] * 3)
    v = np.concatenate([ov, iv]).astype(np.float32)
    t = np.concatenate([ot, it[:, ::-1] + len(ov)]).astype(np.int32)
    E = P.embed(torch.from_numpy(v), torch.from_numpy(t), 8, 0, 2, 19)
    assert np.all(E.links["q"].cpu().numpy() == 0.5)
    blocks = E.fetch_blocks()[0].cpu().numpy()
    loc = np.stack([np.arange(64) % 4, (np.arange(64) // 4) % 4, np.arange(64) // 16], 1)
    gg = 4 * blocks[:, None, :] + loc[None]
    cav = torch.from_numpy(np.all((gg >= 12) & (gg < 20), axis=2).reshape(-1)).cuda()
    pop_d, _ = _fluid_pops(P, E, 19, seed=3)
    m0 = pop_d[:, cav].double().sum().item()
    a, b, pre = pop_d, torch.empty_like(pop_d), torch.empty_like(pop_d)
    for _ in range(50):
        P.emb_lbm_step(E.forest, 19, E.links, 1.2, a, out=b, pre=pre)
        a, b = b, a
    m = a[:, cav].double().sum().item()
    assert abs(m - m0) <= 2e-6 * m0  # float32 rounding over 50 steps; halfway walls conserve mass exactly
