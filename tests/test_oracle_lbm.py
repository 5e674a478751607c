"""Pins of the oracle's lattice-Boltzmann step (streaming, Bouzidi bounce-back from the
cut-link table, BGK collision) against closed forms:

- the rest state w_i is a fixed point of the whole step, walls included;
- without collision a single population moves one cell along its direction;
- a population running into a wall half a cell away comes back reversed into its own
  cell (q = 1/2: the linear rule reduces to simple bounce-back);
- a cavity closed by such walls keeps its mass exactly under streaming and collision.
"""
from __future__ import annotations

import numpy as np

from synth.meshes import axis_box, icosphere

GRID = 1 << 20


def _setup(orc, v, t, R, levels, lattice):
    o = orc.embed(v, t, R, levels, 2, lattice)
    return o["blocks"][levels], o["masks"][levels], o["links"]


def _cell_of(orc, blocks, g):
    """Cell id of the level cell with integer coordinates g (x, y, z)."""
    b = np.array(g) // 4
    idx = orc._block_index(blocks)[tuple(b.tolist())]
    loc = np.array(g) - 4 * b
    return idx * 64 + int(loc[0] + 4 * loc[1] + 16 * loc[2])


def _hollow_box():
    # solid shell between [8/32, 24/32]^3 (outward) and [12/32, 20/32]^3 (inward): the
    # cavity inside is fluid and every face lies on a cell boundary for R = 8, level 0
    outer_v, outer_t = axis_box([8 * GRID // 32] * 3, [24 * GRID // 32] * 3)
    inner_v, inner_t = axis_box([12 * GRID // 32] * 3, [20 * GRID // 32] * 3)
    v = np.concatenate([outer_v, inner_v]).astype(np.float32)
    t = np.concatenate([outer_t, inner_t[:, ::-1] + len(outer_v)]).astype(np.int32)
    return v, t


def test_rest_state_is_a_fixed_point(orc):
    v, t = icosphere(2, radius=0.3, centre=(0.5, 0.5, 0.5))
    blocks, mask, links = _setup(orc, v, t, 2, 1, 19)
    fluid = orc.unpack_masks(mask).reshape(-1) == 0
    w = orc.lattice_weights(19)
    pop = np.where(fluid[None, :], w[:, None], 0.0)
    out = orc.lbm_step(2, 1, blocks, mask, links, pop, 1.3, 19)
    assert len(links["q"]) > 0
    np.testing.assert_allclose(out, pop, rtol=0, atol=1e-15)


def test_weights_sum_to_one_with_zero_mean_and_unit_third_variance(orc):
    for lat in (19, 27):
        w = orc.lattice_weights(lat)
        C = orc.directions()[:lat].astype(np.float64)
        assert abs(w.sum() - 1) < 1e-15
        np.testing.assert_allclose(w @ C, 0, atol=1e-16)
        np.testing.assert_allclose((w[:, None, None] * C[:, :, None] * C[:, None, :]).sum(0), np.eye(3) / 3, atol=1e-15)


def test_a_pulse_streams_one_cell(orc):
    v, t = _hollow_box()
    blocks, mask, links = _setup(orc, v, t, 8, 0, 27)
    n = len(blocks) * 64
    C = orc.directions()
    for i in (1, 8, 20):  # an axis, an edge and a corner direction
        pop = np.zeros((27, n))
        x0 = np.array([15, 16, 15])  # inside the cavity, two cells from every wall
        pop[i, _cell_of(orc, blocks, x0)] = 1.0
        out = orc.lbm_step(8, 0, blocks, mask, links, pop, 0.0, 27)
        expect = np.zeros_like(pop)
        expect[i, _cell_of(orc, blocks, x0 + C[i])] = 1.0
        np.testing.assert_array_equal(out, expect)


def test_a_pulse_bounces_off_a_halfway_wall(orc):
    v, t = _hollow_box()
    blocks, mask, links = _setup(orc, v, t, 8, 0, 27)
    assert np.all(links["q"] == 0.5)  # every face lies on a cell boundary
    n = len(blocks) * 64
    pop = np.zeros((27, n))
    x0 = _cell_of(orc, blocks, [19, 16, 16])  # the last cavity cell before the +x wall
    pop[1, x0] = 1.0  # moving +x, into the wall
    out = orc.lbm_step(8, 0, blocks, mask, links, pop, 0.0, 27)
    expect = np.zeros_like(pop)
    expect[2, x0] = 1.0  # back along -x, in the same cell
    np.testing.assert_array_equal(out, expect)


def test_cavity_mass_is_conserved(orc):
    v, t = _hollow_box()
    blocks, mask, links = _setup(orc, v, t, 8, 0, 19)
    n = len(blocks) * 64
    rng = np.random.default_rng(5)
    fluid = orc.unpack_masks(mask).reshape(-1) == 0
    g = (4 * blocks[:, None, :] + np.stack([np.arange(64) % 4, (np.arange(64) // 4) % 4, np.arange(64) // 16], 1)[None])
    cav = np.all((g >= 12) & (g < 20), axis=2).reshape(-1)
    assert cav.sum() == 512 and np.all(fluid[cav])
    pop = np.where(fluid[None, :], orc.lattice_weights(19)[:, None] * rng.uniform(0.9, 1.1, (19, n)), 0.0)
    m0 = pop[:, cav].sum()
    for _ in range(3):
        pop = orc.lbm_step(8, 0, blocks, mask, links, pop, 1.4, 19)
    assert abs(pop[:, cav].sum() - m0) <= 1e-12 * m0


def test_full_relaxation_gives_the_equilibrium_moments(orc):
    # a uniform state off equilibrium: after one step with omega = 1 the cells away from
    # the walls hold f_eq(rho, u), whose moments are rho, rho u and rho (u u + I/3)
    v, t = _hollow_box()
    blocks, mask, links = _setup(orc, v, t, 8, 0, 27)
    n = len(blocks) * 64
    fluid = orc.unpack_masks(mask).reshape(-1) == 0
    rng = np.random.default_rng(9)
    f0 = orc.lattice_weights(27) * rng.uniform(0.7, 1.3, 27)
    pop = np.where(fluid[None, :], f0[:, None], 0.0)
    out = orc.lbm_step(8, 0, blocks, mask, links, pop, 1.0, 27)
    C = orc.directions()[:27].astype(np.float64)
    rho = f0.sum()
    u = (C.T @ f0) / rho
    x = _cell_of(orc, blocks, [15, 16, 16])  # two cells from every wall: pulled values are uniform
    f = out[:, x]
    assert abs(f.sum() - rho) < 1e-14
    np.testing.assert_allclose(C.T @ f, rho * u, atol=1e-14)
    np.testing.assert_allclose((f[:, None, None] * C[:, :, None] * C[:, None, :]).sum(0),
                               rho * (np.outer(u, u) + np.eye(3) / 3), atol=1e-14)
