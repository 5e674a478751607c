"""Named synthetic workloads (mesh recipe + forest spec), batch meshes, populations.

The paper's Stanford models are not available; seeded radial meshes with the
same triangle counts stand in for them (Table 1 gives 112,394 and 7,218,906
triangles).  Seeds are NumPy PCG64: the workload with index k uses seed
20251201 + k, batch mesh j uses 20251300 + j.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .meshes import icosphere, radial_star


@dataclass(frozen=True)
class Workload:
    name: str
    mesh: dict                      # keyword arguments of the generator
    generator: str                  # "icosphere" | "radial_star"
    R: int                          # root blocks per axis
    levels: int                     # number of refinement levels (finest level index)
    band: int = 2                   # near-wall distance in finest cells
    lattices: tuple = (19,)
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def build_mesh(self):
        if self.generator == "icosphere":
            return icosphere(**self.mesh)
        if self.generator == "radial_star":
            return radial_star(**self.mesh)
        raise ValueError(self.generator)


def _sig_sq(c, p):
    return lambda l: c / (l ** p)


WORKLOADS = {
    # 320-triangle icosphere, root 2^3 blocks, levels 0..2, D3Q19 (small case)
    "icosphere_320": Workload(
        "icosphere_320", dict(subdiv=2, radius=0.3, seed=20251202), "icosphere", R=2, levels=2,
        lattices=(19,)),
    # ~112K-triangle radial star (bunny-sized), root 16^3, levels 0..3
    "star_112k": Workload(
        "star_112k", dict(n_theta=237, n_phi=236, lmax=8, sigma=_sig_sq(0.05, 2), seed=20251203),
        "radial_star", R=16, levels=3, lattices=(19, 27)),
    # ~7.2M-triangle anisotropic radial star (dragon-sized), root 32^3, levels 0..4, D3Q27
    "star_7m": Workload(
        "star_7m", dict(n_theta=1897, n_phi=1898, lmax=32, sigma=_sig_sq(0.08, 1.5), seed=20251204,
                        scale=(1.0, 0.6, 0.4)),
        "radial_star", R=32, levels=4, lattices=(27,)),
    # profiling case: the 7.2M form at 3.0M triangles (144 MB of records, more than the
    # 129 MB L2), root 32^3, levels 0..4, D3Q27
    "star_3m": Workload(
        "star_3m", dict(n_theta=1225, n_phi=1224, lmax=32, sigma=_sig_sq(0.08, 1.5), seed=20251205,
                        scale=(1.0, 0.6, 0.4)),
        "radial_star", R=32, levels=4, lattices=(27,)),
    # differentiation case: the 112K mesh, root 16^3, levels 0..3, D3Q19
    "diff_112k": Workload(
        "diff_112k", dict(n_theta=237, n_phi=236, lmax=8, sigma=_sig_sq(0.05, 2), seed=20251203),
        "radial_star", R=16, levels=3, lattices=(19,), extra=dict(pop_seed=20251206, w_seed=20251207)),
    # small parity cases that the oracle runs in full
    "star_1k": Workload(
        "star_1k", dict(n_theta=24, n_phi=24, lmax=8, sigma=_sig_sq(0.05, 2), seed=20251210),
        "radial_star", R=4, levels=3, lattices=(19, 27)),
    "star_4k_r3": Workload(
        "star_4k_r3", dict(n_theta=46, n_phi=44, lmax=12, sigma=_sig_sq(0.08, 1.5), seed=20251211,
                           scale=(1.0, 0.7, 0.5), rotate=True),
        "radial_star", R=3, levels=3, lattices=(27,)),
    "star_20k": Workload(
        "star_20k", dict(n_theta=101, n_phi=100, lmax=16, sigma=_sig_sq(0.08, 1.5), seed=20251212,
                         scale=(1.0, 0.6, 0.4)),
        "radial_star", R=8, levels=3, lattices=(27,)),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def batch_meshes(n: int = 48, base_seed: int = 20251300, t_min: float = 1e3, t_max: float = 5e5):
    """The batched workload: n radial meshes of log-uniform triangle counts.

    Returns a list of dicts with keys verts, tris, R, levels.  Mesh j uses
    seed base_seed + j; rejected draws (bounding box not inside (0,1)^3) are
    redrawn from the same generator.
    """
    out = []
    for j in range(n):
        rng = np.random.default_rng(base_seed + j)
        while True:
            T = int(round(math.exp(rng.uniform(math.log(t_min), math.log(t_max)))))
            n_phi = max(3, int(round(math.sqrt(T / 2.0))))
            n_theta = max(2, int(round(T / (2.0 * n_phi))) + 1)
            base = float(rng.uniform(0.15, 0.4))
            R = int(rng.integers(8, 25))
            levels = int(rng.integers(2, 5))
            sub = int(rng.integers(0, 2**31 - 1))
            try:
                v, t = radial_star(n_theta, n_phi, lmax=8, sigma=_sig_sq(0.05, 2), seed=sub,
                                   base_radius=base, jitter=0.01, rotate=True)
            except ValueError:
                continue
            out.append(dict(verts=v, tris=t, R=R, levels=levels, band=2, lattice=19))
            break
    return out


# lattice data used only to synthesise populations (an input, not method arithmetic)
D3Q27_DIRS = np.array(
    [[0, 0, 0],
     [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
     [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
     [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
     [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1],
     [1, 1, 1], [-1, -1, -1], [1, 1, -1], [-1, -1, 1], [1, -1, 1], [-1, 1, -1], [-1, 1, 1], [1, -1, -1]],
    dtype=np.int64)
D3Q19_WEIGHTS = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, dtype=np.float64)
D3Q27_WEIGHTS = np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8, dtype=np.float64)


def populations(n_cells: int, seed: int, u=(0.05, 0.0, 0.0), noise: float = 0.01, lattice: int = 19) -> np.ndarray:
    """Populations [lattice, n_cells] float32 (D3Q19 or D3Q27): a uniform flow state,
    equilibrium(rho=1, u) * (1 + noise N(0,1)) per population."""
    rng = np.random.default_rng(seed)
    c = D3Q27_DIRS[:lattice].astype(np.float64)
    w = D3Q19_WEIGHTS if lattice == 19 else D3Q27_WEIGHTS
    u = np.asarray(u, dtype=np.float64)
    cu = c @ u
    feq = w * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * float(u @ u))
    z = rng.standard_normal((lattice, n_cells))
    return (feq[:, None] * (1.0 + noise * z)).astype(np.float32)


def link_weights(n_links: int, seed: int) -> np.ndarray:
    """Per-link weights w_k ~ N(0, 1) for the loss sum_k w_k q_k (float32)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n_links).astype(np.float32)
