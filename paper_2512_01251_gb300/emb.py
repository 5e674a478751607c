"""Python binding of libemb: the C ABI calls under the same names, taking torch
CUDA tensors (argument marshalling only), plus ``embed``, which chains the calls
of the whole path (bin -> voxelize -> refine flags -> refine, per level, then the
cut-link table) the way Sec. 3.4 orders them.

Status codes other than EMB_OK raise ``EmbError``.  Device-side errors are
collected by ``emb_status_get`` (``embed`` checks it once at the end).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import torch

from ._lib import load

EMB_OK = 0
EMB_ERR_BAD_INPUT = -1
EMB_ERR_NOT_WATERTIGHT = -2
EMB_ERR_CAPACITY = -3
EMB_ERR_CUDA = -4
EMB_ERR_TIMEOUT = -5
EMB_ERR_RANGE = -6
EMB_ERR_STATE = -7
EMB_ERR_BOUNDS = -8


class EmbError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        name = load().emb_status_string(code).decode()
        super().__init__(f"{where}: {name} ({code})")


def _check(code: int, where: str):
    if code != EMB_OK:
        raise EmbError(code, where)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _out_ptr(t: torch.Tensor | None):
    """An output buffer: a CUDA tensor, or a host tensor that the library checks (it takes
    page-locked host memory and refuses pageable memory)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _sync(stream=None):
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()


class _Handle:
    _destroy = None

    def __init__(self, h, keep=()):
        self.h = h
        self._keep = keep

    def close(self):
        if self.h:
            getattr(load(), self._destroy)(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh(_Handle):
    _destroy = "emb_mesh_destroy"


class Forest(_Handle):
    _destroy = "emb_forest_destroy"


class Bins(_Handle):
    _destroy = "emb_bins_destroy"


class Batch(_Handle):
    _destroy = "emb_batch_destroy"


# --------------------------------------------------------------------------- #
# the C ABI, one wrapper per call
# --------------------------------------------------------------------------- #
def emb_status_get(stream=None) -> int:
    out = ctypes.c_int32(0)
    _check(load().emb_status_get(_stream(stream), ctypes.byref(out)), "emb_status_get")
    return out.value


def emb_launch_count() -> int:
    out = ctypes.c_int64(0)
    _check(load().emb_launch_count(ctypes.byref(out)), "emb_launch_count")
    return out.value


def emb_directions() -> list:
    buf = (ctypes.c_int32 * 81)()
    _check(load().emb_directions(buf), "emb_directions")
    return [tuple(buf[3 * i:3 * i + 3]) for i in range(27)]


EMB_PROBE_XLINE, EMB_PROBE_SEGMENT, EMB_PROBE_PAIR, EMB_PROBE_BOX = 0, 1, 2, 3


def emb_probe_predicates(kind: int, queries: torch.Tensor, stream=None):
    """The library's device predicates on (n, 15) int64 queries (layout in emb.h):
    returns (hit int32, q float32) tensors."""
    queries = queries.to(device="cuda", dtype=torch.int64).contiguous()
    n = queries.shape[0]
    hit = torch.empty(n, dtype=torch.int32, device="cuda")
    q = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(load().emb_probe_predicates(int(kind), _ptr(queries), n, _ptr(hit), _ptr(q), _stream(stream)),
           "emb_probe_predicates")
    return hit, q


def emb_mesh_create(verts: torch.Tensor, tris: torch.Tensor, R: int, check_watertight: bool = True,
                    stream=None) -> Mesh:
    verts = verts.to(device="cuda", dtype=torch.float32).contiguous()
    tris = tris.to(device="cuda", dtype=torch.int32).contiguous()
    h = ctypes.c_void_p()
    rc = load().emb_mesh_create(_ptr(verts), _ptr(tris), verts.shape[0], tris.shape[0], int(R),
                                int(bool(check_watertight)), _stream(stream), ctypes.byref(h))
    _check(rc, "emb_mesh_create")
    m = Mesh(h)
    m.V, m.T, m.R = verts.shape[0], tris.shape[0], int(R)
    return m


def emb_mesh_update(mesh: Mesh, verts: torch.Tensor, stream=None):
    """New positions for the mesh's vertices (same triangles); asynchronous, no allocation."""
    verts = verts.to(device="cuda", dtype=torch.float32).contiguous()
    _check(load().emb_mesh_update(mesh.h, _ptr(verts), verts.shape[0], _stream(stream)), "emb_mesh_update")
    mesh._moved_verts = verts  # kept alive until the next update (the kernel may still be queued)


def emb_forest_root(R: int, max_level: int, stream=None) -> Forest:
    h = ctypes.c_void_p()
    _check(load().emb_forest_root(int(R), int(max_level), _stream(stream), ctypes.byref(h)), "emb_forest_root")
    f = Forest(h)
    f.R, f.max_level = int(R), int(max_level)
    return f


def emb_forest_refine(forest: Forest, level: int, flags: torch.Tensor, stream=None):
    _check(load().emb_forest_refine(forest.h, int(level), _ptr(flags), _stream(stream)), "emb_forest_refine")


def emb_forest_num_blocks(forest: Forest, level: int) -> int:
    out = ctypes.c_int64(0)
    _check(load().emb_forest_num_blocks(forest.h, int(level), ctypes.byref(out)), "emb_forest_num_blocks")
    return out.value


def emb_forest_blocks(forest: Forest, level: int, stream=None) -> torch.Tensor:
    n = emb_forest_num_blocks(forest, level)
    out = torch.empty((n, 3), dtype=torch.int32, device="cuda")
    _check(load().emb_forest_blocks(forest.h, int(level), _ptr(out), _stream(stream)), "emb_forest_blocks")
    return out


def emb_forest_neighbors(forest: Forest, level: int, stream=None) -> torch.Tensor:
    n = emb_forest_num_blocks(forest, level)
    out = torch.empty((n, 26), dtype=torch.int32, device="cuda")
    _check(load().emb_forest_neighbors(forest.h, int(level), _ptr(out), _stream(stream)), "emb_forest_neighbors")
    return out


def emb_forest_masks(forest: Forest, level: int, stream=None) -> torch.Tensor:
    n = emb_forest_num_blocks(forest, level)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    _check(load().emb_forest_masks(forest.h, int(level), _ptr(out), _stream(stream)), "emb_forest_masks")
    return out


EMB_BIN_FILTER_COMPACT, EMB_BIN_FILTER_ONLY, EMB_BIN_NO_FILTER = 0, 1, 2


def emb_bin(mesh: Mesh, forest: Forest, level: int, lattice: int = 19, stream=None,
            mode: int = EMB_BIN_FILTER_COMPACT) -> Bins:
    """mode: EMB_BIN_FILTER_COMPACT (default), or the ablations EMB_BIN_FILTER_ONLY / EMB_BIN_NO_FILTER."""
    h = ctypes.c_void_p()
    if mode == EMB_BIN_FILTER_COMPACT:
        _check(load().emb_bin(mesh.h, forest.h, int(level), int(lattice), _stream(stream), ctypes.byref(h)), "emb_bin")
    else:
        _check(load().emb_bin_ex(mesh.h, forest.h, int(level), int(lattice), int(mode), _stream(stream),
                                 ctypes.byref(h)), "emb_bin_ex")
    b = Bins(h, keep=(mesh, forest))
    b.level = int(level)
    return b


def emb_bins_stats(bins: Bins):
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().emb_bins_stats(bins.h, ctypes.byref(a), ctypes.byref(b)), "emb_bins_stats")
    return a.value, b.value


def emb_bins_copy(bins: Bins, forest: Forest | None = None, stream=None) -> dict:
    """Filtered triangle ids and, at the finest level, the CSR bins (int32 tensors)."""
    nf, npairs = emb_bins_stats(bins)
    out = dict(filtered=torch.empty(max(nf, 1), dtype=torch.int32, device="cuda"))
    want_csr = forest is not None
    if want_csr:
        n = emb_forest_num_blocks(forest, bins.level)
        out["off"] = torch.empty(n + 1, dtype=torch.int32, device="cuda")
        out["ent"] = torch.empty(max(npairs, 1), dtype=torch.int32, device="cuda")
    _check(load().emb_bins_copy(bins.h, _ptr(out["filtered"]), _ptr(out.get("off")), _ptr(out.get("ent")),
                                _stream(stream)), "emb_bins_copy")
    out["filtered"] = out["filtered"][:nf]
    if want_csr:
        out["ent"] = out["ent"][:npairs]
    return out


def emb_voxelize(forest: Forest, bins: Bins, level: int, out: torch.Tensor | None = None, stream=None):
    """Solid mask words of `level` (int64 tensor holding the uint64 bit patterns)."""
    n = emb_forest_num_blocks(forest, level)
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device="cuda")
    elif out.numel() < n:
        raise EmbError(EMB_ERR_CAPACITY, "emb_voxelize: the output holds fewer words than the level has blocks")
    _check(load().emb_voxelize(forest.h, bins.h, int(level), _out_ptr(out), _stream(stream)), "emb_voxelize")
    return out[:n]


def emb_voxelize_guard(forest: Forest, bins: Bins, out_solid: torch.Tensor | None = None,
                       out_guard: torch.Tensor | None = None, stream=None):
    """The paper's guard-cell voxelizer on the finest level (the ablation of the exact
    one): (solid words, guard words) as int64 tensors holding the uint64 patterns."""
    n = emb_forest_num_blocks(forest, bins.level)
    if out_solid is None:
        out_solid = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    if out_guard is None:
        out_guard = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    _check(load().emb_voxelize_guard(forest.h, bins.h, _ptr(out_solid), _ptr(out_guard), _stream(stream)),
           "emb_voxelize_guard")
    return out_solid[:n], out_guard[:n]


def emb_refine_flags(forest: Forest, bins: Bins, level: int, band: int, out: torch.Tensor | None = None,
                     stream=None):
    if out is None:
        out = torch.empty(emb_forest_num_blocks(forest, level), dtype=torch.uint8, device="cuda")
    _check(load().emb_refine_flags(forest.h, bins.h, int(level), int(band), _ptr(out), _stream(stream)),
           "emb_refine_flags")
    return out


def emb_refine_flags_paper(forest: Forest, level: int, d_spec: float, out: torch.Tensor | None = None, stream=None):
    """The paper's block-layer refinement rules (Sec. 3.4, Eq. N_prop); d_spec in units of the unit domain."""
    if out is None:
        out = torch.empty(max(1, emb_forest_num_blocks(forest, level)), dtype=torch.uint8, device="cuda")
    _check(load().emb_refine_flags_paper(forest.h, int(level), float(d_spec), _ptr(out), _stream(stream)),
           "emb_refine_flags_paper")
    return out[:emb_forest_num_blocks(forest, level)]


def emb_cutlinks_count(forest: Forest, lattice: int, stream=None) -> int:
    out = ctypes.c_int64(0)
    _check(load().emb_cutlinks_count(forest.h, int(lattice), ctypes.byref(out), _stream(stream)), "emb_cutlinks_count")
    return out.value


def emb_cutlinks_prepare(forest: Forest, lattice: int, stream=None) -> None:
    """Enqueue the candidate cells of the link table without reading the count back."""
    _check(load().emb_cutlinks_prepare(forest.h, int(lattice), _stream(stream)), "emb_cutlinks_prepare")


def emb_cutlinks(forest: Forest, bins: Bins, lattice: int, capacity: int | None = None, out: dict | None = None,
                 stream=None, sync: bool = True) -> dict:
    """Cut-link table {cell int32, dir uint8, q float32, tri int32, count int64}.

    Without `capacity` the count is read back first (emb_cutlinks_count) and the
    table is sized to it.  With `capacity` nothing is read back before the launch;
    with `sync` the call then waits for the stream, reads the count and returns the
    table cut to it (EmbError EMB_ERR_CAPACITY when it held more links than
    `capacity`); without `sync` it returns the whole buffers at once and the caller
    cuts them to out["count"] once the stream has passed the call.
    """
    exact = capacity is None
    if exact:
        capacity = emb_cutlinks_count(forest, lattice, stream)
    if out is None:
        out = dict(cell=torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda"),
                   dir=torch.empty(max(capacity, 1), dtype=torch.uint8, device="cuda"),
                   q=torch.empty(max(capacity, 1), dtype=torch.float32, device="cuda"),
                   tri=torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda"),
                   count=torch.zeros(1, dtype=torch.int64, device="cuda"))
    rc = load().emb_cutlinks(forest.h, bins.h, int(lattice), _out_ptr(out["cell"]), _out_ptr(out["dir"]),
                             _out_ptr(out["q"]), _out_ptr(out["tri"]), int(capacity), _out_ptr(out["count"]),
                             _stream(stream))
    _check(rc, "emb_cutlinks")
    if exact:
        n = capacity
    elif sync:
        _sync(stream)
        n = int(out["count"][0].item())
        if n > capacity:
            raise EmbError(EMB_ERR_CAPACITY, f"emb_cutlinks: {n} links, room for {capacity}")
    else:
        n = capacity
    return {k: (v[:n] if k != "count" else v) for k, v in out.items()}


def emb_mex_force(forest: Forest, lattice: int, cell, dir, q, pop: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(3, dtype=torch.float32, device="cuda")
    _check(load().emb_mex_force(forest.h, int(lattice), _ptr(cell), _ptr(dir), _ptr(q), q.numel(), _ptr(pop),
                                pop.shape[1], _ptr(out), _stream(stream)), "emb_mex_force")
    return out


def emb_mex_force_noalloc(forest: Forest, lattice: int, cell, dir, q, pop: torch.Tensor, out: torch.Tensor,
                          stream=None) -> torch.Tensor:
    """emb_mex_force without any device allocation (for callers that cannot allocate
    mid-run); `out` (3 float32 on the device) must be provided by the caller."""
    _check(load().emb_mex_force_noalloc(forest.h, int(lattice), _ptr(cell), _ptr(dir), _ptr(q), q.numel(), _ptr(pop),
                                        pop.shape[1], _ptr(out), _stream(stream)), "emb_mex_force_noalloc")
    return out


def emb_mex_force_backward(forest: Forest, lattice: int, cell, dir, q, pop: torch.Tensor, gF: torch.Tensor,
                           out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty_like(q)
    gF = gF.to(device="cuda", dtype=torch.float32).contiguous()
    _check(load().emb_mex_force_backward(forest.h, int(lattice), _ptr(cell), _ptr(dir), _ptr(q), q.numel(),
                                         _ptr(pop), pop.shape[1], _ptr(gF), _ptr(out), _stream(stream)),
           "emb_mex_force_backward")
    return out


def emb_lbm_step(forest: Forest, lattice: int, links: dict, omega: float, pop: torch.Tensor,
                 out: torch.Tensor | None = None, pre: torch.Tensor | None = None, phases: int = 7, stream=None):
    """One lattice-Boltzmann step on the finest level with Bouzidi bounce-back from the link table.
    pop: (lattice, stride) float32 post-collision populations; returns those one step later."""
    if out is None:
        out = torch.empty_like(pop)
    if pre is None:
        pre = torch.empty_like(pop)
    n = links["q"].numel()
    _check(load().emb_lbm_step(forest.h, int(lattice), _ptr(links["cell"]), _ptr(links["dir"]), _ptr(links["q"]), n,
                               float(omega), _ptr(pop), _ptr(pre), _ptr(out), pop.shape[1], int(phases),
                               _stream(stream)), "emb_lbm_step")
    return out


def emb_cutlinks_backward(mesh: Mesh, forest: Forest, cell, dir, q, tri, gq: torch.Tensor,
                          out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty((mesh.V, 3), dtype=torch.float32, device="cuda")
    gq = gq.to(device="cuda", dtype=torch.float32).contiguous()
    _check(load().emb_cutlinks_backward(mesh.h, forest.h, _ptr(cell), _ptr(dir), _ptr(q), _ptr(tri), q.numel(),
                                        _ptr(gq), _ptr(out), _stream(stream)), "emb_cutlinks_backward")
    return out


# --------------------------------------------------------------------------- #
# the whole path
# --------------------------------------------------------------------------- #
@dataclass
class Embedding:
    mesh: Mesh
    forest: Forest
    levels: int
    lattice: int
    blocks: list = field(default_factory=list)   # per level (n, 3) int32, filled by fetch_blocks
    masks: list = field(default_factory=list)    # per level int64 mask words
    flags: list = field(default_factory=list)    # per level < finest, uint8
    links: dict | None = None
    bins: list = field(default_factory=list)
    stats: dict = field(default_factory=dict)

    def fetch_blocks(self):
        self.blocks = [emb_forest_blocks(self.forest, L) for L in range(self.levels + 1)]
        return self.blocks

    def units(self) -> int:
        """Cells over all levels plus cut links (the throughput unit)."""
        cells = sum(64 * emb_forest_num_blocks(self.forest, L) for L in range(self.levels + 1))
        return cells + (0 if self.links is None else int(self.links["q"].numel()))


def embed(verts: torch.Tensor, tris: torch.Tensor, R: int, levels: int, band: int = 2, lattice: int = 19,
          check_watertight: bool = True, mesh: Mesh | None = None, keep_bins: bool = False,
          check_status: bool = True, stream=None, bin_mode: int = EMB_BIN_FILTER_COMPACT,
          d_spec: float | None = None, links_out: dict | None = None,
          finest_mask_out: torch.Tensor | None = None) -> Embedding:
    """Embed a closed mesh into a forest with root R^3 blocks and levels 0..levels.

    Per level: emb_bin, emb_voxelize, then (below the finest level)
    emb_refine_flags and emb_forest_refine; at the finest level the cut-link
    table of `lattice` (19 or 27).  With d_spec, the refinement follows the
    paper's block-layer rules (emb_refine_flags_paper) instead of `band`.
    links_out (cell, dir, q, tri int tensors and a count int64 tensor, each large enough)
    and finest_mask_out receive the link table and the finest solid mask; they may be
    page-locked host tensors, which the library then fills over the host link.
    """
    forest = emb_forest_root(R, levels, stream)  # first: it runs while the mesh check reads back
    if mesh is None:
        mesh = emb_mesh_create(verts, tris, R, check_watertight, stream)
    E = Embedding(mesh=mesh, forest=forest, levels=levels, lattice=lattice)
    for L in range(levels + 1):
        bins = emb_bin(mesh, forest, L, lattice, stream, mode=bin_mode)
        E.masks.append(emb_voxelize(forest, bins, L, out=finest_mask_out if L == levels else None, stream=stream))
        if L < levels:
            fl = (emb_refine_flags(forest, bins, L, band, stream=stream) if d_spec is None
                  else emb_refine_flags_paper(forest, L, d_spec, stream=stream))
            E.flags.append(fl)
            emb_forest_refine(forest, L, fl, stream)
        else:
            if links_out is None:
                E.links = emb_cutlinks(forest, bins, lattice, stream=stream)
            else:
                # the buffers' size is the capacity: the count stays on the device
                # until the table is written
                cap = min(links_out[k].numel() for k in ("cell", "dir", "q", "tri"))
                try:
                    E.links = emb_cutlinks(forest, bins, lattice, capacity=cap, out=links_out, stream=stream)
                except EmbError as e:
                    if e.code == EMB_ERR_CAPACITY:
                        emb_status_get(stream)  # the status the short table left
                        raise EmbError(EMB_ERR_CAPACITY, "embed: links_out holds fewer than the table's links")
                    raise
        if keep_bins:
            E.bins.append(bins)
        else:
            bins.close()
    if check_status:
        st = emb_status_get(stream)
        if st != EMB_OK:
            raise EmbError(st, "embed (device status)")
    return E


# --------------------------------------------------------------------------- #
# incremental re-embedding of a region
# --------------------------------------------------------------------------- #
def emb_forest_root_window(R: int, max_level: int, y0: int, y1: int, z0: int, z1: int, stream=None) -> Forest:
    h = ctypes.c_void_p()
    _check(load().emb_forest_root_window(int(R), int(max_level), int(y0), int(y1), int(z0), int(z1), _stream(stream),
                                         ctypes.byref(h)), "emb_forest_root_window")
    f = Forest(h)
    f.R, f.max_level = int(R), int(max_level)
    return f


def emb_mesh_subset(mesh: Mesh, ylo: int, yhi: int, zlo: int, zhi: int, stream=None):
    """(sub-mesh, map int32 tensor: sub-mesh triangle -> mesh triangle)."""
    tri_map = torch.empty(mesh.T, dtype=torch.int32, device="cuda")
    h = ctypes.c_void_p()
    n = ctypes.c_int64(0)
    _check(load().emb_mesh_subset(mesh.h, int(ylo), int(yhi), int(zlo), int(zhi), _ptr(tri_map), mesh.T,
                                  _stream(stream), ctypes.byref(h), ctypes.byref(n)), "emb_mesh_subset")
    sub = Mesh(h)
    sub.V, sub.T, sub.R = mesh.V, int(n.value), mesh.R
    return sub, tri_map[:n.value]


def emb_splice(forest: Forest, window: Forest, y0: int, y1: int, z0: int, z1: int, links: dict, wlinks: dict,
               tri_map: torch.Tensor | None = None, stream=None) -> dict:
    """Merges `window` into `forest` inside the inner window [y0, y1) x [z0, z1) of root-block
    rows; returns the merged link table."""
    nf, nw = links["q"].numel(), wlinks["q"].numel()
    cap = nf + nw
    out = dict(cell=torch.empty(max(cap, 1), dtype=torch.int32, device="cuda"),
               dir=torch.empty(max(cap, 1), dtype=torch.uint8, device="cuda"),
               q=torch.empty(max(cap, 1), dtype=torch.float32, device="cuda"),
               tri=torch.empty(max(cap, 1), dtype=torch.int32, device="cuda"))
    n = ctypes.c_int64(0)
    args = [_ptr(links[k]) if nf else None for k in ("cell", "dir", "q", "tri")]
    wargs = [_ptr(wlinks[k]) if nw else None for k in ("cell", "dir", "q", "tri")]
    _check(load().emb_splice(forest.h, window.h, int(y0), int(y1), int(z0), int(z1), *args, nf, *wargs, nw,
                             _ptr(tri_map) if tri_map is not None and tri_map.numel() else None,
                             _ptr(out["cell"]), _ptr(out["dir"]), _ptr(out["q"]), _ptr(out["tri"]), cap,
                             ctypes.byref(n), _stream(stream)), "emb_splice")
    return {k: v[:n.value] for k, v in out.items()}


def reembed_window(E: Embedding, verts: torch.Tensor, changed: tuple, band: int = 2, stream=None) -> Embedding:
    """Brings E up to date after the mesh's vertices moved to `verts`, recomputing only the
    region the change can reach (the paper names moving geometry as future work, Sec. 5).

    `changed` = (y_lo, y_hi, z_lo, z_hi): the y-z extent, in root blocks (half-open), of
    every triangle that moved, at its old and at its new position.  The inner window is
    that extent widened by 2 root blocks (the reach of a refine dilation, at most 1.2 root
    blocks, plus the block that holds it); the window forest is 1 root block wider (the
    neighbours of its inner blocks) and is embedded from the triangles that meet it widened
    by 2 more root blocks.  The result is identical to re-embedding the whole mesh."""
    R, Lf = E.forest.R, E.levels
    emb_mesh_update(E.mesh, verts, stream)
    y0, y1, z0, z1 = changed
    iy0, iy1, iz0, iz1 = max(0, y0 - 2), min(R, y1 + 2), max(0, z0 - 2), min(R, z1 + 2)
    wy0, wy1, wz0, wz1 = max(0, iy0 - 1), min(R, iy1 + 1), max(0, iz0 - 1), min(R, iz1 + 1)
    k = (R & -R).bit_length() - 1  # R = r_o 2^k
    W0 = 1 << (20 - k)  # root block width in frame units (4 cells of 2^(18-k))
    sub, tri_map = emb_mesh_subset(E.mesh, (wy0 - 2) * W0, (wy1 + 2) * W0, (wz0 - 2) * W0, (wz1 + 2) * W0, stream)
    fw = emb_forest_root_window(R, Lf, wy0, wy1, wz0, wz1, stream)
    wl = None
    for L in range(Lf + 1):
        bins = emb_bin(sub, fw, L, E.lattice, stream)
        emb_voxelize(fw, bins, L, stream=stream)
        if L < Lf:
            fl = emb_refine_flags(fw, bins, L, band, stream=stream)
            emb_forest_refine(fw, L, fl, stream)
        else:
            wl = emb_cutlinks(fw, bins, E.lattice, stream=stream)
        bins.close()
    E.links = emb_splice(E.forest, fw, iy0, iy1, iz0, iz1, E.links, wl, tri_map, stream)
    E.masks = [emb_forest_masks(E.forest, L, stream) for L in range(Lf + 1)]
    E.flags = []
    E.blocks = []
    fw.close()
    sub.close()
    return E


# --------------------------------------------------------------------------- #
# batches of meshes
# --------------------------------------------------------------------------- #
def emb_batch_create(meshes: list, levels: list, bands: list, lattices: list, stream=None, headroom: int = 0) -> Batch:
    """Plan a batch; headroom (percent) gives the replay's buffers room above the planned
    counts, so that geometry that moves can be replayed without a new plan."""
    n = len(meshes)
    arr = (ctypes.c_void_p * n)(*[m.h for m in meshes])
    lv = (ctypes.c_int32 * n)(*levels)
    bd = (ctypes.c_int32 * n)(*bands)
    lt = (ctypes.c_int32 * n)(*lattices)
    h = ctypes.c_void_p()
    if headroom:
        _check(load().emb_batch_create_ex(arr, lv, bd, lt, n, int(headroom), _stream(stream), ctypes.byref(h)),
               "emb_batch_create_ex")
    else:
        _check(load().emb_batch_create(arr, lv, bd, lt, n, _stream(stream), ctypes.byref(h)), "emb_batch_create")
    b = Batch(h, keep=tuple(meshes))
    b.levels, b.lattices, b.n, b.headroom = list(levels), list(lattices), n, int(headroom)
    return b


def emb_batch_counts(batch: Batch, j: int, stream=None):
    """(blocks per level, links) of mesh j in the last replay."""
    blocks = (ctypes.c_int64 * (batch.levels[j] + 1))()
    links = ctypes.c_int64(0)
    _check(load().emb_batch_counts(batch.h, int(j), _stream(stream), blocks, ctypes.byref(links)), "emb_batch_counts")
    return list(blocks), links.value


def emb_batch_run(batch: Batch, stream=None):
    _check(load().emb_batch_run(batch.h, _stream(stream)), "emb_batch_run")


def emb_batch_capture(batch: Batch, stream=None):
    _check(load().emb_batch_capture(batch.h, _stream(stream)), "emb_batch_capture")


def emb_batch_launch(batch: Batch, stream=None):
    _check(load().emb_batch_launch(batch.h, _stream(stream)), "emb_batch_launch")


def emb_batch_autotune(batch: Batch, stream=None) -> tuple:
    """(streams, tri_block, link CTAs per SM, link placement 0/1/2) of the fastest shape."""
    c = (ctypes.c_int32 * 4)()
    _check(load().emb_batch_autotune(batch.h, _stream(stream), c), "emb_batch_autotune")
    return tuple(c)


EMB_TUNE_FORCE = 1


def emb_batch_autotune_ex(batch: Batch, stream=None, force: bool = False) -> tuple:
    """((streams, tri_block, link CTAs per SM, link placement), taken from the tuning cache)."""
    c = (ctypes.c_int32 * 5)()
    _check(load().emb_batch_autotune_ex(batch.h, _stream(stream), EMB_TUNE_FORCE if force else 0, c),
           "emb_batch_autotune_ex")
    return tuple(c[:4]), bool(c[4])


def emb_batch_configure(batch: Batch, streams: int, tri_block: int, link_ctas: int = 0, per_mesh_links: int = 1):
    c = (ctypes.c_int32 * 4)(streams, tri_block, link_ctas, per_mesh_links)
    _check(load().emb_batch_configure(batch.h, c), "emb_batch_configure")


def emb_batch_info(batch: Batch, j: int):
    blocks = (ctypes.c_int64 * (batch.levels[j] + 1))()
    links = ctypes.c_int64(0)
    _check(load().emb_batch_info(batch.h, int(j), blocks, ctypes.byref(links)), "emb_batch_info")
    return list(blocks), links.value


def emb_batch_results(batch: Batch, j: int, stream=None) -> dict:
    """Mesh j of the last replay: per level (blocks, masks), and its cut-link table."""
    blocks, n = emb_batch_counts(batch, j, stream)
    out = dict(blocks=[], masks=[])
    for L, nb in enumerate(blocks):
        m = torch.empty(max(nb, 1), dtype=torch.int64, device="cuda")
        bc = torch.empty((max(nb, 1), 3), dtype=torch.int32, device="cuda")
        _check(load().emb_batch_results(batch.h, int(j), L, _ptr(m), _ptr(bc), None, None, None, None, _stream(stream)),
               "emb_batch_results")
        out["masks"].append(m[:nb])
        out["blocks"].append(bc[:nb])
    links = dict(cell=torch.empty(max(n, 1), dtype=torch.int32, device="cuda"),
                 dir=torch.empty(max(n, 1), dtype=torch.uint8, device="cuda"),
                 q=torch.empty(max(n, 1), dtype=torch.float32, device="cuda"),
                 tri=torch.empty(max(n, 1), dtype=torch.int32, device="cuda"))
    _check(load().emb_batch_results(batch.h, int(j), 0, None, None, _ptr(links["cell"]), _ptr(links["dir"]),
                                    _ptr(links["q"]), _ptr(links["tri"]), _stream(stream)), "emb_batch_results")
    out["links"] = {k: v[:n] for k, v in links.items()}
    return out

