#!/usr/bin/env python3
"""Throughput of the embedding path on one GB300 (or N replicas, one per GPU).

One step = the whole path on the ~7.2M-triangle radial mesh (root 32^3 blocks,
levels 0..4, band 2, D3Q27): triangle records, then per level binning, solid
voxelization, refine flags and the forest refinement, then the cut-link table.
Metric: cells (64 per block, all levels) plus cut links embedded per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the CPU oracle (exact brute force over every triangle)
on bounded samples of the same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import math
import os
import statistics
import select
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# more hardware work queues than the default 8 for the batched path's 32 streams (a
# setting of this process's CUDA context, read when the context is created)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

from synth import workload  # noqa: E402

METRIC = "cells+cut links embedded/s at 7.2M tris; batched & fwd+bwd vs plain, same GPU"
UNIT = "units/s"
WORKLOAD = "star_7m"
# Nominal 32-bit ALU instruction slots charged per (link, triangle) exact segment test
# (three Pluecker signs in 64-bit arithmetic plus the normal dot product), and per cut
# link for its exact crossing parameter (the int128 plane offsets and the rational
# comparisons between crossings).
KAPPA_SEG = 48
KAPPA_Q = 60


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-extras", action="store_true", help="skip the e2e leg and the CPU baseline")
    ap.add_argument("--legs", default="all",
                    help="comma-separated extra legs to run (e2e, fwd_bwd, batched, ablation, lbm, moving, "
                         "incremental, guard_ablation, replay, cpu_baseline), or 'all'")
    return ap.parse_args()


def workload_config(w, lattice):
    v, t = w.build_mesh()
    return v, t, dict(workload=f"{w.name}: radial star mesh, {len(t)} triangles, root {w.R}^3 blocks of 4^3 "
                                f"cells, levels 0..{w.levels}, band {w.band}, D3Q{lattice}",
                      triangles=int(len(t)), root=w.R, levels=w.levels, band=w.band, lattice=lattice,
                      l2="flushed between steps (256 MB write)")


# --------------------------------------------------------------------------- #
# CPU oracle sample (reference arm and cpu_baseline)
# --------------------------------------------------------------------------- #
def oracle_sample(v, t, w, lattice, n_blocks, seed):
    """Brute-force work for n_blocks finest-level blocks that hold the surface:
    the solid state of their 64 cells and of every lattice neighbour of their
    fluid cells, then q for each cut link.  Returns (units, seconds)."""
    from oracle import oracle as O
    O.lib()
    X = O.int_coords(v, w.R)
    tri9 = O.tri_coords(X, t)
    rng = np.random.default_rng(seed)
    h = O.h_units(w.R, w.levels)
    W = 4 * h
    C = O.directions()
    picks = rng.choice(len(t), n_blocks, replace=False)
    t0 = time.perf_counter()
    units = 0
    for p in picks:
        cen = tri9[p].reshape(3, 3).mean(axis=0)
        blk = (cen // W).astype(np.int64)[None, :]
        P = O.cell_centres(w.R, w.levels, blk)
        s = O.solid(tri9, P)
        fluid = np.nonzero(s == 0)[0]
        cand = (P[fluid][:, None, :] + h * C[None, 1:lattice, :]).reshape(-1, 3)
        cdir = np.tile(np.arange(1, lattice), len(fluid))
        ccell = np.repeat(fluid, lattice - 1)
        uq, inv = np.unique(cand, axis=0, return_inverse=True)
        sn = O.solid(tri9, uq)[inv.reshape(-1)]
        sel = sn == 1
        O.links(tri9, P[ccell[sel]], cdir[sel], h)
        units += 64 + int(sel.sum())
    return units, time.perf_counter() - t0


def oracle_lines_full(v, t, w, lattice):
    """The whole workload by the sorted-line oracle tier (every block, mask, flag and
    link).  Returns (units, seconds)."""
    from oracle import oracle as O
    O.lib()
    t0 = time.perf_counter()
    r = O.embed_lines(v, t, w.R, w.levels, w.band, lattice)
    secs = time.perf_counter() - t0
    return 64 * sum(len(b) for b in r["blocks"]) + len(r["links"]["q"]), secs


def oracle_slab(tri9, w, lattice, z0, z1):
    """The sorted-line tier on the root-block layers z0 <= bz < z1 of the workload: it
    runs on the triangles whose z-range meets those layers widened by three root blocks
    (more than the reach of any refine dilation, mask line or link of a block in the
    layers, so their results are the whole workload's), and only the blocks and links
    inside the layers are counted.  Returns (units, seconds)."""
    from oracle import oracle as O
    O.lib()
    W0 = 4 * O.h_units(w.R, 0)
    t0 = time.perf_counter()
    zs = tri9[:, 2::3]
    sel = (zs.max(axis=1) >= z0 * W0 - 3 * W0) & (zs.min(axis=1) <= z1 * W0 + 3 * W0)
    r = O.embed_lines_tri9(tri9[sel], w.R, w.levels, w.band, lattice)
    secs = time.perf_counter() - t0
    units = 0
    for L, b in enumerate(r["blocks"]):
        units += 64 * int(((b[:, 2] >= z0 << L) & (b[:, 2] < z1 << L)).sum())
    bf = r["blocks"][-1][r["links"]["cell"] // 64]
    units += int(((bf[:, 2] >= z0 << w.levels) & (bf[:, 2] < z1 << w.levels)).sum())
    return units, secs


def omp_threads():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else os.cpu_count()


def body_layers(tri9, w):
    """Root-block layers (bz) that the mesh's z-range touches."""
    from oracle import oracle as O
    W0 = 4 * O.h_units(w.R, 0)
    return int(tri9[:, 2::3].min() // W0), int(tri9[:, 2::3].max() // W0) + 1


def run_reference(args):
    """The oracle arm: each step is the sorted-line oracle tier on two root-block layers
    of the workload (a bounded sample: the layers the step takes move through the body),
    on this host's cores.  Value = units embedded in the sampled layers per second."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.lib()
    w = workload(args.workload)
    lattice = max(w.lattices)
    v, t, cfg = workload_config(w, lattice)
    tri9 = O.tri_coords(O.int_coords(v, w.R), t)
    z_lo, z_hi = body_layers(tri9, w)
    span = 2
    starts = list(range(z_lo, z_hi, span))
    for i in range(args.warmup):
        z0 = starts[i % len(starts)]
        oracle_slab(tri9, w, lattice, z0, z0 + span)
    units = 0
    secs = 0.0
    for i in range(args.steps):
        z0 = starts[i % len(starts)]
        u, s_ = oracle_slab(tri9, w, lattice, z0, z0 + span)
        units += u
        secs += s_
    val = units / secs
    sample = (f"per step {span} root-block layers (z) of the workload, cycling through the {z_hi - z_lo} layers the "
              f"body spans: every block, mask, refine flag and cut link inside them by the sorted-line oracle tier "
              f"(exact integer predicates, FP64 q) on {omp_threads()} host threads")
    line = dict(impl="reference", metric=METRIC, value=val, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * secs / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="int64", data="synthetic", config=cfg,
                cpu_baseline=dict(value=val, unit=UNIT, cores=omp_threads(), kind="oracle", sample=sample),
                e2e=dict(value=val, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- #
# GPU arm
# --------------------------------------------------------------------------- #
class ClockSampler:
    """nvidia-smi samples during the timed region (median SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        """Starts the sampler and returns once its first sample is out: nvidia-smi's own
        start-up (driver queries of the device) then falls before the timed region, where it
        stalled one step by about 7 ms."""
        self.first = ""
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return
        ready, _, _ = select.select([self.p.stdout], [], [], 10.0)
        if ready:
            self.first = self.p.stdout.readline()

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        return parse_clock_samples(self.first + (out or ""))


def parse_clock_samples(text):
    """Median SM clock, maximum clock and the throttle reasons seen in nvidia-smi CSV lines
    of ClockSampler.Q (no header, no units); None when no line parses."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in text.strip().splitlines():
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx = float(f[2])
        except ValueError:
            continue
        for nm, val in zip(names, f[5:9]):
            if val.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return dict(sm_mhz=statistics.median(sm), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


def source_hash(*names):
    """Hash of the kernel's own source files (the ones that hold its body)."""
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2512_01251_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, src_files):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the source is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    if d.get("source_hash") != source_hash(*src_files):
        return None
    return d


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def reduce_over_ranks(dist, total_ms: float, units: float, device: str):
    """Whole-job numbers of N replicas: the slowest rank's time and the sum of the units
    all ranks embedded (one all-reduce each; the only collective of the run)."""
    import torch
    tt = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    uu = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(uu)
    return float(tt.item()), float(uu.item())


def step_roofline(med, T, level_blocks, stats, n_links, tests, hbm_gbs, alu_tops, step_ms, replay_ms=None,
                  link_tris=None):
    """Roofline of the whole step: per call, T_roof = max(algorithmic bytes / HBM peak,
    algorithmic ops / ALU peak); summed over the calls of a step and divided by the
    measured step time.  Bytes per call (B = blocks of the level, T triangles, nf the
    filtered triangles, pairs the finest bin entries):
      mesh records      96 T (indices, vertex gather, records out)
      bin L             48 T + 4 T + 4 nf (records, filter flags, kept ids); at the finest
                        level also 8 pairs + 4 B (pair counts and fill, offsets)
      voxelize L        52 nf + 8 B + 32 B (kept records and ids, masks, line parities in and out)
      refine flags L    48 T + B
      forest refine L   9 B + 8 B_next (flags and keys in, child keys out)
      cut links         27 x 8 B + 4 pairs + 48 Tb + 13 links (mask words, bins, the records
                        of the Tb distinct triangles of the finest bins, the table),
                        ops = tests x KAPPA_SEG + links x KAPPA_Q (Tb = link_tris; the
                        finest level's x-filter count when it is not given)
    Only the cut links carry an op count (the exact segment tests it must run); for the
    other calls the bytes bound is used, which makes their roofline time a lower bound."""
    lf = len(level_blocks) - 1
    rows = {}

    def add(name, ms, by, ops=0.0):
        if ms is None:
            return
        t_roof = max(by / (hbm_gbs * 1e9), ops / (alu_tops * 1e12)) * 1e3
        rows[name] = dict(ms=round(ms, 4), bytes=int(by), ops=float(ops), roof_ms=round(t_roof, 4),
                          frac=round(t_roof / ms, 4) if ms > 0 else None,
                          bound="alu" if ops / (alu_tops * 1e12) > by / (hbm_gbs * 1e9) else "hbm")

    add("mesh", med.get("mesh"), 96 * T)
    for L in range(lf + 1):
        B = level_blocks[L]
        nf, pairs = stats[L]
        by = 48 * T + 4 * T + 4 * nf + ((8 * pairs + 4 * B) if L == lf else 0)
        add(f"bin{L}", med.get(f"bin{L}"), by)
        add(f"voxelize{L}", med.get(f"voxelize{L}"), 52 * nf + 40 * B)
        if L < lf:
            add(f"refine_flags{L}", med.get(f"refine_flags{L}"), 48 * T + B)
            add(f"forest_refine{L}", med.get(f"forest_refine{L}"), 9 * B + 8 * level_blocks[L + 1])
    cl_ms = (med.get("cutlinks_prep") or 0.0) + (med.get("cutlinks_emit") or 0.0)
    Bf = level_blocks[lf]
    tb = stats[lf][0] if link_tris is None else link_tris
    add("cutlinks", cl_ms, 27 * 8 * Bf + 4 * stats[lf][1] + 48 * tb + 13 * n_links,
        tests * KAPPA_SEG + n_links * KAPPA_Q)
    t_roof = sum(r["roof_ms"] for r in rows.values())
    out = dict(step_roof_ms=round(t_roof, 4), step_ms=round(step_ms, 4), step_frac=round(t_roof / step_ms, 4),
               per_call=rows)
    if replay_ms:
        out["replay_ms"] = round(replay_ms, 4)
        out["replay_frac"] = round(t_roof / replay_ms, 4)
    return out


def run_ours(args):
    import torch

    import paper_2512_01251_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload(args.workload)
    lattice = max(w.lattices)
    v, t, cfg = workload_config(w, lattice)
    cfg["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"
    verts = torch.from_numpy(v).cuda()
    tris = torch.from_numpy(t).cuda()
    stream = torch.cuda.current_stream()
    # one-time validation of the input (watertight, snapped)
    P.emb_mesh_create(verts, tris, w.R, check_watertight=True).close()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    names = ["mesh", "bin", "voxelize", "refine_flags", "forest_refine", "cutlinks"]

    link_cap = [None]

    def step(timed=None):
        ev = []

        def mark(name):
            if timed is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                ev.append((name, e))

        mark("start")
        # the root level first: its launches then run while the mesh check's read-back waits
        forest = P.emb_forest_root(w.R, w.levels)
        mesh = P.emb_mesh_create(verts, tris, w.R, check_watertight=False)
        mark("mesh")
        masks, links, stats = [], None, []
        for L in range(w.levels + 1):
            bins = P.emb_bin(mesh, forest, L, lattice)
            mark(f"bin{L}")
            masks.append(P.emb_voxelize(forest, bins, L))
            mark(f"voxelize{L}")
            if L < w.levels:
                fl = P.emb_refine_flags(forest, bins, L, w.band)
                mark(f"refine_flags{L}")
                P.emb_forest_refine(forest, L, fl)
                mark(f"forest_refine{L}")
            else:
                # the count stays on the device: the table's buffers take the previous
                # step's count with headroom (the first step reads it back); the count
                # is read after the step's last event
                P.emb_cutlinks_prepare(forest, lattice)
                mark("cutlinks_prep")
                cap = link_cap[0] if link_cap[0] is not None else P.emb_cutlinks_count(forest, lattice)
                links = P.emb_cutlinks(forest, bins, lattice, capacity=cap, sync=False)
                mark("cutlinks_emit")
                if timed is not None and timed.get("want_bins"):
                    timed["bins"] = P.emb_bins_copy(bins, forest)
            if timed is not None and timed.get("want_bins"):
                stats.append(P.emb_bins_stats(bins))  # reads counts back: outside the timed steps only
            bins.close()
        if timed is not None:
            timed["events"] = ev
        n = int(links["count"].item())
        if n > cap:
            raise RuntimeError(f"link table of {n} links overflowed its {cap} slots")
        link_cap[0] = n + n // 64 + 1024
        links = {k: (v[:n] if k != "count" else v) for k, v in links.items()}
        return mesh, forest, masks, links, stats

    def units_of(forest, links):
        return sum(64 * P.emb_forest_num_blocks(forest, L) for L in range(w.levels + 1)) + links["q"].numel()

    # the warm-up keeps the previous step's results alive, as the timed loop does, so
    # that the memory pool has grown to the timed region's working set before it starts
    prev = None
    for _ in range(args.warmup):
        prev = step()
    torch.cuda.synchronize()
    if P.emb_status_get() != P.EMB_OK:
        raise RuntimeError("device status error during warm-up")

    # ---- timed region: K steps, L2 flushed (untimed) before each
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    # the per-call path reads counts back between its launches: keep the Python garbage
    # collector from pausing the host inside a timed step (collected after the region)
    gc.collect()
    gc.disable()
    clocks.start()
    l0 = P.emb_launch_count()
    step_ms, per_call = [], {}
    units = 0
    last, prev = prev, None
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        info = dict()
        mesh, forest, masks, links, stats = step(info)
        torch.cuda.synchronize()
        ev = info["events"]
        step_ms.append(ev[0][1].elapsed_time(ev[-1][1]))
        for (a, ea), (b, eb) in zip(ev[:-1], ev[1:]):
            per_call.setdefault(b, []).append(ea.elapsed_time(eb))
        units += units_of(forest, links)
        last = (mesh, forest, masks, links, stats, info.get("bins"))
    launches = P.emb_launch_count() - l0
    torch.cuda.synchronize()
    clk = clocks.stop()
    gc.enable()
    if dist is not None:
        dist.barrier()
    st = P.emb_status_get()
    if st != P.EMB_OK:
        raise RuntimeError(f"device status {st} in the timed region")
    # one more step, untimed, that reads the bin statistics back for the roofline and HBM views
    info = dict(want_bins=True)
    mesh, forest, masks, links, stats = step(info)
    torch.cuda.synchronize()
    last = (mesh, forest, masks, links, stats, info.get("bins"))
    total_ms = sum(step_ms)
    if dist is not None:
        total_ms, units = reduce_over_ranks(dist, total_ms, units, "cuda")
    value = units / (total_ms / 1e3)

    # ---- breakdown, roofline of the dominant call
    mesh, forest, masks, links, stats, bins = last
    med = {k: statistics.median(v_) for k, v_ in per_call.items()}
    groups = {}
    for k, ms in med.items():
        g = k.rstrip("0123456789")
        groups[g] = groups.get(g, 0.0) + ms
    pk, pk_src = peaks()
    n_links = int(links["q"].numel())
    lf = w.levels
    off = bins["off"].cpu().numpy().astype(np.int64)
    blk_links = np.bincount(links["cell"].cpu().numpy().astype(np.int64) // 64, minlength=len(off) - 1)
    tests = int((blk_links * np.diff(off)).sum())
    # the triangles the link kernel stages: the distinct ones of the finest bins
    link_tris = int(torch.unique(bins["ent"]).numel()) if bins["ent"].numel() else 0
    emit_ms = med["cutlinks_emit"]
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    clk_mhz = (clk or {}).get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    alu_peak = sm_count * 128 * clk_mhz * 1e6 / 1e12  # Tops/s of 32-bit ALU slots
    achieved = (tests * KAPPA_SEG + n_links * KAPPA_Q) / (emit_ms / 1e3) / 1e12
    traffic = measured_traffic("k_link_emit", ["emb_cutlinks.cu"])
    roofline = dict(kernel="k_link_emit (emb_cutlinks)", bound="alu", achieved=achieved, peak=alu_peak,
                    unit="Tops/s", frac=achieved / alu_peak,
                    traffic=(traffic or {}).get("bytes_per_launch"),
                    basis=(f"({tests} (link, bin triangle) exact segment tests x {KAPPA_SEG} + {n_links} links x "
                           f"{KAPPA_Q}) 32-bit ALU slots / median launch time; peak = {sm_count} SMs x 128 lanes x "
                           f"{clk_mhz:.0f} MHz (SM clock sampled under load; {pk_src} peaks file for HBM)"))
    hbm = pk.get("hbm_gbs", 6800.0)
    T = len(t)
    level_blocks = [P.emb_forest_num_blocks(forest, L) for L in range(lf + 1)]
    # HBM view of the triangle-parallel passes: each reads every 48-byte record once
    hbm_view = {}
    for L in range(lf):
        ms = med.get(f"refine_flags{L}")
        if ms:
            by = 48 * T + level_blocks[L]
            hbm_view[f"refine_flags{L}"] = dict(GBps=by / (ms / 1e3) / 1e9, frac=by / (ms / 1e3) / 1e9 / hbm)
    for L in range(lf + 1):
        ms = med.get(f"bin{L}")
        if ms:
            by = 48 * T + 8 * T + 4 * stats[L][0]
            hbm_view[f"bin{L}"] = dict(GBps=by / (ms / 1e3) / 1e9, frac=by / (ms / 1e3) / 1e9 / hbm)

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="int64", data="synthetic", config=cfg, roofline=roofline, gpu_launches=launches,
                clocks=clk,
                units_per_step=dict(cells=64 * sum(level_blocks), links=n_links, blocks_per_level=level_blocks),
                breakdown_ms={k: round(v_, 4) for k, v_ in groups.items()},
                breakdown_hbm=hbm_view)
    # the paper's protocol (median and its 95 % confidence interval over the timed steps), and
    # the throughput over the four embedding calls alone (binning, voxelization and refine
    # flags on every level, the cut-link count and table), which leaves out the mesh
    # records and the forest refinement that the whole-step value includes
    srt = sorted(step_ms)
    nst = len(srt)
    j = max(0, int(math.floor(nst / 2 - 0.98 * math.sqrt(nst))))
    k = min(nst - 1, int(math.ceil(nst / 2 + 0.98 * math.sqrt(nst))))
    four = sum(groups.get(g_, 0.0) for g_ in ("bin", "voxelize", "refine_flags", "cutlinks_prep", "cutlinks_emit"))
    line["step_ms_stats"] = dict(median=statistics.median(srt), min=srt[0], max=srt[-1],
                                 ci95_median=[srt[j], srt[k]], n=nst,
                                 in_order=[round(x, 3) for x in step_ms])
    line["four_calls"] = dict(ms=round(four, 4),
                             units_per_s=(64 * sum(level_blocks) + n_links) / (four / 1e3) if four else None)
    # the whole step against its roofline (the replay leg below adds the graph-replay time)
    roofline["step"] = step_roofline(med, T, level_blocks, stats, n_links, tests, hbm, alu_peak,
                                     line["step_ms_stats"]["median"], link_tris=link_tris)

    if rank == 0 and not args.no_extras:
        legs = None if args.legs == "all" else set(args.legs.split(","))

        def want(name):
            return legs is None or name in legs

        if want("e2e"):
            line["e2e"] = e2e_leg(P, v, t, w, lattice, args, stream)
        if want("fwd_bwd"):
            line["fwd_bwd"] = fwd_bwd_leg(P)
        if want("batched"):
            line["batched"] = batch_leg(P)
        if want("ablation"):
            line["ablation"] = ablation_leg(P, verts, tris, w, lattice)
        if want("lbm"):
            line["lbm"] = lbm_leg(P)
        if want("moving"):
            line["moving"] = moving_leg(P)
        if want("incremental"):
            line["incremental"] = incremental_leg(P)
        if want("guard_ablation"):
            line["guard_ablation"] = guard_leg(P, verts, tris, w, lattice)
        if want("replay"):
            line["replay"] = replay_leg(P, verts, tris, w, lattice, line["ms_per_step"])
            line["roofline"]["step"] = step_roofline(med, T, level_blocks, stats, n_links, tests, hbm, alu_peak,
                                                     line["step_ms_stats"]["median"], line["replay"]["ms"],
                                                     link_tris=link_tris)
        if want("cpu_baseline"):
            units_b, secs_b = oracle_lines_full(v, t, w, lattice)
            units_a, secs_a = oracle_sample(v, t, w, lattice, 4, seed=7)
            full_units = 64 * sum(level_blocks) + n_links
            line["cpu_baseline"] = dict(
                value=units_b / secs_b, unit=UNIT, cores=omp_threads(), kind="oracle",
                sample=(f"the whole workload ({units_b} units) by the sorted-line oracle tier: every block, mask, "
                        f"refine flag and cut link, exact integer predicates, FP64 q; {secs_b:.1f} s"),
                brute_force=dict(value=units_a / secs_a, unit=UNIT, cores=omp_threads(),
                                 sample=(f"extrapolated: 4 surface blocks of the finest level by brute force over all "
                                         f"{len(t)} triangles ({units_a} units in {secs_a:.1f} s); at that rate the "
                                         f"full step of {full_units} units would take "
                                         f"{full_units / (units_a / secs_a) / 3600:.0f} h")))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def fwd_bwd_leg(P, reps=10):
    """Differentiation workload: the ~112K-triangle mesh, root 16^3, levels 0..3, D3Q19, populations
    = equilibrium(rho=1, u=(0.05,0,0)) * (1 + 0.01 N(0,1)).  Forward = cut-link table + force;
    backward = dF/dq + dq/dV reduced per vertex.  Median CUDA-event times over `reps`."""
    import torch

    from synth import link_weights, populations
    w = workload("diff_112k")
    v, t = w.build_mesh()
    verts = torch.from_numpy(v).cuda()
    tris = torch.from_numpy(t).cuda()
    E = P.embed(verts, tris, w.R, w.levels, w.band, 19, keep_bins=True)
    fin = E.bins[-1]
    n = E.links["q"].numel()
    nblk = P.emb_forest_num_blocks(E.forest, w.levels)
    pop = torch.from_numpy(populations(nblk * 64, seed=w.extra["pop_seed"])).cuda()
    gq_w = torch.from_numpy(link_weights(n, seed=w.extra["w_seed"])).cuda()
    gF = torch.tensor([1.0, 0.0, 0.0], device="cuda")
    L = dict(cell=torch.empty(n, dtype=torch.int32, device="cuda"), dir=torch.empty(n, dtype=torch.uint8, device="cuda"),
             q=torch.empty(n, dtype=torch.float32, device="cuda"), tri=torch.empty(n, dtype=torch.int32, device="cuda"),
             count=torch.zeros(1, dtype=torch.int64, device="cuda"))
    F = torch.empty(3, dtype=torch.float32, device="cuda")
    gq = torch.empty(n, dtype=torch.float32, device="cuda")
    gv = torch.empty((len(v), 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    fw, bw, em = [], [], []
    for i in range(reps + 2):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record(stream)
        P.emb_cutlinks(E.forest, fin, 19, capacity=n, out=L, sync=False)
        P.emb_mex_force(E.forest, 19, L["cell"], L["dir"], L["q"], pop, out=F)
        e1.record(stream)
        P.emb_mex_force_backward(E.forest, 19, L["cell"], L["dir"], L["q"], pop, gF, out=gq)
        gq.add_(gq_w)  # d/dq of F_x + sum_k w_k q_k
        P.emb_cutlinks_backward(E.mesh, E.forest, L["cell"], L["dir"], L["q"], L["tri"], gq, out=gv)
        e2.record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            fw.append(e0.elapsed_time(e1))
            bw.append(e1.elapsed_time(e2))
    for i in range(reps + 1):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        P.embed(verts, tris, w.R, w.levels, w.band, 19, check_watertight=False, check_status=False)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= 1:
            em.append(a.elapsed_time(b))
    fmed, bmed, emed = statistics.median(fw), statistics.median(bw), statistics.median(em)
    return dict(workload=f"diff_112k: {len(t)} triangles, root {w.R}^3, levels 0..{w.levels}, D3Q19, {n} cut links",
                forward_ms=round(fmed, 4), backward_ms=round(bmed, 4), backward_over_forward=round(bmed / fmed, 3),
                embed_ms=round(emed, 4), backward_over_embed=round(bmed / emed, 3),
                forward="emb_cutlinks + emb_mex_force", backward="emb_mex_force_backward + emb_cutlinks_backward")


def lbm_leg(P, reps=20):
    """The link table's consumer on the differentiation workload (diff_112k, D3Q19): one
    lattice-Boltzmann step on the finest level, timed per pass with CUDA events (median):
    pull streaming and BGK collision over every cell, the Bouzidi pass over the cut links,
    and the momentum-exchange force.  'boundary_share' = (Bouzidi + force) / whole."""
    import torch

    from synth import populations
    w = workload("diff_112k")
    v, t = w.build_mesh()
    E = P.embed(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), w.R, w.levels, w.band, 19)
    nblk = P.emb_forest_num_blocks(E.forest, w.levels)
    ncell = nblk * 64
    pop = torch.from_numpy(populations(ncell, seed=w.extra["pop_seed"])).cuda()
    out, pre = torch.empty_like(pop), torch.empty_like(pop)
    F = torch.empty(3, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    calls = {
        "stream": lambda: P.emb_lbm_step(E.forest, 19, E.links, 1.2, pop, out=out, pre=pre, phases=1),
        "bouzidi": lambda: P.emb_lbm_step(E.forest, 19, E.links, 1.2, pop, out=out, pre=pre, phases=2),
        "collide": lambda: P.emb_lbm_step(E.forest, 19, E.links, 1.2, pop, out=out, pre=pre, phases=4),
        "force": lambda: P.emb_mex_force(E.forest, 19, E.links["cell"], E.links["dir"], E.links["q"], pop, out=F),
        "step": lambda: P.emb_lbm_step(E.forest, 19, E.links, 1.2, pop, out=out, pre=pre, phases=7),
    }
    ms = {}
    for name, fn in calls.items():
        fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms[name] = round(statistics.median(ts), 4)
    hbm = peaks()[0].get("hbm_gbs", 6800.0)
    cell_bytes = 19 * 4 * 2  # one population read and one written per direction and cell
    gbps = {k: ncell * cell_bytes / (ms[k] / 1e3) / 1e9 for k in ("stream", "collide")}
    whole = ms["step"] + ms["force"]
    return dict(workload=f"diff_112k: {len(t)} triangles, {ncell} finest cells, {E.links['q'].numel()} cut links, D3Q19",
                ms=ms, boundary_share=round((ms["bouzidi"] + ms["force"]) / whole, 4),
                stream_GBps=round(gbps["stream"], 1), collide_GBps=round(gbps["collide"], 1),
                hbm_frac=dict(stream=round(gbps["stream"] / hbm, 3), collide=round(gbps["collide"] / hbm, 3)),
                timing=f"CUDA events, median of {reps}; bytes = 2 x 19 x 4 per cell and pass")


def moving_leg(P, reps=10):
    """A moving body re-embedded every step (star_112k, root 16^3, levels 0..3, D3Q19):
    the mesh shifts by one root block along x and back, so every count of a plan holds
    and the planned replay applies.  Per step: emb_mesh_update, then either the per-call
    path (embed) or the captured graph of the planned replay; CUDA events, median."""
    import torch

    w = workload("star_112k")
    v, t = w.build_mesh()
    pos = [torch.from_numpy(v).cuda(), torch.from_numpy(v + np.float32(1.0 / w.R) * np.array([1, 0, 0], np.float32)).cuda()]
    tris = torch.from_numpy(t).cuda()
    mesh = P.emb_mesh_create(pos[0], tris, w.R)
    s = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(s):
        B = P.emb_batch_create([mesh], [w.levels], [w.band], [19], stream=s)
        P.emb_batch_capture(B, s)
        for name in ("per_call", "replay"):
            ts = []
            for r in range(reps + 2):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                P.emb_mesh_update(mesh, pos[r % 2], s)
                if name == "per_call":
                    P.embed(pos[r % 2], tris, w.R, w.levels, w.band, 19, mesh=mesh, check_status=False, stream=s)
                else:
                    P.emb_batch_launch(B, s)
                b.record(s)
                s.synchronize()
                if r >= 2:
                    ts.append(a.elapsed_time(b))
            out[name] = round(statistics.median(ts), 4)
        st = P.emb_status_get(s)
        # a body whose counts change every step (scaled by 0.97, 1.0, 1.03 about the
        # domain centre, in turn): the per-call path against one captured graph of a
        # replay planned with 30 % headroom
        from synth.meshes import snap
        scaled = [torch.from_numpy(snap((v.astype(np.float64) - 0.5) * f + 0.5)).cuda() for f in (0.97, 1.0, 1.03)]
        HB = P.emb_batch_create([mesh], [w.levels], [w.band], [19], stream=s, headroom=30)
        P.emb_batch_capture(HB, s)
        links = set()
        for name in ("per_call_scaled", "headroom_replay"):
            ts = []
            for r in range(reps + 3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                P.emb_mesh_update(mesh, scaled[r % 3], s)
                if name == "per_call_scaled":
                    P.embed(scaled[r % 3], tris, w.R, w.levels, w.band, 19, mesh=mesh, check_status=False, stream=s)
                else:
                    P.emb_batch_launch(HB, s)
                b.record(s)
                s.synchronize()
                if name == "headroom_replay" and r < 3:
                    links.add(P.emb_batch_counts(HB, 0, s)[1])
                if r >= 3:
                    ts.append(a.elapsed_time(b))
            out[name] = round(statistics.median(ts), 4)
        hst = P.emb_status_get(s)
    return dict(workload=f"star_112k shifted by one root block each step: {len(t)} triangles, D3Q19",
                per_call_ms=out["per_call"], replay_ms=out["replay"], speedup=round(out["per_call"] / out["replay"], 2),
                status=st, timing=f"mesh update + re-embedding per step, CUDA events, median of {reps}",
                headroom=dict(workload="star_112k scaled by 0.97, 1.0, 1.03 in turn (the counts change every step)",
                              per_call_ms=out["per_call_scaled"], headroom_replay_ms=out["headroom_replay"],
                              speedup=round(out["per_call_scaled"] / out["headroom_replay"], 2),
                              link_counts_seen=sorted(links), headroom_pct=30, status=hst))


def incremental_leg(P, reps=6):
    """A local deformation of the bench workload (the ~7.2M-triangle mesh, D3Q27): a cap
    of vertices pushed in and out along their radial directions, step after step.  The
    windowed re-embedding (reembed_window: a window forest of the root-block rows the
    change can reach, the triangles near it, emb_splice) against a full re-embedding
    through the per-call path.  Host wall clock around synchronised calls (both paths
    synchronise inside)."""
    import torch

    from synth import bump
    w = workload("star_7m")
    v, t = w.build_mesh()
    tt = torch.from_numpy(t).cuda()
    E = P.embed(torch.from_numpy(v).cuda(), tt, w.R, w.levels, w.band, 27)
    inc, full, sizes = [], [], []
    for i in range(reps + 2):
        v_new, moved = bump(v, (0.2, 1.0, 0.3), 0.995, 300 if i % 2 == 0 else -300)
        hit = np.isin(t, moved).any(axis=1)
        pts = np.concatenate([v[t[hit]].reshape(-1, 3), v_new[t[hit]].reshape(-1, 3)])
        lo, hi = np.floor(pts.min(axis=0) * w.R).astype(int), np.floor(pts.max(axis=0) * w.R).astype(int) + 1
        ext = (int(lo[1]), int(hi[1]), int(lo[2]), int(hi[2]))
        vn = torch.from_numpy(v_new).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.reembed_window(E, vn, ext, w.band)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        F = P.embed(vn, tt, w.R, w.levels, w.band, 27, check_watertight=False, check_status=False)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if i >= 2:
            inc.append(1e3 * (t1 - t0))
            full.append(1e3 * (t2 - t1))
            sizes.append(ext)
        same = F.links["q"].numel() == E.links["q"].numel()
        del F
        v = v_new
    st = P.emb_status_get()
    mi, mf = statistics.median(inc), statistics.median(full)
    return dict(workload=(f"star_7m ({len(t)} triangles, root 32^3, levels 0..4, D3Q27): a cap of {len(moved)} "
                          "vertices pushed by +-300 grid units per step"),
                changed_rows=f"y {sizes[-1][0]}..{sizes[-1][1]}, z {sizes[-1][2]}..{sizes[-1][3]} of {w.R}",
                incremental_ms=round(mi, 4), full_ms=round(mf, 4), speedup=round(mf / mi, 2),
                same_link_count=bool(same), status=st,
                timing=f"host wall clock around synchronised calls, median of {reps}")


def replay_leg(P, verts, tris, w, lattice, step_ms, reps=10):
    """The bench workload as a planned replay (a batch of one mesh, captured in a CUDA graph):
    the same kernels recompute the whole embedding from the triangle records, without the
    count read-backs of the per-call path (the counts come from the plan, made once outside
    the timing, and are checked on the device).  Reported beside the per-call step, not in
    place of it: it shows what the host round trips of the per-call path cost."""
    import torch
    mesh = P.emb_mesh_create(verts, tris, w.R, check_watertight=False)
    B = P.emb_batch_create([mesh], [w.levels], [w.band], [lattice])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        P.emb_batch_capture(B, s)
        P.emb_batch_launch(B, s)
        s.synchronize()
        ts = []
        flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")  # 256 MB, larger than L2
        for i in range(reps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            P.emb_batch_launch(B, s)
            b.record(s)
            s.synchronize()
            ts.append(a.elapsed_time(b))
        st = P.emb_status_get(s)
    med = statistics.median(ts)
    return dict(ms=round(med, 4), per_call_step_ms=round(step_ms, 4), host_round_trips_ms=round(step_ms - med, 4),
                status=st, timing=f"graph launch, CUDA events, median of {reps}, L2 flushed before each")


def ablation_leg(P, verts, tris, w, lattice, reps=3):
    """The paper's binning variants (Sec. 4: 'n', 'r', 'rc') on the bench workload: 'rc'
    = exact x-line filter and compacted id list (the default), 'r' = the filter's flags
    tested by the voxelizer without compaction, 'n' = no filter.  Median CUDA-event time
    of emb_bin + emb_voxelize per level, and the triangles the filter keeps per level."""
    import torch
    stream = torch.cuda.current_stream()
    out, kept = {}, []
    for name, mode in (("rc", P.EMB_BIN_FILTER_COMPACT), ("r", P.EMB_BIN_FILTER_ONLY), ("n", P.EMB_BIN_NO_FILTER)):
        runs = []
        for rep in range(reps + 1):
            mesh = P.emb_mesh_create(verts, tris, w.R, check_watertight=False)
            forest = P.emb_forest_root(w.R, w.levels)
            ev, keep = [], []
            for L in range(w.levels + 1):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                bins = P.emb_bin(mesh, forest, L, lattice, mode=mode)
                P.emb_voxelize(forest, bins, L)
                b.record(stream)
                ev.append((a, b))
                if L < w.levels:
                    P.emb_forest_refine(forest, L, P.emb_refine_flags(forest, bins, L, w.band))
                keep.append(bins)
            torch.cuda.synchronize()
            if rep > 0:
                runs.append([a.elapsed_time(b) for a, b in ev])
            if mode == P.EMB_BIN_FILTER_COMPACT and rep == reps:
                kept = [P.emb_bins_stats(bb)[0] for bb in keep]
            for bb in keep:
                bb.close()
        per_level = [statistics.median(r[L] for r in runs) for L in range(w.levels + 1)]
        out[name] = dict(ms_per_level=[round(x, 4) for x in per_level], ms_total=round(sum(per_level), 4))
    out["kept_per_level"] = kept
    out["triangles"] = len(tris)
    out["timing"] = "emb_bin + emb_voxelize per level, CUDA events, median of %d" % reps
    return out


def guard_leg(P, v, t, w, lattice, reps=10):
    """The paper's guard-cell voxelizer (binary32 nearest face, internal and external
    propagation) against the exact parity voxelizer on the finest level of the bench
    workload: median CUDA-event time of each on the same bins, and the cells on which
    the two disagree."""
    import torch
    stream = torch.cuda.current_stream()
    E = P.embed(v, t, w.R, w.levels, w.band, lattice, keep_bins=True, check_watertight=False)
    L = w.levels
    fin = E.bins[-1]
    exact = E.masks[L].clone()
    n = exact.numel()
    solid = torch.empty(n, dtype=torch.int64, device="cuda")
    guard = torch.empty(n, dtype=torch.int64, device="cuda")
    vox = torch.empty(n, dtype=torch.int64, device="cuda")

    def timed(fn):
        runs = []
        for rep in range(reps + 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            if rep >= 2:
                runs.append(a.elapsed_time(b))
        return statistics.median(runs)

    g_ms = timed(lambda: P.emb_voxelize_guard(E.forest, fin, solid, guard))
    e_ms = timed(lambda: P.emb_voxelize(E.forest, fin, L, vox))
    st = P.emb_status_get()

    def popc(x):
        return int(np.unpackbits(x.cpu().numpy().view(np.uint8)).sum())

    return dict(level=L, blocks=n, guard_ms=round(g_ms, 4), exact_ms=round(e_ms, 4),
                solid_cells_exact=popc(exact), guard_cells=popc(guard),
                cells_differing=popc(solid ^ exact), solid_only_in_guard=popc(solid & ~exact),
                solid_only_in_exact=popc(exact & ~solid), exact_rerun_identical=bool(torch.equal(vox, exact)),
                status=st, timing=f"CUDA events, median of {reps}; both on the finest bins of the step")


def batch_leg(P, reps=5):
    """The batched workload: 48 seeded radial meshes (triangle counts log-uniform in
    1e3..5e5, random rotations, radii 0.15..0.4), each in its own forest (root 8^3..24^3,
    2..4 levels, band 2, D3Q19).  Plain = the per-call path mesh after mesh on one stream;
    batched = the captured graph of the planned replay (autotuned launch shape).  Both
    start from triangle records already on the device."""
    import torch

    from synth import batch_meshes
    cases = batch_meshes(48)
    meshes = [P.emb_mesh_create(torch.from_numpy(c["verts"]), torch.from_numpy(c["tris"]), c["R"]) for c in cases]
    verts = [torch.from_numpy(c["verts"]).cuda() for c in cases]
    tris = [torch.from_numpy(c["tris"]).cuda() for c in cases]

    def plain_once():
        units = 0
        for c, m, v_, t_ in zip(cases, meshes, verts, tris):
            E = P.embed(v_, t_, c["R"], c["levels"], c["band"], c["lattice"], mesh=m, check_status=False)
            units += E.units()
        return units

    plain_once()
    torch.cuda.synchronize()
    pt = []
    for _ in range(reps):
        t0 = time.perf_counter()
        units = plain_once()
        torch.cuda.synchronize()
        pt.append(1e3 * (time.perf_counter() - t0))
    B = P.emb_batch_create(meshes, [c["levels"] for c in cases], [c["band"] for c in cases],
                           [c["lattice"] for c in cases])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        choice = P.emb_batch_autotune(B, s)
        P.emb_batch_capture(B, s)
        P.emb_batch_launch(B, s)
        s.synchronize()
        bt = []
        for _ in range(reps):
            t0 = time.perf_counter()
            P.emb_batch_launch(B, s)
            s.synchronize()
            bt.append(1e3 * (time.perf_counter() - t0))
        st_ = P.emb_status_get(s)
    bunits = sum(64 * sum(P.emb_batch_info(B, j)[0]) + P.emb_batch_info(B, j)[1] for j in range(len(cases)))
    pm, bm = statistics.median(pt), statistics.median(bt)
    return dict(workload=f"batch_48: 48 radial meshes, {sum(len(c['tris']) for c in cases)} triangles in total, "
                         f"roots 8^3..24^3, 2..4 levels, D3Q19",
                plain_ms=round(pm, 3), batched_ms=round(bm, 3), speedup=round(pm / bm, 2),
                plain_units_per_s=units / (pm / 1e3), batched_units_per_s=bunits / (bm / 1e3),
                same_units=bool(units == bunits), status=st_,
                autotuned=dict(streams=choice[0], tri_block=choice[1], link_ctas_per_sm=choice[2],
                               link_placement=["joint", "per mesh", "per mesh, low priority"][choice[3]]),
                timing="host wall clock around a synchronised run (the plain path synchronises inside)")


def e2e_leg(P, v, t, w, lattice, args, stream):
    """Same metric through the public API with host inputs and a host copy of the result:
    pinned host -> device copies of the mesh, the embedding, and the cut-link table (cell,
    dir, q) and the finest solid mask in pinned host memory, all inside the timed region.
    The library writes those outputs straight into the page-locked host buffers over the
    host link (the link kernel's stores, and one asynchronous copy of the mask), so no
    device -> host copy of the table follows the kernel.  The pinned buffers are allocated
    once, after a first embedding sizes them, as a caller that embeds repeatedly would;
    the step time is the median over the timed steps."""
    import torch

    hv = torch.from_numpy(v).pin_memory()
    ht = torch.from_numpy(t).pin_memory()
    h2d = hv.numel() * 4 + ht.numel() * 4
    # sizes from one embedding before the loop
    E0 = P.embed(hv.to("cuda"), ht.to("cuda"), w.R, w.levels, w.band, lattice, check_watertight=False)
    n, nm = E0.links["q"].numel(), E0.masks[-1].numel()
    del E0
    links_out = dict(cell=torch.empty(n, dtype=torch.int32, pin_memory=True),
                     dir=torch.empty(n, dtype=torch.uint8, pin_memory=True),
                     q=torch.empty(n, dtype=torch.float32, pin_memory=True),
                     tri=torch.empty(n, dtype=torch.int32, device="cuda"),  # the argmin faces stay on the device
                     count=torch.zeros(1, dtype=torch.int64, device="cuda"))
    mask_out = torch.empty(nm, dtype=torch.int64, pin_memory=True)
    times, units = [], []
    for i in range(args.warmup + max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dv = hv.to("cuda", non_blocking=True)
        dt = ht.to("cuda", non_blocking=True)
        E = P.embed(dv, dt, w.R, w.levels, w.band, lattice, check_watertight=False, check_status=False,
                    links_out=links_out, finest_mask_out=mask_out)
        torch.cuda.synchronize()
        dt_s = time.perf_counter() - t0
        if E.links["q"].numel() != n or E.masks[-1].numel() != nm:
            raise RuntimeError("the table changed size between steps")
        if i >= args.warmup:
            times.append(dt_s)
            units.append(E.units())
    d2h = n * (4 + 1 + 4) + nm * 8
    med = statistics.median(times)
    return dict(value=statistics.median(units) / med, unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                ms_per_step=1e3 * med, outputs="cell, dir, q and the finest mask written into page-locked host memory")


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
