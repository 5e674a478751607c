/*
 * emb.h -- C ABI of libemb: GB300 embedding of a closed triangle mesh into a
 * block-structured forest of octrees (arXiv 2512.01251).
 *
 * The library implements the data-parallel path of the paper's geometry module:
 * hierarchical spatial binning (Sec. 3.3), solid voxelization by ray casting
 * (Sec. 3.4, "Partial Surface Voxelization" and "External Cell Flag
 * Propagation"), near-wall refinement flags (Sec. 3.4, "Refinement Flagging"),
 * and the flattened link-length table for interpolated bounce-back (Sec. 3.4,
 * "Link-Length Computation"), plus the momentum-exchange force with Bouzidi
 * interpolation and the adjoint of q with respect to the vertices.
 *
 * Conventions shared by every call
 *   - Pointers named d_* are CUDA device pointers owned by the caller; the
 *     library never frees them.  Handles (emb_mesh, emb_forest, emb_bins) own
 *     library-allocated device memory, released by the matching *_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls enqueue work on it and return an immediate status for argument and
 *     launch errors; errors detected inside kernels are recorded in a device
 *     status word read (and cleared) by emb_status_get.  Calls that must size a
 *     library allocation (mesh creation, forest refinement, binning, link
 *     counting) synchronise the stream once to read a count back.
 *   - Integer frame: with R = r_o 2^k root blocks per axis (r_o odd), vertex
 *     coordinate v (a multiple of 2^-20 in (0,1)) maps to v 2^20 r_o.  Level L
 *     cells have size 2^(18-k-L) and centres at odd multiples of 2^(17-k-L);
 *     k + L <= 17 is required (EMB_ERR_RANGE otherwise).
 *   - Blocks of 4x4x4 cells; cell t = x + 4y + 16z inside a block (the LINEAR
 *     map of Alg. 3).  The blocks of a level are numbered in (z, y, x) order
 *     of their block coordinates; the global cell id at the finest level is
 *     block_id * 64 + t.
 *   - Lattice directions (index: vector), opposite pairs adjacent:
 *     0 rest; 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z;
 *     7 (1,1,0), 8 (-1,-1,0), 9 (1,-1,0), 10 (-1,1,0), 11 (1,0,1), 12 (-1,0,-1),
 *     13 (1,0,-1), 14 (-1,0,1), 15 (0,1,1), 16 (0,-1,-1), 17 (0,1,-1), 18 (0,-1,1);
 *     19 (1,1,1), 20 (-1,-1,-1), 21 (1,1,-1), 22 (-1,-1,1), 23 (1,-1,1),
 *     24 (-1,1,-1), 25 (-1,1,1), 26 (1,-1,-1).  D3Q19 uses 0..18, D3Q27 0..26.
 *   - Every inside/outside, crossing and overlap decision is exact (integer
 *     predicates with a fixed symbolic perturbation of the query points), so
 *     masks, flags, forests and link sets are deterministic and bit-exact.
 */
#ifndef EMB_H
#define EMB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t emb_status;
#define EMB_OK 0
#define EMB_ERR_BAD_INPUT (-1)      /* argument out of range, unsnapped vertex, bad triangle id */
#define EMB_ERR_NOT_WATERTIGHT (-2) /* an edge is not shared by exactly two oppositely oriented faces */
#define EMB_ERR_CAPACITY (-3)       /* caller buffer too small; the required size was written */
#define EMB_ERR_CUDA (-4)           /* a CUDA runtime call failed */
#define EMB_ERR_TIMEOUT (-5)        /* a bounded device wait gave up (reserved: no call of this
                                       library waits on the device) */
#define EMB_ERR_RANGE (-6)          /* the level is too fine for the integer frame */
#define EMB_ERR_STATE (-7)          /* call order violated, or an internal invariant failed */
#define EMB_ERR_BOUNDS (-8)         /* a library built with -DEMB_CHECK found an index out of
                                       range (the access was skipped; device status only) */

typedef struct emb_mesh_s *emb_mesh;
typedef struct emb_forest_s *emb_forest;
typedef struct emb_bins_s *emb_bins;

/* Human-readable name of a status code (static string). */
const char *emb_status_string(emb_status s);

/* Synchronises `stream`, then returns in *out the first error recorded by a
 * kernel since the last call (EMB_OK if none) and clears it. */
emb_status emb_status_get(void *stream, emb_status *out);

/* Writes the 27 lattice vectors (27 x 3 int32, host memory) in the order above. */
emb_status emb_directions(int32_t *h_out);

/* Diagnostics (no counterpart in the paper): number of kernels this library has
 * launched in the process so far, counted on the host at each launch site. */
emb_status emb_launch_count(int64_t *h_out);

/* Diagnostics for tests: evaluates the library's exact device predicates on n
 * caller-given queries (no counterpart in the paper; these are the decisions of
 * Sec. 3.3-3.4 taken in isolation, so that they can be checked against a host
 * evaluation on adversarial and extreme inputs).  d_in: n x 15 int64 per query
 * (device): a triangle A, B, C in frame units (9 values, each in [0, 2^25)), then
 *   EMB_PROBE_XLINE:   [9] unused, [10] y, [11] z of a +x line; hit = the perturbed
 *                      line crosses the triangle (filter and voxelizer test);
 *   EMB_PROBE_SEGMENT: [9..11] P, [12] direction 1..26, [13] h > 0; hit = the
 *                      perturbed segment P -> P + h c crosses the triangle, q = its
 *                      parameter rounded to float (the link kernel's exact rescan);
 *   EMB_PROBE_PAIR:    same query through the link kernel's per-pair path (32-bit
 *                      moments when every vertex is within 2^14 of P);
 *   EMB_PROBE_BOX:     [9..11] lo, [12..14] hi; hit = the triangle meets the closed
 *                      box (binning and refine-flag test).
 * d_hit: n int32 (0, 1, or -1 for a direction or h out of range); d_q: n floats (-1
 * where not hit).  Points and box corners within 2^25 of the triangle.  Enqueues only.
 * Errors: EMB_ERR_BAD_INPUT (kind, n < 0, null pointers with n > 0). */
#define EMB_PROBE_XLINE 0
#define EMB_PROBE_SEGMENT 1
#define EMB_PROBE_PAIR 2
#define EMB_PROBE_BOX 3
emb_status emb_probe_predicates(int32_t kind, const int64_t *d_in, int64_t n, int32_t *d_hit, float *d_q, void *stream);

/* ---------------------------------------------------------------- mesh ---- */
/* Geometry input (Sec. 3.1): a closed, oriented triangle mesh given as an index
 * list.  d_verts: V x 3 float32, each coordinate a multiple of 2^-20 strictly
 * inside (0,1); d_tris: T x 3 int32 vertex ids, counter-clockwise seen from
 * outside.  R: root blocks per axis of the forests this mesh will be embedded
 * in (fixes the integer frame).  check_watertight != 0 verifies on the GPU that
 * every directed edge occurs once and its reverse once (Sec. 3.4 requires a
 * watertight, non-self-intersecting surface).  Builds library-owned 48-byte
 * records {X,Y,Z,vertex id} x 3 per triangle.  Synchronises the stream.
 * Errors: EMB_ERR_BAD_INPUT, EMB_ERR_NOT_WATERTIGHT, EMB_ERR_RANGE, EMB_ERR_CUDA. */
emb_status emb_mesh_create(const float *d_verts, const int32_t *d_tris, int64_t V, int64_t T, int32_t R,
                           int32_t check_watertight, void *stream, emb_mesh *out);
void emb_mesh_destroy(emb_mesh m);

/* Moving geometry (the paper's future work, Sec. 5, re-embedding a moving body):
 * new positions for the same V vertices, same triangles.  d_verts: V x 3
 * float32 under the rules of emb_mesh_create.  Rewrites the mesh's records in
 * place on `stream`; enqueues one kernel, allocates nothing and does not
 * synchronise, so it can precede a batch replay (or be captured with one) every
 * step.  A coordinate off the 2^-20 grid or outside (0,1) leaves its record
 * unchanged and raises EMB_ERR_BAD_INPUT in the device status word.  Forests,
 * bins and link tables built before the call describe the old positions; a
 * batch replay recomputes everything and reports EMB_ERR_STATE on the device
 * when a count no longer matches its plan (re-create the batch then).
 * Errors (immediate): EMB_ERR_BAD_INPUT (null handle or pointer, V differs from
 * the mesh's), EMB_ERR_CUDA. */
emb_status emb_mesh_update(emb_mesh m, const float *d_verts, int64_t V, void *stream);

/* -------------------------------------------------------------- forest ---- */
/* Root grid of R^3 blocks (Sec. 3.2) with room for levels 0..max_level.
 * Errors: EMB_ERR_BAD_INPUT (R < 1, max_level < 0 or > 15), EMB_ERR_RANGE. */
emb_status emb_forest_root(int32_t R, int32_t max_level, void *stream, emb_forest *out);
void emb_forest_destroy(emb_forest f);

/* Creates level+1 from the refinement flags of `level` (d_flags: one uint8 per
 * level block, nonzero = refine): 8 children per flagged block, numbered in
 * (z, y, x) order, plus their lookup index (a rank bitmap of the level's dense block
 * positions, or a hash where there are more than 2^32 of them).  This is the forest harness
 * (the paper delegates it to its AMR pipeline, Sec. 3.2 steps 1-8); it keeps no
 * ghost/interface metadata.  Where the child level takes a rank bitmap the call
 * returns without waiting: the child count travels to a pinned host slot behind the
 * child keys, and the next call on this forest (any entry point that takes it) waits
 * for it first, except emb_bin / emb_bin_ex: below the finest level they are the x-line
 * filter alone (it does not depend on the blocks) and do not wait; at the finest level
 * they wait after enqueueing the filter.  So the GPU has work while the count travels.
 * With a hashed child level the call waits for the count itself.
 * Errors: EMB_ERR_STATE (level not the current finest, or beyond max_level). */
emb_status emb_forest_refine(emb_forest f, int32_t level, const uint8_t *d_flags, void *stream);

/* Number of blocks at `level` (host value; 0 if the level does not exist). */
emb_status emb_forest_num_blocks(emb_forest f, int32_t level, int64_t *h_out);

/* Copies the block coordinates (n x 3 int32: bx, by, bz) of `level` into d_out. */
emb_status emb_forest_blocks(emb_forest f, int32_t level, int32_t *d_out, void *stream);

/* Copies the neighbour table of `level` into d_out (n x 26 int32): entry
 * [b*26 + i-1] is the id of the block at offset c_i from block b, or -1 if it
 * does not exist at this level (Sec. 3.2: neighbour links over the full halo). */
emb_status emb_forest_neighbors(emb_forest f, int32_t level, int32_t *d_out, void *stream);

/* Copies the solid mask words of `level` (written by emb_voxelize) into d_out. */
emb_status emb_forest_masks(emb_forest f, int32_t level, uint64_t *d_out, void *stream);

/* ---------------------------------------------------------------- bins ---- */
/* Spatial binning on `level` (Sec. 3.3, steps 1-9 and Alg. 1-2):
 *  (1) filter: keeps the triangles crossed by at least one x-line through level
 *      cell centres (the 1-D ray-indicator filter, exact), as a compact id list
 *      in ascending order;
 *  (2) at the finest level of the forest (level == max_level): per-block bins in
 *      CSR form holding every non-degenerate triangle that overlaps the block box
 *      dilated by half a cell (Alg. 2 dilates bins by the cell size; a link from
 *      a cell centre, itself half a cell inside the block, reaches at most one
 *      cell further, so half a cell suffices), built by one counting pass that
 *      also lists the pairs, an exclusive scan and a scatter; ids within a bin
 *      are unordered.
 * `lattice` (19 or 27) is recorded for emb_cutlinks.  Enqueues only: the counts
 * stay on the device until emb_bins_stats, emb_bins_copy or emb_cutlinks reads
 * them (synchronising `stream`).  The finest bins start from a pair list of
 * 4 T + 2^20 entries; when that proves too small, the first of those readers
 * rebuilds them with the exact size before using them.
 * Errors: EMB_ERR_BAD_INPUT, EMB_ERR_STATE (level missing, mesh/forest frame mismatch). */
emb_status emb_bin(emb_mesh m, emb_forest f, int32_t level, int32_t lattice, void *stream, emb_bins *out);

/* emb_bin with a choice of the filter step, for the ablation of Sec. 4 (the
 * paper's binning variants 'n', 'r' and 'rc'):
 *   EMB_BIN_FILTER_COMPACT  exact x-line filter, compacted id list (emb_bin);
 *   EMB_BIN_FILTER_ONLY     the same filter, kept as per-triangle flags that the
 *                           voxelizer tests, without compaction ('r');
 *   EMB_BIN_NO_FILTER       every triangle goes to the voxelizer ('n').
 * The filter is exact, so all three give the same masks; only the work differs.
 * Errors: those of emb_bin, and EMB_ERR_BAD_INPUT for an unknown mode. */
#define EMB_BIN_FILTER_COMPACT 0
#define EMB_BIN_FILTER_ONLY 1
#define EMB_BIN_NO_FILTER 2
emb_status emb_bin_ex(emb_mesh m, emb_forest f, int32_t level, int32_t lattice, int32_t mode, void *stream,
                      emb_bins *out);
void emb_bins_destroy(emb_bins b);

/* Host statistics: filtered triangles and (at the finest level) bin entries.
 * Synchronises the stream of emb_bin on first use. */
emb_status emb_bins_stats(emb_bins b, int64_t *h_filtered, int64_t *h_pairs);

/* Copies the bins out (Sec. 3.3's bins_face_ids / _N arrays): d_filtered gets the
 * filtered triangle ids (h_filtered entries), d_off the CSR offsets (blocks + 1
 * entries) and d_ent the triangle ids of every bin (h_pairs entries, unordered
 * within a bin).  Any pointer may be NULL; offsets exist only at the finest level. */
emb_status emb_bins_copy(emb_bins b, uint32_t *d_filtered, uint32_t *d_off, uint32_t *d_ent, void *stream);

/* ------------------------------------------------------------ voxelize ---- */
/* Solid voxelization of `level` (Sec. 3.4): a cell is solid iff its centre is
 * inside the surface.  Each filtered triangle casts the +x lines through the
 * level's cell centres that cross it; the crossing's block records which of its
 * four cells on that line lie before the hit and flips the line's block parity.
 * A segmented suffix-XOR of the line parities along each (y, z) row of blocks
 * then completes every line (the role of the external propagation of Alg. 4).
 * Writes one uint64 per level block (bit t = cell t solid) into d_solid_mask
 * (may be NULL; device memory or page-locked host memory, EMB_ERR_BAD_INPUT for
 * pageable memory) and keeps a copy in the forest.
 * Exact for any forest: a crossing inside a block position the level does not have
 * (a region left coarser) is carried along its row to the blocks on its left.
 * Errors: EMB_ERR_STATE (bins of another level, missing level). */
emb_status emb_voxelize(emb_forest f, emb_bins b, int32_t level, uint64_t *d_solid_mask, void *stream);

/* The paper's own voxelizer, for the ablation of the exact one above (Sec. 3.4,
 * "Partial Surface Voxelization" with Alg. 3, and "External Cell Flag
 * Propagation"), on the finest level of the forest (`b` = its bins):
 *  (1) every cell takes the nearest face of its block's bin that its +x line meets,
 *      in binary32: signed distance d = ((v1 - c) . n) / n_x to the face's plane
 *      (n the unit normal), point-in-face by overlap of the face with a box of
 *      half-width 2^-23 around the line, equal |d| to the lowest face id; the cell
 *      is solid if n_x d > 0, a guard otherwise, untouched if no face is met;
 *  (2) internal propagation along x inside each block (three rounds: a fluid cell
 *      next to a guard becomes a guard, then a non-guard cell next to a solid
 *      becomes solid);
 *  (3) external propagation along +x, then (max_level > 0) along -x: each run of
 *      consecutive blocks is walked from its first block, a solid status turning
 *      the next block's row solid except at guards; a run whose first block borders
 *      a hole left by a coarser block with a solid cell (the masks of the coarser
 *      levels decide) starts from the solid.
 * d_solid_mask gets the solid cells (the paper's masks once guards turn back into
 * fluid), d_guard_mask the guard cells, one uint64 per finest block each, distinct
 * device buffers owned by the caller.  The forest's own masks are not changed.
 * Enqueues only (after completing the bins, as emb_cutlinks does).
 * Errors: EMB_ERR_BAD_INPUT (NULL or equal outputs), EMB_ERR_STATE (bins of another
 * level, coarser masks missing; on the device: a bin entry outside the mesh). */
emb_status emb_voxelize_guard(emb_forest f, emb_bins b, uint64_t *d_solid_mask, uint64_t *d_guard_mask,
                              void *stream);

/* -------------------------------------------------------------- refine ---- */
/* Near-wall refinement flags of `level` < max_level (Sec. 3.4, "Refinement
 * Flagging"; near-wall criterion d_spec): flag = some triangle overlaps the
 * closed block box dilated by (rho_L - 1/2) cells, where rho = band at level
 * max_level-1 and rho_L = max(band, rho_{L+1}/2 + 5/2) above it.  This keeps the
 * 2:1 balance of Sec. 3.2 and leaves every unrefined block free of the surface.
 * d_flags: one uint8 per level block (1 = refine), overwritten.
 * Errors: EMB_ERR_BAD_INPUT (band < 1), EMB_ERR_STATE, EMB_ERR_RANGE. */
emb_status emb_refine_flags(emb_forest f, emb_bins b, int32_t level, int32_t band, uint8_t *d_flags,
                            void *stream);

/* The paper's own refinement rules for `level` < max_level (Sec. 3.4, "Refinement
 * Flagging and Propagation", Eq. N_prop), an alternative to emb_refine_flags.
 * From the level's masks (emb_voxelize first): a block is solid if one of its cells
 * is solid, fully fluid otherwise; solid blocks with a fully fluid neighbour form the
 * solid boundary and are marked; every block next to one is marked; then
 * N_prop = 1 + floor(d_spec R / sqrt(2)) propagation rounds (Eq. N_prop with the
 * block length 1/(R 2^L): its 2^L factors cancel) mark each unmarked block next to a
 * marked one, fully fluid blocks in every round and solid blocks in the first only
 * (two layers into the body).  Blocks on the refinement interface (an in-domain
 * neighbour position without a block of the level) are never marked.  d_spec:
 * near-wall distance in units of the unit domain, >= 0.  Unlike the distance rule,
 * unrefined blocks may contain surface; the voxelizer and the cut links handle that
 * (a neighbour cell in a missing block counts as fluid).  d_flags: one uint8 per
 * level block, overwritten.  Needs no bins.
 * Errors: EMB_ERR_BAD_INPUT (d_spec negative or not finite, null d_flags),
 * EMB_ERR_STATE (level not the finest built, or not voxelized). */
emb_status emb_refine_flags_paper(emb_forest f, int32_t level, double d_spec, uint8_t *d_flags, void *stream);

/* ------------------------------------------------- incremental re-embedding ---- */
/* A window of root-block rows: the root blocks with y0 <= by < y1 and z0 <= bz < z1,
 * every bx (0 <= y0 < y1 <= R, 0 <= z0 < z1 <= R).  A forest started from a window
 * is embedded by the ordinary calls (emb_bin ... emb_cutlinks); its x-rows of cells are
 * whole, so the voxelizer's row parity is exact inside it.  The paper names moving
 * geometry as future work (Sec. 5); this is the region-limited re-embedding a
 * locally moving or deforming surface needs.  Errors as emb_forest_root, plus
 * EMB_ERR_BAD_INPUT for an empty or out-of-range window. */
emb_status emb_forest_root_window(int32_t R, int32_t max_level, int32_t y0, int32_t y1, int32_t z0, int32_t z1,
                                  void *stream, emb_forest *out);

/* The triangles of m whose bounding box meets the slab ylo <= y <= yhi, zlo <= z <= zhi
 * (frame units, the integer coordinates of the records: a vertex coordinate v maps to
 * v 2^20 r_o with R = r_o 2^k), as a new mesh handle for embedding a window (its
 * records are copies, in the order of m; the subset is not closed, which the window's
 * whole x-rows do not need).  d_map (device, optional, map_capacity entries) receives
 * for each subset triangle its id in m; *h_count (host) the subset size.  Synchronises.
 * Errors: EMB_ERR_BAD_INPUT, EMB_ERR_CAPACITY (d_map too small; nothing created),
 * EMB_ERR_STATE (no triangle meets the slab). */
emb_status emb_mesh_subset(emb_mesh m, int64_t ylo, int64_t yhi, int64_t zlo, int64_t zhi, int32_t *d_map,
                           int64_t map_capacity, void *stream, emb_mesh *out, int64_t *h_count);

/* Splices the embedding of a window forest w into the forest f (same R and levels,
 * both refined to their finest level and voxelized on every level): on every level
 * the blocks of f whose root ancestor lies in the inner window [y0, y1) x [z0, z1)
 * (all bx) are replaced by the blocks of w there, with their solid masks, in (z, y, x)
 * order; f's level index is rebuilt and its neighbour table and link candidates are
 * dropped.  The link tables (sorted by (cell, dir), cells numbered on the finest level
 * of their own forest) are merged into o_* (device, capacity entries): the links of f
 * outside the inner window and those of w inside it, renumbered to the merged finest
 * level, in (cell, dir) order; w_tri_map (device, optional) maps w's triangle ids to
 * the caller's (w was embedded from a subset of the triangles).  *h_count (host)
 * receives the merged link count.  The result equals an embedding of the whole mesh
 * when every change of the mesh since f was embedded lies inside the inner window
 * widened by 2 root blocks in y and z, the window of w holds the inner window widened
 * by 1 root block, and w was embedded from every triangle that meets the window of w
 * widened by 2 root blocks (refine dilations reach at most 1.2 root blocks, a link one
 * finest cell).  Synchronises (the merged counts size the levels).
 * Errors: EMB_ERR_BAD_INPUT, EMB_ERR_STATE (forests not matching, not refined or not
 * voxelized), EMB_ERR_CAPACITY (nothing written to o_*; f already spliced). */
emb_status emb_splice(emb_forest f, emb_forest w, int32_t y0, int32_t y1, int32_t z0, int32_t z1,
                      const int32_t *f_cell, const uint8_t *f_dir, const float *f_q, const int32_t *f_tri, int64_t f_n,
                      const int32_t *w_cell, const uint8_t *w_dir, const float *w_q, const int32_t *w_tri, int64_t w_n,
                      const int32_t *w_tri_map, int32_t *o_cell, uint8_t *o_dir, float *o_q, int32_t *o_tri,
                      int64_t capacity, int64_t *h_count, void *stream);

/* ------------------------------------------------------------ cut links ---- */
/* Number of cut links at the finest level for `lattice` (19 or 27): pairs
 * (fluid cell, direction i) whose neighbour along c_i is solid (Sec. 3.4,
 * "Boundary Cell Identification").  Needs emb_voxelize of the finest level.
 * Synchronises; the count is returned in *h_count. */
emb_status emb_cutlinks_count(emb_forest f, int32_t lattice, int64_t *h_count, void *stream);

/* The same work as emb_cutlinks_count (the finest level's neighbour table and the
 * candidate cells of `lattice`), enqueued on `stream` without reading the count back:
 * nothing synchronises.  A later emb_cutlinks on the same forest and lattice reuses
 * it; emb_cutlinks_count afterwards only reads the count.  Errors: EMB_ERR_BAD_INPUT
 * (lattice), EMB_ERR_STATE (finest level not voxelized). */
emb_status emb_cutlinks_prepare(emb_forest f, int32_t lattice, void *stream);

/* The flat link-length table (Sec. 3.4, "Link-Length Computation"): for every
 * cut link, d_cell = finest cell id, d_dir = direction, d_q = distance from the
 * cell centre to the nearest crossed face along the link divided by the link
 * length (in [0,1]), d_tri = that face's triangle id (lowest id on exact ties).
 * Ordered by (cell, dir).  `b` must be the bins of the finest level.  *d_count
 * (device int64, may be NULL) receives the number of links.  The call reads nothing
 * back unless the candidates have yet to be built (it then builds them without a
 * read-back, as emb_cutlinks_prepare does): so the host does not wait for the GPU.
 * If the count exceeds `capacity`: when the count is already known on the host
 * (emb_cutlinks_count before), nothing is enqueued but the status and count writes,
 * and EMB_ERR_CAPACITY is returned; otherwise the links at table positions below
 * `capacity` are written, none past it, *d_count still receives the required size
 * and the device status becomes EMB_ERR_CAPACITY (read it with emb_status_get).
 * A finest-level bin may hold at most 2^24 triangles (16,777,216 faces overlapping
 * one block); the links of a block with a larger bin are not written and the device
 * status becomes EMB_ERR_CAPACITY (refine further so that the bins shrink).
 * The five output buffers may be device memory or page-locked host memory (e.g.
 * cudaHostAlloc): the kernel then writes the table straight into host memory over the
 * host link, with no copy after it.  Any other host memory (pageable) is refused with
 * EMB_ERR_BAD_INPUT before anything is enqueued. */
emb_status emb_cutlinks(emb_forest f, emb_bins b, int32_t lattice, int32_t *d_cell, uint8_t *d_dir,
                        float *d_q, int32_t *d_tri, int64_t capacity, int64_t *d_count, void *stream);

/* -------------------------------------------------- force and adjoints ---- */
/* Momentum-exchange force on the body (Sec. 2.2 cites momentum exchange and
 * Bouzidi interpolated bounce-back; linear rule): per link (x_f, i, q),
 *   F += c_i (f_i(x_f) + g),  g = 2q f_i(x_f) + (1-2q) f_i(x_f - c_i)       (q < 1/2)
 *                             g = f_i(x_f)/(2q) + (2q-1)/(2q) f_-i(x_f)     (q >= 1/2)
 *                             g = f_i(x_f)  when q < 1/2 and x_f - c_i is not a
 *                                           fluid cell of the finest level.
 * d_pop: D3Q19/D3Q27 populations (post-collision), layout [Q][pop_stride]
 * indexed by finest cell id (pop_stride >= 64 * blocks).  d_F: 3 floats.
 * Deterministic fixed-order reduction (no float atomics). */
emb_status emb_mex_force(emb_forest f, int32_t lattice, const int32_t *d_cell, const uint8_t *d_dir,
                         const float *d_q, int64_t n, const float *d_pop, int64_t pop_stride, float *d_F,
                         void *stream);

/* d_gq[k] = d_gF . dF/dq_k for the force above (d_gF: 3 floats). */
emb_status emb_mex_force_backward(emb_forest f, int32_t lattice, const int32_t *d_cell, const uint8_t *d_dir,
                                  const float *d_q, int64_t n, const float *d_pop, int64_t pop_stride,
                                  const float *d_gF, float *d_gq, void *stream);

/* Allocation-free variant of emb_mex_force, for callers that cannot call
 * cudaMalloc: a solver time loop that reserved all device memory up front through
 * its own pool, or code that must not pay a driver allocation (latency, implicit
 * device synchronisation) inside a time step.  The paper has no counterpart; this
 * is a deployment convenience.  Same arguments and result as emb_mex_force, within
 * float rounding: the per-CTA partial sums (one per 256 links) go to a fixed
 * 192 KB array inside the library instead of a stream-ordered allocation, so the
 * partial sums are grouped differently.  The call allocates nothing, and nothing in
 * the array needs to start at zero (each call writes every partial it reads).
 * Limits and rules:
 *   - n <= 2,097,152 links, else EMB_ERR_CAPACITY before any work is enqueued;
 *   - the finest level's neighbour table must already exist, built by
 *     emb_cutlinks_count, emb_cutlinks, emb_mex_force or emb_forest_neighbors on
 *     this forest; else EMB_ERR_STATE;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture;
 *   - all calls share the one array, so calls that overlap on the GPU (other
 *     streams, other threads) race: serialise them;
 *   - the looked-up address belongs to the device's primary context: after
 *     cudaDeviceReset (or anything else that destroys that context) the next call
 *     looks it up again, because the library keys its cache on the context. */
emb_status emb_mex_force_noalloc(emb_forest f, int32_t lattice, const int32_t *d_cell, const uint8_t *d_dir,
                                 const float *d_q, int64_t n, const float *d_pop, int64_t pop_stride, float *d_F,
                                 void *stream);

/* ------------------------------------------------------------- solver ---- */
/* One lattice-Boltzmann step on the finest level, the consumer of the link table
 * (Sec. 2.2: interpolated bounce-back with the link fractions q; the paper cites
 * the method and prints no formula).  Populations are SoA float32, pop[i * stride
 * + cell] for the lattice's directions (order of emb_directions), cell = block *
 * 64 + x + 4 y + 16 z on the finest level; d_pop holds post-collision values at t,
 * d_pop_out receives them at t + 1, d_pre is caller scratch of the same size; the
 * three buffers must differ.  phases (bits, 7 = the whole step): 1 pull streaming
 * into d_pre (from the cell x - c_i when it is a fluid cell of the level, the cell's
 * own value when its block is missing: zero gradient at the edge of the level, the
 * coupling to coarser levels being out of scope); 2 at every cut link (x, d, q),
 * the population entering x against c_d by the linear Bouzidi rule of
 * emb_mex_force; 4 BGK collision with relaxation omega in [0, 2) and the standard
 * D3Q19 / D3Q27 weights at fluid cells, 0 at solid ones.  The link table is the one
 * of emb_cutlinks for this forest and lattice.  Enqueues only (builds the finest
 * neighbour table on first use).
 * Errors: EMB_ERR_BAD_INPUT (lattice, omega, phases, stride, aliasing, null
 * pointers; device status for a link outside the level), EMB_ERR_STATE (no finest
 * masks). */
emb_status emb_lbm_step(emb_forest f, int32_t lattice, const int32_t *d_cell, const uint8_t *d_dir, const float *d_q,
                        int64_t n_links, float omega, const float *d_pop, float *d_pre, float *d_pop_out,
                        int64_t pop_stride, int32_t phases, void *stream);

/* Adjoint of the link table with respect to the vertex positions (world
 * units): d_gverts (V x 3 float32, overwritten) = sum_k d_gq[k] dq_k/dV with
 * dq/dV_j = lambda_j n / (h n.c) for the three vertices of link k's triangle
 * (lambda: barycentric coordinates of the hit point, n: face normal, h: cell
 * size).  Summed per vertex in link order (segmented, no float atomics). */
emb_status emb_cutlinks_backward(emb_mesh m, emb_forest f, const int32_t *d_cell, const uint8_t *d_dir,
                                 const float *d_q, const int32_t *d_tri, int64_t n, const float *d_gq,
                                 float *d_gverts, void *stream);

/* --------------------------------------------------------------- batch ---- */
/* Batched embedding of up to 64 meshes (no counterpart in the paper, which embeds
 * one geometry at a time; this serves workloads with many bodies).
 *
 * emb_batch_create plans: it embeds every mesh once through the per-call path
 * above (synchronising), records every count, and allocates every buffer a replay
 * needs.  meshes[j] is used by reference (keep it alive); levels[j] is the finest
 * level, bands[j] the near-wall band, lattices[j] 19 or 27.
 *
 * emb_batch_run replays the whole batch with no allocation and no host
 * synchronisation: per-mesh pipelines on several internal streams, every count
 * recomputed on the device checked against the plan (device status
 * EMB_ERR_STATE on a difference, e.g. moved geometry), and the cut links of all
 * meshes either from one persistent kernel launch over a shared (mesh, block)
 * work queue after all pipelines ("joint" placement) or from one launch per mesh
 * on that mesh's stream right after its pipeline, its grid sized to the mesh's
 * work ("per-mesh" placement, which overlaps link work with other meshes'
 * pipelines).  Results are identical to the per-call path in either placement.
 * `stream` must not be the legacy default stream for emb_batch_capture.
 *
 * emb_batch_capture records emb_batch_run into a CUDA graph; emb_batch_launch
 * replays that graph on `stream`.
 *
 * emb_batch_autotune times a small set of launch shapes on this batch (as captured
 * graphs when `stream` can be captured, else as stream launches) and keeps the
 * fastest; h_choice (4 int32, may be NULL) receives the chosen stream count
 * (1..32), thread-block size of the triangle-parallel kernels (128, 256 or 512),
 * resident link CTAs per SM (0 = as many as fit) and link placement (0 joint,
 * 1 per mesh on its pipeline's stream, 2 per mesh on a low-priority stream of its
 * own, so that the link kernels yield SMs to the pipelines still running).  It synchronises and drops a captured graph.
 * A tuned shape is cached under (SM count, floor(log2) of the batch's triangles,
 * floor(log2) of its mesh count, largest lattice); a later batch with the same key takes
 * the cached shape without timing.  With the environment variable EMB_TUNE_CACHE set to
 * a file path, the cache is read from that file at first use and rewritten after every
 * timing run (plain text, one line of 8 integers per key; lines that name no valid
 * shape are ignored; a file that cannot be opened only disables persistence).
 * emb_batch_autotune_ex does the same with `flags` (EMB_TUNE_FORCE: time even when a
 * shape is cached; other bits: EMB_ERR_BAD_INPUT) and h_choice of 5 int32 (may be
 * NULL): the 4 values above and 1 when the shape came from the cache, else 0.
 * emb_batch_autotune is emb_batch_autotune_ex with flags 0 and the first 4 values.
 * emb_batch_configure
 * sets such a 4-value shape directly (host array; EMB_ERR_BAD_INPUT outside the
 * ranges above) and drops a captured graph; it enqueues nothing.
 *
 * emb_batch_create_ex is emb_batch_create with `headroom` percent (0..1000) of room in
 * the replay's buffers (a replay whose buffers carry headroom; moving geometry, Sec. 5).
 * Every planned count becomes a capacity of count x (1 + headroom/100) + 64: flagged
 * blocks per refined level (8 child blocks each), bin entries, blocks with links and
 * links.  A replay then accepts any counts up to those capacities: each level's block
 * count is formed and read on the device, and a count above its capacity sets
 * EMB_ERR_CAPACITY (the results are then incomplete, never out of bounds).  With
 * headroom 0 the counts must match the plan exactly (EMB_ERR_STATE otherwise).
 * emb_batch_counts: the blocks per level (levels[j] + 1 int64) and links of mesh j in
 * the last replay (host arrays, either may be NULL); with headroom they are read from the
 * device, which synchronises `stream`.
 *
 * emb_batch_info: planned blocks per level (levels[j] + 1 int64) and link count of
 * mesh j (host): the capacities of a batch with headroom.  emb_batch_results copies mesh
 * j's results of the last replay into caller buffers (any pointer may be NULL), as many
 * as emb_batch_counts reports (with headroom it reads them, synchronising `stream`): the
 * solid mask words and block coordinates (bx, by, bz int32) of `level`, and the cut-link
 * table. */
typedef struct emb_batch_s *emb_batch;
emb_status emb_batch_create(const emb_mesh *meshes, const int32_t *levels, const int32_t *bands,
                            const int32_t *lattices, int32_t n, void *stream, emb_batch *out);
emb_status emb_batch_create_ex(const emb_mesh *meshes, const int32_t *levels, const int32_t *bands,
                               const int32_t *lattices, int32_t n, int32_t headroom, void *stream, emb_batch *out);
emb_status emb_batch_counts(emb_batch b, int32_t j, void *stream, int64_t *h_blocks, int64_t *h_links);
emb_status emb_batch_run(emb_batch b, void *stream);
emb_status emb_batch_capture(emb_batch b, void *stream);
emb_status emb_batch_launch(emb_batch b, void *stream);
#define EMB_TUNE_FORCE 1
emb_status emb_batch_autotune(emb_batch b, void *stream, int32_t *h_choice);
emb_status emb_batch_autotune_ex(emb_batch b, void *stream, int32_t flags, int32_t *h_choice);
emb_status emb_batch_configure(emb_batch b, const int32_t *h_choice);
emb_status emb_batch_info(emb_batch b, int32_t j, int64_t *h_blocks, int64_t *h_links);
emb_status emb_batch_results(emb_batch b, int32_t j, int32_t level, uint64_t *d_mask, int32_t *d_blocks,
                             int32_t *d_cell, uint8_t *d_dir, float *d_q, int32_t *d_tri, void *stream);
void emb_batch_destroy(emb_batch b);

#ifdef __cplusplus
}
#endif

#endif /* EMB_H */
