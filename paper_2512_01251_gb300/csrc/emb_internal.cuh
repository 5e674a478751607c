// Internal definitions shared by the translation units of libemb (sm_103a).
//
// Holds the handle layouts, the device status word, the level hash and the
// exact integer predicates used by the kernels.  Predicates evaluate signs in
// int64 / __int128 with the query point pushed by (e, e^2, e^3), e -> 0+
// (simulation of simplicity), so that no query point ever lies on a plane,
// edge or vertex of the mesh and every decision has one answer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/emb.h"

#define EMB_MAX_LEVELS 16

typedef __int128 i128;

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
#define EMB_CUDA_TRY(expr)                                 \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) {                           \
            emb_note_cuda_error(_e, #expr, __FILE__, __LINE__); \
            return EMB_ERR_CUDA;                           \
        }                                                  \
    } while (0)

void emb_note_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Every kernel launch goes through EMB_LAUNCH((kernel), grid, block, smem, stream)(args), which
// bumps a host-side counter read by emb_launch_count.
void emb_count_launch();
#define EMB_STRIP(...) __VA_ARGS__
#define EMB_LAUNCH(kern, ...) emb_count_launch(), EMB_STRIP kern<<<__VA_ARGS__>>>
int *emb_status_word();  // device pointer of the current device's status word (lazily created)
// Stream-ordered allocation from the library's memory pool of the current device.  The
// pool keeps freed memory for reuse instead of returning it to the driver at every
// synchronisation (the default pool's behaviour), so a call that follows a host
// synchronisation does not map fresh pages for its scratch.
cudaError_t emb_malloc_raw(void **p, size_t bytes, cudaStream_t s);
template <class T>
static inline cudaError_t emb_malloc_async(T **p, size_t bytes, cudaStream_t s)
{
    return emb_malloc_raw((void **)p, bytes, s);
}
cudaStream_t emb_stream(void *s);

__device__ __forceinline__ void emb_set_status(int *st, int code)
{
    atomicCAS(st, 0, code);
}

// Bounds mode.  A library built with -DEMB_CHECK checks each index that a kernel
// derives from data (block ids from the level index or the neighbour table, work-item
// blocks, bin triangle ids) before it is used: one out of range records
// EMB_ERR_BOUNDS in the device status word and the access is skipped, so a bad index
// shows up as a status instead of a fault.  The default build compiles the checks out.
#ifdef EMB_CHECK
__device__ __forceinline__ bool emb_ck(uint64_t i, uint64_t n, int *st)
{
    if (i < n) return true;
    if (st) emb_set_status(st, EMB_ERR_BOUNDS);
    return false;
}
#else
__device__ __forceinline__ bool emb_ck(uint64_t, uint64_t, int *) { return true; }
#endif

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct emb_mesh_s {
    int32_t R, r_o, k;
    int64_t V, T;
    int4 *rec;      // T x 3 records {X, Y, Z, vertex id}
    int device;
};

struct EmbLevel {
    int64_t n = 0;
    int64_t nb_axis = 0;       // blocks per axis at this level (R << L)
    uint64_t *key = nullptr;   // block keys, ascending ((bz << 42) | (by << 21) | bx)
    uint64_t *hkey = nullptr;  // open-addressing hash: key -> block id
    int32_t *hval = nullptr;
    int64_t hcap = 0;          // power of two
    uint64_t *mask = nullptr;  // solid mask per block (after emb_voxelize)
    int32_t *nbr = nullptr;    // n x 26 neighbour ids (built on demand)
    // rank bitmap over the dense (bz, by, bx) positions of the level: bit = block exists;
    // blocks are numbered in that linear order, so a block's id is the rank of its bit
    uint64_t *bits = nullptr;
    uint32_t *wpre = nullptr;  // exclusive popcount prefix per 64-bit word
    int mask_valid = 0;
    // a replay with headroom: n is the capacity, *d_n (device) the blocks of this replay;
    // passes over the level's blocks stop at min(n, *d_n)
    const uint32_t *d_n = nullptr;
};

__device__ __forceinline__ int64_t emb_count(int64_t n, const uint32_t *d_n)
{
    return d_n && (int64_t)*d_n < n ? (int64_t)*d_n : n;
}

#define EMB_BITMAP_MAX_BITS (1ll << 32)

// Block lookup of one level, passed by value to kernels: the rank bitmap when it
// exists (two loads, L2-resident at the sizes used here), else the hash.
struct EmbLookup {
    const uint64_t *hkey;
    const int32_t *hval;
    int64_t hcap;
    const uint64_t *bits;
    const uint32_t *wpre;
    int64_t nb;
    int64_t n;  // blocks of the level (ids below n)
    int *st;    // device status word (bounds mode)
};

static inline EmbLookup emb_lookup_of(const EmbLevel &lv)
{
    EmbLookup l;
    l.hkey = lv.hkey;
    l.hval = lv.hval;
    l.hcap = lv.hcap;
    l.bits = lv.bits;
    l.wpre = lv.wpre;
    l.nb = lv.nb_axis;
    l.n = lv.n;
    l.st = emb_status_word();
    return l;
}

struct emb_forest_s {
    int32_t R, r_o, k, max_level, top;
    EmbLevel lv[EMB_MAX_LEVELS];
    // cut-link candidates at the finest level (built by emb_cutlinks_count / emb_cutlinks)
    uint64_t *cand = nullptr;     // per finest block x 26 directions: fluid cells whose neighbour along c_d is solid
    uint32_t *blk_off = nullptr;  // per finest block: exclusive link offset (n+1 entries)
    uint32_t *work = nullptr;     // ids of finest blocks with at least one link; count at work_n[0]
    uint32_t *work_n = nullptr;
    unsigned int *next = nullptr; // work-queue cursor of the persistent link kernel
    int32_t cand_lattice = 0;
    int64_t n_links = -1;
    int device;
    // pinned slot for reading the flagged count back while the child level is built
    int rb_slot = -1;
    uint64_t *rb_h = nullptr;
    cudaEvent_t rb_ev = nullptr;
    // the level whose block count is still on its way to rb_h (-1: none); taken by
    // emb_forest_settle, which every entry point that needs a forest's counts calls
    // before it uses them
    int32_t n_pending = -1;
};

struct emb_bins_s {
    emb_mesh m;
    emb_forest f;
    int32_t level, lattice;
    cudaStream_t s = nullptr;   // stream of emb_bin (for reading the counts back)
    uint32_t *flist = nullptr;  // filtered triangle ids (ascending), T + 1 entries
    uint32_t *keep = nullptr;   // filter mode without compaction: per-triangle filter flags
    uint32_t *off = nullptr;    // finest level only: CSR offsets (n_blocks + 1)
    uint32_t *ent = nullptr;    // triangle ids, ent_cap entries
    uint64_t ent_cap = 0;
    uint64_t list_cap = 0;      // capacity of the pair list used by emb_bin
    // device counts: filtered triangles, bin entries (uint32 each), pair-list requests (uint64)
    unsigned char *dcount = nullptr;
    // host copies, valid once `known` (emb_bins_sync)
    bool known = false;
    int64_t nf = 0, npairs = 0;
    // pinned slot the counts are copied into as soon as the bins are enqueued
    int rb_slot = -1;
    uint64_t *rb_h = nullptr;
    cudaEvent_t rb_ev = nullptr;
};
// Reads the counts of b back (synchronising b's stream) and, at the finest level,
// redoes the bins with an exact pair list if the first one was too small.
emb_status emb_bins_sync(emb_bins b);

// Geometry of one level in frame units.
struct LevelGeom {
    long long h, half, W;  // cell size, half cell, block width (powers of two)
    long long ncell;       // cells per axis
    long long nb;          // blocks per axis
    int lh, lW;            // log2 h, log2 W
};

static inline LevelGeom level_geom(const emb_forest_s *f, int L)
{
    LevelGeom g;
    g.lh = 18 - f->k - L;
    g.lW = g.lh + 2;
    g.h = 1ll << g.lh;
    g.half = g.h >> 1;
    g.W = 4 * g.h;
    g.nb = (long long)f->R << L;
    g.ncell = 4 * g.nb;
    return g;
}

// ---------------------------------------------------------------------------
// small host helpers (defined in emb_common.cu)
// ---------------------------------------------------------------------------
// Waits for a block count emb_forest_refine left on its way back, and stores it
// (emb_forest.cu).
emb_status emb_forest_settle(emb_forest f);
#define EMB_SETTLE(f_)                                         \
    do {                                                       \
        const emb_status rs_ = emb_forest_settle(f_);          \
        if (rs_ != EMB_OK) return rs_;                         \
    } while (0)
// Scans: d_out gets n + 1 entries (exclusive sums, total at n).  emb_scan_u32
// allocates its scratch and can read the total back (synchronising); emb_scan_into
// only enqueues, with emb_scan_tmp_words(n) words of caller scratch.
emb_status emb_scan_u32(const uint32_t *d_in, uint32_t *d_out, int64_t n, uint64_t *h_total, cudaStream_t s);
emb_status emb_scan_into(const uint32_t *d_in, uint32_t *d_out, int64_t n, uint64_t *tmp, cudaStream_t s);
// emb_scan_into that also checks the total against a planned count (EMB_ERR_STATE on the
// device when they differ), for planned replays; EMB_NO_EXPECT skips the check.
#define EMB_NO_EXPECT 0xFFFFFFFFFFFFFFFFull
emb_status emb_scan_into_expect(const uint32_t *d_in, uint32_t *d_out, int64_t n, uint64_t *tmp, uint64_t expect,
                                cudaStream_t s);
int64_t emb_scan_tmp_words(int64_t n);
// Level index (hash + rank bitmap) and neighbour table.
int64_t emb_hash_capacity(int64_t n);
int64_t emb_bitmap_words(int64_t nb);
emb_status emb_enq_level_index(EmbLevel &lv, uint32_t *pc, uint64_t *tmp, cudaStream_t s);
emb_status emb_build_hash(EmbLevel &lv, cudaStream_t s);
emb_status emb_build_index_counted(EmbLevel &lv, const uint32_t *nflags, int64_t cap, cudaStream_t s);
// Device address of a caller output buffer (device memory, or page-locked host memory
// through its mapping); EMB_ERR_BAD_INPUT for pageable memory.  NULL stays NULL.
emb_status emb_device_view(void *p, void **dp);
// A pinned host slot (8 words) and its event for a count read-back; -1 when none is free.
int emb_readback_acquire(uint64_t **h, cudaEvent_t *ev);
void emb_readback_release(int slot);
emb_status emb_enq_neighbors(EmbLevel &lv, cudaStream_t s);
emb_status emb_build_neighbors(EmbLevel &lv, cudaStream_t s);
int emb_grid(int64_t n, int block);
int emb_sm_count();
// Forest steps (enqueue only; buffers supplied by the caller).
emb_status emb_enq_root_keys(int64_t R, uint64_t *key, cudaStream_t s);
emb_status emb_enq_flag_ranks(const EmbLevel &P, const uint8_t *d_flags, uint32_t *cnt, uint32_t *rank, uint64_t *tmp,
                              cudaStream_t s, uint64_t expect = EMB_NO_EXPECT);
emb_status emb_enq_children(const EmbLevel &P, const uint8_t *d_flags, const uint32_t *rank, uint64_t *ckey, int64_t Cn,
                            bool planned, cudaStream_t s);
// Binning, voxelization and refine flags (enqueue only).
struct LevelGeom;
emb_status emb_enq_filter(const int4 *rec, int64_t T, LevelGeom g, uint32_t *flag, uint32_t *pos, uint32_t *flist,
                          uint64_t *tmp, int block, cudaStream_t s, uint64_t expect = EMB_NO_EXPECT);
struct EmbBigQ;
emb_status emb_enq_bin_pairs(const int4 *rec, int64_t T, LevelGeom g, const EmbLevel &lv, uint32_t *cnt, uint32_t *off,
                             uint2 *list_bs, uint32_t *list_tri, unsigned long long *list_n, uint64_t list_cap,
                             uint64_t *tmp, const EmbBigQ &Q, cudaStream_t s, uint64_t expect = EMB_NO_EXPECT);
emb_status emb_enq_bin_scatter(const uint2 *list_bs, const uint32_t *list_tri, const unsigned long long *list_n,
                               uint64_t list_cap, const uint32_t *off, uint32_t *ent, uint64_t ent_cap, cudaStream_t s);
emb_status emb_enq_voxelize(const int4 *rec, int64_t T, const uint32_t *flist, int64_t nf, const uint32_t *d_nf,
                            const uint32_t *keep, LevelGeom g, const EmbLevel &lv, unsigned long long *s_acc,
                            unsigned int *p_acc, unsigned int *t_acc, const EmbBigQ &Q, int block, cudaStream_t s);
emb_status emb_enq_refine(const int4 *rec, int64_t T, LevelGeom g, long long dil, const EmbLevel &lv, uint8_t *flags,
                          unsigned long long *fbits, const EmbBigQ &Q, cudaStream_t s);
long long emb_refine_dilation(const emb_forest_s *f, int L, int band);

// Cut links: per-mesh arguments of the persistent link kernel, passed by value as
// a table so one launch can serve a whole batch of meshes.
#define EMB_MAX_BATCH 64
struct LinkMesh {
    const uint64_t *key;       // finest block keys
    const uint64_t *cand;      // 26 direction words per block
    const uint32_t *blk_off;   // link offsets per block
    const uint32_t *bin_off;   // CSR bins
    const uint32_t *bin_ent;
    uint64_t ent_cap;          // bin entries that exist
    const int4 *rec;           // triangle records
    uint32_t T;                // their count
    // work items (block, first | end << 8): the cells with links of rank [first, end)
    // among the block's; one per block with links (its count at *work_n), plus the
    // further parts of heavy blocks in `extra` (EMB_BIG_NONE = unused entry)
    const uint2 *witem;
    const uint32_t *work_n;
    const uint2 *extra;
    const unsigned long long *extra_n;  // extra entries requested (valid: min(extra_n, extra_cap))
    uint32_t extra_cap;
    int32_t *o_cell;
    uint8_t *o_dir;
    float *o_q;
    int32_t *o_tri;
    LevelGeom g;
    uint32_t cap;              // capacity of the output table
    int64_t nblk;              // finest blocks (bounds mode)
};
struct LinkTable {
    int n;
    LinkMesh m[EMB_MAX_BATCH];
};
emb_status emb_enq_link_prep(const EmbLevel &lv, int lattice, uint64_t *cand, uint32_t *cnt, uint32_t *flag,
                             uint32_t *work_n, uint32_t *work, uint32_t *blk_off, uint64_t *tmp, cudaStream_t s,
                             uint64_t expect_work = EMB_NO_EXPECT, uint64_t expect_links = EMB_NO_EXPECT);
emb_status emb_enq_link_split(const EmbLevel &lv, const uint32_t *work, const uint32_t *work_n, const uint64_t *cand,
                              const uint32_t *blk_off, const uint32_t *bin_off, uint2 *witem, uint2 *extra,
                              unsigned long long *extra_n, uint32_t extra_cap, cudaStream_t s);
int64_t emb_link_extra_capacity(int64_t n);
emb_status emb_enq_link_emit(const LinkTable &tab, unsigned int *next, int ctas_per_sm, cudaStream_t s,
                             int64_t items);
emb_status emb_link_emit_init();
size_t emb_link_emit_smem();

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#define EMB_KEY_BITS 21
#define EMB_KEY_MASK ((1ull << EMB_KEY_BITS) - 1ull)
#define EMB_HASH_EMPTY 0xFFFFFFFFFFFFFFFFull

__host__ __device__ __forceinline__ uint64_t emb_key(int64_t bx, int64_t by, int64_t bz)
{
    return ((uint64_t)bz << (2 * EMB_KEY_BITS)) | ((uint64_t)by << EMB_KEY_BITS) | (uint64_t)bx;
}

__host__ __device__ __forceinline__ uint64_t emb_hash_mix(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Block id of key in a level hash, or -1.  Probing is bounded by the table size.
__device__ __forceinline__ int32_t emb_hash_find(const uint64_t *__restrict__ hkey, const int32_t *__restrict__ hval,
                                                 int64_t hcap, uint64_t key)
{
    uint64_t m = (uint64_t)hcap - 1;
    uint64_t s = emb_hash_mix(key) & m;
    for (int64_t i = 0; i < hcap; ++i) {
        uint64_t k = __ldg(hkey + s);
        if (k == key) return __ldg(hval + s);
        if (k == EMB_HASH_EMPTY) return -1;
        s = (s + 1) & m;
    }
    return -1;
}

// Block id at (bx, by, bz) of a level, or -1 (coordinates must lie in [0, nb)).
__device__ __forceinline__ int32_t emb_lookup(const EmbLookup &l, int64_t bx, int64_t by, int64_t bz)
{
    int32_t id;
    if (l.bits) {
        const int64_t lin = (bz * l.nb + by) * l.nb + bx;
        if (!emb_ck((uint64_t)lin, (uint64_t)l.nb * l.nb * l.nb, l.st)) return -1;
        // the word and its rank prefix are independent loads: both issued before the test
        const uint64_t w = __ldg(l.bits + (lin >> 6));
        const uint32_t pre = __ldg(l.wpre + (lin >> 6));
        const int sh = (int)(lin & 63);
        if (!((w >> sh) & 1ull)) return -1;
        id = (int32_t)(pre + __popcll(w & ((1ull << sh) - 1ull)));
    } else {
        id = emb_hash_find(l.hkey, l.hval, l.hcap, emb_key(bx, by, bz));
    }
    if (id >= 0 && !emb_ck((uint64_t)id, (uint64_t)l.n, l.st)) return -1;
    return id;
}

// First index in the ascending a[0, n) whose value is not below v.
static __device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *__restrict__ a, int64_t n, uint64_t v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// floor(a / 2^s) and ceil(a / 2^s) for signed a (arithmetic shifts; the cell and
// block widths of every level are powers of two).
__device__ __forceinline__ int64_t emb_floor_shr(int64_t a, int s) { return a >> s; }
__device__ __forceinline__ int64_t emb_ceil_shr(int64_t a, int s) { return -((-a) >> s); }

__device__ __forceinline__ int sgn_ll(long long v) { return (v > 0) - (v < 0); }
__device__ __forceinline__ int sgn_i128(i128 v) { return (v > 0) - (v < 0); }

// Lattice vectors in the order documented in emb.h.  Component d of c_i is
// ((K_d >> 2i) & 3) - 1 with the three packed constants below (pure ALU, so a
// divergent index costs no memory access).
#define EMB_DIR_KX 0x20889548889549ull
#define EMB_DIR_KY 0xa088895609495ull
#define EMB_DIR_KZ 0x8a0a0a0954955ull
__host__ __device__ __forceinline__ void emb_dir(int i, int &cx, int &cy, int &cz)
{
    cx = (int)((EMB_DIR_KX >> (2 * i)) & 3ull) - 1;
    cy = (int)((EMB_DIR_KY >> (2 * i)) & 3ull) - 1;
    cz = (int)((EMB_DIR_KZ >> (2 * i)) & 3ull) - 1;
}

// Set of directions (bit i = direction i) whose component on `axis` equals `val`.
__host__ __device__ constexpr uint32_t emb_dirs_with(int axis, int val)
{
    uint32_t m = 0;
    for (int i = 0; i < 27; ++i) {
        unsigned long long K = axis == 0 ? EMB_DIR_KX : (axis == 1 ? EMB_DIR_KY : EMB_DIR_KZ);
        if ((int)((K >> (2 * i)) & 3ull) - 1 == val) m |= 1u << i;
    }
    return m;
}

// Orientation of the perturbed query (py + e^2, pz + e^3) against the yz
// projection of edge U -> V:  (V-U)_y (P-U)_z - (V-U)_z (P-U)_y, with the
// e^2 coefficient -(V-U)_z and the e^3 coefficient (V-U)_y deciding ties.
__device__ __forceinline__ int emb_orient_yz(int uy, int uz, int vy, int vz, int py, int pz)
{
    long long ey = (long long)vy - uy, ez = (long long)vz - uz;
    long long o = ey * ((long long)pz - uz) - ez * ((long long)py - uy);
    if (o != 0) return o > 0 ? 1 : -1;
    if (ez != 0) return ez > 0 ? -1 : 1;
    return ey > 0 ? 1 : (ey < 0 ? -1 : 0);
}

// i128 from the product of two int64.
__device__ __forceinline__ i128 mul128(long long a, long long b) { return (i128)a * (i128)b; }

// Float approximation of a non-negative i128 (relative error below 2^-23).
__device__ __forceinline__ float i128_to_float(i128 v)
{
    unsigned long long hi = (unsigned long long)(v >> 64);
    unsigned long long lo = (unsigned long long)v;
    return (float)hi * 18446744073709551616.0f + (float)lo;
}

// Exact overlap of a triangle with the closed box [lo, hi] (separating axes:
// the box normals, the face normal and the 9 edge x axis products), computed
// in coordinates relative to the box's low corner.
static __device__ __noinline__ bool emb_tri_box(const int4 &A, const int4 &B, const int4 &C, long long lx, long long ly,
                                            long long lz, long long hx, long long hy, long long hz)
{
    long long v[3][3] = {{A.x - lx, A.y - ly, A.z - lz}, {B.x - lx, B.y - ly, B.z - lz}, {C.x - lx, C.y - ly, C.z - lz}};
    long long E[3] = {hx - lx, hy - ly, hz - lz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        long long mn = min(v[0][d], min(v[1][d], v[2][d]));
        long long mx = max(v[0][d], max(v[1][d], v[2][d]));
        if (mn > E[d] || mx < 0) return false;
    }
    long long f[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        f[0][d] = v[1][d] - v[0][d];
        f[1][d] = v[2][d] - v[1][d];
        f[2][d] = v[0][d] - v[2][d];
    }
    // face normal: the triangle projects to the single value n.v0
    long long n0 = f[0][1] * f[1][2] - f[0][2] * f[1][1];
    long long n1 = f[0][2] * f[1][0] - f[0][0] * f[1][2];
    long long n2 = f[0][0] * f[1][1] - f[0][1] * f[1][0];
    {
        i128 p = mul128(n0, v[0][0]) + mul128(n1, v[0][1]) + mul128(n2, v[0][2]);
        i128 t0 = mul128(n0, E[0]), t1 = mul128(n1, E[1]), t2 = mul128(n2, E[2]);
        i128 bmin = (t0 < 0 ? t0 : 0) + (t1 < 0 ? t1 : 0) + (t2 < 0 ? t2 : 0);
        i128 bmax = (t0 > 0 ? t0 : 0) + (t1 > 0 ? t1 : 0) + (t2 > 0 ? t2 : 0);
        if (p < bmin || p > bmax) return false;
    }
    // edge axes e_d x f_j: (e_x x f) = (0, -f_z, f_y), (e_y x f) = (f_z, 0, -f_x), (e_z x f) = (-f_y, f_x, 0)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            long long a[3];
            if (d == 0) { a[0] = 0; a[1] = -f[j][2]; a[2] = f[j][1]; }
            else if (d == 1) { a[0] = f[j][2]; a[1] = 0; a[2] = -f[j][0]; }
            else { a[0] = -f[j][1]; a[1] = f[j][0]; a[2] = 0; }
            long long p0 = a[0] * v[0][0] + a[1] * v[0][1] + a[2] * v[0][2];
            long long p1 = a[0] * v[1][0] + a[1] * v[1][1] + a[2] * v[1][2];
            long long p2 = a[0] * v[2][0] + a[1] * v[2][1] + a[2] * v[2][2];
            long long pmin = min(p0, min(p1, p2)), pmax = max(p0, max(p1, p2));
            long long t0 = a[0] * E[0], t1 = a[1] * E[1], t2 = a[2] * E[2];
            long long bmin = min(t0, 0ll) + min(t1, 0ll) + min(t2, 0ll);
            long long bmax = max(t0, 0ll) + max(t1, 0ll) + max(t2, 0ll);
            if (pmax < bmin || pmin > bmax) return false;
        }
    }
    return true;
}

__device__ __forceinline__ bool emb_point_in_box(const int4 &P, long long lx, long long ly, long long lz, long long hx,
                                                 long long hy, long long hz)
{
    return P.x >= lx && P.x <= hx && P.y >= ly && P.y <= hy && P.z >= lz && P.z <= hz;
}

// Enumerate the block range [b0, b1] along one axis whose boxes dilated by dil
// meet the interval [mn, mx] (block width 2^lW, nb blocks on the axis).
__device__ __forceinline__ void emb_block_range(long long mn, long long mx, int lW, long long dil, long long nb,
                                                long long &b0, long long &b1)
{
    b0 = emb_ceil_shr(mn - dil - (1ll << lW), lW);
    b1 = emb_floor_shr(mx + dil, lW);
    if (b0 < 0) b0 = 0;
    if (b1 > nb - 1) b1 = nb - 1;
}

// Range of line indices j with centre (2j+1) half inside [mn, mx], clamped (cell size 2^lh).
__device__ __forceinline__ void line_range(long long mn, long long mx, int lh, long long half, long long ncell,
                                           long long &j0, long long &j1)
{
    j0 = emb_ceil_shr(mn - half, lh);
    j1 = emb_floor_shr(mx - half, lh);
    if (j0 < 0) j0 = 0;
    if (j1 > ncell - 1) j1 = ncell - 1;
}

// ---------------------------------------------------------------------------
// warp-cooperative visit of (triangle, block) overlaps
// ---------------------------------------------------------------------------
// A warp takes 32 consecutive triangles (neighbours in a mesh's storage order
// are usually neighbours in space) and stages them in shared memory.  The refine
// kernel may form the union of the block ranges their dilated boxes can touch and
// let each lane test whole blocks of that union against all 32 triangles, which
// trades 32 independent lookups per candidate block for one; when the union is
// large (above EMB_WU_MAX blocks) or loose (more than an eighth of the warp's
// summed per-triangle candidates), and always in the finest-level binning, the
// warp's (triangle, candidate block) pairs are spread evenly over its lanes instead.
#define EMB_WU_WARPS 4
// Division by a per-triangle divisor d >= 1 in the pair-spreading loops, through its
// reciprocal m = ceil(2^32 / d) (emb_recip, once per triangle): q = floor(r m / 2^32)
// is floor(r / d) or one more (r m / 2^32 lies in [r / d, r / d + r / 2^32)), and
// the one multiply-compare takes the excess back; exact while r + d < 2^32.
__device__ __forceinline__ uint32_t emb_recip(uint32_t d) { return d > 1u ? 0xFFFFFFFFu / d + 1u : 0u; }
__device__ __forceinline__ uint32_t emb_div_recip(uint32_t r, uint32_t d, uint32_t m)
{
    uint32_t q = __umulhi(r, m);
    q -= (uint32_t)(q * d > r);
    return d > 1u ? q : r;
}
#define EMB_WU_MAX 2048

struct WuTri {
    int4 A[32], B[32], C[32];
    int lo[3][32], hi[3][32];
};

// Overlap of triangle j of the tile with the closed box [l, u] (exact).
__device__ __forceinline__ bool wu_overlap(const WuTri &S, int j, long long lx, long long ly, long long lz, long long ux,
                                           long long uy, long long uz)
{
    if (S.lo[0][j] > ux || S.hi[0][j] < lx || S.lo[1][j] > uy || S.hi[1][j] < ly || S.lo[2][j] > uz || S.hi[2][j] < lz)
        return false;
    const int4 A = S.A[j], B = S.B[j], C = S.C[j];
    return emb_point_in_box(A, lx, ly, lz, ux, uy, uz) || emb_point_in_box(B, lx, ly, lz, ux, uy, uz) ||
           emb_point_in_box(C, lx, ly, lz, ux, uy, uz) || emb_tri_box(A, B, C, lx, ly, lz, ux, uy, uz);
}

// ---------------------------------------------------------------------------
// work split of large triangles
// ---------------------------------------------------------------------------
// The triangle-parallel kernels give each triangle to one thread.  A triangle
// with more than EMB_BIG_ITEMS items (x-lines, or candidate blocks) would keep
// its thread busy long after the rest of the grid is done (a coarse mesh on a
// fine level), so the thread instead appends ceil(items / EMB_BIG_CHUNK) chunk
// entries to a queue, and a second kernel walks every chunk with one warp.  A
// thread that finds the queue full walks its items itself: the queue's size
// affects the speed only, never the result.
#define EMB_BIG_ITEMS 64
#define EMB_BIG_CHUNK 512
#define EMB_BIG_NONE 0xFFFFFFFFu
struct EmbBigQ {
    uint2 *q;               // entries (triangle, chunk | chunk count << 16); EMB_BIG_NONE = unused
    unsigned long long *n;  // entries requested (may exceed cap)
    uint32_t cap;           // 0: no queue, every thread walks its own items
};

// Reserves the chunks of triangle t; false when they do not fit.
__device__ __forceinline__ bool emb_bigq_push(const EmbBigQ &Q, uint32_t t, unsigned long long items)
{
    if (Q.cap == 0) return false;
    unsigned long long nch = (items + EMB_BIG_CHUNK - 1) / EMB_BIG_CHUNK;
    if (nch > 0xFFFFull) nch = 0xFFFFull;
    const unsigned long long base = atomicAdd(Q.n, nch);
    if (base + nch > Q.cap) {
        for (unsigned long long e = base; e < Q.cap; ++e) Q.q[e] = make_uint2(EMB_BIG_NONE, 0u);
        return false;
    }
    for (uint32_t c = 0; c < (uint32_t)nch; ++c) Q.q[base + c] = make_uint2(t, c | ((uint32_t)nch << 16));
    return true;
}

// Items [i0, i1) of the chunk described by an entry's second word.
__device__ __forceinline__ void emb_bigq_range(uint32_t y, unsigned long long items, unsigned long long &i0,
                                               unsigned long long &i1)
{
    const unsigned long long c = y & 0xFFFFu, nch = y >> 16;
    const unsigned long long span = (items + nch - 1) / nch;
    i0 = c * span;
    i1 = i0 + span < items ? i0 + span : items;
}

// Entries to walk (entries beyond the capacity were never written).
__device__ __forceinline__ unsigned long long emb_bigq_count(const EmbBigQ &Q)
{
    const unsigned long long n = *Q.n;
    return n < Q.cap ? n : Q.cap;
}

// Host side (emb_common.cu): capacity for T triangles, allocation, per-launch reset.
int64_t emb_bigq_capacity(int64_t T);
emb_status emb_bigq_alloc(EmbBigQ &Q, int64_t T, cudaStream_t s);  // stream-ordered
void emb_bigq_free(EmbBigQ &Q, cudaStream_t s);
#define EMB_BIG_GRID 1216   // CTAs of the chunk kernels (8 per SM on 152 SMs)
#define EMB_BIG_BLOCK 128
