// Boundary-cell identification and the flat link-length table (Sec. 3.4,
// "Boundary Cell Identification", "Memory Allocations for Boundary Cells",
// "Link-Length Computation").
//
// k_link_cand: per finest block and direction, the 64-bit word of fluid cells
//   whose neighbour along that direction is solid, from the 27 mask words of the
//   block and its 26 neighbours by 3-D bit shifts.
// Counts per block -> exclusive scan -> link offsets (block-granular, in block
//   order, so the table is sorted by (cell, direction)).
// k_link_split: a block whose links times bin triangles is large becomes several
//   work items, each a contiguous range of its boundary cells.
// k_link_emit: one warp per work item (details at the kernel).  Exact
//   Pluecker sides for the line, exact plane sides for the two segment ends
//   (query points pushed by (e, e^2, e^3)), and an exact rational comparison of
//   t = N / (h M) between crossings (lowest triangle id on equality).  q = t is
//   rounded to float once.
#include "emb_internal.cuh"

#define LINK_TILE 64

// Neighbour-solid words by 3-D bit shifts.  A block's 64 cells are bit t =
// x + 4y + 16z of its mask word; shifting the 4x4x4 bit cube by one cell along an
// axis takes three cell layers from the block itself and the fourth from the
// neighbouring block on that side.
#define EMB_X0 0x1111111111111111ull
#define EMB_X3 0x8888888888888888ull
#define EMB_Y0 0x000F000F000F000Full
#define EMB_Y3 0xF000F000F000F000ull
#define EMB_Z0 0x000000000000FFFFull
#define EMB_Z3 0xFFFF000000000000ull

// bit t of the result = bit of cell (t + e_axis * s) where the cell lies in `cur`
// or, across the face, in `nxt` (the neighbour block on the +s side).
__device__ __forceinline__ uint64_t shift_axis(uint64_t cur, uint64_t nxt, int axis, int s)
{
    if (axis == 0) return s > 0 ? (((cur >> 1) & ~EMB_X3) | ((nxt << 3) & EMB_X3)) : (((cur << 1) & ~EMB_X0) | ((nxt >> 3) & EMB_X0));
    if (axis == 1) return s > 0 ? (((cur >> 4) & ~EMB_Y3) | ((nxt << 12) & EMB_Y3)) : (((cur << 4) & ~EMB_Y0) | ((nxt >> 12) & EMB_Y0));
    return s > 0 ? (((cur >> 16) & ~EMB_Z3) | ((nxt << 48) & EMB_Z3)) : (((cur << 16) & ~EMB_Z0) | ((nxt >> 48) & EMB_Z0));
}

// Per finest block: word d-1 (d = 1 .. lattice-1) has bit t set iff cell t is fluid
// and its neighbour along c_d is solid.  A missing neighbour block counts as fluid:
// a fluid cell with a solid neighbour is within one link of the surface, and the
// refine rule makes every block within that reach exist.  One thread per block; the
// CTA reads its blocks' rows of the neighbour table and writes their rows of direction
// words through shared memory, so that both go with coalesced accesses (rows of the
// output are padded to 27 words there, against bank conflicts).
#define CAND_BLOCK 128
__global__ void __launch_bounds__(CAND_BLOCK) k_link_cand(const uint64_t *__restrict__ mask,
                                                           const int32_t *__restrict__ nbr, int64_t n, int lattice,
                                                           uint64_t *__restrict__ cand, uint32_t *__restrict__ blk_cnt,
                                                           int *st, const uint32_t *d_n)
{
    __shared__ uint64_t stage[CAND_BLOCK * 27];
    int32_t *const srow = (int32_t *)stage;  // first the neighbour rows (26 ids a block)
    const int64_t cnt = emb_count(n, d_n);
    const int64_t b0 = (int64_t)blockIdx.x * CAND_BLOCK;
    if (b0 >= cnt) return;  // the whole CTA
    const int nloc = (int)(cnt - b0 < CAND_BLOCK ? cnt - b0 : CAND_BLOCK);
    const int tid = threadIdx.x;
    for (int j = tid; j < nloc * 26; j += CAND_BLOCK) srow[j] = nbr[b0 * 26 + j];
    __syncthreads();
    const int64_t b = b0 + tid;
    uint64_t W[27];  // mask words by offset code (ox+1) + 3(oy+1) + 9(oz+1)
    if (tid < nloc) {
        W[13] = mask[b];
#pragma unroll
        for (int i = 1; i < 27; ++i) {
            int cx, cy, cz;
            emb_dir(i, cx, cy, cz);
            const int32_t id = srow[tid * 26 + i - 1];
            W[(cx + 1) + 3 * (cy + 1) + 9 * (cz + 1)] = id >= 0 && emb_ck((uint64_t)id, (uint64_t)n, st) ? mask[id] : 0ull;
        }
    }
    __syncthreads();  // the neighbour rows are overwritten below
    if (tid < nloc) {
        const uint64_t fluid = ~W[13];
        uint32_t count = 0;
#pragma unroll
        for (int d = 1; d < 27; ++d) {
            if (d >= lattice) {
                stage[tid * 27 + d - 1] = 0;
                continue;
            }
            int cx, cy, cz;
            emb_dir(d, cx, cy, cz);
            // shift along x for every (y, z) block layer touched, then along y, then along z
            uint64_t Y[2][2];
#pragma unroll
            for (int jy = 0; jy < 2; ++jy)
#pragma unroll
                for (int jz = 0; jz < 2; ++jz) {
                    const int oy = jy ? cy : 0, oz = jz ? cz : 0;
                    const uint64_t cur = W[1 + 3 * (oy + 1) + 9 * (oz + 1)];
                    Y[jy][jz] = cx ? shift_axis(cur, W[(cx + 1) + 3 * (oy + 1) + 9 * (oz + 1)], 0, cx) : cur;
                }
            uint64_t Z[2];
#pragma unroll
            for (int jz = 0; jz < 2; ++jz) Z[jz] = cy ? shift_axis(Y[0][jz], Y[1][jz], 1, cy) : Y[0][jz];
            const uint64_t nb_solid = cz ? shift_axis(Z[0], Z[1], 2, cz) : Z[0];
            const uint64_t c = fluid & nb_solid;
            stage[tid * 27 + d - 1] = c;
            count += __popcll(c);
        }
        blk_cnt[b] = count;
    }
    __syncthreads();
    for (int j = tid; j < nloc * 26; j += CAND_BLOCK) {
        const int r = j / 26;
        cand[b0 * 26 + j] = stage[r * 27 + (j - r * 26)];
    }
}

// One warp per work item: a finest block with links, or one part of a heavy block
// (a contiguous range of its cells with links, see k_link_split).  The item's
// cells that have cut links are taken in chunks of up to 32 (slot j = the j-th
// such cell of the chunk).  The block's bin is staged 32 triangles at a time into
// the warp's shared-memory tile.  A triangle can only cross a link from cell
// centre P if its bounding box meets the cube [P - h, P + h]; because the cells
// form a 4x4x4 lattice, the set of cells passing that test is a sub-box, built as
// a 64-bit mask with a few bit operations.  The surviving (triangle, cell) pairs
// of a tile are spread over the 32 lanes with a prefix sum.  Per pair, with the
// vertices relative to P, the moments m_i of the three edges are formed once; the
// three Pluecker signs c . m_i test the lines of all 13 direction pairs (c and -c
// share the line) at once.  When every vertex lies within 2^14 of P the moments fit
// 32-bit integers; otherwise they are formed in 64 bits by widening products
// (coarse frames, where h itself is 2^14 or more, take this path).  A pair whose
// lines hit is queued in the warp's shared memory (tile index, cell, hit
// directions); the queue is drained 32 hits at a time, one hit per lane, which
// checks the ends of the segment against the plane (D = n . (A - P) against
// D - h n.c, in 64 bits, or 128 bits on the wide path) and rounds q.  A zero
// Pluecker value sends its direction through the exact per-direction test with the
// full tie-break at once.  Crossings are appended to a per-cell bucket; afterwards
// the owner lane of each cell keeps, per direction, the nearest one (exact rational
// comparison when a link crosses more than one face), and the warp writes the
// chunk's links, which are consecutive in the table (the direction words fix each
// cell's offset whichever warp handles it), one link per lane.  A bucket that
// overflows sends its cell through an exact per-cell scan of the whole bin instead.
// Sizes: 4 warps per CTA; a warp's tile of 32 triangles, 20 hit slots per cell and the
// byte-wide best-hit indices (shared with the hit queue) take 9 KB of shared memory, so
// six CTAs would fit on an SM.  The launch bound asks for five, which leaves 96
// registers a thread: with the queue's shorter instruction stream the spills of the
// 80-register build cost more than the sixth CTA gains (3.76 -> 3.43 ms on the 7.2M
// step).  Fewer hit slots let more CTAs fit but send many more cells of a D3Q27
// workload through the per-cell rescan, which costs far more than it saves.
#define LE_WARPS 4
#define LE_TILE 32
#define LE_BCAP 20
// Largest finest-level bin the link kernel takes (hit records hold the bin-local
// triangle index in 24 bits); a larger bin sets EMB_ERR_CAPACITY.
#define EMB_BIN_MAX_ENTRIES (1u << 24)
// A block is split into about (links x bin triangles) / LE_SPLIT_COST parts, at
// most one per three links and LE_SPLIT_MAX in all.
#define LE_SPLIT_COST 16384
#define LE_SPLIT_MAX 64

struct TriT {
    int ax, ay, az, bx, by, bz, cx, cy, cz, id;
    int lox, loy, loz, hix, hiy, hiz;
    long long nx, ny, nz;
};

struct LeWarp {
    TriT tile[LE_TILE];
    uint2 hit[LE_BCAP][32];  // per slot: (bin-local index | direction << 24, q bits)
    union {
        signed char best[27][32];  // resolution: per (direction, slot) the index of the nearest hit
        uint2 hq[32];              // tile passes: queued pairs (tile index | cell << 5 | slot << 11 | wide << 16, line hits)
    };
    int hcnt[32];
    uint32_t cm[32];         // candidate directions of each slot's cell
};

// Directions whose component on one axis lies in an allowed subset of {-1, 0, +1}.
__device__ __forceinline__ uint32_t dirs_allowed(int axis, bool neg, bool zero, bool pos)
{
    const uint32_t N = axis == 0 ? emb_dirs_with(0, -1) : (axis == 1 ? emb_dirs_with(1, -1) : emb_dirs_with(2, -1));
    const uint32_t Z = axis == 0 ? emb_dirs_with(0, 0) : (axis == 1 ? emb_dirs_with(1, 0) : emb_dirs_with(2, 0));
    const uint32_t P = axis == 0 ? emb_dirs_with(0, 1) : (axis == 1 ? emb_dirs_with(1, 1) : emb_dirs_with(2, 1));
    return (neg ? N : 0u) | (zero ? Z : 0u) | (pos ? P : 0u);
}

__device__ __forceinline__ long long cdot(int cx, int cy, int cz, long long x, long long y, long long z)
{
    long long s = 0;
    if (cx) s = cx > 0 ? s + x : s - x;
    if (cy) s = cy > 0 ? s + y : s - y;
    if (cz) s = cz > 0 ? s + z : s - z;
    return s;
}

// Perturbed Pluecker sign for edge U -> V given s = c . ((U-P) x (V-P)) and the edge vector d = V - U:
// a zero is resolved by e . (c x d), e = (e, e^2, e^3).
__device__ __forceinline__ int plk_resolve(long long s, int cx, int cy, int cz, long long dx, long long dy, long long dz)
{
    if (s != 0) return s > 0 ? 1 : -1;
    long long w0 = cy * dz - cz * dy;
    if (w0) return w0 > 0 ? 1 : -1;
    long long w1 = cz * dx - cx * dz;
    if (w1) return w1 > 0 ? 1 : -1;
    long long w2 = cx * dy - cy * dx;
    return w2 > 0 ? 1 : (w2 < 0 ? -1 : 0);
}

// Sign of (X - n . e): X when nonzero, else minus the first nonzero normal component.
__device__ __forceinline__ int side_sign(i128 X, long long nx, long long ny, long long nz)
{
    if (X != 0) return X > 0 ? 1 : -1;
    if (nx) return nx > 0 ? -1 : 1;
    if (ny) return ny > 0 ? -1 : 1;
    return nz > 0 ? -1 : 1;
}

// Position of the r-th (0-based) set bit of m (m has more than r set bits).
__device__ __forceinline__ int select64(unsigned long long m, int r)
{
    int pos = 0;
#pragma unroll
    for (int w = 32; w >= 1; w >>= 1) {
        unsigned long long lowm = m & ((1ull << w) - 1ull);
        int c = __popcll(lowm);
        if (r >= c) {
            r -= c;
            m >>= w;
            pos += w;
        } else {
            m = lowm;
        }
    }
    return pos;
}


// Position of the r-th (0-based) set bit of the 32-bit m (m has more than r set bits).
__device__ __forceinline__ int select32(uint32_t m, int r)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t lowm = m & ((1u << w) - 1u);
        const int c = __popc(lowm);
        if (r >= c) {
            r -= c;
            m >>= w;
            pos += w;
        } else {
            m = lowm;
        }
    }
    return pos;
}

// 32 x 32 bit-matrix transpose across a warp: lane r holds row r (bit c = entry
// (r, c)); lane c receives column c (bit r = entry (r, c)).  Five stages, each
// swapping the off-diagonal sub-blocks of the current size between lane pairs.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane)
{
    const uint32_t mk[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int j = 16 >> k;
        const uint32_t m = mk[k];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

// Bits [lo, hi] of a 64-bit word (0 <= lo <= hi <= 63).
__device__ __forceinline__ unsigned long long bit_range(int lo, int hi)
{
    unsigned long long top = hi >= 63 ? ~0ull : ((1ull << (hi + 1)) - 1ull);
    return top & ~((1ull << lo) - 1ull);
}

// Exact crossing parameter t = N / (h M) of the segment P -> P + h c with a triangle
// already known to be crossed (recomputed from its record).
__device__ __forceinline__ void tri_NM(const int4 *__restrict__ rec, int tr, long long px, long long py, long long pz,
                                       int cx, int cy, int cz, i128 &N, long long &M)
{
    int4 A = rec[3 * (int64_t)tr], B = rec[3 * (int64_t)tr + 1], C = rec[3 * (int64_t)tr + 2];
    long long ux = (long long)B.x - A.x, uy = (long long)B.y - A.y, uz = (long long)B.z - A.z;
    long long vx = (long long)C.x - A.x, vy = (long long)C.y - A.y, vz = (long long)C.z - A.z;
    long long nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    long long nc = cdot(cx, cy, cz, nx, ny, nz);
    i128 D = mul128(nx, A.x - px) + mul128(ny, A.y - py) + mul128(nz, A.z - pz);
    N = nc > 0 ? D : -D;
    M = nc > 0 ? nc : -nc;
}

// Exact test of the segment P -> P + h c (perturbed) against a triangle given its
// vertices relative to P, its normal and the edge moments; fills D on first use.
__device__ __forceinline__ bool seg_cross(int cx, int cy, int cz, long long h, long long ax, long long ay, long long az,
                                          long long bx, long long by, long long bz, long long qx, long long qy,
                                          long long qz, long long nx, long long ny, long long nz, long long m1x,
                                          long long m1y, long long m1z, long long m2x, long long m2y, long long m2z,
                                          long long m3x, long long m3y, long long m3z, i128 &D, bool &haveD)
{
    const long long nc = cdot(cx, cy, cz, nx, ny, nz);
    if (nc == 0) return false;
    const int sn = nc > 0 ? 1 : -1;
    if (plk_resolve(cdot(cx, cy, cz, m1x, m1y, m1z), cx, cy, cz, bx - ax, by - ay, bz - az) != sn) return false;
    if (plk_resolve(cdot(cx, cy, cz, m2x, m2y, m2z), cx, cy, cz, qx - bx, qy - by, qz - bz) != sn) return false;
    if (plk_resolve(cdot(cx, cy, cz, m3x, m3y, m3z), cx, cy, cz, ax - qx, ay - qy, az - qz) != sn) return false;
    if (!haveD) {
        D = mul128(nx, ax) + mul128(ny, ay) + mul128(nz, az);
        haveD = true;
    }
    if (side_sign(D, nx, ny, nz) != sn) return false;                 // t <= 0
    if (side_sign(D - mul128(h, nc), nx, ny, nz) != -sn) return false;  // t >= 1
    return true;
}

// Nearest crossed triangle of every candidate direction in `cm` for cell centre P,
// by a plain exact scan of the whole bin (used for cells whose bucket overflowed).
__device__ __noinline__ void scan_cell_slow(const uint32_t *__restrict__ bin_ent, uint32_t e0, uint32_t e1,
                                            const int4 *__restrict__ rec, uint32_t T, long long px, long long py,
                                            long long pz, long long h, uint32_t cm, int *bestT)
{
    for (int d = 0; d < 27; ++d) bestT[d] = -1;
    for (uint32_t e = e0; e < e1; ++e) {
        const int id = (int)bin_ent[e];
        if ((uint32_t)id >= T) continue;
        const int4 A = rec[3 * (int64_t)id], B = rec[3 * (int64_t)id + 1], C = rec[3 * (int64_t)id + 2];
        const long long ax = A.x - px, ay = A.y - py, az = A.z - pz;
        const long long bx = B.x - px, by = B.y - py, bz = B.z - pz;
        const long long qx = C.x - px, qy = C.y - py, qz = C.z - pz;
        const long long ux = bx - ax, uy = by - ay, uz = bz - az, vx = qx - ax, vy = qy - ay, vz = qz - az;
        const long long nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
        const long long m1x = ay * bz - az * by, m1y = az * bx - ax * bz, m1z = ax * by - ay * bx;
        const long long m2x = by * qz - bz * qy, m2y = bz * qx - bx * qz, m2z = bx * qy - by * qx;
        const long long m3x = qy * az - qz * ay, m3y = qz * ax - qx * az, m3z = qx * ay - qy * ax;
        i128 D = 0;
        bool haveD = false;
        uint32_t mm = cm;
        while (mm) {
            const int d = __ffs(mm) - 1;
            mm &= mm - 1;
            int cx, cy, cz;
            emb_dir(d, cx, cy, cz);
            if (!seg_cross(cx, cy, cz, h, ax, ay, az, bx, by, bz, qx, qy, qz, nx, ny, nz, m1x, m1y, m1z, m2x, m2y, m2z,
                           m3x, m3y, m3z, D, haveD))
                continue;
            bool better = bestT[d] < 0;
            if (!better) {
                i128 No, Nn;
                long long Mo, Mn;
                tri_NM(rec, bestT[d], px, py, pz, cx, cy, cz, No, Mo);
                tri_NM(rec, id, px, py, pz, cx, cy, cz, Nn, Mn);
                const i128 l = Nn * (i128)Mo, r = No * (i128)Mn;
                better = l < r || (l == r && id < bestT[d]);
            }
            if (better) bestT[d] = id;
        }
    }
}

// A cell whose bucket overflowed: exact per-cell scan of the whole bin, links written directly.
__device__ __noinline__ void emit_cell_slow(const LinkMesh &M, uint32_t e0, uint32_t e1, long long px, long long py,
                                           long long pz, long long h, uint32_t cm, uint32_t o0, int64_t cell, int *st)
{
    int bestT[27];
    scan_cell_slow(M.bin_ent, e0, e1, M.rec, M.T, px, py, pz, h, cm, bestT);
    uint32_t mm = cm, o = o0;
    while (mm) {
        const int d = __ffs(mm) - 1;
        mm &= mm - 1;
        if (o >= M.cap) {
            emb_set_status(st, EMB_ERR_CAPACITY);
            ++o;
            continue;
        }
        const int tr = bestT[d];
        float q = -1.0f;
        if (tr >= 0) {
            int cx, cy, cz;
            emb_dir(d, cx, cy, cz);
            i128 N;
            long long Mq;
            tri_NM(M.rec, tr, px, py, pz, cx, cy, cz, N, Mq);
            q = __fdiv_rn(i128_to_float(N), (float)Mq * (float)h);
        } else {
            emb_set_status(st, EMB_ERR_STATE);
        }
        M.o_cell[o] = (int32_t)cell;
        M.o_dir[o] = (uint8_t)d;
        M.o_q[o] = q;
        M.o_tri[o] = tr;
        ++o;
    }
}

__device__ __forceinline__ int side_sign64(long long X, long long nx, long long ny, long long nz)
{
    if (X != 0) return X > 0 ? 1 : -1;
    if (nx) return nx > 0 ? -1 : 1;
    if (ny) return ny > 0 ? -1 : 1;
    return nz > 0 ? -1 : 1;
}

// Segment ends of a line hit of the narrow path (every vertex offset from P within
// 2^14, so |n| < 3 * 2^29 per component): direction d's line is known to cross the
// triangle, at t = D / (h c . n) with D = n . (A - P).  The link crosses iff t lies in
// (0, 1) under the perturbation; then q = t rounded to float.  D < 3 * 2^31 * 2^14 and
// h c . n < 2^18 * 9 * 2^29 fit 64 bits.
__device__ __forceinline__ bool hit_segment(const TriT &T, long long px, long long py, long long pz, int d, long long h,
                                            float *q)
{
    const int nx = (int)T.nx, ny = (int)T.ny, nz = (int)T.nz;
    const long long D = (long long)nx * (int)(T.ax - px) + (long long)ny * (int)(T.ay - py) +
                        (long long)nz * (int)(T.az - pz);
    int cx, cy, cz;
    emb_dir(d, cx, cy, cz);
    const long long nc = (long long)cx * nx + (long long)cy * ny + (long long)cz * nz;
    const int sn = nc > 0 ? 1 : -1;
    if (side_sign64(D, nx, ny, nz) != sn) return false;           // t <= 0
    if (side_sign64(D - h * nc, nx, ny, nz) != -sn) return false;  // t >= 1
    const long long N = sn > 0 ? D : -D, Mq = nc > 0 ? nc : -nc;
    *q = __fdiv_rn((float)N, (float)Mq * (float)h);
    return true;
}

// The same for a line hit of the 64-bit path (coordinates below 2^25, so offsets fit 32
// bits, |n| < 3 * 2^51 and c . n < 9 * 2^51): D = n . (A - P) in 128 bits.
__device__ __noinline__ bool hit_segment_wide(const TriT &T, long long px, long long py, long long pz, int d,
                                                 long long h, float *q)
{
    const long long nx = T.nx, ny = T.ny, nz = T.nz;
    const i128 D = mul128(nx, (int)(T.ax - px)) + mul128(ny, (int)(T.ay - py)) + mul128(nz, (int)(T.az - pz));
    int cx, cy, cz;
    emb_dir(d, cx, cy, cz);
    const long long nc = cx * nx + cy * ny + cz * nz;
    const int sn = nc > 0 ? 1 : -1;
    if (side_sign(D, nx, ny, nz) != sn) return false;                  // t <= 0
    if (side_sign(D - mul128(h, nc), nx, ny, nz) != -sn) return false;  // t >= 1
    const i128 N = sn > 0 ? D : -D;
    const long long Mq = nc > 0 ? nc : -nc;
    *q = __fdiv_rn(i128_to_float(N), (float)Mq * (float)h);
    return true;
}

// Exact segment test for a pair whose vertices are not all within 2^14 of P
// (128-bit plane offsets, 64-bit Pluecker products); returns t = N / (h M).
__device__ __noinline__ bool pair_cross_wide(const TriT &T, long long px, long long py, long long pz, int cx, int cy,
                                             int cz, long long h, float *q)
{
    const long long ax = T.ax - px, ay = T.ay - py, az = T.az - pz;
    const long long bx = T.bx - px, by = T.by - py, bz = T.bz - pz;
    const long long qx = T.cx - px, qy = T.cy - py, qz = T.cz - pz;
    const long long m1x = ay * bz - az * by, m1y = az * bx - ax * bz, m1z = ax * by - ay * bx;
    const long long m2x = by * qz - bz * qy, m2y = bz * qx - bx * qz, m2z = bx * qy - by * qx;
    const long long m3x = qy * az - qz * ay, m3y = qz * ax - qx * az, m3z = qx * ay - qy * ax;
    i128 D = 0;
    bool haveD = false;
    if (!seg_cross(cx, cy, cz, h, ax, ay, az, bx, by, bz, qx, qy, qz, T.nx, T.ny, T.nz, m1x, m1y, m1z, m2x, m2y, m2z, m3x,
                   m3y, m3z, D, haveD))
        return false;
    const long long nc = cdot(cx, cy, cz, T.nx, T.ny, T.nz);
    const i128 N = nc > 0 ? D : -D;
    const long long M = nc > 0 ? nc : -nc;
    *q = __fdiv_rn(i128_to_float(N), (float)M * (float)h);
    return true;
}

// The line tests of one (triangle, cell centre P) pair on the candidate directions
// ccm.  The directions whose line crosses the triangle come back in `lines` (`wide`
// says which path found them); the caller finishes each with the segment-end test
// hit_segment or hit_segment_wide, so that a warp can run those 32 at a time.  When
// every vertex lies within 2^14 of P the moments fit 32-bit integers; otherwise they
// are formed in 64 bits by widening products.  A zero Pluecker value sends its
// direction through the exact per-direction test with the full tie-break, and a
// crossing found there is passed to emit(d, q) at once.
template <class Emit>
__device__ __forceinline__ void link_pair(const TriT &T, long long px, long long py, long long pz, uint32_t ccm,
                                          long long h, Emit emit, uint32_t &lines, bool &wide)
{
    lines = 0;
    wide = false;
    // coordinates and cell centres lie below 2^25: the offsets fit 32 bits
    const int LIM = 1 << 14;
    const int pxi = (int)px, pyi = (int)py, pzi = (int)pz;
    const int l0 = T.lox - pxi, h0 = T.hix - pxi, l1 = T.loy - pyi, h1 = T.hiy - pyi, l2 = T.loz - pzi,
              h2 = T.hiz - pzi;
    const bool narrow = l0 > -LIM && h0 < LIM && l1 > -LIM && h1 < LIM && l2 > -LIM && h2 < LIM;
    if (narrow) {
        // Every vertex offset a, b, q lies in (-2^14, 2^14), so in 32-bit integers:
        //   moment components (a x b etc.): |a_y b_z - a_z b_y| < 2 * 2^28 = 2^29;
        //   V_k = c . m_k over the at most three nonzero components of c: < 3 * 2^29 < 2^31;
        //   n = m1 + m2 + m3 per component: < 3 * 2^29 < 2^31.
        // c . n is NOT formed in 32 bits: for a corner direction it reaches 9 * 2^29 > 2^31.
        // The line test needs only the signs of V1, V2, V3 (n = m1 + m2 + m3, so c . n =
        // V1 + V2 + V3, which has their common sign when they agree and are nonzero, and a
        // line parallel to the face cannot have three nonzero V of one sign).
        const int ax = (int)(T.ax - px), ay = (int)(T.ay - py), az = (int)(T.az - pz);
        const int bx = (int)(T.bx - px), by = (int)(T.by - py), bz = (int)(T.bz - pz);
        const int qx = (int)(T.cx - px), qy = (int)(T.cy - py), qz = (int)(T.cz - pz);
        const int m1x = ay * bz - az * by, m1y = az * bx - ax * bz, m1z = ax * by - ay * bx;
        const int m2x = by * qz - bz * qy, m2y = bz * qx - bx * qz, m2z = bx * qy - by * qx;
        const int m3x = qy * az - qz * ay, m3y = qz * ax - qx * az, m3z = qx * ay - qy * ax;
        // line tests for the 13 direction pairs (odd index d and its opposite d + 1):
        // all 13 lines, without branches (the lanes hold different cells, so a
        // per-direction branch would diverge); non-candidates are masked off
        uint32_t line = 0, degen = 0;
#pragma unroll
        for (int r = 0; r < 13; ++r) {
            const int d = 2 * r + 1;
            int cx, cy, cz;
            emb_dir(d, cx, cy, cz);
            const int V1 = cx * m1x + cy * m1y + cz * m1z;
            const int V2 = cx * m2x + cy * m2y + cz * m2z;
            const int V3 = cx * m3x + cy * m3y + cz * m3z;
            const uint32_t ok = ((ccm >> d) & 3u) != 0u;
            const uint32_t zero = (V1 == 0) | (V2 == 0) | (V3 == 0);
            const uint32_t same = ((V1 ^ V2) | (V1 ^ V3)) >= 0;
            // a zero V (the perturbation decides) goes to the exact per-direction test,
            // which also rejects a line parallel to the face
            degen |= (ok & zero) << d;
            line |= (ok & (zero ^ 1u) & same) << d;
        }
        // members of line-hit pairs that are candidates (their segment ends are tested later)
        lines = (line | (line << 1)) & ccm;
        // a zero Pluecker value: resolve the pair's directions exactly
        uint32_t mm = (degen | (degen << 1)) & ccm;
        while (mm) {
            const int d = __ffs(mm) - 1;
            mm &= mm - 1;
            int cx, cy, cz;
            emb_dir(d, cx, cy, cz);
            float q;
            if (!pair_cross_wide(T, px, py, pz, cx, cy, cz, h, &q)) continue;
            emit(d, q);
        }
    } else {
        // coordinates are below 2^25, so offsets fit 32 bits: moments (below 2^51)
        // and their signed sums in 64 bits from widening products
        const int ax = (int)(T.ax - px), ay = (int)(T.ay - py), az = (int)(T.az - pz);
        const int bx = (int)(T.bx - px), by = (int)(T.by - py), bz = (int)(T.bz - pz);
        const int qx = (int)(T.cx - px), qy = (int)(T.cy - py), qz = (int)(T.cz - pz);
        const long long m1x = (long long)ay * bz - (long long)az * by,
                        m1y = (long long)az * bx - (long long)ax * bz,
                        m1z = (long long)ax * by - (long long)ay * bx;
        const long long m2x = (long long)by * qz - (long long)bz * qy,
                        m2y = (long long)bz * qx - (long long)bx * qz,
                        m2z = (long long)bx * qy - (long long)by * qx;
        const long long m3x = (long long)qy * az - (long long)qz * ay,
                        m3y = (long long)qz * ax - (long long)qx * az,
                        m3z = (long long)qx * ay - (long long)qy * ax;
        const long long nx = m1x + m2x + m3x, ny = m1y + m2y + m3y, nz = m1z + m2z + m3z;
        uint32_t line = 0, degen = 0;
#pragma unroll
        for (int r = 0; r < 13; ++r) {
            const int d = 2 * r + 1;
            if (!(ccm & (3u << d))) continue;
            int cx, cy, cz;
            emb_dir(d, cx, cy, cz);
            const long long NC = cx * nx + cy * ny + cz * nz;
            const long long V1 = cx * m1x + cy * m1y + cz * m1z;
            const long long V2 = cx * m2x + cy * m2y + cz * m2z;
            const long long V3 = cx * m3x + cy * m3y + cz * m3z;
            if (NC == 0) continue;
            if (V1 == 0 || V2 == 0 || V3 == 0) {
                degen |= 1u << d;
                continue;
            }
            if (((V1 ^ NC) | (V2 ^ NC) | (V3 ^ NC)) >= 0) line |= 1u << d;
        }
        lines = (line | (line << 1)) & ccm;
        wide = true;
        uint32_t mm = (degen | (degen << 1)) & ccm;
        while (mm) {
            const int d = __ffs(mm) - 1;
            mm &= mm - 1;
            int cx, cy, cz;
            emb_dir(d, cx, cy, cz);
            float q;
            if (!pair_cross_wide(T, px, py, pz, cx, cy, cz, h, &q)) continue;
            emit(d, q);
        }
    }
}

#ifndef LE_MINB
#define LE_MINB 5
#endif
__global__ void __launch_bounds__(LE_WARPS * 32, LE_MINB) k_link_emit(const __grid_constant__ LinkTable tab,
                                                                unsigned int *__restrict__ next, int *st)
{
    extern __shared__ __align__(16) unsigned char le_smem[];
    __shared__ uint32_t s_pre[EMB_MAX_BATCH + 1];  // work items of meshes before j
    __shared__ uint32_t s_ext[EMB_MAX_BATCH];      // extra parts of mesh j (they come first in its range)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    LeWarp &S = reinterpret_cast<LeWarp *>(le_smem)[w];
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int j = 0; j < tab.n; ++j) {
            const LinkMesh &M = tab.m[j];
            const unsigned long long ne = M.extra_n ? *M.extra_n : 0ull;
            s_ext[j] = (uint32_t)(ne < M.extra_cap ? ne : M.extra_cap);
            s_pre[j] = acc;
            acc += *M.work_n + s_ext[j];
        }
        s_pre[tab.n] = acc;
    }
    __syncthreads();
    // persistent warps: take the next (mesh, part of a block with links) item of the shared work queue
    for (;;) {
        unsigned int widx = 0;
        if (lane == 0) widx = atomicAdd(next, 1u);
        widx = __shfl_sync(0xffffffffu, widx, 0);
        if (widx >= s_pre[tab.n]) return;
        int mj = 0;
        while (mj + 1 < tab.n && s_pre[mj + 1] <= widx) ++mj;
        const LinkMesh &M = tab.m[mj];
        const uint32_t *__restrict__ bin_ent = M.bin_ent;
        const int4 *__restrict__ rec = M.rec;
        const uint32_t local = widx - s_pre[mj];
        const uint2 E = local < s_ext[mj] ? M.extra[local] : M.witem[local - s_ext[mj]];
        if (E.x == EMB_BIG_NONE) continue;
        const int64_t b = E.x;
        if (!emb_ck((uint64_t)b, (uint64_t)M.nblk, st)) continue;
        const uint32_t base = M.blk_off[b];
        // candidate directions of cells lane and 32 + lane: lane d < 26 holds direction
        // word d + 1; a 32 x 32 bit transpose of the low and of the high halves gives
        // each lane the column of its two cells
        const uint64_t wd = lane < 26 ? M.cand[b * 26 + lane] : 0ull;
        const uint32_t c0 = warp_transpose32((uint32_t)wd, lane) << 1;
        const uint32_t c1 = warp_transpose32((uint32_t)(wd >> 32), lane) << 1;
        const unsigned long long bmask =
            ((unsigned long long)__ballot_sync(0xffffffffu, c1 != 0) << 32) | __ballot_sync(0xffffffffu, c0 != 0);
        const int nbc = __popcll(bmask);
        // exclusive link offsets of cells lane and 32 + lane, in cell order
        uint32_t k0 = __popc(c0), k1 = __popc(c1), i0 = k0, i1 = k1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t0 = __shfl_up_sync(0xffffffffu, i0, o), t1 = __shfl_up_sync(0xffffffffu, i1, o);
            if (lane >= o) {
                i0 += t0;
                i1 += t1;
            }
        }
        const uint32_t tot0 = __shfl_sync(0xffffffffu, i0, 31);
        const uint32_t ex0 = i0 - k0, ex1 = tot0 + i1 - k1;
        const uint64_t bk = M.key[b];
        const long long h = M.g.h, half = M.g.half;
        const long long X0 = 4 * (long long)(bk & EMB_KEY_MASK) * h, Y0 = 4 * (long long)((bk >> EMB_KEY_BITS) & EMB_KEY_MASK) * h,
                        Z0 = 4 * (long long)(bk >> (2 * EMB_KEY_BITS)) * h;
        // the bin, clamped to the entries that exist (a replay whose counts left its plan
        // reports that through its count checks; its passes must stay in bounds)
        const uint32_t e1 = (uint64_t)M.bin_off[b + 1] < M.ent_cap ? M.bin_off[b + 1] : (uint32_t)M.ent_cap;
        const uint32_t e0 = M.bin_off[b] < e1 ? M.bin_off[b] : e1;
        if (e1 - e0 > EMB_BIN_MAX_ENTRIES) {
            // a hit record keeps the bin-local triangle index in 24 bits
            if (lane == 0) emb_set_status(st, EMB_ERR_CAPACITY);
            continue;
        }
        const int lh = __ffsll(h) - 1;  // h is a power of two
        // this item's cells with links: ranks [kb0, kb1) among the set bits of bmask
        const int kb0 = (int)(E.y & 0xFFu), kb1 = min(nbc, (int)((E.y >> 8) & 0xFFu));
        for (int cb = kb0; cb < kb1; cb += 32) {
            // the chunk's cells: set bits cb .. cb + 31 of bmask
            const int lo_bit = select64(bmask, cb);
            const int ncc = min(32, kb1 - cb);
            const int hi_bit = select64(bmask, cb + ncc - 1);
            const unsigned long long cmask = bmask & bit_range(lo_bit, hi_bit);
            // slot lane: its cell, candidates and link offset
            const bool active = lane < ncc;
            const int t = active ? select64(cmask, lane) : 0;
            const uint32_t cm_lo = __shfl_sync(0xffffffffu, c0, t & 31), cm_hi = __shfl_sync(0xffffffffu, c1, t & 31);
            const uint32_t ex_lo = __shfl_sync(0xffffffffu, ex0, t & 31), ex_hi = __shfl_sync(0xffffffffu, ex1, t & 31);
            const uint32_t cm = active ? (t < 32 ? cm_lo : cm_hi) : 0u;
            const uint32_t off = t < 32 ? ex_lo : ex_hi;
            S.cm[lane] = cm;
            S.hcnt[lane] = 0;
            __syncwarp();
            for (uint32_t e = e0; e < e1; e += LE_TILE) {
                // stage triangle `lane` of this tile and the chunk cells its reach box touches
                unsigned long long pm = 0;
                const uint32_t id = e + lane < e1 ? bin_ent[e + lane] : 0xFFFFFFFFu;
                if (id < M.T) {
                    const int4 A = rec[3 * (int64_t)id], B = rec[3 * (int64_t)id + 1], C = rec[3 * (int64_t)id + 2];
                    TriT s;
                    s.ax = A.x; s.ay = A.y; s.az = A.z;
                    s.bx = B.x; s.by = B.y; s.bz = B.z;
                    s.cx = C.x; s.cy = C.y; s.cz = C.z;
                    s.id = (int)id;
                    s.lox = min(A.x, min(B.x, C.x)); s.hix = max(A.x, max(B.x, C.x));
                    s.loy = min(A.y, min(B.y, C.y)); s.hiy = max(A.y, max(B.y, C.y));
                    s.loz = min(A.z, min(B.z, C.z)); s.hiz = max(A.z, max(B.z, C.z));
                    // edge vectors in 32 bits (coordinates below 2^25), products widened to 64
                    const int ux = B.x - A.x, uy = B.y - A.y, uz = B.z - A.z;
                    const int vx = C.x - A.x, vy = C.y - A.y, vz = C.z - A.z;
                    s.nx = (long long)uy * vz - (long long)uz * vy;
                    s.ny = (long long)uz * vx - (long long)ux * vz;
                    s.nz = (long long)ux * vy - (long long)uy * vx;
                    S.tile[lane] = s;
                    // cell i (centre X0 + (2i+1) half) reaches the box iff lo - h <= centre <= hi + h
                    // in 32 bits: coordinates and block origins lie below 2^25, h below 2^19
                    int r0[3], r1[3];
                    const int hh = (int)h + (int)half;
                    const int lo3[3] = {s.lox - (int)X0, s.loy - (int)Y0, s.loz - (int)Z0};
                    const int hi3[3] = {s.hix - (int)X0, s.hiy - (int)Y0, s.hiz - (int)Z0};
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int a_ = lo3[d] - hh;             // ceil(a / h)
                        const int c_ = hi3[d] + (int)h - (int)half;  // floor(c / h)
                        const int i0_ = -((-a_) >> lh), i1_ = c_ >> lh;
                        r0[d] = i0_ < 0 ? 0 : (i0_ > 4 ? 4 : i0_);
                        r1[d] = i1_ > 3 ? 3 : (i1_ < -1 ? -1 : i1_);
                    }
                    if (r0[0] <= r1[0] && r0[1] <= r1[1] && r0[2] <= r1[2]) {
                        const unsigned long long X = (unsigned long long)(((1u << (r1[0] + 1)) - 1u) & ~((1u << r0[0]) - 1u)) *
                                                     0x1111111111111111ull;
                        const unsigned long long Y = (((1ull << (4 * r1[1] + 4)) - 1ull) & ~((1ull << (4 * r0[1])) - 1ull)) *
                                                     0x0001000100010001ull;
                        const unsigned long long Z = bit_range(16 * r0[2], 16 * r1[2] + 15);
                        pm = X & Y & Z & cmask;
                    }
                }
                __syncwarp();
                // spread the tile's (triangle, cell) pairs over the lanes
                const int np = __popcll(pm);
                int incl = np;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int tt = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += tt;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                // the segment-end tests of the narrow path's line hits, queued per pair in
                // S.hq and run 32 hits at a time: lane g takes hit g of the queue
                int qn = 0;
                auto flush = [&]() {
                    __syncwarp();
                    const uint2 qe = lane < qn ? S.hq[lane] : make_uint2(0u, 0u);
                    const int nq = __popc(qe.y);
                    int qi = nq;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int tt = __shfl_up_sync(0xffffffffu, qi, o);
                        if (lane >= o) qi += tt;
                    }
                    const int qt = __shfl_sync(0xffffffffu, qi, 31);
                    for (int g0 = 0; g0 < qt; g0 += 32) {
                        const int g = g0 + lane;
                        int ei = 0;
#pragma unroll
                        for (int step = 16; step >= 1; step >>= 1) {
                            const int v = __shfl_sync(0xffffffffu, qi, ei + step - 1);
                            if (v <= g) ei += step;
                        }
                        ei = ei > 31 ? 31 : ei;
                        const int qex = __shfl_sync(0xffffffffu, qi - nq, ei);
                        const uint32_t qm = __shfl_sync(0xffffffffu, qe.y, ei), qx = __shfl_sync(0xffffffffu, qe.x, ei);
                        if (g >= qt) continue;
                        const int d = select32(qm, g - qex);
                        const int ti = (int)(qx & 31u), cell = (int)((qx >> 5) & 63u), slot = (int)((qx >> 11) & 31u);
                        const int px = (int)X0 + (2 * (cell & 3) + 1) * (int)half,
                                  py = (int)Y0 + (2 * ((cell >> 2) & 3) + 1) * (int)half,
                                  pz = (int)Z0 + (2 * (cell >> 4) + 1) * (int)half;
                        float q;
                        const bool ok = (qx >> 16) ? hit_segment_wide(S.tile[ti], px, py, pz, d, h, &q)
                                                   : hit_segment(S.tile[ti], px, py, pz, d, h, &q);
                        if (!ok) continue;
                        const int kk = atomicAdd(&S.hcnt[slot], 1);
                        if (kk < LE_BCAP)
                            S.hit[kk][slot] = make_uint2((e - e0 + (uint32_t)ti) | ((uint32_t)d << 24), __float_as_uint(q));
                    }
                    __syncwarp();
                    qn = 0;
                };
                for (int s0 = 0; s0 < total; s0 += 32) {
                    const int gidx = s0 + lane;
                    int lo = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        int v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                        if (v <= gidx) lo += step;
                    }
                    const int ti = lo > 31 ? 31 : lo;
                    const int excl_i = __shfl_sync(0xffffffffu, incl - np, ti);
                    const unsigned long long pmi = ((unsigned long long)__shfl_sync(0xffffffffu, (unsigned)(pm >> 32), ti) << 32) |
                                                   (unsigned long long)__shfl_sync(0xffffffffu, (unsigned)pm, ti);
                    uint32_t dm = 0, qx = 0;
                    bool wide = false;
                    if (gidx < total) {
                        const int cell = select64(pmi, gidx - excl_i);
                        const int slot = __popcll(cmask & ((1ull << cell) - 1ull));
                        const TriT &T = S.tile[ti];
                        const int px = (int)X0 + (2 * (cell & 3) + 1) * (int)half,
                                  py = (int)Y0 + (2 * ((cell >> 2) & 3) + 1) * (int)half,
                                  pz = (int)Z0 + (2 * (cell >> 4) + 1) * (int)half;
                        const uint32_t ccm = S.cm[slot];
                        const uint32_t local = e - e0 + (uint32_t)ti;
                        link_pair(
                            T, px, py, pz, ccm, h,
                            [&](int d, float q) {
                                const int kk = atomicAdd(&S.hcnt[slot], 1);
                                if (kk < LE_BCAP)
                                    S.hit[kk][slot] = make_uint2(local | ((uint32_t)d << 24), __float_as_uint(q));
                            },
                            dm, wide);
                        qx = (uint32_t)ti | ((uint32_t)cell << 5) | ((uint32_t)slot << 11) | ((uint32_t)wide << 16);
                    }
                    const unsigned qb = __ballot_sync(0xffffffffu, dm != 0);
                    if (qn + __popc(qb) > 32) flush();
                    if (dm) S.hq[qn + __popc(qb & ((1u << lane) - 1u))] = make_uint2(qx, dm);
                    qn += __popc(qb);
                }
                if (qn) flush();  // before the next tile replaces S.tile
                __syncwarp();
            }
            // resolve: the owner lane of each cell keeps, per direction, the nearest crossing
            // (`got` marks the directions with a kept hit)
            const int nh = active ? S.hcnt[lane] : 0;
            uint32_t got = 0;
            if (active) {
                const long long px = X0 + (2 * (t & 3) + 1) * half, py = Y0 + (2 * ((t >> 2) & 3) + 1) * half,
                                pz = Z0 + (2 * (t >> 4) + 1) * half;
                if (nh > LE_BCAP) {
                    emit_cell_slow(M, e0, e1, px, py, pz, h, cm, base + off, b * 64 + t, st);
                } else {
                    for (int k = 0; k < nh; ++k) {
                        const uint2 hv = S.hit[k][lane];
                        const int d = (int)(hv.x >> 24);
                        bool better = !((got >> d) & 1u);
                        if (!better) {
                            const int prev = S.best[d][lane];
                            // several faces cross this link: compare t exactly
                            int cx, cy, cz;
                            emb_dir(d, cx, cy, cz);
                            const int tn = (int)bin_ent[e0 + (hv.x & 0xFFFFFFu)];
                            const int to = (int)bin_ent[e0 + (S.hit[prev][lane].x & 0xFFFFFFu)];
                            if (!emb_ck((uint32_t)tn, M.T, st) || !emb_ck((uint32_t)to, M.T, st)) continue;
                            i128 Nn, No;
                            long long Mn, Mo;
                            tri_NM(rec, tn, px, py, pz, cx, cy, cz, Nn, Mn);
                            tri_NM(rec, to, px, py, pz, cx, cy, cz, No, Mo);
                            const i128 l = Nn * (i128)Mo, rr = No * (i128)Mn;
                            better = l < rr || (l == rr && tn < to);
                        }
                        if (better) {
                            S.best[d][lane] = (signed char)k;
                            got |= 1u << d;
                        }
                    }
                }
            }
            __syncwarp();
            // write the chunk's links: they are consecutive in the table (slot s holds links
            // off_s .. off_s + popc(cm_s) - 1 of the block), so the lanes take them in turn
            // and the stores coalesce; a cell written by the overflow path above is skipped
            const int nl = __popc(cm);
            int lincl = nl;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int tt = __shfl_up_sync(0xffffffffu, lincl, o);
                if (lane >= o) lincl += tt;
            }
            const int ltotal = __shfl_sync(0xffffffffu, lincl, 31);
            const uint32_t o_first = base + __shfl_sync(0xffffffffu, off, 0);
            for (int j0 = 0; j0 < ltotal; j0 += 32) {
                const int j = j0 + lane;
                int sl = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int v = __shfl_sync(0xffffffffu, lincl, sl + step - 1);
                    if (v <= j) sl += step;
                }
                sl = sl > 31 ? 31 : sl;
                const int s_excl = __shfl_sync(0xffffffffu, lincl - nl, sl);
                const uint32_t s_cm = __shfl_sync(0xffffffffu, cm, sl), s_got = __shfl_sync(0xffffffffu, got, sl);
                const int s_nh = __shfl_sync(0xffffffffu, nh, sl), s_t = __shfl_sync(0xffffffffu, t, sl);
                if (j >= ltotal || s_nh > LE_BCAP) continue;
                const uint32_t o = o_first + (uint32_t)j;
                if (o >= M.cap) {
                    emb_set_status(st, EMB_ERR_CAPACITY);
                    continue;
                }
                const int d = select32(s_cm, j - s_excl);
                int tr = -1;
                float q = -1.0f;
                if ((s_got >> d) & 1u) {
                    const uint2 hv = S.hit[S.best[d][sl]][sl];
                    tr = (int)bin_ent[e0 + (hv.x & 0xFFFFFFu)];
                    q = __uint_as_float(hv.y);
                } else {
                    emb_set_status(st, EMB_ERR_STATE);  // a fluid-to-solid link must cross the surface
                }
                M.o_cell[o] = (int32_t)(b * 64 + s_t);
                M.o_dir[o] = (uint8_t)d;
                M.o_q[o] = q;
                M.o_tri[o] = tr;
            }
            __syncwarp();
        }
    }
}

__global__ void k_store_count(const uint32_t *__restrict__ blk_off, int64_t n, int64_t *__restrict__ d_count)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *d_count = (int64_t)blk_off[n];
}

__global__ void k_set_status(int *st, int code) { emb_set_status(st, code); }

// EMB_ERR_CAPACITY when the block offsets count any link (a call with room for none).
__global__ void k_count_check(const uint32_t *__restrict__ blk_off, int64_t n, int *st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && blk_off[n] > 0) emb_set_status(st, EMB_ERR_CAPACITY);
}

__global__ void k_nonempty(const uint32_t *__restrict__ cnt, int64_t n, uint32_t *__restrict__ flag)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = cnt[i] ? 1u : 0u;
}

__global__ void k_compact_ids(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos, int64_t n,
                              uint32_t *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = (uint32_t)i;
}

static void free_candidates(emb_forest f, cudaStream_t s)
{
    if (f->cand) cudaFreeAsync(f->cand, s);
    f->cand = nullptr;
    uint32_t **bufs[] = {&f->blk_off, &f->work, &f->work_n};
    for (uint32_t **p : bufs) {
        if (*p) cudaFreeAsync(*p, s);
        *p = nullptr;
    }
}

// Link preparation for the finest level (enqueue only, neighbour table in place):
// cand (26 n words), cnt and flag (n + 1 uint32, scratch), work_n (n + 1: the
// work-list scan, count at work_n[n]), work (n), blk_off (n + 1: link offsets,
// total at blk_off[n]), tmp (scan scratch for n).
emb_status emb_enq_link_prep(const EmbLevel &lv, int lattice, uint64_t *cand, uint32_t *cnt, uint32_t *flag,
                             uint32_t *work_n, uint32_t *work, uint32_t *blk_off, uint64_t *tmp, cudaStream_t s,
                             uint64_t expect_work, uint64_t expect_links)
{
    EMB_CUDA_TRY(cudaMemsetAsync(cnt, 0, (lv.n + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(cudaMemsetAsync(flag, 0, (lv.n + 1) * sizeof(uint32_t), s));
    if (lv.n > 0) {
        EMB_LAUNCH((k_link_cand), emb_grid(lv.n, CAND_BLOCK), CAND_BLOCK, 0, s)(lv.mask, lv.nbr, lv.n, lattice, cand, cnt,
                                                                  emb_status_word(), lv.d_n);
        EMB_LAUNCH((k_nonempty), emb_grid(lv.n, 256), 256, 0, s)(cnt, lv.n, flag);
    }
    emb_status rc = emb_scan_into_expect(flag, work_n, lv.n, tmp, expect_work, s);
    if (rc != EMB_OK) return rc;
    if (lv.n > 0) EMB_LAUNCH((k_compact_ids), emb_grid(lv.n, 256), 256, 0, s)(flag, work_n, lv.n, work);
    EMB_CUDA_TRY(cudaGetLastError());
    return emb_scan_into_expect(cnt, blk_off, lv.n, tmp, expect_links, s);
}

// Work items (thread per block with links): block b with l links, a bin of nt
// triangles and nbc cells with links costs about l * nt exact tests and is cut
// into P = min(ceil(l nt / LE_SPLIT_COST), nbc, LE_SPLIT_MAX) parts of
// ceil(nbc / P) consecutive cells.  The first part is the block's own item; the
// others are appended to `extra`, and when that is full the block stays whole,
// which changes the speed only.  The lanes of a warp take their extra slots with one
// atomic (a single counter taken once per heavy block serialised the kernel).
__global__ void k_link_split(const uint32_t *__restrict__ work, const uint32_t *__restrict__ work_n,
                             const uint64_t *__restrict__ cand, const uint32_t *__restrict__ blk_off,
                             const uint32_t *__restrict__ bin_off, int64_t n, uint2 *__restrict__ witem,
                             uint2 *__restrict__ extra, unsigned long long *__restrict__ extra_n, uint32_t cap)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool live = i < n && i < (int64_t)*work_n;
    if (__ballot_sync(0xffffffffu, live) == 0u) return;  // the whole warp
    const uint32_t b = live ? work[i] : 0u;
    uint32_t nbc = 0;
    unsigned long long P = 0;
    if (live) {
        uint64_t bm = 0;
        for (int d = 0; d < 26; ++d) bm |= cand[(int64_t)b * 26 + d];
        nbc = (uint32_t)__popcll(bm);
        const unsigned long long l = blk_off[b + 1] - blk_off[b], nt = bin_off[b + 1] - bin_off[b];
        P = (l * nt + LE_SPLIT_COST - 1) / LE_SPLIT_COST;
        P = P < nbc ? P : nbc;
        P = P < LE_SPLIT_MAX ? P : LE_SPLIT_MAX;
    }
    uint32_t span = nbc;
    if (P > 1) {
        span = (uint32_t)((nbc + P - 1) / P);
        P = (nbc + span - 1) / span;  // no empty part
    }
    // the warp's extra slots: one atomic, each lane's range from an exclusive prefix
    const uint32_t want = P > 1 ? (uint32_t)(P - 1) : 0u;
    uint32_t incl = want;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long wbase = 0;
    if (lane == 31 && total > 0) wbase = atomicAdd(extra_n, (unsigned long long)total);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    if (!live) return;
    if (P > 1) {
        const unsigned long long base = wbase + (incl - want);
        if (base + P - 1 > cap) {
            for (unsigned long long e = base; e < cap; ++e) extra[e] = make_uint2(EMB_BIG_NONE, 0u);
            span = nbc;
        } else {
            for (uint32_t p = 1; p < (uint32_t)P; ++p) {
                const uint32_t k0 = p * span, k1 = k0 + span < nbc ? k0 + span : nbc;
                extra[base + p - 1] = make_uint2(b, k0 | (k1 << 8));
            }
        }
    }
    witem[i] = make_uint2(b, 0u | (span << 8));
}

int64_t emb_link_extra_capacity(int64_t n)
{
    const int64_t c = 2 * n + 4096;
    return c < (1 << 20) ? c : (1 << 20);
}

// Enqueue only: after emb_enq_link_prep and the finest bins; witem holds n entries.
emb_status emb_enq_link_split(const EmbLevel &lv, const uint32_t *work, const uint32_t *work_n, const uint64_t *cand,
                              const uint32_t *blk_off, const uint32_t *bin_off, uint2 *witem, uint2 *extra,
                              unsigned long long *extra_n, uint32_t extra_cap, cudaStream_t s)
{
    EMB_CUDA_TRY(cudaMemsetAsync(extra_n, 0, sizeof(unsigned long long), s));
    if (lv.n > 0)
        EMB_LAUNCH((k_link_split), emb_grid(lv.n, 256), 256, 0, s)(work, work_n, cand, blk_off, bin_off, lv.n, witem,
                                                                   extra, extra_n, extra_cap);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

size_t emb_link_emit_smem() { return LE_WARPS * sizeof(LeWarp); }

static int g_le_per_sm = 0, g_le_sms = 0;

// Kernel attributes and occupancy of the link kernel (once per process; call
// before any stream capture).
emb_status emb_link_emit_init()
{
    if (g_le_per_sm) return EMB_OK;
    const size_t smem = emb_link_emit_smem();
    EMB_CUDA_TRY(cudaFuncSetAttribute(k_link_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, per_sm = 0;
    EMB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_link_emit, LE_WARPS * 32, smem));
    EMB_CUDA_TRY(cudaGetDevice(&dev));
    EMB_CUDA_TRY(cudaDeviceGetAttribute(&g_le_sms, cudaDevAttrMultiProcessorCount, dev));
    g_le_per_sm = per_sm < 1 ? 1 : per_sm;
    return EMB_OK;
}

// One persistent launch over the meshes of `tab`; `next` is the queue cursor.
// The grid fills every SM (ctas_per_sm resident CTAs each, 0 = as many as fit)
// unless the work is smaller: with `items` > 0 (the blocks with links, known to
// the caller) it stops at about items_per_warp items per warp, so that a small
// mesh leaves SMs to the kernels of other streams.
emb_status emb_enq_link_emit(const LinkTable &tab, unsigned int *next, int ctas_per_sm, cudaStream_t s, int64_t items)
{
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    emb_status rc = emb_link_emit_init();
    if (rc != EMB_OK) return rc;
    const size_t smem = emb_link_emit_smem();
    const int use = ctas_per_sm > 0 && ctas_per_sm < g_le_per_sm ? ctas_per_sm : g_le_per_sm;
    int64_t grid = (int64_t)use * g_le_sms;
    if (items > 0) {
        const int64_t items_per_warp = 4;
        const int64_t need = (items + LE_WARPS * items_per_warp - 1) / (LE_WARPS * items_per_warp);
        if (need < grid) grid = need;
    }
    EMB_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(unsigned int), s));
    EMB_LAUNCH((k_link_emit), (int)grid, LE_WARPS * 32, smem, s)(tab, next, st);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

// f->n_links: -1 no candidates; -2 candidates built, the link count still on the device
// (blk_off[n]); >= 0 the count, read back.  With read_count the count is read back
// (synchronising s); without it nothing is read back.
#define EMB_LINKS_ON_DEVICE (-2)
static emb_status build_candidates(emb_forest f, int lattice, cudaStream_t s, bool read_count)
{
    int L = f->max_level;
    if (f->top != L || !f->lv[L].mask_valid) return EMB_ERR_STATE;
    if ((f->n_links >= 0 || f->n_links == EMB_LINKS_ON_DEVICE) && f->cand_lattice == lattice && f->cand) {
        if (f->n_links >= 0 || !read_count) return EMB_OK;
        uint32_t total = 0;
        EMB_CUDA_TRY(cudaMemcpyAsync(&total, f->blk_off + f->lv[L].n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        EMB_CUDA_TRY(cudaStreamSynchronize(s));
        f->n_links = (int64_t)total;
        return EMB_OK;
    }
    EmbLevel &lv = f->lv[L];
    emb_status rc = emb_build_neighbors(lv, s);
    if (rc != EMB_OK) return rc;
    free_candidates(f, s);
    EMB_CUDA_TRY(emb_malloc_async(&f->cand, (lv.n * 26 + 1) * sizeof(uint64_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&f->blk_off, (lv.n + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&f->work_n, (lv.n + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&f->work, (lv.n + 1) * sizeof(uint32_t), s));
    if (!f->next) EMB_CUDA_TRY(cudaMalloc(&f->next, sizeof(unsigned int)));
    uint32_t *cnt = nullptr, *flag = nullptr;
    uint64_t *tmp = nullptr;
    EMB_CUDA_TRY(emb_malloc_async(&cnt, (lv.n + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&flag, (lv.n + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&tmp, emb_scan_tmp_words(lv.n) * sizeof(uint64_t), s));
    rc = emb_enq_link_prep(lv, lattice, f->cand, cnt, flag, f->work_n, f->work, f->blk_off, tmp, s);
    if (rc != EMB_OK) return rc;
    EMB_CUDA_TRY(cudaFreeAsync(cnt, s));
    EMB_CUDA_TRY(cudaFreeAsync(flag, s));
    EMB_CUDA_TRY(cudaFreeAsync(tmp, s));
    f->cand_lattice = lattice;
    f->n_links = EMB_LINKS_ON_DEVICE;
    if (!read_count) return EMB_OK;
    uint32_t total = 0;
    EMB_CUDA_TRY(cudaMemcpyAsync(&total, f->blk_off + lv.n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    EMB_CUDA_TRY(cudaStreamSynchronize(s));
    f->n_links = (int64_t)total;
    return EMB_OK;
}

extern "C" emb_status emb_cutlinks_count(emb_forest f, int32_t lattice, int64_t *h_count, void *stream)
{
    if (!f || !h_count || (lattice != 19 && lattice != 27)) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    emb_status rc = build_candidates(f, lattice, emb_stream(stream), true);
    if (rc != EMB_OK) return rc;
    *h_count = f->n_links;
    return EMB_OK;
}

extern "C" emb_status emb_cutlinks_prepare(emb_forest f, int32_t lattice, void *stream)
{
    if (!f || (lattice != 19 && lattice != 27)) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    return build_candidates(f, lattice, emb_stream(stream), false);
}

extern "C" emb_status emb_cutlinks(emb_forest f, emb_bins b, int32_t lattice, int32_t *d_cell, uint8_t *d_dir, float *d_q,
                                   int32_t *d_tri, int64_t capacity, int64_t *d_count, void *stream)
{
    if (!f || !b || (lattice != 19 && lattice != 27) || capacity < 0) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    if (b->f != f || b->level != f->max_level || f->top != f->max_level) return EMB_ERR_STATE;
    {
        // the outputs may be page-locked host memory: the kernel then writes the table
        // straight over the host link, with no copy after it
        void *v[5];
        if (emb_device_view(d_cell, &v[0]) != EMB_OK || emb_device_view(d_dir, &v[1]) != EMB_OK ||
            emb_device_view(d_q, &v[2]) != EMB_OK || emb_device_view(d_tri, &v[3]) != EMB_OK ||
            emb_device_view(d_count, &v[4]) != EMB_OK)
            return EMB_ERR_BAD_INPUT;
        d_cell = (int32_t *)v[0];
        d_dir = (uint8_t *)v[1];
        d_q = (float *)v[2];
        d_tri = (int32_t *)v[3];
        d_count = (int64_t *)v[4];
    }
    cudaStream_t s = emb_stream(stream);
    if (f->lv[f->max_level].n == 0) {
        // an empty finest level (nothing was refined down to it): no links
        if (d_count) EMB_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int64_t), s));
        f->n_links = 0;
        return EMB_OK;
    }
    if (!b->off) return EMB_ERR_STATE;
    {
        // complete bins (a pair list that proved too small is redone here)
        const emb_status rb = emb_bins_sync(b);
        if (rb != EMB_OK) return rb;
    }
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    // without a count read back before (emb_cutlinks_count), the count stays on the
    // device: the kernel writes no link past `capacity` and sets EMB_ERR_CAPACITY
    emb_status rc = build_candidates(f, lattice, s, false);
    if (rc != EMB_OK) return rc;
    EmbLevel &lv = f->lv[f->max_level];
    if (d_count) EMB_LAUNCH((k_store_count), 1, 32, 0, s)(f->blk_off, lv.n, d_count);
    if (f->n_links >= 0 && f->n_links > capacity) {
        EMB_LAUNCH((k_set_status), 1, 1, 0, s)(st, EMB_ERR_CAPACITY);
        EMB_CUDA_TRY(cudaGetLastError());
        return EMB_ERR_CAPACITY;
    }
    if (f->n_links == 0) return EMB_OK;
    if (capacity == 0) {
        // nothing may be written: the count on the device decides whether that is an error
        EMB_LAUNCH((k_count_check), 1, 32, 0, s)(f->blk_off, lv.n, st);
        EMB_CUDA_TRY(cudaGetLastError());
        return EMB_OK;
    }
    if (!d_cell || !d_dir || !d_q || !d_tri) return EMB_ERR_BAD_INPUT;
    LinkTable tab;
    tab.n = 1;
    LinkMesh &M = tab.m[0];
    M.key = lv.key;
    M.cand = f->cand;
    M.blk_off = f->blk_off;
    M.bin_off = b->off;
    M.bin_ent = b->ent;
    M.ent_cap = (uint64_t)b->npairs;  // complete after emb_bins_sync
    M.rec = b->m->rec;
    M.T = (uint32_t)b->m->T;
    M.work_n = f->work_n + lv.n;
    M.o_cell = d_cell;
    M.o_dir = d_dir;
    M.o_q = d_q;
    M.o_tri = d_tri;
    M.g = level_geom(f, f->max_level);
    M.cap = (uint32_t)(capacity < 0xFFFFFFFFll ? capacity : 0xFFFFFFFFll);
    M.nblk = lv.n;
    // parts of heavy blocks
    const int64_t xcap = emb_link_extra_capacity(lv.n);
    char *sp = nullptr;
    const size_t a_w = ((size_t)(lv.n + 1) * sizeof(uint2) + 255) & ~(size_t)255;
    EMB_CUDA_TRY(emb_malloc_async((void **)&sp, 256 + a_w + (size_t)xcap * sizeof(uint2), s));
    unsigned long long *xn = (unsigned long long *)sp;
    uint2 *witem = (uint2 *)(sp + 256);
    uint2 *extra = (uint2 *)(sp + 256 + a_w);
    rc = emb_enq_link_split(lv, f->work, f->work_n + lv.n, f->cand, f->blk_off, b->off, witem, extra, xn, (uint32_t)xcap,
                            s);
    if (rc == EMB_OK) {
        M.witem = witem;
        M.extra = extra;
        M.extra_n = xn;
        M.extra_cap = (uint32_t)xcap;
        rc = emb_enq_link_emit(tab, f->next, 0, s, 0);
    }
    cudaFreeAsync(sp, s);
    if (rc != EMB_OK) return rc;
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

// ---------------------------------------------------------------------------
// Predicate probe: the device predicates of the path on caller-given queries
// ---------------------------------------------------------------------------
// One thread per query of 15 int64 (layout in emb.h, emb_probe_predicates).
__global__ void k_probe(int kind, const long long *__restrict__ in, int64_t n, int32_t *__restrict__ hit,
                        float *__restrict__ qout)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long *r = in + 15 * i;
    const int4 A = make_int4((int)r[0], (int)r[1], (int)r[2], 0), B = make_int4((int)r[3], (int)r[4], (int)r[5], 0),
               C = make_int4((int)r[6], (int)r[7], (int)r[8], 0);
    int h_ = 0;
    float q_ = -1.0f;
    if (kind == EMB_PROBE_XLINE) {
        // the x-line test of the filter and the voxelizer
        const long long nx = ((long long)B.y - A.y) * ((long long)C.z - A.z) - ((long long)B.z - A.z) * ((long long)C.y - A.y);
        if (nx != 0) {
            const int sx = nx > 0 ? 1 : -1, py = (int)r[10], pz = (int)r[11];
            h_ = emb_orient_yz(A.y, A.z, B.y, B.z, py, pz) == sx && emb_orient_yz(B.y, B.z, C.y, C.z, py, pz) == sx &&
                 emb_orient_yz(C.y, C.z, A.y, A.z, py, pz) == sx;
        }
    } else if (kind == EMB_PROBE_BOX) {
        // the overlap test of the binning and the refine flags (closed box [lo, hi])
        h_ = emb_point_in_box(A, r[9], r[10], r[11], r[12], r[13], r[14]) ||
             emb_point_in_box(B, r[9], r[10], r[11], r[12], r[13], r[14]) ||
             emb_point_in_box(C, r[9], r[10], r[11], r[12], r[13], r[14]) ||
             emb_tri_box(A, B, C, r[9], r[10], r[11], r[12], r[13], r[14]);
    } else {
        const long long px = r[9], py = r[10], pz = r[11], h = r[13];
        const int d = (int)r[12];
        if (r[12] < 1 || r[12] > 26 || h <= 0) {
            h_ = -1;  // not a query of this kind
        } else if (kind == EMB_PROBE_SEGMENT) {
            // the exact per-direction test of the link kernel's rescan path
            const long long ax = A.x - px, ay = A.y - py, az = A.z - pz;
            const long long bx = B.x - px, by = B.y - py, bz = B.z - pz;
            const long long qx = C.x - px, qy = C.y - py, qz = C.z - pz;
            const long long ux = bx - ax, uy = by - ay, uz = bz - az, vx = qx - ax, vy = qy - ay, vz = qz - az;
            const long long nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
            const long long m1x = ay * bz - az * by, m1y = az * bx - ax * bz, m1z = ax * by - ay * bx;
            const long long m2x = by * qz - bz * qy, m2y = bz * qx - bx * qz, m2z = bx * qy - by * qx;
            const long long m3x = qy * az - qz * ay, m3y = qz * ax - qx * az, m3z = qx * ay - qy * ax;
            int cx, cy, cz;
            emb_dir(d, cx, cy, cz);
            i128 D = 0;
            bool haveD = false;
            if (seg_cross(cx, cy, cz, h, ax, ay, az, bx, by, bz, qx, qy, qz, nx, ny, nz, m1x, m1y, m1z, m2x, m2y, m2z,
                          m3x, m3y, m3z, D, haveD)) {
                const long long nc = cdot(cx, cy, cz, nx, ny, nz);
                const i128 N = nc > 0 ? D : -D;
                const long long M = nc > 0 ? nc : -nc;
                h_ = 1;
                q_ = __fdiv_rn(i128_to_float(N), (float)M * (float)h);
            }
        } else {
            // the link kernel's per-pair path (32-bit moments within 2^14 of P, else 64-bit)
            TriT T;
            T.ax = A.x; T.ay = A.y; T.az = A.z;
            T.bx = B.x; T.by = B.y; T.bz = B.z;
            T.cx = C.x; T.cy = C.y; T.cz = C.z;
            T.id = 0;
            T.lox = min(A.x, min(B.x, C.x)); T.hix = max(A.x, max(B.x, C.x));
            T.loy = min(A.y, min(B.y, C.y)); T.hiy = max(A.y, max(B.y, C.y));
            T.loz = min(A.z, min(B.z, C.z)); T.hiz = max(A.z, max(B.z, C.z));
            const long long ux = (long long)B.x - A.x, uy = (long long)B.y - A.y, uz = (long long)B.z - A.z;
            const long long vx = (long long)C.x - A.x, vy = (long long)C.y - A.y, vz = (long long)C.z - A.z;
            T.nx = uy * vz - uz * vy;
            T.ny = uz * vx - ux * vz;
            T.nz = ux * vy - uy * vx;
            uint32_t dm = 0;
            bool wide = false;
            link_pair(
                T, px, py, pz, 1u << d, h,
                [&](int dd, float qq) {
                    if (dd == d) {
                        h_ = 1;
                        q_ = qq;
                    }
                },
                dm, wide);
            float qq;
            if (((dm >> d) & 1u) &&
                (wide ? hit_segment_wide(T, px, py, pz, d, h, &qq) : hit_segment(T, px, py, pz, d, h, &qq))) {
                h_ = 1;
                q_ = qq;
            }
        }
    }
    hit[i] = h_;
    qout[i] = q_;
}

extern "C" emb_status emb_probe_predicates(int32_t kind, const int64_t *d_in, int64_t n, int32_t *d_hit, float *d_q,
                                           void *stream)
{
    if (kind < EMB_PROBE_XLINE || kind > EMB_PROBE_BOX || n < 0) return EMB_ERR_BAD_INPUT;
    if (n == 0) return EMB_OK;
    if (!d_in || !d_hit || !d_q) return EMB_ERR_BAD_INPUT;
    EMB_LAUNCH((k_probe), emb_grid(n, 128), 128, 0, emb_stream(stream))(kind, (const long long *)d_in, n, d_hit, d_q);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}
