// Spatial binning (Sec. 3.3).
//
// Step 1, the filter (the 1-D ray indicator of Alg. 1): a triangle takes part
// in voxelizing level L only if some +x line through level-L cell centres
// crosses it.  The test is exact and the survivors are compacted into an
// ascending id list by flag / exclusive scan / scatter (no sort).
//
// Steps 2-9 at the finest level (Alg. 2): every triangle is paired with the
// existing blocks whose box, dilated by half a cell, it overlaps (exact
// separating-axis test).  A link P -> P + h c starts at a cell centre, at least
// h/2 inside the block, and has L-infinity length h, so it stays inside the box
// dilated by h/2.  One pass over the geometry counts the pairs per block with
// integer atomics (the count is also the pair's slot in its block) and appends
// (block, slot, triangle) to a pair list; offsets come from an exclusive scan and
// a scatter of the list fills the CSR bins.
#include <stdlib.h>
#include <string.h>

#include "emb_internal.cuh"

// Exact x-line filter of triangle t: 1 iff its yz-projection contains the centre of
// some x-line of the level (perturbed orientation tests, Sec. 3.4 parity rule).  In
// 32-bit arithmetic: coordinates lie below 2^25, the orientation products are widened
// to 64 bits.
__device__ __forceinline__ int orient_yz32(int uy, int uz, int vy, int vz, int py, int pz)
{
    const int ey = vy - uy, ez = vz - uz;
    const long long o = (long long)ey * (pz - uz) - (long long)ez * (py - uy);
    if (o != 0) return o > 0 ? 1 : -1;
    if (ez != 0) return ez > 0 ? -1 : 1;
    return ey > 0 ? 1 : (ey < 0 ? -1 : 0);
}
__device__ __forceinline__ uint32_t xline_hit32(const int4 *__restrict__ rec, int64_t t, const LevelGeom &g)
{
    const int4 A = rec[3 * t], B = rec[3 * t + 1], C = rec[3 * t + 2];
    const long long nx = (long long)(B.y - A.y) * (C.z - A.z) - (long long)(B.z - A.z) * (C.y - A.y);
    if (nx == 0) return 0;
    const int sx = nx > 0 ? 1 : -1;
    const int lh = g.lh, half = (int)g.half, nc = (int)g.ncell;
    const int mny = min(A.y, min(B.y, C.y)), mxy = max(A.y, max(B.y, C.y));
    const int mnz = min(A.z, min(B.z, C.z)), mxz = max(A.z, max(B.z, C.z));
    int j0 = -((-(mny - half)) >> lh), j1 = (mxy - half) >> lh;
    int k0 = -((-(mnz - half)) >> lh), k1 = (mxz - half) >> lh;
    j0 = j0 < 0 ? 0 : j0;
    k0 = k0 < 0 ? 0 : k0;
    j1 = j1 > nc - 1 ? nc - 1 : j1;
    k1 = k1 > nc - 1 ? nc - 1 : k1;
    if (j1 < j0 || k1 < k0) return 0;
    // the line nearest the centroid first: it settles a large triangle in one test
    int jc = ((A.y + B.y + C.y) >> lh) / 3, kc = ((A.z + B.z + C.z) >> lh) / 3;
    jc = jc < j0 ? j0 : (jc > j1 ? j1 : jc);
    kc = kc < k0 ? k0 : (kc > k1 ? k1 : kc);
    {
        const int py = (2 * jc + 1) * half, pz = (2 * kc + 1) * half;
        if (orient_yz32(A.y, A.z, B.y, B.z, py, pz) == sx && orient_yz32(B.y, B.z, C.y, C.z, py, pz) == sx &&
            orient_yz32(C.y, C.z, A.y, A.z, py, pz) == sx)
            return 1;
    }
    for (int k = k0; k <= k1; ++k) {
        const int pz = (2 * k + 1) * half;
        for (int j = j0; j <= j1; ++j) {
            const int py = (2 * j + 1) * half;
            if (orient_yz32(A.y, A.z, B.y, B.z, py, pz) == sx && orient_yz32(B.y, B.z, C.y, C.z, py, pz) == sx &&
                orient_yz32(C.y, C.z, A.y, A.z, py, pz) == sx)
                return 1;
        }
    }
    return 0;
}

// Per-triangle filter flags (the ablation that keeps the list uncompacted).
__global__ void k_xfilter(const int4 *__restrict__ rec, int64_t T, LevelGeom g, uint32_t *__restrict__ flag)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    flag[t] = xline_hit32(rec, t, g);
}

// The filter as one bit per triangle: warp word t / 32 (bit t % 32) and its popcount.
// The block size is a multiple of 32, so a warp covers triangles 32 w .. 32 w + 31.
__global__ void k_xfilter_bits(const int4 *__restrict__ rec, int64_t T, LevelGeom g, uint32_t *__restrict__ word,
                               uint32_t *__restrict__ wcnt)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t hit = t < T ? xline_hit32(rec, t, g) : 0u;
    const uint32_t m = __ballot_sync(0xffffffffu, hit != 0u);
    if ((threadIdx.x & 31) == 0 && t < T) {
        word[t >> 5] = m;
        wcnt[t >> 5] = (uint32_t)__popc(m);
    }
}

// Kept triangles in ascending order, one thread per filter word: the set bits of word
// w go, in order, to the places from the exclusive prefix of its word; the kept count
// is stored at count.
__global__ void k_compact_bits(const uint32_t *__restrict__ word, const uint32_t *__restrict__ wpos, int64_t T,
                               uint32_t *__restrict__ flist, uint32_t *count)
{
    const int64_t W = (T + 31) >> 5;
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    uint32_t m = word[w];
    uint32_t o = wpos[w];
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        flist[o++] = (uint32_t)(32 * w + b);
    }
    if (w == 0) *count = wpos[W];
}

__global__ void k_compact(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos, int64_t n,
                          uint32_t *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = (uint32_t)i;
}

// Triangle t as the binning pass sees it: false for a degenerate triangle (zero
// normal, never crossed by a link), else its vertices and candidate block ranges.
__device__ __forceinline__ bool bin_setup(const int4 *__restrict__ rec, int64_t t, const LevelGeom &g, long long dil,
                                          int4 &A, int4 &B, int4 &C, long long b0[3], long long b1[3])
{
    A = rec[3 * t];
    B = rec[3 * t + 1];
    C = rec[3 * t + 2];
    long long ux = (long long)B.x - A.x, uy = (long long)B.y - A.y, uz = (long long)B.z - A.z;
    long long vx = (long long)C.x - A.x, vy = (long long)C.y - A.y, vz = (long long)C.z - A.z;
    if (uy * vz - uz * vy == 0 && uz * vx - ux * vz == 0 && ux * vy - uy * vx == 0) return false;
    emb_block_range(min(A.x, min(B.x, C.x)), max(A.x, max(B.x, C.x)), g.lW, dil, g.nb, b0[0], b1[0]);
    emb_block_range(min(A.y, min(B.y, C.y)), max(A.y, max(B.y, C.y)), g.lW, dil, g.nb, b0[1], b1[1]);
    emb_block_range(min(A.z, min(B.z, C.z)), max(A.z, max(B.z, C.z)), g.lW, dil, g.nb, b0[2], b1[2]);
    return true;
}

__device__ __forceinline__ unsigned long long box_items(const long long b0[3], const long long b1[3])
{
    if (b1[0] < b0[0] || b1[1] < b0[1] || b1[2] < b0[2]) return 0;
    return (unsigned long long)(b1[0] - b0[0] + 1) * (unsigned long long)(b1[1] - b0[1] + 1) *
           (unsigned long long)(b1[2] - b0[2] + 1);
}


// The pair kernel's set-up in 32-bit arithmetic (coordinates, block origins, widths and
// dilations below 2^25 in magnitude; the degenerate test widens its products to 64 bits).
__device__ __forceinline__ bool bin_setup32(const int4 *__restrict__ rec, int64_t t, int lW, int dil, int nb, int4 &A,
                                            int4 &B, int4 &C, int b0[3], int b1[3])
{
    A = rec[3 * t];
    B = rec[3 * t + 1];
    C = rec[3 * t + 2];
    const int ux = B.x - A.x, uy = B.y - A.y, uz = B.z - A.z;
    const int vx = C.x - A.x, vy = C.y - A.y, vz = C.z - A.z;
    if ((long long)uy * vz - (long long)uz * vy == 0 && (long long)uz * vx - (long long)ux * vz == 0 &&
        (long long)ux * vy - (long long)uy * vx == 0)
        return false;
    const int mn[3] = {min(A.x, min(B.x, C.x)), min(A.y, min(B.y, C.y)), min(A.z, min(B.z, C.z))};
    const int mx[3] = {max(A.x, max(B.x, C.x)), max(A.y, max(B.y, C.y)), max(A.z, max(B.z, C.z))};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        b0[d] = -((-(mn[d] - dil - (1 << lW))) >> lW);  // ceil
        b1[d] = (mx[d] + dil) >> lW;                    // floor
        if (b0[d] < 0) b0[d] = 0;
        if (b1[d] > nb - 1) b1[d] = nb - 1;
    }
    return true;
}
__device__ __forceinline__ bool bin_pt32(const int4 &P, int lx, int ly, int lz, int hx, int hy, int hz)
{
    return P.x >= lx && P.x <= hx && P.y >= ly && P.y <= hy && P.z >= lz && P.z <= hz;
}

// Pair list of one binning pass: entry e is (block, slot in the block) and the triangle.
struct PairList {
    uint2 *bs;
    uint32_t *tri;
    unsigned long long *n;  // entries requested (may exceed cap)
    uint64_t cap;
    __device__ __forceinline__ void put(unsigned long long e, uint32_t id, uint32_t slot, uint32_t t) const
    {
        if (e < cap) {
            bs[e] = make_uint2(id, slot);
            tri[e] = t;
        }
    }
};

// Pair (t, block (bx, by, bz)) if the block exists and t overlaps its dilated box.
__device__ __forceinline__ void bin_block(const int4 &A, const int4 &B, const int4 &C, uint32_t t, long long bx,
                                          long long by, long long bz, const LevelGeom &g, long long dil,
                                          const EmbLookup &lk, uint32_t *__restrict__ cnt, const PairList &PL)
{
    const int32_t id = emb_lookup(lk, bx, by, bz);
    if (id < 0) return;
    const long long lx = bx * g.W - dil, ly = by * g.W - dil, lz = bz * g.W - dil;
    const long long hx = lx + g.W + 2 * dil, hy = ly + g.W + 2 * dil, hz = lz + g.W + 2 * dil;
    if (!(emb_point_in_box(A, lx, ly, lz, hx, hy, hz) || emb_point_in_box(B, lx, ly, lz, hx, hy, hz) ||
          emb_point_in_box(C, lx, ly, lz, hx, hy, hz) || emb_tri_box(A, B, C, lx, ly, lz, hx, hy, hz)))
        return;
    const uint32_t slot = atomicAdd(cnt + id, 1u);
    PL.put(atomicAdd(PL.n, 1ull), (uint32_t)id, slot, t);
}

// Per warp: (triangle lane, bx, by, bz) and block id of pairs whose triangle has no vertex
// in the dilated block, waiting for the separating-axis test.
struct SatQueue {
    int4 e[EMB_WU_WARPS][64];
    int32_t id[EMB_WU_WARPS][64];
};

// Per warp: pairs (block, slot; triangle) waiting to be appended to the pair list, so
// that the list's one counter is taken once per 32 or more pairs instead of once per
// round (a counter that every warp takes each round serialised the kernel).
struct PairBuf {
    uint2 bs[EMB_WU_WARPS][64];
    uint32_t tri[EMB_WU_WARPS][64];
};

// Appends the buffered pairs of warp w to the list with one atomic; coalesced stores.
__device__ __forceinline__ void pair_flush(PairBuf &PB, int w, int &bn, int lane, const PairList &PL)
{
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(PL.n, (unsigned long long)bn);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int j = lane; j < bn; j += 32) {
        const uint2 v = PB.bs[w][j];
        PL.put(base + (unsigned long long)j, v.x, v.y, PB.tri[w][j]);
    }
    __syncwarp();
    bn = 0;
}

// Appends the pairs of the lanes with `hit` through the warp's buffer: each pair takes
// its slot in its block at once (lanes that hit the same block with one atomic); the
// buffer is flushed once it holds 32 pairs or more (bn, warp-uniform, is below 32 on
// entry, so 64 entries suffice).
__device__ __forceinline__ void bin_append_buf(bool hit, int32_t id, uint32_t tri, int lane, uint32_t *__restrict__ cnt,
                                               PairBuf &PB, int w, int &bn, const PairList &PL)
{
    const unsigned hm = __ballot_sync(0xffffffffu, hit);
    if (!hm) return;
    if (hit) {
        const unsigned grp = __match_any_sync(hm, id);
        const int lead = __ffs(grp) - 1;
        uint32_t first = 0;
        if (lane == lead) first = atomicAdd(cnt + id, (uint32_t)__popc(grp));
        first = __shfl_sync(grp, first, lead);
        const int pos = bn + __popc(hm & ((1u << lane) - 1u));
        PB.bs[w][pos] = make_uint2((uint32_t)id, first + (uint32_t)__popc(grp & ((1u << lane) - 1u)));
        PB.tri[w][pos] = tri;
    }
    bn += __popc(hm);
    if (bn >= 32) pair_flush(PB, w, bn, lane, PL);
}

// The separating-axis test of the first n queued pairs, one per lane.
__device__ __forceinline__ void bin_sat_batch(const SatQueue &Q2, int w, int n, int lane, const WuTri &S, int64_t t0,
                                              const LevelGeom &g, long long dil, uint32_t *__restrict__ cnt,
                                              PairBuf &PB, int &bn, const PairList &PL)
{
    bool hit = false;
    int32_t id = -1;
    int ti = 0;
    if (lane < n) {
        const int4 e = Q2.e[w][lane];
        id = Q2.id[w][lane];
        ti = e.x;
        const long long lx = (long long)e.y * g.W - dil, ly = (long long)e.z * g.W - dil, lz = (long long)e.w * g.W - dil;
        const long long hx = lx + g.W + 2 * dil, hy = ly + g.W + 2 * dil, hz = lz + g.W + 2 * dil;
        hit = emb_tri_box(S.A[ti], S.B[ti], S.C[ti], lx, ly, lz, hx, hy, hz);
    }
    bin_append_buf(hit, id, (uint32_t)(t0 + ti), lane, cnt, PB, w, bn, PL);
}

// The (triangle, candidate block) pairs of 32 consecutive triangles, spread evenly over
// the warp's lanes by a prefix sum of the lanes' candidate counts, so that every lane
// tests one pair per round (a triangle with very many candidates goes to the chunk queue
// instead), the pairs buffered per warp for the list.  A pair whose triangle has a vertex
// in the dilated block is decided at once; the others wait in a per-warp queue and take
// the full separating-axis test 32 at a time, so that the lanes run it together.  (Visiting the union of the 32
// triangles' candidate blocks instead, one lane per block against all 32 triangles,
// measured slower here: the lanes' overlap tests diverge.)  Degenerate triangles (zero
// normal) are never crossed by a link and are left out.  Eight CTAs per SM (64
// registers, a few spills) hide the lookup and atomic latencies better than the six
// that 80 registers allow (finest-level binning 1.060 -> 1.024 ms on the 7.2M mesh).
__global__ void __launch_bounds__(EMB_WU_WARPS * 32, 8) k_bin_pairs(const int4 *__restrict__ rec, int64_t T, LevelGeom g,
                                                                 long long dil, EmbLookup lk, uint32_t *__restrict__ cnt,
                                                                 PairList PL, EmbBigQ Q)
{
    __shared__ WuTri tiles[EMB_WU_WARPS];
    __shared__ SatQueue Q2;
    __shared__ PairBuf PB;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WuTri &S = tiles[w];
    int qn = 0;  // pairs queued for the full overlap test (warp-uniform)
    int bn = 0;  // pairs buffered for the list (warp-uniform)
    const int64_t t0 = ((int64_t)blockIdx.x * EMB_WU_WARPS + w) * 32;
    const int64_t t = t0 + lane;
    const int dil32 = (int)dil, W32 = (int)g.W;
    int b0[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, b1[3] = {-1, -1, -1};
    int4 A = make_int4(0, 0, 0, 0), B = A, C = A;
    const bool valid = t < T && bin_setup32(rec, t, g.lW, dil32, (int)g.nb, A, B, C, b0, b1);
    S.A[lane] = A;
    S.B[lane] = B;
    S.C[lane] = C;
    __syncwarp();
    const unsigned long long own =
        valid && b1[0] >= b0[0] && b1[1] >= b0[1] && b1[2] >= b0[2]
            ? (unsigned long long)(b1[0] - b0[0] + 1) * (unsigned long long)(b1[1] - b0[1] + 1) *
                  (unsigned long long)(b1[2] - b0[2] + 1)
            : 0ull;
    const bool mine = valid && own > 0 && !(own > EMB_BIG_ITEMS && emb_bigq_push(Q, (uint32_t)t, own));
    const uint32_t k = mine ? (uint32_t)own : 0u;
    uint32_t incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
    const int ox = (int)b0[0], oy = (int)b0[1], oz = (int)b0[2];
    const int onx = mine ? (int)(b1[0] - b0[0] + 1) : 1, ony = mine ? (int)(b1[1] - b0[1] + 1) : 1;
    const uint32_t omx = emb_recip((uint32_t)onx), omy = emb_recip((uint32_t)ony);
    for (uint32_t s0 = 0; s0 < wtot; s0 += 32) {
        const uint32_t gi = s0 + lane;
        int lo = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
            if (v <= gi) lo += step;
        }
        const int ti = lo > 31 ? 31 : lo;
        const uint32_t first = __shfl_sync(0xffffffffu, incl, ti) - __shfl_sync(0xffffffffu, k, ti);
        const int bx0 = __shfl_sync(0xffffffffu, ox, ti), by0 = __shfl_sync(0xffffffffu, oy, ti),
                  bz0 = __shfl_sync(0xffffffffu, oz, ti), nbx = __shfl_sync(0xffffffffu, onx, ti),
                  nby = __shfl_sync(0xffffffffu, ony, ti);
        const uint32_t mbx = __shfl_sync(0xffffffffu, omx, ti), mby = __shfl_sync(0xffffffffu, omy, ti);
        bool hit = false, need = false;
        int32_t id = -1;
        int bxi = 0, byi = 0, bzi = 0;
        if (gi < wtot) {
            const uint32_t r = gi - first, rr = emb_div_recip(r, (uint32_t)nbx, mbx), cx = r - rr * (uint32_t)nbx,
                           cz = emb_div_recip(rr, (uint32_t)nby, mby), cy = rr - cz * (uint32_t)nby;
            bxi = bx0 + (int)cx;
            byi = by0 + (int)cy;
            bzi = bz0 + (int)cz;
            id = emb_lookup(lk, bxi, byi, bzi);
            if (id >= 0) {
                const int lx = bxi * W32 - dil32, ly = byi * W32 - dil32, lz = bzi * W32 - dil32;
                const int hx = lx + W32 + 2 * dil32, hy = ly + W32 + 2 * dil32, hz = lz + W32 + 2 * dil32;
                hit = bin_pt32(S.A[ti], lx, ly, lz, hx, hy, hz) || bin_pt32(S.B[ti], lx, ly, lz, hx, hy, hz) ||
                      bin_pt32(S.C[ti], lx, ly, lz, hx, hy, hz);
                need = !hit;
            }
        }
        bin_append_buf(hit, id, (uint32_t)(t0 + ti), lane, cnt, PB, w, bn, PL);
        // pairs that need the full overlap test wait until a whole warp's worth is queued
        const unsigned nm = __ballot_sync(0xffffffffu, need);
        if (need) {
            const int pos = qn + __popc(nm & ((1u << lane) - 1u));
            Q2.e[w][pos] = make_int4(ti, bxi, byi, bzi);
            Q2.id[w][pos] = id;
        }
        qn += __popc(nm);
        __syncwarp();
        if (qn >= 32) {
            bin_sat_batch(Q2, w, 32, lane, S, t0, g, dil, cnt, PB, bn, PL);
            int4 e = make_int4(0, 0, 0, 0);
            int32_t idn = 0;
            if (lane < qn - 32) {
                e = Q2.e[w][32 + lane];
                idn = Q2.id[w][32 + lane];
            }
            __syncwarp();
            if (lane < qn - 32) {
                Q2.e[w][lane] = e;
                Q2.id[w][lane] = idn;
            }
            qn -= 32;
            __syncwarp();
        }
    }
    if (qn > 0) bin_sat_batch(Q2, w, qn, lane, S, t0, g, dil, cnt, PB, bn, PL);
    if (bn > 0) pair_flush(PB, w, bn, lane, PL);
}

// Decomposition of candidate index i of the box [b0, b1] (x fastest) and its step by 32.
struct BoxWalk {
    long long nx, ny, x, y, z, dx, dy, dz;
    __device__ __forceinline__ void start(const long long b0[3], const long long b1[3], unsigned long long i)
    {
        nx = b1[0] - b0[0] + 1;
        ny = b1[1] - b0[1] + 1;
        x = (long long)(i % (unsigned long long)nx);
        const unsigned long long r = i / (unsigned long long)nx;
        y = (long long)(r % (unsigned long long)ny);
        z = (long long)(r / (unsigned long long)ny);
        dx = 32 % nx;
        dy = (32 / nx) % ny;
        dz = (32 / nx) / ny;
    }
    __device__ __forceinline__ void step()
    {
        x += dx;
        y += dy;
        z += dz;
        if (x >= nx) {
            x -= nx;
            ++y;
        }
        if (y >= ny) {
            y -= ny;
            ++z;
        }
    }
};

// The queued chunks of large triangles, one warp per chunk.
__global__ void __launch_bounds__(EMB_BIG_BLOCK) k_bin_pairs_big(const int4 *__restrict__ rec, LevelGeom g, long long dil,
                                                                 EmbLookup lk, uint32_t *__restrict__ cnt, PairList PL,
                                                                 EmbBigQ Q)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long nq = emb_bigq_count(Q);
    const unsigned long long nw = (unsigned long long)gridDim.x * (EMB_BIG_BLOCK / 32);
    for (unsigned long long e = (unsigned long long)blockIdx.x * (EMB_BIG_BLOCK / 32) + (threadIdx.x >> 5); e < nq;
         e += nw) {
        const uint2 E = Q.q[e];
        if (E.x == EMB_BIG_NONE) continue;
        int4 A, B, C;
        long long b0[3], b1[3];
        if (!bin_setup(rec, E.x, g, dil, A, B, C, b0, b1)) continue;
        unsigned long long i0, i1;
        emb_bigq_range(E.y, box_items(b0, b1), i0, i1);
        BoxWalk bw;
        bw.start(b0, b1, i0 + lane);
        for (unsigned long long it = i0 + lane; it < i1; it += 32, bw.step())
            bin_block(A, B, C, E.x, b0[0] + bw.x, b0[1] + bw.y, b0[2] + bw.z, g, dil, lk, cnt, PL);
    }
}

// Step 1 (enqueue only): flag, pos, flist hold T + 1 uint32; the kept count ends at
// pos[T]; tmp is scan scratch for T entries.  The filter is kept as one bit per
// triangle (flag[0, W) the W = ceil(T / 32) words, flag[W, 2W) their popcounts,
// 2W <= T + 1), whose popcounts are scanned into pos[0, W]; the compaction then
// reads the words instead of a 32-bit flag per triangle.
emb_status emb_enq_filter(const int4 *rec, int64_t T, LevelGeom g, uint32_t *flag, uint32_t *pos, uint32_t *flist,
                          uint64_t *tmp, int block, cudaStream_t s, uint64_t expect)
{
    const int64_t W = (T + 31) / 32;
    const int bs = block < 32 ? 32 : block - block % 32;
    if (T > 0) EMB_LAUNCH((k_xfilter_bits), emb_grid(T, bs), bs, 0, s)(rec, T, g, flag, flag + W);
    emb_status rc = emb_scan_into_expect(flag + W, pos, W, tmp, expect, s);
    if (rc != EMB_OK) return rc;
    if (T > 0) EMB_LAUNCH((k_compact_bits), emb_grid(W, 256), 256, 0, s)(flag, pos, T, flist, pos + T);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

// The filter with a 32-bit flag per triangle kept in flag (the mode without compaction).
static emb_status enq_filter_flags(const int4 *rec, int64_t T, LevelGeom g, uint32_t *flag, uint32_t *pos,
                                   uint32_t *flist, uint64_t *tmp, int block, cudaStream_t s)
{
    EMB_LAUNCH((k_xfilter), emb_grid(T, block), block, 0, s)(rec, T, g, flag);
    emb_status rc = emb_scan_into_expect(flag, pos, T, tmp, EMB_NO_EXPECT, s);
    if (rc != EMB_OK) return rc;
    EMB_LAUNCH((k_compact), emb_grid(T, 256), 256, 0, s)(flag, pos, T, flist);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

// The pair list into the CSR bins: entry e goes to off[block] + slot (below ent_cap).
__global__ void k_bin_scatter(const uint2 *__restrict__ bs, const uint32_t *__restrict__ tri,
                              const unsigned long long *__restrict__ n, uint64_t cap, const uint32_t *__restrict__ off,
                              uint32_t *__restrict__ ent, uint64_t ent_cap)
{
    const unsigned long long m = *n < cap ? *n : cap;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const uint2 v = bs[e];
        const uint64_t p = (uint64_t)off[v.x] + v.y;
        if (p < ent_cap) ent[p] = tri[e];
    }
}

// Steps 2-9 at the finest level, geometry half (enqueue only): cnt holds n + 1 uint32
// and receives the pairs per block, off their n + 1 offsets (total at off[n]); the
// list holds list_cap entries (list_n counts the requests); tmp: scan scratch for n.
emb_status emb_enq_bin_pairs(const int4 *rec, int64_t T, LevelGeom g, const EmbLevel &lv, uint32_t *cnt, uint32_t *off,
                             uint2 *list_bs, uint32_t *list_tri, unsigned long long *list_n, uint64_t list_cap,
                             uint64_t *tmp, const EmbBigQ &Q, cudaStream_t s, uint64_t expect)
{
    EMB_CUDA_TRY(cudaMemsetAsync(cnt, 0, (lv.n + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(cudaMemsetAsync(list_n, 0, sizeof(unsigned long long), s));
    const EmbLookup lk = emb_lookup_of(lv);
    const PairList PL = {list_bs, list_tri, list_n, list_cap};
    if (Q.cap) EMB_CUDA_TRY(cudaMemsetAsync(Q.n, 0, sizeof(unsigned long long), s));
    if (T > 0)
        EMB_LAUNCH((k_bin_pairs), emb_grid(T, 32 * EMB_WU_WARPS), 32 * EMB_WU_WARPS, 0, s)(rec, T, g, g.half, lk, cnt, PL,
                                                                                           Q);
    if (Q.cap) EMB_LAUNCH((k_bin_pairs_big), EMB_BIG_GRID, EMB_BIG_BLOCK, 0, s)(rec, g, g.half, lk, cnt, PL, Q);
    return emb_scan_into_expect(cnt, off, lv.n, tmp, expect, s);
}

// Scatter half: ent holds ent_cap entries.
emb_status emb_enq_bin_scatter(const uint2 *list_bs, const uint32_t *list_tri, const unsigned long long *list_n,
                               uint64_t list_cap, const uint32_t *off, uint32_t *ent, uint64_t ent_cap, cudaStream_t s)
{
    int64_t grid = (int64_t)((list_cap + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    EMB_LAUNCH((k_bin_scatter), (int)grid, 256, 0, s)(list_bs, list_tri, list_n, list_cap, off, ent, ent_cap);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

// The finest level's bins with a pair list of list_cap entries into ent (ent_cap
// entries), all enqueued on s; the device counts land in b->dcount.
static emb_status bin_finest(emb_bins b, uint64_t list_cap, uint64_t ent_cap, cudaStream_t s)
{
    const emb_mesh m = b->m;
    const EmbLevel &lv = b->f->lv[b->level];
    const LevelGeom g = level_geom(b->f, b->level);
    emb_status rc = EMB_OK;
    uint32_t *cnt = nullptr;
    uint64_t *tmp = nullptr;
    char *list = nullptr;
    EmbBigQ Q = {nullptr, nullptr, 0};
    const size_t a_bs = ((size_t)list_cap * sizeof(uint2) + 255) & ~(size_t)255;
    if (emb_malloc_async(&cnt, (lv.n + 1) * sizeof(uint32_t), s) != cudaSuccess ||
        emb_malloc_async(&tmp, emb_scan_tmp_words(lv.n) * sizeof(uint64_t), s) != cudaSuccess ||
        emb_malloc_async((void **)&list, 256 + a_bs + (size_t)list_cap * sizeof(uint32_t), s) != cudaSuccess)
        rc = EMB_ERR_CUDA;
    if (rc == EMB_OK && !b->off && emb_malloc_async(&b->off, (lv.n + 1) * sizeof(uint32_t), s) != cudaSuccess)
        rc = EMB_ERR_CUDA;
    if (rc == EMB_OK && b->ent_cap != ent_cap) {
        if (b->ent) cudaFreeAsync(b->ent, s);
        b->ent = nullptr;
        b->ent_cap = ent_cap;
        if (emb_malloc_async(&b->ent, ((size_t)ent_cap + 1) * sizeof(uint32_t), s) != cudaSuccess) rc = EMB_ERR_CUDA;
    }
    if (rc == EMB_OK) rc = emb_bigq_alloc(Q, m->T, s);
    unsigned long long *ln = (unsigned long long *)list;
    uint2 *lbs = (uint2 *)(list + 256);
    uint32_t *ltri = (uint32_t *)(list + 256 + a_bs);
    if (rc == EMB_OK) rc = emb_enq_bin_pairs(m->rec, m->T, g, lv, cnt, b->off, lbs, ltri, ln, list_cap, tmp, Q, s);
    if (rc == EMB_OK) rc = emb_enq_bin_scatter(lbs, ltri, ln, list_cap, b->off, b->ent, ent_cap, s);
    if (rc == EMB_OK &&
        (cudaMemcpyAsync(b->dcount + 4, b->off + lv.n, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(b->dcount + 8, ln, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s) != cudaSuccess))
        rc = EMB_ERR_CUDA;
    b->list_cap = list_cap;
    emb_bigq_free(Q, s);
    if (list) cudaFreeAsync(list, s);
    if (cnt) cudaFreeAsync(cnt, s);
    if (tmp) cudaFreeAsync(tmp, s);
    return rc;
}

// Every triangle id (the list of the modes without compaction), and its count.
__global__ void k_iota(uint32_t *__restrict__ out, int64_t n, uint32_t *__restrict__ count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)i;
    if (i == 0) *count = (uint32_t)n;
}

extern "C" emb_status emb_bin(emb_mesh m, emb_forest f, int32_t level, int32_t lattice, void *stream, emb_bins *out)
{
    return emb_bin_ex(m, f, level, lattice, EMB_BIN_FILTER_COMPACT, stream, out);
}

// No host synchronisation: the filtered count and, at the finest level, the bin
// sizes stay on the device until emb_bins_sync reads them.  The finest bins start
// from a pair list of 4 T + 2^20 entries; if that proved too small, emb_bins_sync
// (called by every consumer that needs complete bins) redoes them exactly.
extern "C" emb_status emb_bin_ex(emb_mesh m, emb_forest f, int32_t level, int32_t lattice, int32_t mode, void *stream,
                                 emb_bins *out)
{
    if (!m || !f || !out) return EMB_ERR_BAD_INPUT;
    if (lattice != 19 && lattice != 27) return EMB_ERR_BAD_INPUT;
    if (mode != EMB_BIN_FILTER_COMPACT && mode != EMB_BIN_FILTER_ONLY && mode != EMB_BIN_NO_FILTER) return EMB_ERR_BAD_INPUT;
    if (level < 0 || level > f->top) return EMB_ERR_STATE;
    if (m->R != f->R) return EMB_ERR_STATE;
    *out = nullptr;
    cudaStream_t s = emb_stream(stream);
    emb_bins b = new emb_bins_s();
    b->m = m;
    b->f = f;
    b->level = level;
    b->lattice = lattice;
    b->s = s;
    LevelGeom g = level_geom(f, level);
    const EmbLevel &lv = f->lv[level];
    emb_status rc = EMB_OK;
    uint32_t *flag = nullptr, *pos = nullptr;
    uint64_t *tmp = nullptr;
    // step 1: exact x-line filter, compacted in ascending order
    // every buffer is stream-ordered on s: the bins are freed the same way, without a
    // device synchronisation (the flags of the mode without compaction live in the bins)
    if (emb_malloc_async(&flag, (m->T + 1) * sizeof(uint32_t), s) != cudaSuccess ||
        emb_malloc_async(&pos, (m->T + 1) * sizeof(uint32_t), s) != cudaSuccess ||
        emb_malloc_async(&tmp, emb_scan_tmp_words(m->T) * sizeof(uint64_t), s) != cudaSuccess ||
        emb_malloc_async(&b->flist, (m->T + 1) * sizeof(uint32_t), s) != cudaSuccess ||
        emb_malloc_async(&b->dcount, 16, s) != cudaSuccess) {
        emb_bins_destroy(b);
        return EMB_ERR_CUDA;
    }
    EMB_CUDA_TRY(cudaMemsetAsync(b->dcount, 0, 16, s));
    if (mode == EMB_BIN_FILTER_COMPACT) {
        rc = emb_enq_filter(m->rec, m->T, g, flag, pos, b->flist, tmp, 256, s);
        if (rc == EMB_OK && cudaMemcpyAsync(b->dcount, pos + m->T, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            rc = EMB_ERR_CUDA;
    } else {
        // ablations: the filter flags kept per triangle without compaction, or no filter
        if (mode == EMB_BIN_FILTER_ONLY) {
            rc = enq_filter_flags(m->rec, m->T, g, flag, pos, b->flist, tmp, 256, s);
            b->keep = flag;
            flag = nullptr;
        }
        if (rc == EMB_OK) EMB_LAUNCH((k_iota), emb_grid(m->T, 256), 256, 0, s)(b->flist, m->T, (uint32_t *)b->dcount);
    }
    // the finest level's bins need its exact block count: a count the forest still
    // waits for is taken now, with the filter queued (below the finest level the bins are
    // the filter alone, and the next call that needs the count takes it)
    if (rc == EMB_OK && level == f->max_level) rc = emb_forest_settle(f);
    // steps 2-9 at the finest level: CSR bins of link-relevant triangles per block
    if (rc == EMB_OK && level == f->max_level && lv.n > 0) {
        const uint64_t cap = (uint64_t)4 * m->T + (1 << 20);
        rc = bin_finest(b, cap, cap, s);
    }
    if (flag) cudaFreeAsync(flag, s);
    cudaFreeAsync(pos, s);
    cudaFreeAsync(tmp, s);
    // the counts travel to a pinned slot behind the bins, so that emb_bins_sync only
    // waits for them instead of synchronising the stream
    if (rc == EMB_OK) {
        b->rb_slot = emb_readback_acquire(&b->rb_h, &b->rb_ev);
        if (b->rb_slot >= 0 && (cudaMemcpyAsync(b->rb_h, b->dcount, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                                cudaEventRecord(b->rb_ev, s) != cudaSuccess))
            rc = EMB_ERR_CUDA;
    }
    if (rc == EMB_OK && cudaGetLastError() != cudaSuccess) rc = EMB_ERR_CUDA;
    if (rc != EMB_OK) {
        emb_bins_destroy(b);
        return rc;
    }
    *out = b;
    return EMB_OK;
}

emb_status emb_bins_sync(emb_bins b)
{
    if (b->known) return EMB_OK;
    unsigned char h[16];
    if (b->rb_slot >= 0) {
        EMB_CUDA_TRY(cudaEventSynchronize(b->rb_ev));
        memcpy(h, (const void *)b->rb_h, 16);
    } else {
        EMB_CUDA_TRY(cudaMemcpyAsync(h, b->dcount, 16, cudaMemcpyDeviceToHost, b->s));
        EMB_CUDA_TRY(cudaStreamSynchronize(b->s));
    }
    uint32_t nf = 0, np = 0;
    unsigned long long lreq = 0;
    memcpy(&nf, h, 4);
    memcpy(&np, h + 4, 4);
    memcpy(&lreq, h + 8, 8);
    if (b->off && lreq > b->list_cap) {
        // the pair list was too small: the bins once more, with its exact size
        emb_status rc = bin_finest(b, lreq, lreq, b->s);
        if (rc != EMB_OK) return rc;
        EMB_CUDA_TRY(cudaMemcpyAsync(h, b->dcount, 16, cudaMemcpyDeviceToHost, b->s));
        EMB_CUDA_TRY(cudaStreamSynchronize(b->s));
        memcpy(&np, h + 4, 4);
    }
    b->nf = nf;
    b->npairs = np;
    b->known = true;
    return EMB_OK;
}

// Stream-ordered frees on the stream of emb_bin: no device synchronisation, so a
// pipeline that drops each level's bins keeps the GPU busy.
extern "C" void emb_bins_destroy(emb_bins b)
{
    if (!b) return;
    void *bufs[] = {b->flist, b->off, b->ent, b->dcount, b->keep};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, b->s);
    emb_readback_release(b->rb_slot);  // reused only once its event has completed
    delete b;
}

extern "C" emb_status emb_bins_stats(emb_bins b, int64_t *h_filtered, int64_t *h_pairs)
{
    if (!b) return EMB_ERR_BAD_INPUT;
    if (b) EMB_SETTLE(b->f);
    emb_status rc = emb_bins_sync(b);
    if (rc != EMB_OK) return rc;
    if (h_filtered) *h_filtered = b->nf;
    if (h_pairs) *h_pairs = b->npairs;
    return EMB_OK;
}

extern "C" emb_status emb_bins_copy(emb_bins b, uint32_t *d_filtered, uint32_t *d_off, uint32_t *d_ent, void *stream)
{
    if (!b) return EMB_ERR_BAD_INPUT;
    if (b) EMB_SETTLE(b->f);
    emb_status rc = emb_bins_sync(b);
    if (rc != EMB_OK) return rc;
    cudaStream_t s = emb_stream(stream);
    if (d_filtered && b->nf > 0)
        EMB_CUDA_TRY(cudaMemcpyAsync(d_filtered, b->flist, b->nf * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    if ((d_off || d_ent) && !b->off) return EMB_ERR_STATE;
    if (d_off)
        EMB_CUDA_TRY(cudaMemcpyAsync(d_off, b->off, (b->f->lv[b->level].n + 1) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    if (d_ent && b->npairs > 0)
        EMB_CUDA_TRY(cudaMemcpyAsync(d_ent, b->ent, b->npairs * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    return EMB_OK;
}
