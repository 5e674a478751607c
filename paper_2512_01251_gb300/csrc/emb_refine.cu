// Near-wall refinement flags (Sec. 3.4, "Refinement Flagging and Propagation").
//
// The paper marks solid-boundary blocks and propagates flags block by block a
// number of layers set by the near-wall distance (Eq. N_prop).  Here the
// criterion is evaluated directly and exactly: block B of level L is flagged iff
// some triangle overlaps B's closed box dilated by (rho_L - 1/2) h_L, i.e. iff a
// cell centre of B lies within L-infinity distance rho_L h_L of the surface.
// rho equals `band` one level above the finest and grows towards the root as
// rho_L = max(band, rho_{L+1}/2 + 5/2), which keeps all 26 neighbours of every
// refined block present (2:1 balance) and leaves unrefined blocks surface-free.
//
// Warp-cooperative over 32 consecutive triangles (see emb_internal.cuh): when the
// union of their candidate blocks is at most an eighth of their summed candidates,
// each block of the union is looked up once and tested against the 32 triangles;
// otherwise the warp's (triangle, candidate block) pairs are spread evenly over its
// lanes, and a triangle with very many candidates goes in queued chunks to whole
// warps.  Flags are idempotent byte stores.
#include <math.h>

#include "emb_internal.cuh"

#ifndef REFINE_MINB
#define REFINE_MINB 4
#endif

__device__ __forceinline__ void refine_setup(const int4 *__restrict__ rec, int64_t t, const LevelGeom &g, long long dil,
                                             int4 &A, int4 &B, int4 &C, long long b0[3], long long b1[3])
{
    A = rec[3 * t];
    B = rec[3 * t + 1];
    C = rec[3 * t + 2];
    emb_block_range(min(A.x, min(B.x, C.x)), max(A.x, max(B.x, C.x)), g.lW, dil, g.nb, b0[0], b1[0]);
    emb_block_range(min(A.y, min(B.y, C.y)), max(A.y, max(B.y, C.y)), g.lW, dil, g.nb, b0[1], b1[1]);
    emb_block_range(min(A.z, min(B.z, C.z)), max(A.z, max(B.z, C.z)), g.lW, dil, g.nb, b0[2], b1[2]);
}

__device__ __forceinline__ unsigned long long refine_items(const long long b0[3], const long long b1[3])
{
    if (b1[0] < b0[0] || b1[1] < b0[1] || b1[2] < b0[2]) return 0;
    return (unsigned long long)(b1[0] - b0[0] + 1) * (unsigned long long)(b1[1] - b0[1] + 1) *
           (unsigned long long)(b1[2] - b0[2] + 1);
}

// Flagged blocks of the level as one bit per dense position (bx + nb (by + nb bz)),
// when the level is small enough to have one: the common "already flagged" case
// then costs one cached load instead of a block lookup and a flag load.
struct FlagBits {
    unsigned long long *w;  // null: no dense bits, test the flag bytes
    long long nb;
    // A plain (L1-cached) load: a word cached before another SM set a bit only sends
    // the candidate through the full test, which decides exactly.
    __device__ __forceinline__ bool test(long long bx, long long by, long long bz, unsigned long long &pos) const
    {
        pos = (unsigned long long)((bz * nb + by) * nb + bx);
        return (w[pos >> 6] >> (pos & 63)) & 1ull;
    }
    __device__ __forceinline__ void set(unsigned long long pos) const { atomicOr(w + (pos >> 6), 1ull << (pos & 63)); }
};

// Id of block (bx, by, bz) if it exists and is not flagged yet, else -1; pos receives
// its dense position.  With both dense bitmaps (flagged bits and the level's rank
// bitmap) the flagged word, the existence word and its rank prefix are independent
// loads issued together, and the flag byte is not read: a flagged word read before
// another SM set the bit only sends the block through the exact test once more, whose
// flag store is idempotent.  Otherwise: the flagged bit, the lookup, the flag byte.
__device__ __forceinline__ int32_t refine_candidate(const EmbLookup &lk, const FlagBits &fb,
                                                    const uint8_t *__restrict__ flags, long long bx, long long by,
                                                    long long bz, unsigned long long &pos)
{
    if (fb.w && lk.bits) {
        pos = (unsigned long long)((bz * fb.nb + by) * fb.nb + bx);
        if (!emb_ck(pos, (uint64_t)lk.nb * lk.nb * lk.nb, lk.st)) return -1;
        const unsigned long long fw = fb.w[pos >> 6];
        const uint64_t ew = __ldg(lk.bits + (pos >> 6));
        const uint32_t pre = __ldg(lk.wpre + (pos >> 6));
        const int sh = (int)(pos & 63);
        if (((fw >> sh) & 1ull) || !((ew >> sh) & 1ull)) return -1;
        const int32_t id = (int32_t)(pre + (uint32_t)__popcll(ew & ((1ull << sh) - 1ull)));
        return emb_ck((uint64_t)id, (uint64_t)lk.n, lk.st) ? id : -1;
    }
    if (fb.w && fb.test(bx, by, bz, pos)) return -1;
    const int32_t id = emb_lookup(lk, bx, by, bz);
    if (id < 0 || *((volatile const uint8_t *)flags + id)) return -1;
    return id;
}

// Flag block (bx, by, bz) if it exists, is not flagged yet and the triangle meets its dilated box.
__device__ __forceinline__ void refine_block(const int4 &A, const int4 &B, const int4 &C, long long bx, long long by,
                                             long long bz, const LevelGeom &g, long long dil, const EmbLookup &lk,
                                             uint8_t *__restrict__ flags, const FlagBits &fb)
{
    unsigned long long pos = 0;
    const int32_t id = refine_candidate(lk, fb, flags, bx, by, bz, pos);
    if (id < 0) return;
    const long long lx = bx * g.W - dil, ly = by * g.W - dil, lz = bz * g.W - dil;
    const long long hx = lx + g.W + 2 * dil, hy = ly + g.W + 2 * dil, hz = lz + g.W + 2 * dil;
    if (emb_point_in_box(A, lx, ly, lz, hx, hy, hz) || emb_point_in_box(B, lx, ly, lz, hx, hy, hz) ||
        emb_point_in_box(C, lx, ly, lz, hx, hy, hz) || emb_tri_box(A, B, C, lx, ly, lz, hx, hy, hz)) {
        flags[id] = 1;
        if (fb.w) fb.set(pos);
    }
}


// 32-bit forms of the per-block arithmetic: coordinates, block origins, widths and
// dilations all lie below 2^25 in magnitude, block indices below 2^21.
__device__ __forceinline__ void ref_range(int mn, int mx, int lW, int dil, int nb, int &b0, int &b1)
{
    b0 = -((-(mn - dil - (1 << lW))) >> lW);  // ceil
    b1 = (mx + dil) >> lW;                    // floor
    if (b0 < 0) b0 = 0;
    if (b1 > nb - 1) b1 = nb - 1;
}
__device__ __forceinline__ bool ref_pt(const int4 &P, int lx, int ly, int lz, int hx, int hy, int hz)
{
    return P.x >= lx && P.x <= hx && P.y >= ly && P.y <= hy && P.z >= lz && P.z <= hz;
}
__device__ __forceinline__ bool ref_overlap(const WuTri &S, int j, int lx, int ly, int lz, int ux, int uy, int uz)
{
    if (S.lo[0][j] > ux || S.hi[0][j] < lx || S.lo[1][j] > uy || S.hi[1][j] < ly || S.lo[2][j] > uz || S.hi[2][j] < lz)
        return false;
    const int4 A = S.A[j], B = S.B[j], C = S.C[j];
    return ref_pt(A, lx, ly, lz, ux, uy, uz) || ref_pt(B, lx, ly, lz, ux, uy, uz) || ref_pt(C, lx, ly, lz, ux, uy, uz) ||
           emb_tri_box(A, B, C, lx, ly, lz, ux, uy, uz);
}
__device__ __forceinline__ void ref_block(const int4 &A, const int4 &B, const int4 &C, int bx, int by, int bz, int W,
                                          int dil, const EmbLookup &lk, uint8_t *__restrict__ flags, const FlagBits &fb)
{
    unsigned long long pos = 0;
    const int32_t id = refine_candidate(lk, fb, flags, bx, by, bz, pos);
    if (id < 0) return;
    const int lx = bx * W - dil, ly = by * W - dil, lz = bz * W - dil;
    const int hx = lx + W + 2 * dil, hy = ly + W + 2 * dil, hz = lz + W + 2 * dil;
    if (ref_pt(A, lx, ly, lz, hx, hy, hz) || ref_pt(B, lx, ly, lz, hx, hy, hz) || ref_pt(C, lx, ly, lz, hx, hy, hz) ||
        emb_tri_box(A, B, C, lx, ly, lz, hx, hy, hz)) {
        flags[id] = 1;
        if (fb.w) fb.set(pos);
    }
}

// Persistent warps over tiles of 32 consecutive triangles; each warp loads the
// records of its next tile before it works on the current one, so that the loads
// are in flight during the work (a warp otherwise spends most of its life after its
// loads, in dependent lookups, and the record stream runs far below HBM speed).
__global__ void __launch_bounds__(EMB_WU_WARPS * 32, REFINE_MINB) k_refine(const int4 *__restrict__ rec, int64_t T, LevelGeom g,
                                                              long long dil, EmbLookup lk, uint8_t *__restrict__ flags,
                                                              FlagBits fb, EmbBigQ Q)
{
    __shared__ WuTri tiles[EMB_WU_WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WuTri &S = tiles[w];
    const int64_t ntiles = (T + 31) / 32;
    const int64_t stride = (int64_t)gridDim.x * EMB_WU_WARPS;
    int64_t tile = (int64_t)blockIdx.x * EMB_WU_WARPS + w;
    int4 nA = make_int4(0, 0, 0, 0), nB = nA, nC = nA;
    if (tile < ntiles && tile * 32 + lane < T) {
        const int64_t t = tile * 32 + lane;
        nA = rec[3 * t];
        nB = rec[3 * t + 1];
        nC = rec[3 * t + 2];
    }
    for (; tile < ntiles; tile += stride) {
        const int64_t t = tile * 32 + lane;
        const bool valid = t < T;
        const int4 A = nA, B = nB, C = nC;
        {
            const int64_t tn = (tile + stride) * 32 + lane;
            if (tile + stride < ntiles && tn < T) {
                nA = rec[3 * tn];
                nB = rec[3 * tn + 1];
                nC = rec[3 * tn + 2];
            }
        }
        const int dil32 = (int)dil, W32 = (int)g.W, nb32 = (int)g.nb;
        int b0[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, b1[3] = {-1, -1, -1};
        if (valid) {
            ref_range(min(A.x, min(B.x, C.x)), max(A.x, max(B.x, C.x)), g.lW, dil32, nb32, b0[0], b1[0]);
            ref_range(min(A.y, min(B.y, C.y)), max(A.y, max(B.y, C.y)), g.lW, dil32, nb32, b0[1], b1[1]);
            ref_range(min(A.z, min(B.z, C.z)), max(A.z, max(B.z, C.z)), g.lW, dil32, nb32, b0[2], b1[2]);
        }
        __syncwarp();  // the previous tile's lanes are done with S
        S.A[lane] = A;
        S.B[lane] = B;
        S.C[lane] = C;
        S.lo[0][lane] = valid ? min(A.x, min(B.x, C.x)) : 0x7fffffff;
        S.hi[0][lane] = valid ? max(A.x, max(B.x, C.x)) : -0x7fffffff;
        S.lo[1][lane] = min(A.y, min(B.y, C.y));
        S.hi[1][lane] = max(A.y, max(B.y, C.y));
        S.lo[2][lane] = min(A.z, min(B.z, C.z));
        S.hi[2][lane] = max(A.z, max(B.z, C.z));
        __syncwarp();
        int u0[3], u1[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            u0[d] = __reduce_min_sync(0xffffffffu, b0[d]);
            u1[d] = __reduce_max_sync(0xffffffffu, b1[d]);
        }
        const long long nx = u1[0] - u0[0] + 1, ny = u1[1] - u0[1] + 1, nz = u1[2] - u0[2] + 1;
        if (nx <= 0 || ny <= 0 || nz <= 0) continue;
        const long long total = nx * ny * nz;
        // per-triangle candidates summed over the warp: the union pays off only when it is
        // much smaller (eight times: measured against two and four, and against sixteen)
        const unsigned long long own =
            valid && b1[0] >= b0[0] && b1[1] >= b0[1] && b1[2] >= b0[2]
                ? (unsigned long long)(b1[0] - b0[0] + 1) * (unsigned long long)(b1[1] - b0[1] + 1) *
                      (unsigned long long)(b1[2] - b0[2] + 1)
                : 0ull;
        const unsigned own_sum = __reduce_add_sync(0xffffffffu, (unsigned)min(own, 1ull << 20));
        if (total <= EMB_WU_MAX && 8 * total <= (long long)own_sum) {
            // total <= EMB_WU_MAX: decode the union index in 32-bit arithmetic.  Each lane
            // takes a union block; the blocks that exist and are not flagged yet are then
            // tested one at a time by the whole warp, each lane against its own triangle.
            const unsigned ux = (unsigned)nx, uxy = (unsigned)(nx * ny);
            const unsigned mx = emb_recip(ux), mxy = emb_recip(uxy);
            for (unsigned c0 = 0; c0 < (unsigned)total; c0 += 32) {
                const unsigned c = c0 + lane;
                int bx = 0, by = 0, bz = 0;
                unsigned long long pos = 0;
                int32_t id = -1;
                if (c < (unsigned)total) {
                    const unsigned cz = emb_div_recip(c, uxy, mxy), cr = c - cz * uxy, cy = emb_div_recip(cr, ux, mx);
                    bx = u0[0] + (int)(cr - cy * ux);
                    by = u0[1] + (int)cy;
                    bz = u0[2] + (int)cz;
                    id = refine_candidate(lk, fb, flags, bx, by, bz, pos);
                }
                unsigned m = __ballot_sync(0xffffffffu, id >= 0);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const int lx = __shfl_sync(0xffffffffu, bx, src) * W32 - dil32,
                              ly = __shfl_sync(0xffffffffu, by, src) * W32 - dil32,
                              lz = __shfl_sync(0xffffffffu, bz, src) * W32 - dil32;
                    const bool hit = ref_overlap(S, lane, lx, ly, lz, lx + W32 + 2 * dil32, ly + W32 + 2 * dil32,
                                                 lz + W32 + 2 * dil32);
                    if (__any_sync(0xffffffffu, hit) && lane == src) {
                        flags[id] = 1;
                        if (fb.w) fb.set(pos);
                    }
                }
            }
            continue;
        }
        // large or loose union: the warp's (triangle, candidate block) pairs spread evenly over
        // the lanes (a triangle with very many candidates goes to the chunk queue instead)
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
            if (gi < wtot) {
                const uint32_t r = gi - first, rr = emb_div_recip(r, (uint32_t)nbx, mbx), cx = r - rr * (uint32_t)nbx,
                               cz = emb_div_recip(rr, (uint32_t)nby, mby), cy = rr - cz * (uint32_t)nby;
                ref_block(S.A[ti], S.B[ti], S.C[ti], bx0 + (int)cx, by0 + (int)cy, bz0 + (int)cz, W32, dil32, lk, flags,
                          fb);
            }
        }
    }
}

// The queued chunks of large triangles, one warp per chunk (candidates x fastest).
__global__ void __launch_bounds__(EMB_BIG_BLOCK) k_refine_big(const int4 *__restrict__ rec, LevelGeom g, long long dil,
                                                              EmbLookup lk, uint8_t *__restrict__ flags, FlagBits fb,
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
        refine_setup(rec, E.x, g, dil, A, B, C, b0, b1);
        unsigned long long i0, i1;
        emb_bigq_range(E.y, refine_items(b0, b1), i0, i1);
        const long long nx = b1[0] - b0[0] + 1, ny = b1[1] - b0[1] + 1;
        const unsigned long long first = i0 + lane;
        long long x = (long long)(first % (unsigned long long)nx);
        long long y = (long long)((first / (unsigned long long)nx) % (unsigned long long)ny);
        long long z = (long long)((first / (unsigned long long)nx) / (unsigned long long)ny);
        const long long dx = 32 % nx, dy = (32 / nx) % ny, dz = (32 / nx) / ny;
        for (unsigned long long it = first; it < i1; it += 32) {
            refine_block(A, B, C, b0[0] + x, b0[1] + y, b0[2] + z, g, dil, lk, flags, fb);
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
    }
}

// (rho_L - 1/2) h_L in frame units, or -1 if it is not an integer.
long long emb_refine_dilation(const emb_forest_s *f, int L, int band)
{
    const int sh = 16;  // rho is kept as an integer multiple of 2^-16
    long long rho = (long long)band << sh;
    for (int l = f->max_level - 1; l > L; --l) {
        long long cand = rho / 2 + (5ll << (sh - 1));
        rho = cand > ((long long)band << sh) ? cand : ((long long)band << sh);
    }
    long long h = 1ll << (18 - f->k - L);
    long long num = (rho - (1ll << (sh - 1))) * h;
    if (num % (1ll << sh) != 0) return -1;
    return num >> sh;
}

// Enqueue only: flags (lv.n bytes) are cleared and set.
emb_status emb_enq_refine(const int4 *rec, int64_t T, LevelGeom g, long long dil, const EmbLevel &lv, uint8_t *flags,
                          unsigned long long *fbits, const EmbBigQ &Q, cudaStream_t s)
{
    if (lv.n == 0) return EMB_OK;
    EMB_CUDA_TRY(cudaMemsetAsync(flags, 0, lv.n, s));
    const EmbLookup lk = emb_lookup_of(lv);
    FlagBits fb = {nullptr, g.nb};
    const int64_t nw = emb_bitmap_words(lv.nb_axis);
    if (fbits && nw > 0) {
        EMB_CUDA_TRY(cudaMemsetAsync(fbits, 0, nw * sizeof(unsigned long long), s));
        fb.w = fbits;
    }
    if (Q.cap) EMB_CUDA_TRY(cudaMemsetAsync(Q.n, 0, sizeof(unsigned long long), s));
    int64_t grid = (T + 32 * EMB_WU_WARPS - 1) / (32 * EMB_WU_WARPS);
    const int64_t resident = (int64_t)emb_sm_count() * REFINE_MINB;
    if (grid > resident) grid = resident;
    if (grid < 1) grid = 1;
    EMB_LAUNCH((k_refine), (int)grid, 32 * EMB_WU_WARPS, 0, s)(rec, T, g, dil, lk, flags, fb, Q);
    if (Q.cap) EMB_LAUNCH((k_refine_big), EMB_BIG_GRID, EMB_BIG_BLOCK, 0, s)(rec, g, dil, lk, flags, fb, Q);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

extern "C" emb_status emb_refine_flags(emb_forest f, emb_bins b, int32_t level, int32_t band, uint8_t *d_flags,
                                       void *stream)
{
    if (!f || !b || band < 1 || band > (1 << 20)) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    if (b->f != f || level < 0 || level > f->top || level >= f->max_level) return EMB_ERR_STATE;
    const EmbLevel &lv = f->lv[level];
    if (lv.n == 0) return EMB_OK;
    if (!d_flags) return EMB_ERR_BAD_INPUT;
    long long dil = emb_refine_dilation(f, level, band);
    if (dil < 0) return EMB_ERR_RANGE;
    cudaStream_t s = emb_stream(stream);
    EmbBigQ Q;
    emb_status rc = emb_bigq_alloc(Q, b->m->T, s);
    if (rc != EMB_OK) return rc;
    unsigned long long *fbits = nullptr;
    const int64_t nw = emb_bitmap_words(lv.nb_axis);
    if (nw > 0 && emb_malloc_async(&fbits, nw * sizeof(unsigned long long), s) != cudaSuccess) fbits = nullptr;
    rc = emb_enq_refine(b->m->rec, b->m->T, level_geom(f, level), dil, lv, d_flags, fbits, Q, s);
    if (fbits) cudaFreeAsync(fbits, s);
    emb_bigq_free(Q, s);
    return rc;
}

// ---------------------------------------------------------------------------
// the paper's refinement rules (Sec. 3.4, "Refinement Flagging and Propagation")
// ---------------------------------------------------------------------------
// Block classes from the masks: solid (a solid cell), fully fluid (none).  cls bit 0:
// solid; bit 1: solid-boundary (solid with a fully fluid neighbour of the level);
// bit 2: eligible (every in-domain neighbour position holds a block of the level,
// always at the root: refining a block on the refinement interface breaks 2:1).
// The solid-boundary blocks are the first marks.
__global__ void k_pf_classify(const uint64_t *__restrict__ key, const uint64_t *__restrict__ mask,
                              const int32_t *__restrict__ nbr, int64_t n, int64_t nb, int root,
                              uint8_t *__restrict__ cls, uint8_t *__restrict__ marks)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const uint64_t k = key[b];
    const int64_t bx = (int64_t)(k & EMB_KEY_MASK), by = (int64_t)((k >> EMB_KEY_BITS) & EMB_KEY_MASK),
                  bz = (int64_t)(k >> (2 * EMB_KEY_BITS));
    const bool solid = mask[b] != 0;
    bool eligible = true, fluid_nbr = false;
    for (int d = 1; d < 27; ++d) {
        int cx, cy, cz;
        emb_dir(d, cx, cy, cz);
        const int64_t x = bx + cx, y = by + cy, z = bz + cz;
        if (x < 0 || y < 0 || z < 0 || x >= nb || y >= nb || z >= nb) continue;
        const int32_t j = nbr[b * 26 + d - 1];
        if (j < 0) {
            if (!root) eligible = false;
        } else if (mask[j] == 0) {
            fluid_nbr = true;
        }
    }
    const bool sb = solid && fluid_nbr;
    cls[b] = (uint8_t)((solid ? 1 : 0) | (sb ? 2 : 0) | (eligible ? 4 : 0));
    marks[b] = (uint8_t)(sb && eligible);
}

// One propagation step: out = in, plus every eligible block in scope next to a block
// whose `want` bits are set in cls (the adjacency step: want = solid-boundary, every
// class in scope) or that is marked in `in` (the propagation rounds: want = 0, scope =
// fully fluid blocks, and solid ones in the first round).
__global__ void k_pf_step(const int32_t *__restrict__ nbr, int64_t n, const uint8_t *__restrict__ cls, int want,
                          int solid_in_scope, const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    uint8_t m = in[b];
    const uint8_t c = cls[b];
    if (!m && (c & 4) && (!(c & 1) || solid_in_scope)) {
        for (int d = 0; d < 26 && !m; ++d) {
            const int32_t j = nbr[b * 26 + d];
            if (j >= 0 && (want ? (cls[j] & want) : in[j])) m = 1;
        }
    }
    out[b] = m;
}

extern "C" emb_status emb_refine_flags_paper(emb_forest f, int32_t level, double d_spec, uint8_t *d_flags, void *stream)
{
    if (!f || !(d_spec >= 0.0) || d_spec > 1e6) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    if (level < 0 || level != f->top || level >= f->max_level) return EMB_ERR_STATE;
    EmbLevel &lv = f->lv[level];
    if (!lv.mask_valid) return EMB_ERR_STATE;
    if (lv.n == 0) return EMB_OK;
    if (!d_flags) return EMB_ERR_BAD_INPUT;
    cudaStream_t s = emb_stream(stream);
    // Eq. N_prop: 1 + floor(2^-L d_spec / (sqrt(2) Dx_{b,L})), Dx_{b,L} = 4 Dx_L = 1 / (R 2^L)
    // for d_spec in units of the unit domain: the 2^L factors cancel
    const double np_d = floor((d_spec * (double)f->R) / sqrt(2.0));
    if (np_d > 1e6) return EMB_ERR_BAD_INPUT;
    const int nprop = 1 + (int)np_d;
    emb_status rc = emb_build_neighbors(lv, s);
    if (rc != EMB_OK) return rc;
    uint8_t *cls = nullptr, *tmp = nullptr;
    EMB_CUDA_TRY(emb_malloc_async(&cls, lv.n, s));
    EMB_CUDA_TRY(emb_malloc_async(&tmp, lv.n, s));
    const int grid = emb_grid(lv.n, 256);
    EMB_LAUNCH((k_pf_classify), grid, 256, 0, s)(lv.key, lv.mask, lv.nbr, lv.n, lv.nb_axis, level == 0 ? 1 : 0, cls,
                                                 d_flags);
    // blocks next to the solid boundary (both classes), then the rounds, ping-pong
    EMB_LAUNCH((k_pf_step), grid, 256, 0, s)(lv.nbr, lv.n, cls, 2, 1, d_flags, tmp);
    uint8_t *a = tmp, *b = d_flags;
    for (int r = 0; r < nprop; ++r) {
        EMB_LAUNCH((k_pf_step), grid, 256, 0, s)(lv.nbr, lv.n, cls, 0, r == 0 ? 1 : 0, a, b);
        uint8_t *t = a;
        a = b;
        b = t;
    }
    if (a != d_flags) EMB_CUDA_TRY(cudaMemcpyAsync(d_flags, a, lv.n, cudaMemcpyDeviceToDevice, s));
    EMB_CUDA_TRY(cudaGetLastError());
    EMB_CUDA_TRY(cudaFreeAsync(cls, s));
    EMB_CUDA_TRY(cudaFreeAsync(tmp, s));
    return EMB_OK;
}
