// Solid voxelization of one level (Sec. 3.4, "Partial Surface Voxelization" and
// "External Cell Flag Propagation").
//
// A cell is solid iff its centre lies inside the closed surface, i.e. iff the
// +x ray from the (perturbed) centre crosses the surface an odd number of times.
// The work is split along each x-line of cell centres:
//   k_vox (triangle-parallel over the filtered list): every crossing of a level
//     x-line with a triangle is owned by the block whose box [lo, lo + W) holds
//     the crossing's x.  The owner XORs two things: for each of its four cells on
//     that line, whether the crossing lies beyond the cell centre (bit of s), and
//     the line's block parity (bit of p).
//   k_xscan (one thread per x-row of blocks): walking the row from +x to -x,
//     solid = s XOR (parity of every crossing in the blocks further along +x).
// Rows are contiguous and x-ordered in the level's block list.  Under the distance
// refine rule, unrefined gaps between blocks of a row contain no surface; under the
// paper's block-layer rule they may, and a crossing in a gap joins the line parity of
// the next block of the row (or a tail word of the row's last block that the row scan
// starts from), so the scan sees every crossing either way.  Block-local parity plays the role of the
// paper's internal propagation, and the suffix scan that of Alg. 4's
// neighbour-to-neighbour walk along +x.
#include "emb_internal.cuh"

// One triangle as the voxelizer sees it: its x-lines (j, k) in [j0, j1] x [k0, k1]
// and the x-range [bx0, bx1] of blocks its crossings can fall in.
struct VoxTri {
    int4 A, B, C;
    long long nx, ny, nz;
    int sx;
    long long j0, j1, k0, k1, bx0, bx1;
};

// false for a triangle parallel to x (no line crosses it)
__device__ __forceinline__ bool vox_setup(const int4 *__restrict__ rec, int64_t t, const LevelGeom &g, VoxTri &V)
{
    V.A = rec[3 * t];
    V.B = rec[3 * t + 1];
    V.C = rec[3 * t + 2];
    const int4 A = V.A, B = V.B, C = V.C;
    long long ux = (long long)B.x - A.x, uy = (long long)B.y - A.y, uz = (long long)B.z - A.z;
    long long vx = (long long)C.x - A.x, vy = (long long)C.y - A.y, vz = (long long)C.z - A.z;
    V.nx = uy * vz - uz * vy;
    V.ny = uz * vx - ux * vz;
    V.nz = ux * vy - uy * vx;
    if (V.nx == 0) return false;
    V.sx = V.nx > 0 ? 1 : -1;
    line_range(min(A.y, min(B.y, C.y)), max(A.y, max(B.y, C.y)), g.lh, g.half, g.ncell, V.j0, V.j1);
    line_range(min(A.z, min(B.z, C.z)), max(A.z, max(B.z, C.z)), g.lh, g.half, g.ncell, V.k0, V.k1);
    V.bx0 = emb_floor_shr(min(A.x, min(B.x, C.x)), g.lW);
    V.bx1 = emb_floor_shr(max(A.x, max(B.x, C.x)), g.lW);
    if (V.bx0 < 0) V.bx0 = 0;
    if (V.bx1 > g.nb - 1) V.bx1 = g.nb - 1;
    return true;
}

__device__ __forceinline__ unsigned long long vox_items(const VoxTri &V)
{
    if (V.j1 < V.j0 || V.k1 < V.k0) return 0;
    return (unsigned long long)(V.j1 - V.j0 + 1) * (unsigned long long)(V.k1 - V.k0 + 1);
}

// Parity sinks of one voxelization: per block the cell bits s and the line parity p,
// and per block the row tail t (crossings beyond the last block of its row, read by
// the row scan of that last block); the level's sorted keys locate them.
struct VoxAcc {
    unsigned long long *s;
    unsigned int *p, *t;
    const uint64_t *key;
    int64_t n;
};

// A crossing inside a block position the level does not have (a region left coarser by
// the refinement rule): it flips every cell of the row to its left, so it joins the line
// parity of the next block of the row to its right, or the row tail of the row's last
// block when there is none.
__device__ __noinline__ void vox_gap(const VoxAcc &acc, long long bx, long long by, long long bz, int line)
{
    const uint64_t row = (uint64_t)emb_key(0, by, bz) >> EMB_KEY_BITS;
    const int64_t nx = lower_bound_u64(acc.key, acc.n, emb_key(bx + 1, by, bz));
    if (nx < acc.n && (acc.key[nx] >> EMB_KEY_BITS) == row) atomicXor(acc.p + nx, 1u << line);
    else if (nx > 0 && (acc.key[nx - 1] >> EMB_KEY_BITS) == row) atomicXor(acc.t + nx - 1, 1u << line);
}

// The crossing of line (j, k) with the triangle, if any, recorded in its owner block.
__device__ __forceinline__ void vox_line(const VoxTri &V, const LevelGeom &g, const EmbLookup &lk, long long j,
                                         long long k, const VoxAcc &acc, int *st)
{
    unsigned long long *__restrict__ s_acc = acc.s;
    unsigned int *__restrict__ p_acc = acc.p;
    const int4 A = V.A, B = V.B, C = V.C;
    const int sx = V.sx;
    const int pz = (int)((2 * k + 1) * g.half), py = (int)((2 * j + 1) * g.half);
    if (emb_orient_yz(A.y, A.z, B.y, B.z, py, pz) != sx || emb_orient_yz(B.y, B.z, C.y, C.z, py, pz) != sx ||
        emb_orient_yz(C.y, C.z, A.y, A.z, py, pz) != sx)
        return;
    // n . (A - (x, py, pz)) = D_yz + n_x (A_x - x); the crossing is at x_hit with
    // x_hit - x = D(x) / n_x.
    const i128 Dyz = mul128(V.ny, (long long)A.y - py) + mul128(V.nz, (long long)A.z - pz);
    for (long long bx = V.bx0; bx <= V.bx1; ++bx) {
        const long long lo = bx * g.W;
        const i128 Dlo = Dyz + mul128(V.nx, (long long)A.x - lo);
        if (sgn_i128(Dlo) * sx < 0) continue;                     // x_hit < lo
        if (sgn_i128(Dlo - mul128(V.nx, g.W)) * sx >= 0) continue;  // x_hit >= lo + W
        const int32_t id = emb_lookup(lk, bx, j >> 2, k >> 2);
        if (id < 0) {
            vox_gap(acc, bx, j >> 2, k >> 2, (int)((j & 3) + 4 * (k & 3)));
            return;
        }
        // cell q of this line (centre lo + (2q+1) half) lies before the crossing iff
        // the perturbed centre sees the plane ahead: sign(D) == sign(n_x), D == 0 -> no
        unsigned long long bits = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const i128 Dq = Dlo - mul128(V.nx, (2 * q + 1) * g.half);
            if (sgn_i128(Dq) == sx) bits |= 1ull << q;
        }
        const int line = (int)((j & 3) + 4 * (k & 3));
        if (!emb_ck((uint64_t)id, (uint64_t)acc.n, st)) return;
        if (bits) atomicXor(s_acc + id, bits << (4 * line));
        atomicXor(p_acc + id, 1u << line);
        return;
    }
    emb_set_status(st, EMB_ERR_STATE);  // no block owns the crossing
}

__global__ void k_vox(const int4 *__restrict__ rec, int64_t T, const uint32_t *__restrict__ flist, int64_t nf,
                      const uint32_t *__restrict__ d_nf, const uint32_t *__restrict__ keep, LevelGeom g, EmbLookup lk,
                      VoxAcc acc, EmbBigQ Q, int *st)
{
    // nf: the planned count of a replay, or T when the count is still on the device;
    // d_nf: the count the filter found.  Grid-stride, so that a level with few kept
    // triangles does not launch a thread per triangle of the mesh.
    int64_t n = nf;
    if (d_nf && (int64_t)*d_nf < n) n = (int64_t)*d_nf;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = flist[i];
        if ((int64_t)t >= T) continue;
        if (keep && !keep[t]) continue;  // filtered out, the list not compacted
        VoxTri V;
        if (!vox_setup(rec, t, g, V)) continue;
        const unsigned long long items = vox_items(V);
        if (items > EMB_BIG_ITEMS && emb_bigq_push(Q, t, items)) continue;
        for (long long k = V.k0; k <= V.k1; ++k)
            for (long long j = V.j0; j <= V.j1; ++j) vox_line(V, g, lk, j, k, acc, st);
    }
}

// The queued chunks of large triangles, one warp per chunk (lines in j-major order).
__global__ void __launch_bounds__(EMB_BIG_BLOCK) k_vox_big(const int4 *__restrict__ rec, LevelGeom g, EmbLookup lk,
                                                           VoxAcc acc, EmbBigQ Q, int *st)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long nq = emb_bigq_count(Q);
    const unsigned long long nw = (unsigned long long)gridDim.x * (EMB_BIG_BLOCK / 32);
    for (unsigned long long e = (unsigned long long)blockIdx.x * (EMB_BIG_BLOCK / 32) + (threadIdx.x >> 5); e < nq;
         e += nw) {
        const uint2 E = Q.q[e];
        if (E.x == EMB_BIG_NONE) continue;
        VoxTri V;
        if (!vox_setup(rec, E.x, g, V)) continue;
        const unsigned long long items = vox_items(V);
        unsigned long long i0, i1;
        emb_bigq_range(E.y, items, i0, i1);
        const unsigned long long nj = (unsigned long long)(V.j1 - V.j0 + 1);
        const unsigned long long first = i0 + lane;
        long long jj = (long long)(first % nj), kk = (long long)(first / nj);
        const long long dj = (long long)(32 % nj), dk = (long long)(32 / nj);
        for (unsigned long long it = first; it < i1; it += 32) {
            vox_line(V, g, lk, V.j0 + jj, V.k0 + kk, acc, st);
            jj += dj;
            kk += dk;
            if (jj >= (long long)nj) {
                jj -= (long long)nj;
                ++kk;
            }
        }
    }
}

// Bit l of a 16-bit line set -> the four cell bits 4l .. 4l+3.
__device__ __forceinline__ unsigned long long spread_lines(unsigned int p)
{
    unsigned long long x = p & 0xFFFFu;
    x = (x | (x << 24)) & 0x000000FF000000FFull;
    x = (x | (x << 12)) & 0x000F000F000F000Full;
    x = (x | (x << 6)) & 0x0303030303030303ull;
    x = (x | (x << 3)) & 0x1111111111111111ull;
    return x * 0xFull;
}

__global__ void k_xscan(const uint64_t *__restrict__ key, int64_t n, const unsigned long long *__restrict__ s_acc,
                        const unsigned int *__restrict__ p_acc, const unsigned int *__restrict__ t_acc,
                        uint64_t *__restrict__ mask, const uint32_t *d_n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    n = emb_count(n, d_n);
    if (i >= n) return;
    uint64_t row = key[i] >> EMB_KEY_BITS;
    if (i + 1 < n && (key[i + 1] >> EMB_KEY_BITS) == row) return;  // only the row's last (+x-most) block walks
    unsigned int acc = t_acc[i];  // crossings beyond the row's last block
    // the walk loads 8 blocks at a time (those past the row's first block are read and
    // dropped), so that it waits on memory once per 8 blocks instead of once per block
    for (int64_t j = i;; j -= 8) {
        uint64_t kk[8];
        unsigned long long ss[8];
        unsigned int pp[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t jj = j - u;
            kk[u] = jj >= 0 ? key[jj] : ~0ull;  // ~0 >> EMB_KEY_BITS is no row
            ss[u] = jj >= 0 ? s_acc[jj] : 0ull;
            pp[u] = jj >= 0 ? p_acc[jj] : 0u;
        }
        bool end = false;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            end = end || (kk[u] >> EMB_KEY_BITS) != row;
            if (!end) {
                mask[j - u] = ss[u] ^ spread_lines(acc);
                acc ^= pp[u];
            }
        }
        if (end) break;
    }
}

// Enqueue only: s_acc (n uint64) and p_acc (n uint32) are scratch; writes lv.mask.
emb_status emb_enq_voxelize(const int4 *rec, int64_t T, const uint32_t *flist, int64_t nf, const uint32_t *d_nf,
                            const uint32_t *keep, LevelGeom g, const EmbLevel &lv, unsigned long long *s_acc,
                            unsigned int *p_acc, unsigned int *t_acc, const EmbBigQ &Q, int block, cudaStream_t s)
{
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    if (lv.n == 0) return EMB_OK;
    EMB_CUDA_TRY(cudaMemsetAsync(s_acc, 0, lv.n * sizeof(unsigned long long), s));
    EMB_CUDA_TRY(cudaMemsetAsync(p_acc, 0, lv.n * sizeof(unsigned int), s));
    EMB_CUDA_TRY(cudaMemsetAsync(t_acc, 0, lv.n * sizeof(unsigned int), s));
    const VoxAcc acc = {s_acc, p_acc, t_acc, lv.key, lv.n};
    if (nf > 0) {
        const EmbLookup lk = emb_lookup_of(lv);
        if (Q.cap) EMB_CUDA_TRY(cudaMemsetAsync(Q.n, 0, sizeof(unsigned long long), s));
        int64_t grid = emb_grid(nf, block);
        const int64_t full = (int64_t)emb_sm_count() * (2048 / block);  // one resident wave
        if (grid > full) grid = full;
        EMB_LAUNCH((k_vox), (int)grid, block, 0, s)(rec, T, flist, nf, d_nf, keep, g, lk, acc, Q, st);
        if (Q.cap) EMB_LAUNCH((k_vox_big), EMB_BIG_GRID, EMB_BIG_BLOCK, 0, s)(rec, g, lk, acc, Q, st);
    }
    EMB_LAUNCH((k_xscan), emb_grid(lv.n, 256), 256, 0, s)(lv.key, lv.n, s_acc, p_acc, t_acc, lv.mask, lv.d_n);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

extern "C" emb_status emb_voxelize(emb_forest f, emb_bins b, int32_t level, uint64_t *d_solid_mask, void *stream)
{
    if (!f || !b) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    if (b->f != f || b->level != level || level < 0 || level > f->top) return EMB_ERR_STATE;
    void *mask_out = nullptr;
    if (emb_device_view(d_solid_mask, &mask_out) != EMB_OK) return EMB_ERR_BAD_INPUT;
    cudaStream_t s = emb_stream(stream);
    EmbLevel &lv = f->lv[level];
    LevelGeom g = level_geom(f, level);
    if (lv.n == 0) {
        lv.mask_valid = 1;
        return EMB_OK;
    }
    if (!lv.mask) EMB_CUDA_TRY(emb_malloc_async(&lv.mask, lv.n * sizeof(uint64_t), s));
    unsigned long long *s_acc = nullptr;
    unsigned int *p_acc = nullptr, *t_acc = nullptr;
    EMB_CUDA_TRY(emb_malloc_async(&s_acc, lv.n * sizeof(unsigned long long), s));
    EMB_CUDA_TRY(emb_malloc_async(&p_acc, lv.n * sizeof(unsigned int), s));
    EMB_CUDA_TRY(emb_malloc_async(&t_acc, lv.n * sizeof(unsigned int), s));
    EmbBigQ Q;
    emb_status rc = emb_bigq_alloc(Q, b->m->T, s);
    if (rc != EMB_OK) return rc;
    // the filtered count stays on the device: the grid covers every triangle and stops at it
    rc = emb_enq_voxelize(b->m->rec, b->m->T, b->flist, b->known ? b->nf : b->m->T, (const uint32_t *)b->dcount, b->keep,
                          g, lv, s_acc, p_acc, t_acc, Q, 128, s);
    emb_bigq_free(Q, s);
    if (rc != EMB_OK) return rc;
    if (mask_out)  // device memory, or page-locked host memory (an asynchronous copy over the host link)
        EMB_CUDA_TRY(cudaMemcpyAsync(mask_out, lv.mask, lv.n * sizeof(uint64_t), cudaMemcpyDefault, s));
    EMB_CUDA_TRY(cudaFreeAsync(s_acc, s));
    EMB_CUDA_TRY(cudaFreeAsync(p_acc, s));
    EMB_CUDA_TRY(cudaFreeAsync(t_acc, s));
    lv.mask_valid = 1;
    if (level == f->top) f->n_links = -1;
    return EMB_OK;
}
