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
// Rows are contiguous and x-ordered in the level's block list.  Unrefined gaps
// between blocks of a row contain no surface (the refine rule guarantees it), so
// the row scan sees every crossing.  Block-local parity plays the role of the
// paper's internal propagation, and the suffix scan that of Alg. 4's
// neighbour-to-neighbour walk along +x.
#include "emb_internal.cuh"

__global__ void k_vox(const int4 *__restrict__ rec, const uint32_t *__restrict__ flist, int64_t nf, LevelGeom g,
                      EmbLookup lk,
                      unsigned long long *__restrict__ s_acc, unsigned int *__restrict__ p_acc, int *st)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int64_t t = flist[i];
    int4 A = rec[3 * t], B = rec[3 * t + 1], C = rec[3 * t + 2];
    long long ux = (long long)B.x - A.x, uy = (long long)B.y - A.y, uz = (long long)B.z - A.z;
    long long vx = (long long)C.x - A.x, vy = (long long)C.y - A.y, vz = (long long)C.z - A.z;
    long long nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    if (nx == 0) return;
    int sx = nx > 0 ? 1 : -1;
    long long j0, j1, k0, k1;
    line_range(min(A.y, min(B.y, C.y)), max(A.y, max(B.y, C.y)), g.lh, g.half, g.ncell, j0, j1);
    line_range(min(A.z, min(B.z, C.z)), max(A.z, max(B.z, C.z)), g.lh, g.half, g.ncell, k0, k1);
    long long bx0 = emb_floor_shr(min(A.x, min(B.x, C.x)), g.lW), bx1 = emb_floor_shr(max(A.x, max(B.x, C.x)), g.lW);
    if (bx0 < 0) bx0 = 0;
    if (bx1 > g.nb - 1) bx1 = g.nb - 1;
    for (long long k = k0; k <= k1; ++k) {
        int pz = (int)((2 * k + 1) * g.half);
        for (long long j = j0; j <= j1; ++j) {
            int py = (int)((2 * j + 1) * g.half);
            if (emb_orient_yz(A.y, A.z, B.y, B.z, py, pz) != sx || emb_orient_yz(B.y, B.z, C.y, C.z, py, pz) != sx ||
                emb_orient_yz(C.y, C.z, A.y, A.z, py, pz) != sx)
                continue;
            // n . (A - (x, py, pz)) = D_yz + n_x (A_x - x); the crossing is at x_hit with
            // x_hit - x = D(x) / n_x.
            i128 Dyz = mul128(ny, (long long)A.y - py) + mul128(nz, (long long)A.z - pz);
            bool owned = false;
            for (long long bx = bx0; bx <= bx1 && !owned; ++bx) {
                long long lo = bx * g.W;
                i128 Dlo = Dyz + mul128(nx, (long long)A.x - lo);
                if (sgn_i128(Dlo) * sx < 0) continue;                   // x_hit < lo
                if (sgn_i128(Dlo - mul128(nx, g.W)) * sx >= 0) continue;  // x_hit >= lo + W
                owned = true;
                int32_t id = emb_lookup(lk, bx, j >> 2, k >> 2);
                if (id < 0) {
                    emb_set_status(st, EMB_ERR_STATE);  // a crossing outside every block
                    break;
                }
                // cell q of this line (centre lo + (2q+1) half) lies before the crossing iff
                // the perturbed centre sees the plane ahead: sign(D) == sign(n_x), D == 0 -> no
                unsigned long long bits = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    i128 Dq = Dlo - mul128(nx, (2 * q + 1) * g.half);
                    if (sgn_i128(Dq) == sx) bits |= 1ull << q;
                }
                int line = (int)((j & 3) + 4 * (k & 3));
                if (bits) atomicXor(s_acc + id, bits << (4 * line));
                atomicXor(p_acc + id, 1u << line);
            }
            if (!owned) emb_set_status(st, EMB_ERR_STATE);
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
                        const unsigned int *__restrict__ p_acc, uint64_t *__restrict__ mask)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t row = key[i] >> EMB_KEY_BITS;
    if (i + 1 < n && (key[i + 1] >> EMB_KEY_BITS) == row) return;  // only the row's last (+x-most) block walks
    unsigned int acc = 0;
    for (int64_t j = i; j >= 0 && (key[j] >> EMB_KEY_BITS) == row; --j) {
        mask[j] = s_acc[j] ^ spread_lines(acc);
        acc ^= p_acc[j];
    }
}

// Enqueue only: s_acc (n uint64) and p_acc (n uint32) are scratch; writes lv.mask.
emb_status emb_enq_voxelize(const int4 *rec, const uint32_t *flist, int64_t nf, LevelGeom g, const EmbLevel &lv,
                            unsigned long long *s_acc, unsigned int *p_acc, int block, cudaStream_t s)
{
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    if (lv.n == 0) return EMB_OK;
    EMB_CUDA_TRY(cudaMemsetAsync(s_acc, 0, lv.n * sizeof(unsigned long long), s));
    EMB_CUDA_TRY(cudaMemsetAsync(p_acc, 0, lv.n * sizeof(unsigned int), s));
    if (nf > 0)
        EMB_LAUNCH((k_vox), emb_grid(nf, block), block, 0, s)(rec, flist, nf, g, emb_lookup_of(lv), s_acc, p_acc, st);
    EMB_LAUNCH((k_xscan), emb_grid(lv.n, 256), 256, 0, s)(lv.key, lv.n, s_acc, p_acc, lv.mask);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

extern "C" emb_status emb_voxelize(emb_forest f, emb_bins b, int32_t level, uint64_t *d_solid_mask, void *stream)
{
    if (!f || !b) return EMB_ERR_BAD_INPUT;
    if (b->f != f || b->level != level || level < 0 || level > f->top) return EMB_ERR_STATE;
    cudaStream_t s = emb_stream(stream);
    EmbLevel &lv = f->lv[level];
    LevelGeom g = level_geom(f, level);
    if (lv.n == 0) {
        lv.mask_valid = 1;
        return EMB_OK;
    }
    if (!lv.mask) EMB_CUDA_TRY(cudaMalloc(&lv.mask, lv.n * sizeof(uint64_t)));
    unsigned long long *s_acc = nullptr;
    unsigned int *p_acc = nullptr;
    EMB_CUDA_TRY(cudaMallocAsync(&s_acc, lv.n * sizeof(unsigned long long), s));
    EMB_CUDA_TRY(cudaMallocAsync(&p_acc, lv.n * sizeof(unsigned int), s));
    emb_status rc = emb_enq_voxelize(b->m->rec, b->flist, b->nf, g, lv, s_acc, p_acc, 128, s);
    if (rc != EMB_OK) return rc;
    if (d_solid_mask)
        EMB_CUDA_TRY(cudaMemcpyAsync(d_solid_mask, lv.mask, lv.n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    EMB_CUDA_TRY(cudaFreeAsync(s_acc, s));
    EMB_CUDA_TRY(cudaFreeAsync(p_acc, s));
    lv.mask_valid = 1;
    if (level == f->top) f->n_links = -1;
    return EMB_OK;
}
