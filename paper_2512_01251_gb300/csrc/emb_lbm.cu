// One lattice-Boltzmann step on the finest level of a forest: the consumer the
// cut-link table is built for (Sec. 2.2 cites interpolated bounce-back with the link
// fractions q and the momentum exchange; Sec. 3.4 lays the table out for lookup during
// computation).  The paper prints neither the collision model nor Bouzidi's rule; the
// textbook BGK collision with the D3Q19 / D3Q27 weights and the linear Bouzidi rule of
// emb_mex_force are used.  Populations are SoA, pop[i * stride + cell], cell = block *
// 64 + x + 4 y + 16 z on the finest level.  Three passes, each its own kernel so that
// the cost of the boundary treatment can be timed against the rest:
//   k_lbm_stream   pull streaming into pre-collision populations: f_i(x) = f*_i(x - c_i)
//                  when x - c_i is a fluid cell of the level, f*_i(x) when its block is
//                  missing (zero gradient at the edge of the level: the coupling to
//                  coarser levels is out of scope), left for the next pass when solid;
//   k_lbm_bouzidi  per cut link (x, d, q): the population entering x against c_d, from
//                  f*_d(x), f*_d(x - c_d) and f*_-d(x) by the linear rule;
//   k_lbm_collide  BGK f* = f - omega (f - f_eq(rho, u)) at fluid cells, 0 at solid ones.
#include "emb_internal.cuh"

// direction index of a block offset (ox, oy, oz) in {-1,0,1}^3, code (ox+1) + 3(oy+1) + 9(oz+1)
__constant__ int8_t c_lbm_dir_of_offset[27] = {20, 16, 26, 12, 6, 13, 24, 17, 21, 8, 4, 9, 2, 0,
                                               1,  10, 3,  7,  22, 18, 23, 14, 5, 11, 25, 15, 19};

// Cell x - c of cell (b, t): its id, or -1 if it is solid, -2 if its block is missing.
__device__ __forceinline__ int64_t lbm_source(int64_t b, int t, int cx, int cy, int cz, const int32_t *__restrict__ nbr,
                                              const uint64_t *__restrict__ mask)
{
    const int x = (t & 3) - cx, y = ((t >> 2) & 3) - cy, z = (t >> 4) - cz;
    const int ox = x < 0 ? -1 : (x > 3 ? 1 : 0), oy = y < 0 ? -1 : (y > 3 ? 1 : 0), oz = z < 0 ? -1 : (z > 3 ? 1 : 0);
    int64_t nb = b;
    if (ox | oy | oz) {
        nb = nbr[b * 26 + c_lbm_dir_of_offset[(ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)] - 1];
        if (nb < 0) return -2;
    }
    const int lt = (x & 3) + 4 * (y & 3) + 16 * (z & 3);
    if ((mask[nb] >> lt) & 1ull) return -1;
    return nb * 64 + lt;
}

template <int Q>
__global__ void k_lbm_stream(const float *__restrict__ pop, float *__restrict__ pre, int64_t stride, int64_t ncell,
                             const int32_t *__restrict__ nbr, const uint64_t *__restrict__ mask)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ncell) return;
    const int64_t b = x >> 6;
    const int t = (int)(x & 63);
    const bool solid = (mask[b] >> t) & 1ull;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float v = 0.0f;
        if (!solid) {
            int cx, cy, cz;
            emb_dir(i, cx, cy, cz);
            const int64_t s = lbm_source(b, t, cx, cy, cz, nbr, mask);
            v = s >= 0 ? pop[(int64_t)i * stride + s] : (s == -2 ? pop[(int64_t)i * stride + x] : 0.0f);
        }
        pre[(int64_t)i * stride + x] = v;
    }
}

__global__ void k_lbm_bouzidi(const int32_t *__restrict__ cell, const uint8_t *__restrict__ dir,
                              const float *__restrict__ q, int64_t n, const float *__restrict__ pop,
                              float *__restrict__ pre, int64_t stride, int64_t ncell, int lattice,
                              const int32_t *__restrict__ nbr, const uint64_t *__restrict__ mask, int *st)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t c = cell[k];
    const int d = dir[k];
    if (c < 0 || c >= ncell || d < 1 || d >= lattice) {
        emb_set_status(st, EMB_ERR_BAD_INPUT);  // not a link of this level and lattice
        return;
    }
    const int o = (d & 1) ? d + 1 : d - 1;
    int cx, cy, cz;
    emb_dir(d, cx, cy, cz);
    const float f_d = pop[(int64_t)d * stride + c], f_o = pop[(int64_t)o * stride + c];
    const float qq = q[k];
    float g;
    if (qq < 0.5f) {
        const int64_t p = lbm_source(c >> 6, (int)(c & 63), cx, cy, cz, nbr, mask);  // x - c_d
        g = p >= 0 ? 2.0f * qq * f_d + (1.0f - 2.0f * qq) * pop[(int64_t)d * stride + p] : f_d;
    } else {
        g = f_d / (2.0f * qq) + (2.0f * qq - 1.0f) / (2.0f * qq) * f_o;
    }
    pre[(int64_t)o * stride + c] = g;
}

template <int Q>
__global__ void k_lbm_collide(const float *__restrict__ pre, float *__restrict__ out, int64_t stride, int64_t ncell,
                              const uint64_t *__restrict__ mask, float omega)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ncell) return;
    if ((mask[x >> 6] >> (x & 63)) & 1ull) {
#pragma unroll
        for (int i = 0; i < Q; ++i) out[(int64_t)i * stride + x] = 0.0f;
        return;
    }
    float f[Q];
    float rho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int cx, cy, cz;
        emb_dir(i, cx, cy, cz);
        f[i] = pre[(int64_t)i * stride + x];
        rho += f[i];
        jx += cx * f[i];
        jy += cy * f[i];
        jz += cz * f[i];
    }
    const float inv = rho != 0.0f ? 1.0f / rho : 0.0f;
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int cx, cy, cz;
        emb_dir(i, cx, cy, cz);
        const int kind = cx * cx + cy * cy + cz * cz;  // 0 rest, 1 axis, 2 edge, 3 corner
        const float w = Q == 19 ? (kind == 0 ? 1.0f / 3 : (kind == 1 ? 1.0f / 18 : 1.0f / 36))
                                : (kind == 0 ? 8.0f / 27 : (kind == 1 ? 2.0f / 27 : (kind == 2 ? 1.0f / 54 : 1.0f / 216)));
        const float cu = cx * ux + cy * uy + cz * uz;
        const float feq = w * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * usq);
        out[(int64_t)i * stride + x] = f[i] - omega * (f[i] - feq);
    }
}

extern "C" emb_status emb_lbm_step(emb_forest f, int32_t lattice, const int32_t *d_cell, const uint8_t *d_dir,
                                   const float *d_q, int64_t n_links, float omega, const float *d_pop, float *d_pre,
                                   float *d_pop_out, int64_t pop_stride, int32_t phases, void *stream)
{
    if (!f || (lattice != 19 && lattice != 27) || n_links < 0 || !(omega >= 0.0f && omega < 2.0f) || phases < 1 ||
        phases > 7)
        return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    const int L = f->max_level;
    if (f->top != L || !f->lv[L].mask_valid) return EMB_ERR_STATE;
    EmbLevel &lv = f->lv[L];
    const int64_t ncell = lv.n * 64;
    if (pop_stride < ncell) return EMB_ERR_BAD_INPUT;
    if (ncell == 0) return EMB_OK;
    if (!d_pop || !d_pre || !d_pop_out || d_pop == d_pre || d_pre == d_pop_out || d_pop == d_pop_out)
        return EMB_ERR_BAD_INPUT;
    if (n_links > 0 && (!d_cell || !d_dir || !d_q)) return EMB_ERR_BAD_INPUT;
    cudaStream_t s = emb_stream(stream);
    emb_status rc = emb_build_neighbors(lv, s);
    if (rc != EMB_OK) return rc;
    const int grid = emb_grid(ncell, 256);
    if (phases & 1) {
        if (lattice == 19) EMB_LAUNCH((k_lbm_stream<19>), grid, 256, 0, s)(d_pop, d_pre, pop_stride, ncell, lv.nbr, lv.mask);
        else EMB_LAUNCH((k_lbm_stream<27>), grid, 256, 0, s)(d_pop, d_pre, pop_stride, ncell, lv.nbr, lv.mask);
    }
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    if ((phases & 2) && n_links > 0)
        EMB_LAUNCH((k_lbm_bouzidi), emb_grid(n_links, 256), 256, 0, s)(d_cell, d_dir, d_q, n_links, d_pop, d_pre, pop_stride,
                                                                       ncell, lattice, lv.nbr, lv.mask, st);
    if (phases & 4) {
        if (lattice == 19)
            EMB_LAUNCH((k_lbm_collide<19>), grid, 256, 0, s)(d_pre, d_pop_out, pop_stride, ncell, lv.mask, omega);
        else EMB_LAUNCH((k_lbm_collide<27>), grid, 256, 0, s)(d_pre, d_pop_out, pop_stride, ncell, lv.mask, omega);
    }
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}
