// Forest harness (Sec. 3.2): root grid, top-down creation of children from
// refinement flags, per-level coordinate hash and neighbour links.
//
// Blocks of a level are kept in ascending key order, key = (bz, by, bx), so
// every x-row of blocks is contiguous and ordered along +x (the order the
// voxelizer's row scan needs).  Children are written straight into that order:
// with parents sorted, the rank of a child follows from exclusive counts of
// flagged parents before its parent's plane (bz), row (bz, by) and position.
#include <stdlib.h>

#include "emb_internal.cuh"

__global__ void k_root_keys(int64_t R, uint64_t *__restrict__ key)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * R * R) return;
    key[i] = emb_key(i % R, (i / R) % R, i / (R * R));
}

__global__ void k_flags_u32(const uint8_t *__restrict__ f, int64_t n, uint32_t *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = f[i] ? 1u : 0u;
}


__global__ void k_make_children(const uint64_t *__restrict__ key, int64_t n, const uint8_t *__restrict__ flags,
                                const uint32_t *__restrict__ rank, uint64_t *__restrict__ ckey, int64_t Cn)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !flags[p]) return;
    uint64_t k = key[p];
    int64_t bx = (int64_t)(k & EMB_KEY_MASK), by = (int64_t)((k >> EMB_KEY_BITS) & EMB_KEY_MASK),
            bz = (int64_t)(k >> (2 * EMB_KEY_BITS));
    uint64_t row0 = k & ~EMB_KEY_MASK, row1 = row0 + (1ull << EMB_KEY_BITS);
    uint64_t pl0 = k & ~((1ull << (2 * EMB_KEY_BITS)) - 1ull), pl1 = pl0 + (1ull << (2 * EMB_KEY_BITS));
    int64_t rl = lower_bound_u64(key, n, row0), rh = lower_bound_u64(key, n, row1);
    int64_t pll = lower_bound_u64(key, n, pl0), plh = lower_bound_u64(key, n, pl1);
    int64_t r_p = rank[p], r_row = rank[rl], F_row = (int64_t)rank[rh] - r_row;
    int64_t r_pl = rank[pll], F_pl = (int64_t)rank[plh] - r_pl;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int64_t pos = 8 * r_pl + dz * 4 * F_pl + 4 * (r_row - r_pl) + dy * 2 * F_row + 2 * (r_p - r_row) + dx;
                if (pos >= 0 && pos < Cn) ckey[pos] = emb_key(2 * bx + dx, 2 * by + dy, 2 * bz + dz);
            }
}

__global__ void k_unpack_keys(const uint64_t *__restrict__ key, int64_t n, int32_t *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = key[i];
    out[3 * i + 0] = (int32_t)(k & EMB_KEY_MASK);
    out[3 * i + 1] = (int32_t)((k >> EMB_KEY_BITS) & EMB_KEY_MASK);
    out[3 * i + 2] = (int32_t)(k >> (2 * EMB_KEY_BITS));
}

static void free_level(EmbLevel &lv)
{
    if (lv.key) cudaFree(lv.key);
    if (lv.hkey) cudaFree(lv.hkey);
    if (lv.hval) cudaFree(lv.hval);
    if (lv.mask) cudaFree(lv.mask);
    if (lv.nbr) cudaFree(lv.nbr);
    if (lv.bits) cudaFree(lv.bits);
    if (lv.wpre) cudaFree(lv.wpre);
    lv = EmbLevel();
}

extern "C" emb_status emb_forest_root(int32_t R, int32_t max_level, void *stream, emb_forest *out)
{
    if (!out || R < 1 || max_level < 0 || max_level >= EMB_MAX_LEVELS) return EMB_ERR_BAD_INPUT;
    *out = nullptr;
    int32_t r_o = R, k = 0;
    while ((r_o & 1) == 0) {
        r_o >>= 1;
        ++k;
    }
    if (k + max_level > 17 || ((int64_t)R << max_level) >= (1ll << EMB_KEY_BITS) || (int64_t)r_o * (1 << 20) >= (1ll << 25))
        return EMB_ERR_RANGE;
    if ((int64_t)R * R * R > 2147483647ll) return EMB_ERR_BAD_INPUT;
    cudaStream_t s = emb_stream(stream);
    emb_forest f = new emb_forest_s();
    f->R = R;
    f->r_o = r_o;
    f->k = k;
    f->max_level = max_level;
    f->top = 0;
    cudaGetDevice(&f->device);
    EmbLevel &lv = f->lv[0];
    lv.n = (int64_t)R * R * R;
    lv.nb_axis = R;
    if (emb_malloc_async(&lv.key, lv.n * sizeof(uint64_t), s) != cudaSuccess) {
        emb_forest_destroy(f);
        return EMB_ERR_CUDA;
    }
    emb_status rc = emb_enq_root_keys(R, lv.key, s);
    if (rc == EMB_OK) rc = emb_build_hash(lv, s);
    if (rc != EMB_OK) {
        emb_forest_destroy(f);
        return rc;
    }
    *out = f;
    return EMB_OK;
}

// Level arrays come from the stream-ordered pool of the calls that built them; the
// teardown synchronises the device once and returns them all.
extern "C" void emb_forest_destroy(emb_forest f)
{
    if (!f) return;
    cudaDeviceSynchronize();
    for (int L = 0; L < EMB_MAX_LEVELS; ++L) free_level(f->lv[L]);
    if (f->cand) cudaFree(f->cand);
    if (f->blk_off) cudaFree(f->blk_off);
    if (f->work) cudaFree(f->work);
    if (f->work_n) cudaFree(f->work_n);
    if (f->next) cudaFree(f->next);
    emb_readback_release(f->rb_slot);
    delete f;
}

// Refinement in two enqueue-only halves (buffers supplied by the caller):
//  (1) ranks of the flagged blocks of P: cnt, rank hold P.n + 1 uint32; the number
//      of flagged blocks F ends at rank[P.n]; tmp is scan scratch for P.n entries;
//  (2) the 8 F children keys, written in (z, y, x) order into ckey.
emb_status emb_enq_flag_ranks(const EmbLevel &P, const uint8_t *d_flags, uint32_t *cnt, uint32_t *rank, uint64_t *tmp,
                              cudaStream_t s, uint64_t expect)
{
    if (P.n > 0) EMB_LAUNCH((k_flags_u32), emb_grid(P.n, 256), 256, 0, s)(d_flags, P.n, cnt);
    return emb_scan_into_expect(cnt, rank, P.n, tmp, expect, s);
}

// Keys [8 F, Cn) of a planned replay that flagged fewer blocks than its buffers hold
// (a replay with headroom, or one whose counts left its plan): a key above every real
// key, so that the level's keys stay sorted for the binary searches over all Cn of
// them; its coordinates (2^21 - 1 on every axis) fail the range checks of the passes
// that decode keys, and the passes over blocks stop at the device count where there
// is one.
#define EMB_KEY_TAIL 0x7FFFFFFFFFFFFFFFull
__global__ void k_key_tail(uint64_t *__restrict__ ckey, int64_t Cn, const uint32_t *__restrict__ nflags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Cn && i >= 8 * (int64_t)*nflags) ckey[i] = EMB_KEY_TAIL;
}

emb_status emb_enq_children(const EmbLevel &P, const uint8_t *d_flags, const uint32_t *rank, uint64_t *ckey, int64_t Cn,
                            bool planned, cudaStream_t s)
{
    if (P.n > 0 && Cn > 0) EMB_LAUNCH((k_make_children), emb_grid(P.n, 256), 256, 0, s)(P.key, P.n, d_flags, rank, ckey, Cn);
    if (planned && Cn > 0) EMB_LAUNCH((k_key_tail), emb_grid(Cn, 256), 256, 0, s)(ckey, Cn, rank + P.n);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

emb_status emb_enq_root_keys(int64_t R, uint64_t *key, cudaStream_t s)
{
    EMB_LAUNCH((k_root_keys), emb_grid(R * R * R, 256), 256, 0, s)(R, key);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

emb_status emb_forest_settle(emb_forest f)
{
    if (!f || f->n_pending < 0) return EMB_OK;
    EMB_CUDA_TRY(cudaEventSynchronize(f->rb_ev));
    f->lv[f->n_pending].n = 8 * (int64_t)(*(volatile uint32_t *)f->rb_h);
    f->n_pending = -1;
    return EMB_OK;
}

extern "C" emb_status emb_forest_refine(emb_forest f, int32_t level, const uint8_t *d_flags, void *stream)
{
    if (!f) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    if (level < 0 || level != f->top || level >= f->max_level) return EMB_ERR_STATE;
    if (!d_flags && f->lv[level].n > 0) return EMB_ERR_BAD_INPUT;
    cudaStream_t s = emb_stream(stream);
    EmbLevel &P = f->lv[level];
    EmbLevel &C = f->lv[level + 1];
    free_level(C);
    uint32_t *cnt = nullptr, *rank = nullptr;
    uint64_t *tmp = nullptr;
    EMB_CUDA_TRY(emb_malloc_async(&cnt, (P.n + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&rank, (P.n + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&tmp, emb_scan_tmp_words(P.n) * sizeof(uint64_t), s));
    emb_status rc = emb_enq_flag_ranks(P, d_flags, cnt, rank, tmp, s);
    if (rc != EMB_OK) return rc;
    C.nb_axis = P.nb_axis * 2;
    if (f->rb_slot < 0) f->rb_slot = emb_readback_acquire(&f->rb_h, &f->rb_ev);
    if (emb_bitmap_words(C.nb_axis) > 0 && f->rb_slot >= 0) {
        // The child level takes the rank bitmap: its keys (room for 8 per parent) and
        // index are built from the flagged count on the device while that count comes
        // back to the host, so the GPU is not left idle during the read-back.
        EMB_CUDA_TRY(cudaMemcpyAsync(f->rb_h, rank + P.n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        EMB_CUDA_TRY(cudaEventRecord(f->rb_ev, s));
        const int64_t cap = 8 * P.n;
        EMB_CUDA_TRY(emb_malloc_async(&C.key, (cap + 1) * sizeof(uint64_t), s));
        rc = emb_enq_children(P, d_flags, rank, C.key, cap, false, s);
        if (rc == EMB_OK) rc = emb_build_index_counted(C, rank + P.n, cap, s);
        EMB_CUDA_TRY(cudaFreeAsync(cnt, s));
        EMB_CUDA_TRY(cudaFreeAsync(rank, s));
        EMB_CUDA_TRY(cudaFreeAsync(tmp, s));
        if (rc != EMB_OK) return rc;
        // the count is stored when a call first needs it (emb_forest_settle): work that
        // does not need it, such as the next level's x-line filter, is queued first, so
        // that the GPU has it while the count travels
        C.n = 0;
        f->n_pending = level + 1;
    } else {
        uint32_t F = 0;
        EMB_CUDA_TRY(cudaMemcpyAsync(&F, rank + P.n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        EMB_CUDA_TRY(cudaStreamSynchronize(s));
        C.n = 8 * (int64_t)F;
        EMB_CUDA_TRY(emb_malloc_async(&C.key, (C.n + 1) * sizeof(uint64_t), s));
        rc = emb_enq_children(P, d_flags, rank, C.key, C.n, false, s);
        if (rc != EMB_OK) return rc;
        EMB_CUDA_TRY(cudaFreeAsync(cnt, s));
        EMB_CUDA_TRY(cudaFreeAsync(rank, s));
        EMB_CUDA_TRY(cudaFreeAsync(tmp, s));
        rc = emb_build_hash(C, s);
        if (rc != EMB_OK) return rc;
    }
    f->top = level + 1;
    // a new finest level invalidates cached link candidates
    if (f->cand) {
        cudaFreeAsync(f->cand, s);
        f->cand = nullptr;
    }
    if (f->blk_off) {
        cudaFreeAsync(f->blk_off, s);
        f->blk_off = nullptr;
    }
    if (f->work) {
        cudaFreeAsync(f->work, s);
        f->work = nullptr;
    }
    if (f->work_n) {
        cudaFreeAsync(f->work_n, s);
        f->work_n = nullptr;
    }
    f->n_links = -1;
    return EMB_OK;
}

extern "C" emb_status emb_forest_num_blocks(emb_forest f, int32_t level, int64_t *h_out)
{
    if (!f || !h_out || level < 0 || level >= EMB_MAX_LEVELS) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    *h_out = level <= f->top ? f->lv[level].n : 0;
    return EMB_OK;
}

extern "C" emb_status emb_forest_blocks(emb_forest f, int32_t level, int32_t *d_out, void *stream)
{
    EMB_SETTLE(f);
    if (!f || level < 0 || level > f->top) return EMB_ERR_STATE;
    const EmbLevel &lv = f->lv[level];
    if (lv.n == 0) return EMB_OK;
    if (!d_out) return EMB_ERR_BAD_INPUT;
    EMB_LAUNCH((k_unpack_keys), emb_grid(lv.n, 256), 256, 0, emb_stream(stream))(lv.key, lv.n, d_out);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

extern "C" emb_status emb_forest_neighbors(emb_forest f, int32_t level, int32_t *d_out, void *stream)
{
    EMB_SETTLE(f);
    if (!f || level < 0 || level > f->top) return EMB_ERR_STATE;
    EmbLevel &lv = f->lv[level];
    if (lv.n == 0) return EMB_OK;
    if (!d_out) return EMB_ERR_BAD_INPUT;
    cudaStream_t s = emb_stream(stream);
    emb_status rc = emb_build_neighbors(lv, s);
    if (rc != EMB_OK) return rc;
    EMB_CUDA_TRY(cudaMemcpyAsync(d_out, lv.nbr, lv.n * 26 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return EMB_OK;
}

extern "C" emb_status emb_forest_masks(emb_forest f, int32_t level, uint64_t *d_out, void *stream)
{
    EMB_SETTLE(f);
    if (!f || level < 0 || level > f->top || !f->lv[level].mask_valid) return EMB_ERR_STATE;
    const EmbLevel &lv = f->lv[level];
    if (lv.n == 0) return EMB_OK;
    if (!d_out) return EMB_ERR_BAD_INPUT;
    EMB_CUDA_TRY(cudaMemcpyAsync(d_out, lv.mask, lv.n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, emb_stream(stream)));
    return EMB_OK;
}
