// Incremental re-embedding of a moving or deforming body (Sec. 5 names moving
// geometry as future work).
//
// A change of the mesh confined to a region changes the embedding only near that
// region: a refine flag depends on the triangles within its block's dilated box, a
// cell's solid state changes only inside the volume the surface swept, and a link
// only near a changed cell or a moved face.  Rows of cells along +x must still be
// complete for the parity scan, so the region is a window of root-block rows: every
// bx, with y0 <= by < y1 and z0 <= bz < z1.
//
// emb_forest_root_window starts a forest holding only the root blocks of a window;
// the ordinary calls (bin, voxelize, refine flags, forest refinement, cut links)
// then embed the window from the triangles near it.  emb_splice replaces, on every
// level of an existing forest, the blocks inside an inner window by the window
// forest's blocks there, with their solid masks, and merges the two link tables: the
// old links outside the inner window and the window's links inside it, renumbered to
// the merged finest level and ordered by (cell, direction) as a fresh table is.
#include "emb_internal.cuh"

__global__ void k_root_keys_window(int64_t R, int64_t y0, int64_t ny, int64_t z0, int64_t n, uint64_t *__restrict__ key)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t bx = i % R, r = i / R, by = y0 + r % ny, bz = z0 + r / ny;
    key[i] = emb_key(bx, by, bz);
}

extern "C" emb_status emb_forest_root_window(int32_t R, int32_t max_level, int32_t y0, int32_t y1, int32_t z0,
                                             int32_t z1, void *stream, emb_forest *out)
{
    if (!out || R < 1 || max_level < 0 || max_level >= EMB_MAX_LEVELS) return EMB_ERR_BAD_INPUT;
    if (y0 < 0 || z0 < 0 || y1 > R || z1 > R || y0 >= y1 || z0 >= z1) return EMB_ERR_BAD_INPUT;
    *out = nullptr;
    int32_t r_o = R, k = 0;
    while ((r_o & 1) == 0) {
        r_o >>= 1;
        ++k;
    }
    if (k + max_level > 17 || ((int64_t)R << max_level) >= (1ll << EMB_KEY_BITS) || (int64_t)r_o * (1 << 20) >= (1ll << 25))
        return EMB_ERR_RANGE;
    cudaStream_t s = emb_stream(stream);
    emb_forest f = new emb_forest_s();
    f->R = R;
    f->r_o = r_o;
    f->k = k;
    f->max_level = max_level;
    f->top = 0;
    cudaGetDevice(&f->device);
    EmbLevel &lv = f->lv[0];
    lv.n = (int64_t)R * (y1 - y0) * (z1 - z0);
    lv.nb_axis = R;
    if (emb_malloc_async(&lv.key, (lv.n + 1) * sizeof(uint64_t), s) != cudaSuccess) {
        emb_forest_destroy(f);
        return EMB_ERR_CUDA;
    }
    EMB_LAUNCH((k_root_keys_window), emb_grid(lv.n, 256), 256, 0, s)(R, y0, y1 - y0, z0, lv.n, lv.key);
    emb_status rc = cudaGetLastError() == cudaSuccess ? emb_build_hash(lv, s) : EMB_ERR_CUDA;
    if (rc != EMB_OK) {
        emb_forest_destroy(f);
        return rc;
    }
    *out = f;
    return EMB_OK;
}

// ---------------------------------------------------------------------------
// splice
// ---------------------------------------------------------------------------
// Window of root-block rows at level L: the block's root ancestor has y0 <= by < y1
// and z0 <= bz < z1.
struct RowWindow {
    int64_t y0, y1, z0, z1;
    __device__ __forceinline__ bool inside(uint64_t k, int L) const
    {
        const int64_t by = (int64_t)((k >> EMB_KEY_BITS) & EMB_KEY_MASK) >> L, bz = (int64_t)(k >> (2 * EMB_KEY_BITS)) >> L;
        return by >= y0 && by < y1 && bz >= z0 && bz < z1;
    }
};

// sel[i] = 1 for the blocks an old level keeps (outside the window) or a window level
// gives (inside it).
__global__ void k_sp_select(const uint64_t *__restrict__ key, int64_t n, RowWindow W, int L, int want_inside,
                            uint32_t *__restrict__ sel)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sel[i] = (W.inside(key[i], L) ? 1u : 0u) == (uint32_t)want_inside ? 1u : 0u;
}

// Selected keys compacted in order (pos: exclusive scan of sel).
__global__ void k_sp_compact_keys(const uint64_t *__restrict__ key, const uint32_t *__restrict__ sel,
                                  const uint32_t *__restrict__ pos, int64_t n, uint64_t *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && sel[i]) out[pos[i]] = key[i];
}

// Merge by ranks: a selected block of one side goes to its rank on that side plus the
// number of the other side's selected keys below its key (the two sides are disjoint).
// newid[i] = merged id of block i, or -1 when it is not selected.
__global__ void k_sp_place(const uint64_t *__restrict__ key, const uint64_t *__restrict__ mask,
                           const uint32_t *__restrict__ sel, const uint32_t *__restrict__ pos, int64_t n,
                           const uint64_t *__restrict__ other, int64_t n_other, uint64_t *__restrict__ mkey,
                           uint64_t *__restrict__ mmask, int32_t *__restrict__ newid)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!sel[i]) {
        newid[i] = -1;
        return;
    }
    const int64_t p = (int64_t)pos[i] + lower_bound_u64(other, n_other, key[i]);
    mkey[p] = key[i];
    mmask[p] = mask[i];
    newid[i] = (int32_t)p;
}

// First link of every block in a table sorted by cell (cell = block * 64 + t).
__global__ void k_sp_link_starts(const int32_t *__restrict__ cell, int64_t nl, int64_t nblk, uint32_t *__restrict__ start)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nblk) return;
    int64_t lo = 0, hi = nl;
    const int64_t c = b * 64;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)cell[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    start[b] = (uint32_t)lo;
}

// Links per merged block, from the side each merged block came from.
__global__ void k_sp_link_counts(const int32_t *__restrict__ newid, int64_t n, const uint32_t *__restrict__ start,
                                 uint32_t *__restrict__ cnt)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n && newid[b] >= 0) cnt[newid[b]] = start[b + 1] - start[b];
}

// Copies the links of the selected blocks of one side to their merged place.
__global__ void k_sp_link_copy(const int32_t *__restrict__ cell, const uint8_t *__restrict__ dir,
                               const float *__restrict__ q, const int32_t *__restrict__ tri, int64_t nl,
                               const int32_t *__restrict__ newid, const uint32_t *__restrict__ start,
                               const uint32_t *__restrict__ moff, const int32_t *__restrict__ tri_map, int64_t cap,
                               int32_t *__restrict__ o_cell, uint8_t *__restrict__ o_dir, float *__restrict__ o_q,
                               int32_t *__restrict__ o_tri)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nl) return;
    const int64_t b = cell[k] >> 6;
    const int32_t nb = newid[b];
    if (nb < 0) return;
    const int64_t o = (int64_t)moff[nb] + (k - (int64_t)start[b]);
    if (o >= cap) return;
    o_cell[o] = nb * 64 + (cell[k] & 63);
    o_dir[o] = dir[k];
    o_q[o] = q[k];
    o_tri[o] = tri_map && tri[k] >= 0 ? tri_map[tri[k]] : tri[k];
}

extern "C" emb_status emb_splice(emb_forest f, emb_forest w, int32_t y0, int32_t y1, int32_t z0, int32_t z1,
                                 const int32_t *f_cell, const uint8_t *f_dir, const float *f_q, const int32_t *f_tri,
                                 int64_t f_n, const int32_t *w_cell, const uint8_t *w_dir, const float *w_q,
                                 const int32_t *w_tri, int64_t w_n, const int32_t *w_tri_map, int32_t *o_cell,
                                 uint8_t *o_dir, float *o_q, int32_t *o_tri, int64_t capacity, int64_t *h_count,
                                 void *stream)
{
    if (!f || !w || !h_count || f_n < 0 || w_n < 0 || capacity < 0) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    EMB_SETTLE(w);
    if (f->R != w->R || f->max_level != w->max_level) return EMB_ERR_STATE;
    if (y0 < 0 || z0 < 0 || y1 > f->R || z1 > f->R || y0 >= y1 || z0 >= z1) return EMB_ERR_BAD_INPUT;
    const int Lf = f->max_level;
    if (f->top != Lf || w->top != Lf) return EMB_ERR_STATE;
    for (int L = 0; L <= Lf; ++L)
        if (!f->lv[L].mask_valid || !w->lv[L].mask_valid) return EMB_ERR_STATE;
    if ((f_n > 0 && (!f_cell || !f_dir || !f_q || !f_tri)) || (w_n > 0 && (!w_cell || !w_dir || !w_q || !w_tri)))
        return EMB_ERR_BAD_INPUT;
    cudaStream_t s = emb_stream(stream);
    const RowWindow W = {y0, y1, z0, z1};
    emb_status rc = EMB_OK;
    for (int L = 0; L <= Lf && rc == EMB_OK; ++L) {
        EmbLevel &P = f->lv[L];
        const EmbLevel &Q = w->lv[L];
        const int64_t np = P.n, nq = Q.n, nmax = np > nq ? np : nq;
        uint32_t *selP = nullptr, *posP = nullptr, *selQ = nullptr, *posQ = nullptr;
        uint64_t *tmp = nullptr, *cP = nullptr, *cQ = nullptr;
        EMB_CUDA_TRY(emb_malloc_async(&selP, (np + 1) * sizeof(uint32_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&posP, (np + 1) * sizeof(uint32_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&selQ, (nq + 1) * sizeof(uint32_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&posQ, (nq + 1) * sizeof(uint32_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&tmp, emb_scan_tmp_words(nmax) * sizeof(uint64_t), s));
        if (np > 0) EMB_LAUNCH((k_sp_select), emb_grid(np, 256), 256, 0, s)(P.key, np, W, L, 0, selP);
        if (nq > 0) EMB_LAUNCH((k_sp_select), emb_grid(nq, 256), 256, 0, s)(Q.key, nq, W, L, 1, selQ);
        EMB_CUDA_TRY(cudaGetLastError());
        rc = emb_scan_into(selP, posP, np, tmp, s);
        if (rc == EMB_OK) rc = emb_scan_into(selQ, posQ, nq, tmp, s);
        if (rc != EMB_OK) return rc;
        uint32_t kk[2] = {0, 0};
        EMB_CUDA_TRY(cudaMemcpyAsync(&kk[0], posP + np, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        EMB_CUDA_TRY(cudaMemcpyAsync(&kk[1], posQ + nq, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        EMB_CUDA_TRY(cudaStreamSynchronize(s));
        const int64_t kp = kk[0], kq = kk[1], n = kp + kq;
        EMB_CUDA_TRY(emb_malloc_async(&cP, (kp + 1) * sizeof(uint64_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&cQ, (kq + 1) * sizeof(uint64_t), s));
        if (np > 0) EMB_LAUNCH((k_sp_compact_keys), emb_grid(np, 256), 256, 0, s)(P.key, selP, posP, np, cP);
        if (nq > 0) EMB_LAUNCH((k_sp_compact_keys), emb_grid(nq, 256), 256, 0, s)(Q.key, selQ, posQ, nq, cQ);
        uint64_t *mkey = nullptr, *mmask = nullptr;
        int32_t *idP = nullptr, *idQ = nullptr;
        EMB_CUDA_TRY(emb_malloc_async(&mkey, (n + 1) * sizeof(uint64_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&mmask, (n + 1) * sizeof(uint64_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&idP, (np + 1) * sizeof(int32_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&idQ, (nq + 1) * sizeof(int32_t), s));
        if (np > 0)
            EMB_LAUNCH((k_sp_place), emb_grid(np, 256), 256, 0, s)(P.key, P.mask, selP, posP, np, cQ, kq, mkey, mmask, idP);
        if (nq > 0)
            EMB_LAUNCH((k_sp_place), emb_grid(nq, 256), 256, 0, s)(Q.key, Q.mask, selQ, posQ, nq, cP, kp, mkey, mmask, idQ);
        EMB_CUDA_TRY(cudaGetLastError());
        if (L == Lf) {
            // the link tables: per merged block the links of the side it came from
            uint32_t *stP = nullptr, *stQ = nullptr, *cnt = nullptr, *moff = nullptr;
            EMB_CUDA_TRY(emb_malloc_async(&stP, (np + 1) * sizeof(uint32_t), s));
            EMB_CUDA_TRY(emb_malloc_async(&stQ, (nq + 1) * sizeof(uint32_t), s));
            EMB_CUDA_TRY(emb_malloc_async(&cnt, (n + 1) * sizeof(uint32_t), s));
            EMB_CUDA_TRY(emb_malloc_async(&moff, (n + 1) * sizeof(uint32_t), s));
            EMB_CUDA_TRY(cudaMemsetAsync(cnt, 0, (n + 1) * sizeof(uint32_t), s));
            EMB_LAUNCH((k_sp_link_starts), emb_grid(np + 1, 256), 256, 0, s)(f_cell, f_n, np, stP);
            EMB_LAUNCH((k_sp_link_starts), emb_grid(nq + 1, 256), 256, 0, s)(w_cell, w_n, nq, stQ);
            if (np > 0) EMB_LAUNCH((k_sp_link_counts), emb_grid(np, 256), 256, 0, s)(idP, np, stP, cnt);
            if (nq > 0) EMB_LAUNCH((k_sp_link_counts), emb_grid(nq, 256), 256, 0, s)(idQ, nq, stQ, cnt);
            EMB_CUDA_TRY(cudaGetLastError());
            uint64_t *tmp2 = nullptr;
            EMB_CUDA_TRY(emb_malloc_async(&tmp2, emb_scan_tmp_words(n) * sizeof(uint64_t), s));
            rc = emb_scan_into(cnt, moff, n, tmp2, s);
            if (rc != EMB_OK) return rc;
            uint32_t total = 0;
            EMB_CUDA_TRY(cudaMemcpyAsync(&total, moff + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            EMB_CUDA_TRY(cudaStreamSynchronize(s));
            *h_count = (int64_t)total;
            if ((int64_t)total > capacity) {
                rc = EMB_ERR_CAPACITY;
            } else if (total > 0) {
                if (!o_cell || !o_dir || !o_q || !o_tri) return EMB_ERR_BAD_INPUT;
                if (f_n > 0)
                    EMB_LAUNCH((k_sp_link_copy), emb_grid(f_n, 256), 256, 0, s)(f_cell, f_dir, f_q, f_tri, f_n, idP, stP,
                                                                               moff, nullptr, capacity, o_cell, o_dir,
                                                                               o_q, o_tri);
                if (w_n > 0)
                    EMB_LAUNCH((k_sp_link_copy), emb_grid(w_n, 256), 256, 0, s)(w_cell, w_dir, w_q, w_tri, w_n, idQ, stQ,
                                                                               moff, w_tri_map, capacity, o_cell, o_dir,
                                                                               o_q, o_tri);
                EMB_CUDA_TRY(cudaGetLastError());
            }
            cudaFreeAsync(stP, s);
            cudaFreeAsync(stQ, s);
            cudaFreeAsync(cnt, s);
            cudaFreeAsync(moff, s);
            cudaFreeAsync(tmp2, s);
        }
        // the merged level replaces f's level (its index rebuilt, its neighbour table dropped)
        if (rc == EMB_OK) {
            if (P.key) cudaFreeAsync(P.key, s);
            if (P.mask) cudaFreeAsync(P.mask, s);
            if (P.nbr) cudaFreeAsync(P.nbr, s);
            P.key = mkey;
            P.mask = mmask;
            P.nbr = nullptr;
            P.n = n;
            P.mask_valid = 1;
            rc = emb_build_hash(P, s);
        } else {
            cudaFreeAsync(mkey, s);
            cudaFreeAsync(mmask, s);
        }
        void *bufs[] = {selP, posP, selQ, posQ, tmp, cP, cQ, idP, idQ};
        for (void *p : bufs)
            if (p) cudaFreeAsync(p, s);
    }
    // cached link candidates belong to the old finest level
    if (f->cand) cudaFreeAsync(f->cand, s);
    if (f->blk_off) cudaFreeAsync(f->blk_off, s);
    if (f->work) cudaFreeAsync(f->work, s);
    if (f->work_n) cudaFreeAsync(f->work_n, s);
    f->cand = nullptr;
    f->blk_off = nullptr;
    f->work = nullptr;
    f->work_n = nullptr;
    f->n_links = -1;
    EMB_CUDA_TRY(cudaGetLastError());
    return rc;
}

// ---------------------------------------------------------------------------
// triangles near a window
// ---------------------------------------------------------------------------
__global__ void k_sub_flag(const int4 *__restrict__ rec, int64_t T, long long ylo, long long yhi, long long zlo,
                           long long zhi, uint32_t *__restrict__ flag)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int4 A = rec[3 * t], B = rec[3 * t + 1], C = rec[3 * t + 2];
    const long long y0 = min(A.y, min(B.y, C.y)), y1 = max(A.y, max(B.y, C.y));
    const long long z0 = min(A.z, min(B.z, C.z)), z1 = max(A.z, max(B.z, C.z));
    flag[t] = (y1 >= ylo && y0 <= yhi && z1 >= zlo && z0 <= zhi) ? 1u : 0u;
}

__global__ void k_sub_gather(const int4 *__restrict__ rec, const uint32_t *__restrict__ flag,
                             const uint32_t *__restrict__ pos, int64_t T, int4 *__restrict__ out,
                             int32_t *__restrict__ map)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T || !flag[t]) return;
    const int64_t p = pos[t];
    out[3 * p] = rec[3 * t];
    out[3 * p + 1] = rec[3 * t + 1];
    out[3 * p + 2] = rec[3 * t + 2];
    if (map) map[p] = (int32_t)t;
}

extern "C" emb_status emb_mesh_subset(emb_mesh m, int64_t ylo, int64_t yhi, int64_t zlo, int64_t zhi, int32_t *d_map,
                                      int64_t map_capacity, void *stream, emb_mesh *out, int64_t *h_count)
{
    if (!m || !out || !h_count || map_capacity < 0) return EMB_ERR_BAD_INPUT;
    *out = nullptr;
    cudaStream_t s = emb_stream(stream);
    const int64_t T = m->T;
    uint32_t *flag = nullptr, *pos = nullptr;
    uint64_t *tmp = nullptr;
    EMB_CUDA_TRY(emb_malloc_async(&flag, (T + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&pos, (T + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&tmp, emb_scan_tmp_words(T) * sizeof(uint64_t), s));
    EMB_LAUNCH((k_sub_flag), emb_grid(T, 256), 256, 0, s)(m->rec, T, ylo, yhi, zlo, zhi, flag);
    EMB_CUDA_TRY(cudaGetLastError());
    emb_status rc = emb_scan_into(flag, pos, T, tmp, s);
    if (rc != EMB_OK) return rc;
    uint32_t n = 0;
    EMB_CUDA_TRY(cudaMemcpyAsync(&n, pos + T, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    EMB_CUDA_TRY(cudaStreamSynchronize(s));
    *h_count = n;
    if (d_map && (int64_t)n > map_capacity) rc = EMB_ERR_CAPACITY;
    emb_mesh sm = nullptr;
    if (rc == EMB_OK && n > 0) {
        sm = (emb_mesh)calloc(1, sizeof(emb_mesh_s));
        if (!sm) return EMB_ERR_CUDA;
        *sm = *m;
        sm->T = n;
        sm->rec = nullptr;
        if (emb_malloc_async(&sm->rec, (size_t)n * 3 * sizeof(int4), s) != cudaSuccess) {
            free(sm);
            return EMB_ERR_CUDA;
        }
        EMB_LAUNCH((k_sub_gather), emb_grid(T, 256), 256, 0, s)(m->rec, flag, pos, T, sm->rec, d_map);
        EMB_CUDA_TRY(cudaGetLastError());
    }
    cudaFreeAsync(flag, s);
    cudaFreeAsync(pos, s);
    cudaFreeAsync(tmp, s);
    if (rc == EMB_OK && n == 0) rc = EMB_ERR_STATE;  // no triangle near the window
    if (rc != EMB_OK) {
        if (sm) emb_mesh_destroy(sm);
        return rc;
    }
    *out = sm;
    return EMB_OK;
}
