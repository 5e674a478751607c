// Momentum-exchange force with linear Bouzidi interpolated bounce-back, its
// derivative with respect to q, and the adjoint of q with respect to the
// vertices (Sec. 2.2 cites both methods; Sec. 3.4 builds the q table they use).
//
// All reductions have a fixed order: per-CTA trees in FP64 followed by one CTA
// summing the partials in index order, and per-vertex sums taken in ascending
// (link, corner) order.  No floating-point atomics are used.
#include <mutex>

#include "emb_internal.cuh"

#define MEX_BLOCK 256

// direction index of a block offset (ox, oy, oz) in {-1,0,1}^3, code = (ox+1) + 3(oy+1) + 9(oz+1)
__constant__ int8_t c_dir_of_offset[27] = {20, 16, 26, 12, 6, 13, 24, 17, 21, 8, 4, 9, 2, 0,
                                           1,  10, 3,  7,  22, 18, 23, 14, 5, 11, 25, 15, 19};

// Finest-level cell x_f - c_i, or -1 if its block is missing or the cell is solid.
__device__ __forceinline__ int64_t partner_cell(int64_t cell, int cx, int cy, int cz, const int32_t *__restrict__ nbr,
                                                const uint64_t *__restrict__ mask)
{
    int64_t b = cell >> 6;
    int t = (int)(cell & 63);
    int x = (t & 3) - cx, y = ((t >> 2) & 3) - cy, z = (t >> 4) - cz;
    int ox = x < 0 ? -1 : (x > 3 ? 1 : 0), oy = y < 0 ? -1 : (y > 3 ? 1 : 0), oz = z < 0 ? -1 : (z > 3 ? 1 : 0);
    int64_t nb = b;
    if (ox | oy | oz) {
        int d = c_dir_of_offset[(ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)];
        nb = nbr[b * 26 + d - 1];
        if (nb < 0) return -1;
    }
    int lt = (x & 3) + 4 * (y & 3) + 16 * (z & 3);
    if ((mask[nb] >> lt) & 1ull) return -1;
    return nb * 64 + lt;
}

struct LinkTerm {
    double f_i, f_o, f_p;
    bool has;
    int cx, cy, cz;
};

__device__ __forceinline__ LinkTerm link_term(int64_t k, const int32_t *__restrict__ cell, const uint8_t *__restrict__ dir,
                                              const float *__restrict__ pop, int64_t stride,
                                              const int32_t *__restrict__ nbr, const uint64_t *__restrict__ mask)
{
    LinkTerm L;
    int64_t c = cell[k];
    int d = dir[k];
    int o = (d & 1) ? d + 1 : d - 1;
    emb_dir(d, L.cx, L.cy, L.cz);
    L.f_i = pop[(int64_t)d * stride + c];
    L.f_o = pop[(int64_t)o * stride + c];
    int64_t p = partner_cell(c, L.cx, L.cy, L.cz, nbr, mask);
    L.has = p >= 0;
    L.f_p = L.has ? (double)pop[(int64_t)d * stride + p] : 0.0;
    return L;
}

// Fixed-order block reduction of three doubles; thread 0 receives the sums.
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c)
{
    __shared__ double s[3][MEX_BLOCK];
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    s[2][threadIdx.x] = c;
    __syncthreads();
    for (int w = MEX_BLOCK / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
            s[2][threadIdx.x] += s[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    a = s[0][0];
    b = s[1][0];
    c = s[2][0];
}

__global__ void __launch_bounds__(MEX_BLOCK) k_mex_partial(const int32_t *__restrict__ cell, const uint8_t *__restrict__ dir,
                                                           const float *__restrict__ q, int64_t n,
                                                           const float *__restrict__ pop, int64_t stride,
                                                           const int32_t *__restrict__ nbr,
                                                           const uint64_t *__restrict__ mask, double *__restrict__ part)
{
    double fx = 0, fy = 0, fz = 0;
    for (int64_t k = (int64_t)blockIdx.x * MEX_BLOCK + threadIdx.x; k < n; k += (int64_t)gridDim.x * MEX_BLOCK) {
        LinkTerm L = link_term(k, cell, dir, pop, stride, nbr, mask);
        double qq = q[k], g;
        if (qq < 0.5) g = L.has ? 2.0 * qq * L.f_i + (1.0 - 2.0 * qq) * L.f_p : L.f_i;
        else g = L.f_i / (2.0 * qq) + (2.0 * qq - 1.0) / (2.0 * qq) * L.f_o;
        double m = L.f_i + g;
        fx += L.cx * m;
        fy += L.cy * m;
        fz += L.cz * m;
    }
    block_sum3(fx, fy, fz);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = fx;
        part[3 * blockIdx.x + 1] = fy;
        part[3 * blockIdx.x + 2] = fz;
    }
}

__global__ void __launch_bounds__(MEX_BLOCK) k_mex_final(const double *__restrict__ part, int nparts, float *__restrict__ F)
{
    double a = 0, b = 0, c = 0;
    for (int i = threadIdx.x; i < nparts; i += MEX_BLOCK) {
        a += part[3 * i];
        b += part[3 * i + 1];
        c += part[3 * i + 2];
    }
    block_sum3(a, b, c);
    if (threadIdx.x == 0) {
        F[0] = (float)a;
        F[1] = (float)b;
        F[2] = (float)c;
    }
}

__global__ void k_mex_bwd(const int32_t *__restrict__ cell, const uint8_t *__restrict__ dir, const float *__restrict__ q,
                          int64_t n, const float *__restrict__ pop, int64_t stride, const int32_t *__restrict__ nbr,
                          const uint64_t *__restrict__ mask, const float *__restrict__ gF, float *__restrict__ gq)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    LinkTerm L = link_term(k, cell, dir, pop, stride, nbr, mask);
    double qq = q[k], g;
    if (qq < 0.5) g = L.has ? 2.0 * (L.f_i - L.f_p) : 0.0;
    else g = (L.f_o - L.f_i) / (2.0 * qq * qq);
    double s = (double)gF[0] * L.cx + (double)gF[1] * L.cy + (double)gF[2] * L.cz;
    gq[k] = (float)(s * g);
}

static emb_status mex_check(emb_forest f, int lattice, int64_t n, int64_t stride, cudaStream_t s)
{
    if (!f || (lattice != 19 && lattice != 27) || n < 0) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    int L = f->max_level;
    if (f->top != L || !f->lv[L].mask_valid) return EMB_ERR_STATE;
    if (stride < f->lv[L].n * 64) return EMB_ERR_BAD_INPUT;
    return emb_build_neighbors(f->lv[L], s);
}

extern "C" emb_status emb_mex_force(emb_forest f, int32_t lattice, const int32_t *d_cell, const uint8_t *d_dir,
                                    const float *d_q, int64_t n, const float *d_pop, int64_t pop_stride, float *d_F,
                                    void *stream)
{
    cudaStream_t s = emb_stream(stream);
    emb_status rc = mex_check(f, lattice, n, pop_stride, s);
    if (rc != EMB_OK) return rc;
    if (!d_F || (n > 0 && (!d_cell || !d_dir || !d_q || !d_pop))) return EMB_ERR_BAD_INPUT;
    const EmbLevel &lv = f->lv[f->max_level];
    int64_t np64 = (n + MEX_BLOCK - 1) / MEX_BLOCK;
    int nparts = (int)(np64 < 1184 ? np64 : 1184);
    if (nparts < 1) nparts = 1;
    double *part = nullptr;
    EMB_CUDA_TRY(emb_malloc_async(&part, 3 * nparts * sizeof(double), s));
    EMB_LAUNCH((k_mex_partial), nparts, MEX_BLOCK, 0, s)(d_cell, d_dir, d_q, n, d_pop, pop_stride, lv.nbr, lv.mask, part);
    EMB_LAUNCH((k_mex_final), 1, MEX_BLOCK, 0, s)(part, nparts, d_F);
    EMB_CUDA_TRY(cudaGetLastError());
    EMB_CUDA_TRY(cudaFreeAsync(part, s));
    return EMB_OK;
}

extern "C" emb_status emb_mex_force_backward(emb_forest f, int32_t lattice, const int32_t *d_cell, const uint8_t *d_dir,
                                             const float *d_q, int64_t n, const float *d_pop, int64_t pop_stride,
                                             const float *d_gF, float *d_gq, void *stream)
{
    cudaStream_t s = emb_stream(stream);
    emb_status rc = mex_check(f, lattice, n, pop_stride, s);
    if (rc != EMB_OK) return rc;
    if (n == 0) return EMB_OK;
    if (!d_cell || !d_dir || !d_q || !d_pop || !d_gF || !d_gq) return EMB_ERR_BAD_INPUT;
    const EmbLevel &lv = f->lv[f->max_level];
    EMB_LAUNCH((k_mex_bwd), emb_grid(n, 256), 256, 0, s)(d_cell, d_dir, d_q, n, d_pop, pop_stride, lv.nbr, lv.mask, d_gF, d_gq);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of emb_mex_force
// ---------------------------------------------------------------------------
// Some callers cannot call cudaMalloc: a solver time loop that reserved all
// device memory up front through its own pool, or code that must not pay a
// driver allocation (latency, implicit device synchronisation) inside a time
// step.  For them the per-CTA partial sums of the force live in this
// file-scope array instead of a stream-ordered allocation.  Every GPU that loads
// the library holds it (3 x EMB_NOALLOC_MEX_PARTS doubles = 192 KB) until exit.
#define EMB_NOALLOC_MEX_PARTS 8192
static __device__ __align__(256) double g_mex_noalloc_part[3 * EMB_NOALLOC_MEX_PARTS];

static std::mutex g_mex_noalloc_mu;
static double *g_mex_noalloc_ptr[64] = {nullptr};        // device address of the array, per device
static unsigned long long g_mex_noalloc_ctx[64] = {0};   // id of the context it was looked up in

// Unique id of the calling thread's current context (0 when none is current or the
// driver entry points are unavailable).  Context ids are never reused within a
// process, so a reset device (a new primary context) is told apart from the old one.
typedef int (*emb_pfn_ctx_get_current)(void **);
typedef int (*emb_pfn_ctx_get_id)(void *, unsigned long long *);
static unsigned long long current_ctx_id()
{
    static emb_pfn_ctx_get_current get_cur = nullptr;
    static emb_pfn_ctx_get_id get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_cur = (emb_pfn_ctx_get_current)a;
            get_id = (emb_pfn_ctx_get_id)b;
        }
    }
    if (!get_cur || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&ctx) != 0 || !ctx) return 0;
    if (get_id(ctx, &id) != 0) return 0;
    return id;
}

// The array's device address for the current device, looked up once per device
// (and again if that device's context was replaced, e.g. by cudaDeviceReset).  In
// host code the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress with the device current.
static emb_status mex_noalloc_scratch(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return EMB_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mex_noalloc_mu);
    const unsigned long long ctx = current_ctx_id();
    if (!g_mex_noalloc_ptr[dev] || ctx == 0 || ctx != g_mex_noalloc_ctx[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_mex_noalloc_part);
        if (e != cudaSuccess || !p) {
            emb_note_cuda_error(e, "cudaGetSymbolAddress(g_mex_noalloc_part)", __FILE__, __LINE__);
            return EMB_ERR_CUDA;
        }
        g_mex_noalloc_ptr[dev] = (double *)p;
        // the lookup made the device's primary context current if it was not yet
        g_mex_noalloc_ctx[dev] = ctx ? ctx : current_ctx_id();
    }
    *out = g_mex_noalloc_ptr[dev];
    return EMB_OK;
}

extern "C" emb_status emb_mex_force_noalloc(emb_forest f, int32_t lattice, const int32_t *d_cell, const uint8_t *d_dir,
                                            const float *d_q, int64_t n, const float *d_pop, int64_t pop_stride,
                                            float *d_F, void *stream)
{
    if (!f || (lattice != 19 && lattice != 27) || n < 0 || !d_F) return EMB_ERR_BAD_INPUT;
    if (n > 0 && (!d_cell || !d_dir || !d_q || !d_pop)) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    const int L = f->max_level;
    if (f->top != L || !f->lv[L].mask_valid) return EMB_ERR_STATE;
    const EmbLevel &lv = f->lv[L];
    if (pop_stride < lv.n * 64) return EMB_ERR_BAD_INPUT;
    // the neighbour table must already exist (emb_cutlinks or emb_mex_force built it): building it would allocate
    if (lv.n > 0 && !lv.nbr) return EMB_ERR_STATE;
    // one partial sum per CTA of MEX_BLOCK links
    const int64_t nparts64 = n > 0 ? (n + MEX_BLOCK - 1) / MEX_BLOCK : 1;
    if (nparts64 > EMB_NOALLOC_MEX_PARTS) return EMB_ERR_CAPACITY;  // more than 2,097,152 links
    double *part = nullptr;
    emb_status rc = mex_noalloc_scratch(&part);
    if (rc != EMB_OK) return rc;
    cudaStream_t s = emb_stream(stream);
    const int nparts = (int)nparts64;
    EMB_LAUNCH((k_mex_partial), nparts, MEX_BLOCK, 0, s)(d_cell, d_dir, d_q, n, d_pop, pop_stride, lv.nbr, lv.mask, part);
    EMB_LAUNCH((k_mex_final), 1, MEX_BLOCK, 0, s)(part, nparts, d_F);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

// ---------------------------------------------------------------------------
// dq/dV adjoint
// ---------------------------------------------------------------------------
// Per link k and corner j of its triangle: gq_k lambda_j n / (h n.c), world units.
__global__ void k_qbwd_terms(const uint64_t *__restrict__ key, LevelGeom g, double scale, const int32_t *__restrict__ cell,
                             const uint8_t *__restrict__ dir, const float *__restrict__ q, const int32_t *__restrict__ tri,
                             const float *__restrict__ gq, int64_t n, const int4 *__restrict__ rec, int64_t T,
                             float *__restrict__ val, int32_t *__restrict__ vid, uint32_t *__restrict__ vcnt, int *st)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t tr = tri[k];
    if (tr < 0 || tr >= T) {
        emb_set_status(st, EMB_ERR_BAD_INPUT);
        for (int j = 0; j < 3; ++j) vid[3 * k + j] = -1;
        return;
    }
    int4 A = rec[3 * tr], B = rec[3 * tr + 1], C = rec[3 * tr + 2];
    int64_t c = cell[k];
    uint64_t bk = key[c >> 6];
    int t = (int)(c & 63);
    long long gx = 4 * (long long)(bk & EMB_KEY_MASK) + (t & 3);
    long long gy = 4 * (long long)((bk >> EMB_KEY_BITS) & EMB_KEY_MASK) + ((t >> 2) & 3);
    long long gz = 4 * (long long)(bk >> (2 * EMB_KEY_BITS)) + (t >> 4);
    int cx, cy, cz;
    emb_dir(dir[k], cx, cy, cz);
    // coordinates relative to A (exact integers in double)
    double bx = (double)B.x - A.x, by = (double)B.y - A.y, bz = (double)B.z - A.z;
    double qx = (double)C.x - A.x, qy = (double)C.y - A.y, qz = (double)C.z - A.z;
    double s_ = (double)q[k] * (double)g.h;
    double xx = (double)((2 * gx + 1) * g.half - A.x) + s_ * cx;
    double xy = (double)((2 * gy + 1) * g.half - A.y) + s_ * cy;
    double xz = (double)((2 * gz + 1) * g.half - A.z) + s_ * cz;
    double nx = by * qz - bz * qy, ny = bz * qx - bx * qz, nz = bx * qy - by * qx;
    double nn = nx * nx + ny * ny + nz * nz;
    double nc = nx * cx + ny * cy + nz * cz;
    // X = lB B' + lC C':  X x C' = lB n,  B' x X = lC n
    double lB = (nx * (xy * qz - xz * qy) + ny * (xz * qx - xx * qz) + nz * (xx * qy - xy * qx)) / nn;
    double lC = (nx * (by * xz - bz * xy) + ny * (bz * xx - bx * xz) + nz * (bx * xy - by * xx)) / nn;
    double lA = 1.0 - lB - lC;
    double f = (double)gq[k] * scale / ((double)g.h * nc);
    double lam[3] = {lA, lB, lC};
    int ids[3] = {A.w, B.w, C.w};
    for (int j = 0; j < 3; ++j) {
        double w = f * lam[j];
        val[3 * (3 * k + j) + 0] = (float)(w * nx);
        val[3 * (3 * k + j) + 1] = (float)(w * ny);
        val[3 * (3 * k + j) + 2] = (float)(w * nz);
        vid[3 * k + j] = ids[j];
        atomicAdd(vcnt + ids[j], 1u);
    }
}

__global__ void k_qbwd_fill(const int32_t *__restrict__ vid, int64_t m, const uint32_t *__restrict__ voff,
                            uint32_t *__restrict__ cur, uint32_t *__restrict__ slot)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    int32_t v = vid[e];
    if (v < 0) return;
    uint32_t p = atomicAdd(cur + v, 1u);
    slot[voff[v] + p] = (uint32_t)e;
}

// One warp per vertex.  The fill left a vertex's entries unordered in slot[a, b);
// each lane ranks its entries among all of them (entry ids are distinct) and
// stores them at their rank in `sorted`, so sorted[a, b) ascends.  After a warp
// barrier lane l sums the entries of ranks l, l + 32, l + 64, ... in that order
// and the 32 lane sums meet in a fixed butterfly: the result does not depend on
// the order the atomics of the fill happened to take.  Work per vertex is
// c^2 / 32 comparisons per lane for c entries.
__global__ void k_qbwd_reduce(const uint32_t *__restrict__ voff, const uint32_t *__restrict__ slot,
                              uint32_t *__restrict__ sorted, const float *__restrict__ val, int64_t V,
                              float *__restrict__ gv)
{
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= V) return;  // uniform per warp
    const uint32_t a = voff[v], b = voff[v + 1];
    for (uint32_t i = a + lane; i < b; i += 32) {
        const uint32_t e = slot[i];
        uint32_t r = 0;
        for (uint32_t j = a; j < b; ++j) r += slot[j] < e;
        sorted[a + r] = e;
    }
    __syncwarp();
    double sx = 0, sy = 0, sz = 0;
    for (uint32_t i = a + lane; i < b; i += 32) {
        const int64_t e = sorted[i];
        sx += val[3 * e];
        sy += val[3 * e + 1];
        sz += val[3 * e + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    if (lane == 0) {
        gv[3 * v] = (float)sx;
        gv[3 * v + 1] = (float)sy;
        gv[3 * v + 2] = (float)sz;
    }
}

extern "C" emb_status emb_cutlinks_backward(emb_mesh m, emb_forest f, const int32_t *d_cell, const uint8_t *d_dir,
                                            const float *d_q, const int32_t *d_tri, int64_t n, const float *d_gq,
                                            float *d_gverts, void *stream)
{
    if (!m || !f || n < 0 || !d_gverts) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    if (m->R != f->R || f->top != f->max_level) return EMB_ERR_STATE;
    if (n > 0 && (!d_cell || !d_dir || !d_q || !d_tri || !d_gq)) return EMB_ERR_BAD_INPUT;
    if (3 * n >= (1ll << 32)) return EMB_ERR_CAPACITY;
    cudaStream_t s = emb_stream(stream);
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    const EmbLevel &lv = f->lv[f->max_level];
    LevelGeom g = level_geom(f, f->max_level);
    double scale = (double)(1ll << 20) * (double)f->r_o;
    // one scratch allocation: val (9n floats), vid (3n), slot (3n), vcnt and voff (V + 1 each), scan scratch
    const size_t a_val = (size_t)(9 * n + 1) * sizeof(float), a_ent = (size_t)(3 * n + 1) * sizeof(uint32_t),
                 a_v = (size_t)(m->V + 1) * sizeof(uint32_t), a_tmp = emb_scan_tmp_words(m->V) * sizeof(uint64_t);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char *scratch = nullptr;
    EMB_CUDA_TRY(emb_malloc_async((void **)&scratch, up(a_val) + 2 * up(a_ent) + 2 * up(a_v) + up(a_tmp), s));
    float *val = (float *)scratch;
    int32_t *vid = (int32_t *)(scratch + up(a_val));
    uint32_t *slot = (uint32_t *)(scratch + up(a_val) + up(a_ent));
    uint32_t *vcnt = (uint32_t *)(scratch + up(a_val) + 2 * up(a_ent));
    uint32_t *voff = (uint32_t *)(scratch + up(a_val) + 2 * up(a_ent) + up(a_v));
    uint64_t *tmp = (uint64_t *)(scratch + up(a_val) + 2 * up(a_ent) + 2 * up(a_v));
    EMB_CUDA_TRY(cudaMemsetAsync(vcnt, 0, (m->V + 1) * sizeof(uint32_t), s));
    if (n > 0)
        EMB_LAUNCH((k_qbwd_terms), emb_grid(n, 256), 256, 0, s)(lv.key, g, scale, d_cell, d_dir, d_q, d_tri, d_gq, n, m->rec, m->T,
                                                      val, vid, vcnt, st);
    emb_status rc = emb_scan_into(vcnt, voff, m->V, tmp, s);
    if (rc != EMB_OK) {
        cudaFreeAsync(scratch, s);
        return rc;
    }
    EMB_CUDA_TRY(cudaMemsetAsync(vcnt, 0, (m->V + 1) * sizeof(uint32_t), s));
    if (n > 0) EMB_LAUNCH((k_qbwd_fill), emb_grid(3 * n, 256), 256, 0, s)(vid, 3 * n, voff, vcnt, slot);
    // vid is spent after the fill and holds the sorted entries of each vertex
    EMB_LAUNCH((k_qbwd_reduce), emb_grid(32 * m->V, 256), 256, 0, s)(voff, slot, (uint32_t *)vid, val, m->V, d_gverts);
    EMB_CUDA_TRY(cudaGetLastError());
    EMB_CUDA_TRY(cudaFreeAsync(scratch, s));
    return EMB_OK;
}
