// The paper's guard-cell voxelizer (Sec. 3.4, "Partial Surface Voxelization" with
// Alg. 3, and "External Cell Flag Propagation"), built on the finest level of a
// forest as an ablation of the exact parity voxelizer (emb_voxelize).
//
//   k_guard_surface  one warp per block (grid-stride).  The block's bin is staged 32
//                    faces at a time into shared memory, each with its unit normal
//                    computed once; every lane classifies two cells by the nearest
//                    face its x-line meets.  Arithmetic is binary32 with one rounding
//                    per operation in a fixed order (the _rn intrinsics are never
//                    fused into multiply-adds), so the result is reproducible.  The
//                    cells' states go to two words per block (solid, guard), and the
//                    internal propagation runs on those words with shifts inside the
//                    4-bit rows.
//   k_guard_sweep    one thread per run of consecutive blocks along x (the thread of
//                    the run's first block in the sweep's direction) walks the run;
//                    the 16 row statuses are bits of one word, so a block costs a few
//                    word operations.
//
// Equal distances go to the lowest face id, the order in which the paper's sorted
// bins present the faces; the CUDA bins are unordered, so the rule is applied
// explicitly.  The point-in-face test is the paper's triangle / thin-box overlap with
// the box spanning the domain along x: only the axes of the y-z projection can
// separate (y, z and the three edge normals), with half-width 2^-23 (binary32 epsilon).
#include "emb_internal.cuh"

#define GUARD_WARPS 4
#define GUARD_EPS 1.1920928955078125e-7f  // 2^-23
#define GUARD_X0 0x1111111111111111ull    // cell x = 0 of every row
#define GUARD_X3 0x8888888888888888ull    // cell x = 3 of every row

struct GuardFace {
    float ax, ay, az;     // first vertex
    float by, bz, cy, cz; // y-z of the other two
    float nx, ny, nz;     // unit normal
    uint32_t id;
    int valid;
};

// Mesh record coordinate X = m r_o (m = v 2^20, an integer below 2^20) back to the
// binary32 vertex coordinate v = m 2^-20, exactly.
__device__ __forceinline__ float guard_coord(int X, int r_o)
{
    return __fmul_rn((float)(X / r_o), 9.5367431640625e-07f);
}

__device__ __forceinline__ void guard_face_setup(const int4 *__restrict__ rec, uint32_t id, int r_o, GuardFace &F)
{
    const int4 A = rec[3 * (int64_t)id], B = rec[3 * (int64_t)id + 1], C = rec[3 * (int64_t)id + 2];
    const float a0 = guard_coord(A.x, r_o), a1 = guard_coord(A.y, r_o), a2 = guard_coord(A.z, r_o);
    const float b0 = guard_coord(B.x, r_o), b1 = guard_coord(B.y, r_o), b2 = guard_coord(B.z, r_o);
    const float c0 = guard_coord(C.x, r_o), c1 = guard_coord(C.y, r_o), c2 = guard_coord(C.z, r_o);
    const float u0 = __fsub_rn(b0, a0), u1 = __fsub_rn(b1, a1), u2 = __fsub_rn(b2, a2);
    const float w0 = __fsub_rn(c0, a0), w1 = __fsub_rn(c1, a1), w2 = __fsub_rn(c2, a2);
    float n0 = __fsub_rn(__fmul_rn(u1, w2), __fmul_rn(u2, w1));
    float n1 = __fsub_rn(__fmul_rn(u2, w0), __fmul_rn(u0, w2));
    float n2 = __fsub_rn(__fmul_rn(u0, w1), __fmul_rn(u1, w0));
    const float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(n0, n0), __fmul_rn(n1, n1)), __fmul_rn(n2, n2)));
    F.nx = __fdiv_rn(n0, len);
    F.ny = __fdiv_rn(n1, len);
    F.nz = __fdiv_rn(n2, len);
    F.ax = a0;
    F.ay = a1;
    F.az = a2;
    F.by = b1;
    F.bz = b2;
    F.cy = c1;
    F.cz = c2;
    F.id = id;
    F.valid = 1;
}

// Separation of the y-z projection (coordinates relative to the line) by the normal
// of the edge i -> k.
__device__ __forceinline__ bool guard_edge_separates(const float y[3], const float z[3], int i, int k)
{
    const float ey = __fsub_rn(y[k], y[i]), ez = __fsub_rn(z[k], z[i]);
    const float r = __fmul_rn(GUARD_EPS, __fadd_rn(fabsf(ey), fabsf(ez)));
    float lo = 0.0f, hi = 0.0f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float p = __fsub_rn(__fmul_rn(z[m], ey), __fmul_rn(y[m], ez));
        if (m == 0 || p < lo) lo = p;
        if (m == 0 || p > hi) hi = p;
    }
    return lo > r || hi < -r;
}

__device__ __forceinline__ bool guard_in_face(const GuardFace &F, float py, float pz)
{
    const float y[3] = {__fsub_rn(F.ay, py), __fsub_rn(F.by, py), __fsub_rn(F.cy, py)};
    const float z[3] = {__fsub_rn(F.az, pz), __fsub_rn(F.bz, pz), __fsub_rn(F.cz, pz)};
    if (fminf(y[0], fminf(y[1], y[2])) > GUARD_EPS || fmaxf(y[0], fmaxf(y[1], y[2])) < -GUARD_EPS) return false;
    if (fminf(z[0], fminf(z[1], z[2])) > GUARD_EPS || fmaxf(z[0], fmaxf(z[1], z[2])) < -GUARD_EPS) return false;
    return !(guard_edge_separates(y, z, 0, 1) || guard_edge_separates(y, z, 1, 2) || guard_edge_separates(y, z, 2, 0));
}

// One cell against one face: the signed distance along x to the face's plane,
// d = ((v1 - c) . n) / n_x, and the nearest-face update (strictly nearer, or as near
// with a lower id).  st: 0 no face, 1 solid (n_x d > 0), 2 guard.
__device__ __forceinline__ void guard_cell(const GuardFace &F, float px, float py, float pz, float &dmin,
                                           uint32_t &pid, int &st)
{
    const float num = __fadd_rn(__fadd_rn(__fmul_rn(__fsub_rn(F.ax, px), F.nx), __fmul_rn(__fsub_rn(F.ay, py), F.ny)),
                                __fmul_rn(__fsub_rn(F.az, pz), F.nz));
    const float d = __fdiv_rn(num, F.nx);
    const float ad = fabsf(d);
    // pid starts at 0 with dmin = 1: the tie clause cannot admit a face at |d| = 1
    if (!(ad < dmin || (ad == dmin && F.id < pid))) return;
    if (!guard_in_face(F, py, pz)) return;
    dmin = ad;
    pid = F.id;
    st = __fmul_rn(F.nx, d) > 0.0f ? 1 : 2;
}

// Internal propagation inside a block: three rounds, each from the previous round's
// words; a fluid cell next to a guard becomes a guard, then a cell that is not a
// guard next to a solid becomes solid.
__device__ __forceinline__ void guard_internal(uint64_t &S, uint64_t &G)
{
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const uint64_t F = ~(S | G);
        const uint64_t nG = ((G << 1) & ~GUARD_X0) | ((G >> 1) & ~GUARD_X3);
        const uint64_t nS = ((S << 1) & ~GUARD_X0) | ((S >> 1) & ~GUARD_X3);
        const uint64_t G2 = G | (F & nG);
        S = S | (~G2 & nS);
        G = G2;
    }
}

__global__ void __launch_bounds__(32 * GUARD_WARPS)
    k_guard_surface(const int4 *__restrict__ rec, uint32_t T, int r_o, const uint32_t *__restrict__ off,
                    const uint32_t *__restrict__ ent, uint64_t ent_cap, const uint64_t *__restrict__ key, int64_t n,
                    int64_t ncell, uint64_t *__restrict__ S_out, uint64_t *__restrict__ G_out, int *st_word)
{
    __shared__ GuardFace sf[GUARD_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * GUARD_WARPS;
    const float den = (float)(2 * ncell);
    for (int64_t b = (int64_t)blockIdx.x * GUARD_WARPS + w; b < n; b += warps) {
        const uint64_t k = key[b];
        const int64_t bx = (int64_t)(k & 0x1FFFFFull), by = (int64_t)((k >> 21) & 0x1FFFFFull), bz = (int64_t)(k >> 42);
        float px[2], py[2], pz[2], dmin[2] = {1.0f, 1.0f};
        uint32_t pid[2] = {0u, 0u};
        int st[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;
            px[h] = __fdiv_rn((float)(2 * (4 * bx + (t & 3)) + 1), den);
            py[h] = __fdiv_rn((float)(2 * (4 * by + ((t >> 2) & 3)) + 1), den);
            pz[h] = __fdiv_rn((float)(2 * (4 * bz + (t >> 4)) + 1), den);
        }
        uint64_t e0 = off[b], e1 = off[b + 1];
        if (e1 > ent_cap) e1 = ent_cap;
        for (uint64_t e = e0; e < e1; e += 32) {
            const int cnt = (int)min((uint64_t)32, e1 - e);
            if (lane < cnt) {
                const uint32_t id = ent[e + lane];
                if (id < T) {
                    guard_face_setup(rec, id, r_o, sf[w][lane]);
                } else {
                    sf[w][lane].valid = 0;
                    emb_set_status(st_word, EMB_ERR_STATE);
                }
            }
            __syncwarp();
            for (int j = 0; j < cnt; ++j) {
                const GuardFace &F = sf[w][j];
                if (!F.valid) continue;
                guard_cell(F, px[0], py[0], pz[0], dmin[0], pid[0], st[0]);
                guard_cell(F, px[1], py[1], pz[1], dmin[1], pid[1], st[1]);
            }
            __syncwarp();
        }
        uint64_t S = (uint64_t)__ballot_sync(0xffffffffu, st[0] == 1) |
                     ((uint64_t)__ballot_sync(0xffffffffu, st[1] == 1) << 32);
        uint64_t G = (uint64_t)__ballot_sync(0xffffffffu, st[0] == 2) |
                     ((uint64_t)__ballot_sync(0xffffffffu, st[1] == 2) << 32);
        guard_internal(S, G);
        if (lane == 0) {
            S_out[b] = S;
            G_out[b] = G;
        }
    }
}

// Coarser levels of the forest, for the status of a hole: the block at a missing
// position of level L is covered by its nearest existing ancestor, which is solid if
// it has a solid cell.
struct GuardHoles {
    EmbLookup lk[EMB_MAX_LEVELS];
    const uint64_t *mask[EMB_MAX_LEVELS];
    int L;
};

__device__ __forceinline__ bool guard_hole_is_solid(const GuardHoles &H, int64_t x, int64_t y, int64_t z)
{
    for (int l = H.L - 1; l >= 0; --l) {
        const int sh = H.L - l;
        const int32_t id = emb_lookup(H.lk[l], x >> sh, y >> sh, z >> sh);
        if (id >= 0) return H.mask[l][id] != 0ull;
    }
    return false;
}

// The sweep along +x (DIR = 1) or -x (DIR = -1).  A run's first block in the sweep
// direction is the one whose predecessor position holds no block of the level; if
// that position lies in the domain and in a solid hole, the run starts from the
// solid: the rows whose status cell (the face ahead) is not a guard turn their
// non-guard cells solid.  Each following block then takes, row by row, solid where
// the status is solid and the cell is not a guard, and hands on its own status.
template <int DIR>
__global__ void k_guard_sweep(const uint64_t *__restrict__ key, int64_t n, uint64_t *__restrict__ S_io,
                              const uint64_t *__restrict__ G_in, GuardHoles H, int64_t nb)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const uint64_t k = key[b];
    if (DIR > 0 ? (b > 0 && key[b - 1] == k - 1) : (b + 1 < n && key[b + 1] == k + 1)) return;
    const int64_t bx = (int64_t)(k & 0x1FFFFFull), by = (int64_t)((k >> 21) & 0x1FFFFFull), bz = (int64_t)(k >> 42);
    const uint64_t face = DIR > 0 ? GUARD_X3 : GUARD_X0;
    const int64_t before = bx - DIR;
    uint64_t S = S_io[b];
    if (before >= 0 && before < nb && guard_hole_is_solid(H, before, by, bz)) {
        const uint64_t G = G_in[b];
        const uint64_t rows = ~G & face;
        const uint64_t fill = (DIR > 0 ? rows >> 3 : rows) * 0xFull;
        const uint64_t S2 = S | (fill & ~G);
        if (S2 != S) {
            S = S2;
            S_io[b] = S;
        }
    }
    uint64_t status = S & face;
    for (int64_t c = b + DIR; c >= 0 && c < n && key[c] == key[c - DIR] + (uint64_t)(int64_t)DIR; c += DIR) {
        const uint64_t S0 = S_io[c];
        const uint64_t fill = (DIR > 0 ? status >> 3 : status) * 0xFull;
        const uint64_t S1 = S0 | (fill & ~G_in[c]);
        if (S1 != S0) S_io[c] = S1;
        status = S1 & face;
    }
}

extern "C" emb_status emb_voxelize_guard(emb_forest f, emb_bins b, uint64_t *d_solid_mask, uint64_t *d_guard_mask,
                                         void *stream)
{
    if (!f || !b) return EMB_ERR_BAD_INPUT;
    EMB_SETTLE(f);
    const int L = f->max_level;
    if (b->f != f || b->level != L || f->top != L) return EMB_ERR_STATE;
    EmbLevel &lv = f->lv[L];
    if (lv.n == 0) return EMB_OK;
    if (!d_solid_mask || !d_guard_mask || d_solid_mask == d_guard_mask) return EMB_ERR_BAD_INPUT;
    if (!b->off) return EMB_ERR_STATE;
    GuardHoles H;
    H.L = L;
    for (int l = 0; l < L; ++l) {
        if (!f->lv[l].mask_valid) return EMB_ERR_STATE;
        H.lk[l] = emb_lookup_of(f->lv[l]);
        H.mask[l] = f->lv[l].mask;
    }
    const emb_status rb = emb_bins_sync(b);
    if (rb != EMB_OK) return rb;
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    cudaStream_t s = emb_stream(stream);
    const LevelGeom g = level_geom(f, L);
    const int64_t want = (lv.n + GUARD_WARPS - 1) / GUARD_WARPS;
    const int64_t cap = (int64_t)emb_sm_count() * 8;
    const int grid = (int)(want < cap ? want : cap);
    EMB_LAUNCH((k_guard_surface), grid, 32 * GUARD_WARPS, 0, s)(b->m->rec, (uint32_t)b->m->T, b->m->r_o, b->off, b->ent,
                                                                (uint64_t)b->npairs, lv.key, lv.n, g.ncell,
                                                                d_solid_mask, d_guard_mask, st);
    EMB_LAUNCH((k_guard_sweep<1>), emb_grid(lv.n, 256), 256, 0, s)(lv.key, lv.n, d_solid_mask, d_guard_mask, H, g.nb);
    if (L > 0)
        EMB_LAUNCH((k_guard_sweep<-1>), emb_grid(lv.n, 256), 256, 0, s)(lv.key, lv.n, d_solid_mask, d_guard_mask, H,
                                                                         g.nb);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}
