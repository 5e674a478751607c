// Geometry input (Sec. 3.1): snapped vertex check, integer frame, 48-byte
// triangle records, and the watertightness check on the GPU.
#include <stdlib.h>

#include "emb_internal.cuh"

#define MESH_ERR_ID 1         // vertex id out of range
#define MESH_ERR_SNAP 2       // coordinate not a multiple of 2^-20 inside (0,1)
#define MESH_ERR_DUP_EDGE 4   // a directed edge occurs twice
#define MESH_ERR_OPEN_EDGE 8  // a directed edge has no reverse
#define MESH_ERR_DEG_EDGE 16  // an edge joins a vertex to itself

__global__ void k_mesh_records(const float *__restrict__ verts, const int32_t *__restrict__ tris, int64_t V, int64_t T,
                               int32_t r_o, int4 *__restrict__ rec, int *err)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int bad = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int32_t id = tris[3 * t + k];
        if (id < 0 || (int64_t)id >= V) {
            bad |= MESH_ERR_ID;
            rec[3 * t + k] = make_int4(0, 0, 0, -1);
            continue;
        }
        int c[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float m = verts[3 * (int64_t)id + d] * 1048576.0f;  // exact: power-of-two scaling
            if (!(m > 0.0f && m < 1048576.0f && m == truncf(m))) bad |= MESH_ERR_SNAP;
            c[d] = (int)m * r_o;
        }
        rec[3 * t + k] = make_int4(c[0], c[1], c[2], id);
    }
    if (bad) atomicOr(err, bad);
}

// New vertex positions for the same triangles: corner j of triangle t takes the
// coordinates of its vertex id (kept in the record's fourth word).  A coordinate
// that is not a multiple of 2^-20 inside (0,1) leaves the record unchanged and
// raises EMB_ERR_BAD_INPUT in the device status word.
__global__ void k_mesh_move(const float *__restrict__ verts, int64_t V, int64_t T, int32_t r_o, int4 *__restrict__ rec,
                            int *st)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * T) return;
    const int4 r = rec[e];
    if (r.w < 0 || (int64_t)r.w >= V) {
        emb_set_status(st, EMB_ERR_BAD_INPUT);
        return;
    }
    int c[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float m = verts[3 * (int64_t)r.w + d] * 1048576.0f;  // exact: power-of-two scaling
        if (!(m > 0.0f && m < 1048576.0f && m == truncf(m))) ok = false;
        c[d] = ok ? (int)m * r_o : 0;
    }
    if (!ok) {
        emb_set_status(st, EMB_ERR_BAD_INPUT);
        return;
    }
    rec[e] = make_int4(c[0], c[1], c[2], r.w);
}

__global__ void k_edge_insert(const int32_t *__restrict__ tris, int64_t T, unsigned long long *hk, int64_t cap, int *err)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * T) return;
    int64_t t = e / 3;
    int j = (int)(e % 3);
    uint32_t a = (uint32_t)tris[3 * t + j], b = (uint32_t)tris[3 * t + (j + 1) % 3];
    if (a == b) {
        atomicOr(err, MESH_ERR_DEG_EDGE);
        return;
    }
    unsigned long long key = ((unsigned long long)a << 32) | b;
    uint64_t m = (uint64_t)cap - 1, s = emb_hash_mix(key) & m;
    for (int64_t it = 0; it < cap; ++it) {
        unsigned long long prev = atomicCAS(hk + s, (unsigned long long)EMB_HASH_EMPTY, key);
        if (prev == EMB_HASH_EMPTY) return;
        if (prev == key) {
            atomicOr(err, MESH_ERR_DUP_EDGE);
            return;
        }
        s = (s + 1) & m;
    }
    atomicOr(err, MESH_ERR_DUP_EDGE);
}

__global__ void k_edge_check(const int32_t *__restrict__ tris, int64_t T, const unsigned long long *__restrict__ hk,
                             int64_t cap, int *err)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * T) return;
    int64_t t = e / 3;
    int j = (int)(e % 3);
    uint32_t a = (uint32_t)tris[3 * t + j], b = (uint32_t)tris[3 * t + (j + 1) % 3];
    unsigned long long rkey = ((unsigned long long)b << 32) | a;
    uint64_t m = (uint64_t)cap - 1, s = emb_hash_mix(rkey) & m;
    for (int64_t it = 0; it < cap; ++it) {
        unsigned long long k = hk[s];
        if (k == rkey) return;
        if (k == EMB_HASH_EMPTY) break;
        s = (s + 1) & m;
    }
    atomicOr(err, MESH_ERR_OPEN_EDGE);
}

extern "C" emb_status emb_mesh_create(const float *d_verts, const int32_t *d_tris, int64_t V, int64_t T, int32_t R,
                                      int32_t check_watertight, void *stream, emb_mesh *out)
{
    if (!out || !d_verts || !d_tris || V < 3 || T < 1 || R < 1 || V > 2147483647ll || T > (1ll << 30))
        return EMB_ERR_BAD_INPUT;
    *out = nullptr;
    int32_t r_o = R, k = 0;
    while ((r_o & 1) == 0) {
        r_o >>= 1;
        ++k;
    }
    if (k > 17 || (int64_t)r_o * (1 << 20) >= (1ll << 25)) return EMB_ERR_RANGE;
    cudaStream_t s = emb_stream(stream);
    emb_mesh m = (emb_mesh)calloc(1, sizeof(emb_mesh_s));
    if (!m) return EMB_ERR_CUDA;
    m->R = R;
    m->r_o = r_o;
    m->k = k;
    m->V = V;
    m->T = T;
    cudaGetDevice(&m->device);
    int *err = nullptr;
    unsigned long long *hk = nullptr;
    emb_status rc = EMB_OK;
    int herr = 0;
    // records and the error word from the library's pool (stream-ordered on s; the
    // synchronisation below completes them before the mesh is used on any stream)
    if (emb_malloc_async(&m->rec, (size_t)T * 3 * sizeof(int4), s) != cudaSuccess ||
        emb_malloc_async(&err, sizeof(int), s) != cudaSuccess) {
        rc = EMB_ERR_CUDA;
        goto done;
    }
    cudaMemsetAsync(err, 0, sizeof(int), s);
    EMB_LAUNCH((k_mesh_records), emb_grid(T, 256), 256, 0, s)(d_verts, d_tris, V, T, r_o, m->rec, err);
    if (check_watertight) {
        int64_t cap = 1024;
        while (cap < 6 * T) cap <<= 1;
        if (emb_malloc_async(&hk, cap * sizeof(unsigned long long), s) != cudaSuccess) {
            rc = EMB_ERR_CUDA;
            goto done;
        }
        cudaMemsetAsync(hk, 0xFF, cap * sizeof(unsigned long long), s);
        EMB_LAUNCH((k_edge_insert), emb_grid(3 * T, 256), 256, 0, s)(d_tris, T, hk, cap, err);
        EMB_LAUNCH((k_edge_check), emb_grid(3 * T, 256), 256, 0, s)(d_tris, T, hk, cap, err);
        cudaFreeAsync(hk, s);
    }
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rc = EMB_ERR_CUDA;
        goto done;
    }
    if (herr & (MESH_ERR_ID | MESH_ERR_SNAP)) rc = EMB_ERR_BAD_INPUT;
    else if (herr) rc = EMB_ERR_NOT_WATERTIGHT;
done:
    if (err) cudaFreeAsync(err, s);
    if (rc != EMB_OK) {
        emb_mesh_destroy(m);
        return rc;
    }
    *out = m;
    return EMB_OK;
}

extern "C" void emb_mesh_destroy(emb_mesh m)
{
    if (!m) return;
    if (m->rec) cudaFree(m->rec);
    free(m);
}

extern "C" emb_status emb_mesh_update(emb_mesh m, const float *d_verts, int64_t V, void *stream)
{
    if (!m || !d_verts || V != m->V) return EMB_ERR_BAD_INPUT;
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    cudaStream_t s = emb_stream(stream);
    EMB_LAUNCH((k_mesh_move), emb_grid(3 * m->T, 256), 256, 0, s)(d_verts, V, m->T, m->r_o, m->rec, st);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}
