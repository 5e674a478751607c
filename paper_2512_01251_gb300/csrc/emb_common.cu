// Shared plumbing of libemb: device status word, exclusive scan, level hash,
// neighbour tables, and the small query entry points of the C ABI.
#include <stdio.h>
#include <stdlib.h>

#include <atomic>
#include <mutex>

#include "emb_internal.cuh"

// ---------------------------------------------------------------------------
// status word and error notes
// ---------------------------------------------------------------------------
static std::mutex g_status_mu;
static int *g_status_dev[64] = {nullptr};

void emb_note_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    if (getenv("EMB_VERBOSE")) fprintf(stderr, "libemb: %s failed (%s) at %s:%d\n", what, cudaGetErrorString(e), file, line);
}

int *emb_status_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status_dev[dev]) {
        int *p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
        g_status_dev[dev] = p;
    }
    return g_status_dev[dev];
}

cudaStream_t emb_stream(void *s) { return (cudaStream_t)s; }

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {nullptr};

cudaError_t emb_malloc_raw(void **p, size_t bytes, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np = nullptr;
            e = cudaMemPoolCreate(&np, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = UINT64_MAX;  // never trimmed at synchronisations
            e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) return e;
            g_pool[dev] = np;
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

static std::atomic<long long> g_launches{0};

void emb_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" emb_status emb_launch_count(int64_t *h_out)
{
    if (!h_out) return EMB_ERR_BAD_INPUT;
    *h_out = g_launches.load(std::memory_order_relaxed);
    return EMB_OK;
}

int emb_grid(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 2147483647ll) g = 2147483647ll;
    return (int)g;
}

extern "C" const char *emb_status_string(emb_status s)
{
    switch (s) {
    case EMB_OK: return "EMB_OK";
    case EMB_ERR_BAD_INPUT: return "EMB_ERR_BAD_INPUT";
    case EMB_ERR_NOT_WATERTIGHT: return "EMB_ERR_NOT_WATERTIGHT";
    case EMB_ERR_CAPACITY: return "EMB_ERR_CAPACITY";
    case EMB_ERR_CUDA: return "EMB_ERR_CUDA";
    case EMB_ERR_TIMEOUT: return "EMB_ERR_TIMEOUT";
    case EMB_ERR_RANGE: return "EMB_ERR_RANGE";
    case EMB_ERR_STATE: return "EMB_ERR_STATE";
    case EMB_ERR_BOUNDS: return "EMB_ERR_BOUNDS";
    default: return "EMB_ERR_UNKNOWN";
    }
}

extern "C" emb_status emb_status_get(void *stream, emb_status *out)
{
    if (!out) return EMB_ERR_BAD_INPUT;
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    EMB_CUDA_TRY(cudaStreamSynchronize(emb_stream(stream)));
    int v = 0;
    EMB_CUDA_TRY(cudaMemcpy(&v, st, sizeof(int), cudaMemcpyDeviceToHost));
    EMB_CUDA_TRY(cudaMemset(st, 0, sizeof(int)));
    *out = v;
    return EMB_OK;
}

extern "C" emb_status emb_directions(int32_t *h_out)
{
    if (!h_out) return EMB_ERR_BAD_INPUT;
    for (int i = 0; i < 27; ++i) {
        int cx, cy, cz;
        emb_dir(i, cx, cy, cz);
        h_out[3 * i + 0] = cx;
        h_out[3 * i + 1] = cy;
        h_out[3 * i + 2] = cz;
    }
    return EMB_OK;
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 values (three phases: tile sums, scan of sums, apply)
// ---------------------------------------------------------------------------
#define SCAN_BLOCK 512
#define SCAN_ITEMS 8
#define SCAN_TILE (SCAN_BLOCK * SCAN_ITEMS)

// Block-wide exclusive scan of one uint64 per thread; returns the block total in *total.
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *total)
{
    __shared__ uint64_t warp_sums[SCAN_BLOCK / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint64_t s = lane < SCAN_BLOCK / 32 ? warp_sums[lane] : 0;
        uint64_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < SCAN_BLOCK / 32) warp_sums[lane] = si - s;  // exclusive warp offsets
        if (lane == SCAN_BLOCK / 32 - 1) *total = si;
    }
    __syncthreads();
    uint64_t r = warp_sums[w] + inc - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_tile_sums(const uint32_t *__restrict__ in, int64_t n, uint64_t *__restrict__ tile_sum)
{
    __shared__ uint64_t tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += in[base + i];
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(uint64_t *__restrict__ tile_sum, int64_t ntiles, uint64_t *__restrict__ total)
{
    __shared__ uint64_t tot;
    uint64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += SCAN_BLOCK) {
        int64_t i = b + threadIdx.x;
        uint64_t v = i < ntiles ? tile_sum[i] : 0;
        uint64_t ex = block_excl_scan(v, &tot);
        if (i < ntiles) tile_sum[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Writes the tile's exclusive sums from its offset `run`; entry n receives the total,
// which is checked against `expect` unless that is EMB_NO_EXPECT.
__device__ __forceinline__ void scan_write_tile(const uint32_t v[SCAN_ITEMS], int64_t base, int64_t n, uint64_t run,
                                                uint32_t *__restrict__ out, uint64_t expect, int *st)
{
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i <= n) {  // entry n receives the total
            if (run > 0xFFFFFFFFull) emb_set_status(st, EMB_ERR_CAPACITY);
            out[base + i] = (uint32_t)run;
            if (base + i == n && expect != EMB_NO_EXPECT && run != expect) emb_set_status(st, EMB_ERR_STATE);
        }
        run += v[i];
    }
}

__global__ void k_scan_apply(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
                             const uint64_t *__restrict__ tile_off, uint64_t expect, int *st)
{
    __shared__ uint64_t tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        s += v[i];
    }
    const uint64_t run = tile_off[blockIdx.x] + block_excl_scan(s, &tot);
    scan_write_tile(v, base, n, run, out, expect, st);
}

// Apply with the scan of the tile sums folded in: each tile adds up the sums of the
// tiles before it (few enough to read them all), and the last tile stores the total
// after the sums.  With one tile it is the whole scan in one launch.
__global__ void k_scan_apply_fused(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
                                   uint64_t *__restrict__ tile_sum, int64_t ntiles, uint64_t expect, int *st)
{
    __shared__ uint64_t tot, before;
    uint64_t part = 0;
    for (int64_t i = threadIdx.x; i < (int64_t)blockIdx.x; i += SCAN_BLOCK) part += tile_sum[i];
    block_excl_scan(part, &before);
    const uint64_t off = before;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        s += v[i];
    }
    const uint64_t run = off + block_excl_scan(s, &tot);
    if (threadIdx.x == 0 && (int64_t)blockIdx.x == ntiles - 1) tile_sum[ntiles] = off + tot;
    scan_write_tile(v, base, n, run, out, expect, st);
}

int64_t emb_scan_tmp_words(int64_t n) { return (n + 1 + SCAN_TILE - 1) / SCAN_TILE + 1; }

// Above this many tiles the tile sums get a scan of their own.
#define SCAN_FUSE_TILES 1024

// d_out gets n + 1 entries: exclusive prefix sums and, at index n, the total (also in
// tmp[ntiles]); a total other than `expect` raises EMB_ERR_STATE on the device.
// tmp: emb_scan_tmp_words(n) uint64 words of scratch.  Enqueues only: one launch up
// to SCAN_TILE entries, two up to SCAN_FUSE_TILES tiles, three beyond.
emb_status emb_scan_into_expect(const uint32_t *d_in, uint32_t *d_out, int64_t n, uint64_t *tmp, uint64_t expect,
                                cudaStream_t s)
{
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    int64_t ntiles = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles <= SCAN_FUSE_TILES) {
        if (ntiles > 1) EMB_LAUNCH((k_scan_tile_sums), (int)ntiles, SCAN_BLOCK, 0, s)(d_in, n, tmp);
        EMB_LAUNCH((k_scan_apply_fused), (int)ntiles, SCAN_BLOCK, 0, s)(d_in, d_out, n, tmp, ntiles, expect, st);
    } else {
        EMB_LAUNCH((k_scan_tile_sums), (int)ntiles, SCAN_BLOCK, 0, s)(d_in, n, tmp);
        EMB_LAUNCH((k_scan_sums), 1, SCAN_BLOCK, 0, s)(tmp, ntiles, tmp + ntiles);
        EMB_LAUNCH((k_scan_apply), (int)ntiles, SCAN_BLOCK, 0, s)(d_in, d_out, n, tmp, expect, st);
    }
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

emb_status emb_scan_into(const uint32_t *d_in, uint32_t *d_out, int64_t n, uint64_t *tmp, cudaStream_t s)
{
    return emb_scan_into_expect(d_in, d_out, n, tmp, EMB_NO_EXPECT, s);
}

emb_status emb_scan_u32(const uint32_t *d_in, uint32_t *d_out, int64_t n, uint64_t *h_total, cudaStream_t s)
{
    uint64_t *tmp = nullptr;
    int64_t ntiles = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
    EMB_CUDA_TRY(emb_malloc_async(&tmp, emb_scan_tmp_words(n) * sizeof(uint64_t), s));
    emb_status rc = emb_scan_into(d_in, d_out, n, tmp, s);
    if (rc != EMB_OK) return rc;
    if (h_total) {
        EMB_CUDA_TRY(cudaMemcpyAsync(h_total, tmp + ntiles, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        EMB_CUDA_TRY(cudaStreamSynchronize(s));
    }
    EMB_CUDA_TRY(cudaFreeAsync(tmp, s));
    return EMB_OK;
}

// ---------------------------------------------------------------------------
// level hash and neighbour table
// ---------------------------------------------------------------------------
__global__ void k_hash_insert(const uint64_t *__restrict__ key, int64_t n, uint64_t *hkey, int32_t *hval, int64_t hcap,
                              int *st, const uint32_t *d_n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= emb_count(n, d_n)) return;
    uint64_t k = key[i];
    uint64_t m = (uint64_t)hcap - 1, s = emb_hash_mix(k) & m;
    for (int64_t it = 0; it < hcap; ++it) {
        unsigned long long prev = atomicCAS((unsigned long long *)(hkey + s), (unsigned long long)EMB_HASH_EMPTY,
                                            (unsigned long long)k);
        if (prev == EMB_HASH_EMPTY || prev == k) {
            hval[s] = (int32_t)i;
            return;
        }
        s = (s + 1) & m;
    }
    emb_set_status(st, EMB_ERR_STATE);  // table full: cannot happen with capacity >= 2n
}

__global__ void k_bits_set(const uint64_t *__restrict__ key, int64_t n, int64_t nb, unsigned long long *__restrict__ bits,
                           const uint32_t *d_n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= emb_count(n, d_n)) return;
    uint64_t k = key[i];
    int64_t bx = (int64_t)(k & EMB_KEY_MASK), by = (int64_t)((k >> EMB_KEY_BITS) & EMB_KEY_MASK),
            bz = (int64_t)(k >> (2 * EMB_KEY_BITS));
    if (bx >= nb || by >= nb || bz >= nb) return;  // only a replay whose counts left its plan gets here
    int64_t lin = (bz * nb + by) * nb + bx;
    atomicOr(bits + (lin >> 6), 1ull << (lin & 63));
}

// The bits of a child level whose block count, 8 x *nflags (at most cap), is still on
// the device: threads past the count leave the bitmap alone.
__global__ void k_bits_set_counted(const uint64_t *__restrict__ key, const uint32_t *__restrict__ nflags, int64_t cap,
                                   int64_t nb, unsigned long long *__restrict__ bits)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = 8 * (int64_t)*nflags;
    if (i >= n || i >= cap) return;
    uint64_t k = key[i];
    int64_t bx = (int64_t)(k & EMB_KEY_MASK), by = (int64_t)((k >> EMB_KEY_BITS) & EMB_KEY_MASK),
            bz = (int64_t)(k >> (2 * EMB_KEY_BITS));
    if (bx >= nb || by >= nb || bz >= nb) return;
    int64_t lin = (bz * nb + by) * nb + bx;
    atomicOr(bits + (lin >> 6), 1ull << (lin & 63));
}

__global__ void k_word_popc(const uint64_t *__restrict__ bits, int64_t nw, uint32_t *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nw) out[i] = (uint32_t)__popcll(bits[i]);
}

int64_t emb_hash_capacity(int64_t n)
{
    int64_t cap = 1024;
    while (cap < 2 * n) cap <<= 1;
    return cap;
}

int64_t emb_bitmap_words(int64_t nb)
{
    int64_t cells = nb * nb * nb;
    return cells <= EMB_BITMAP_MAX_BITS ? (cells + 63) / 64 : 0;
}

// Rank bitmap of a level whose keys are in place or, where the level's dense positions
// exceed EMB_BITMAP_MAX_BITS, its hash (lookups use whichever exists); buffers sized by
// emb_bitmap_words / emb_hash_capacity; pc: words + 1 uint32, tmp: scan scratch.
emb_status emb_enq_level_index(EmbLevel &lv, uint32_t *pc, uint64_t *tmp, cudaStream_t s)
{
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    int64_t nw = emb_bitmap_words(lv.nb_axis);
    if (!(lv.bits && nw > 0)) {
        EMB_CUDA_TRY(cudaMemsetAsync(lv.hkey, 0xFF, lv.hcap * sizeof(uint64_t), s));
        if (lv.n > 0)
            EMB_LAUNCH((k_hash_insert), emb_grid(lv.n, 256), 256, 0, s)(lv.key, lv.n, lv.hkey, lv.hval, lv.hcap, st, lv.d_n);
    } else {
        EMB_CUDA_TRY(cudaMemsetAsync(lv.bits, 0, nw * sizeof(uint64_t), s));
        if (lv.n > 0)
            EMB_LAUNCH((k_bits_set), emb_grid(lv.n, 256), 256, 0, s)(lv.key, lv.n, lv.nb_axis, (unsigned long long *)lv.bits,
                                                                     lv.d_n);
        EMB_LAUNCH((k_word_popc), emb_grid(nw, 256), 256, 0, s)(lv.bits, nw, pc);
        emb_status rc = emb_scan_into(pc, lv.wpre, nw, tmp, s);
        if (rc != EMB_OK) return rc;
    }
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

// The rank bitmap of level lv (which must have one) from keys whose count, 8 x *nflags
// with at most cap keys, is read on the device: lets the host read the count back while
// the index is being built.
emb_status emb_build_index_counted(EmbLevel &lv, const uint32_t *nflags, int64_t cap, cudaStream_t s)
{
    const int64_t nw = emb_bitmap_words(lv.nb_axis);
    if (nw == 0) return EMB_ERR_STATE;
    if (lv.hkey) EMB_CUDA_TRY(cudaFreeAsync(lv.hkey, s));
    if (lv.hval) EMB_CUDA_TRY(cudaFreeAsync(lv.hval, s));
    if (lv.bits) EMB_CUDA_TRY(cudaFreeAsync(lv.bits, s));
    if (lv.wpre) EMB_CUDA_TRY(cudaFreeAsync(lv.wpre, s));
    lv.hkey = nullptr;
    lv.hval = nullptr;
    lv.hcap = 0;
    uint32_t *pc = nullptr;
    uint64_t *tmp = nullptr;
    EMB_CUDA_TRY(emb_malloc_async(&lv.bits, nw * sizeof(uint64_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&lv.wpre, (nw + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&pc, (nw + 1) * sizeof(uint32_t), s));
    EMB_CUDA_TRY(emb_malloc_async(&tmp, emb_scan_tmp_words(nw) * sizeof(uint64_t), s));
    EMB_CUDA_TRY(cudaMemsetAsync(lv.bits, 0, nw * sizeof(uint64_t), s));
    if (cap > 0)
        EMB_LAUNCH((k_bits_set_counted), emb_grid(cap, 256), 256, 0, s)(lv.key, nflags, cap, lv.nb_axis,
                                                                           (unsigned long long *)lv.bits);
    EMB_LAUNCH((k_word_popc), emb_grid(nw, 256), 256, 0, s)(lv.bits, nw, pc);
    emb_status rc = emb_scan_into(pc, lv.wpre, nw, tmp, s);
    EMB_CUDA_TRY(cudaFreeAsync(pc, s));
    EMB_CUDA_TRY(cudaFreeAsync(tmp, s));
    if (rc != EMB_OK) return rc;
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

// The address a kernel uses for a caller's output buffer: device (or managed) memory as
// it is, page-locked host memory through its device mapping (the kernel then writes
// over the host link); pageable host memory, or an address the runtime does not know,
// is refused before anything is enqueued.
emb_status emb_device_view(void *p, void **dp)
{
    *dp = nullptr;
    if (!p) return EMB_OK;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return EMB_ERR_BAD_INPUT;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        *dp = p;
        return EMB_OK;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *dp = a.devicePointer;
        return EMB_OK;
    }
    return EMB_ERR_BAD_INPUT;
}

// Pinned host words for small count read-backs, each with an event that marks when the
// copy into it has landed (a slab shared by all forests; slots are reused after release).
#define EMB_RB_SLOTS 1024
static std::mutex g_rb_mu;
static uint64_t *g_rb_host = nullptr;
static cudaEvent_t g_rb_ev[EMB_RB_SLOTS];
static int g_rb_dev[EMB_RB_SLOTS];
static bool g_rb_used[EMB_RB_SLOTS];
static bool g_rb_pending[EMB_RB_SLOTS];  // released, but its last copy may still be in flight

int emb_readback_acquire(uint64_t **h, cudaEvent_t *ev)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    std::lock_guard<std::mutex> lk(g_rb_mu);
    if (!g_rb_host) {
        if (cudaHostAlloc((void **)&g_rb_host, EMB_RB_SLOTS * 64, cudaHostAllocPortable) != cudaSuccess) {
            g_rb_host = nullptr;
            return -1;
        }
        for (int i = 0; i < EMB_RB_SLOTS; ++i) {
            g_rb_ev[i] = nullptr;
            g_rb_dev[i] = -1;
            g_rb_used[i] = false;
            g_rb_pending[i] = false;
        }
    }
    for (int i = 0; i < EMB_RB_SLOTS; ++i) {
        if (g_rb_used[i]) continue;
        if (g_rb_pending[i]) {
            if (cudaEventQuery(g_rb_ev[i]) != cudaSuccess) continue;
            g_rb_pending[i] = false;
        }
        if (g_rb_ev[i] && g_rb_dev[i] != dev) {
            cudaEventDestroy(g_rb_ev[i]);
            g_rb_ev[i] = nullptr;
        }
        if (!g_rb_ev[i]) {
            if (cudaEventCreateWithFlags(&g_rb_ev[i], cudaEventDisableTiming) != cudaSuccess) {
                g_rb_ev[i] = nullptr;
                return -1;
            }
            g_rb_dev[i] = dev;
        }
        g_rb_used[i] = true;
        *h = g_rb_host + 8 * i;
        *ev = g_rb_ev[i];
        return i;
    }
    return -1;  // all slots taken: the caller reads the count back the plain way
}

void emb_readback_release(int slot)
{
    if (slot < 0 || slot >= EMB_RB_SLOTS) return;
    std::lock_guard<std::mutex> lk(g_rb_mu);
    g_rb_used[slot] = false;
    g_rb_pending[slot] = true;
}

emb_status emb_build_hash(EmbLevel &lv, cudaStream_t s)
{
    if (lv.hkey) EMB_CUDA_TRY(cudaFreeAsync(lv.hkey, s));
    if (lv.hval) EMB_CUDA_TRY(cudaFreeAsync(lv.hval, s));
    if (lv.bits) EMB_CUDA_TRY(cudaFreeAsync(lv.bits, s));
    if (lv.wpre) EMB_CUDA_TRY(cudaFreeAsync(lv.wpre, s));
    lv.bits = nullptr;
    lv.wpre = nullptr;
    lv.hkey = nullptr;
    lv.hval = nullptr;
    lv.hcap = 0;
    int64_t nw = emb_bitmap_words(lv.nb_axis);
    if (nw == 0) {
        lv.hcap = emb_hash_capacity(lv.n);
        EMB_CUDA_TRY(emb_malloc_async(&lv.hkey, lv.hcap * sizeof(uint64_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&lv.hval, lv.hcap * sizeof(int32_t), s));
    }
    uint32_t *pc = nullptr;
    uint64_t *tmp = nullptr;
    if (nw > 0) {
        EMB_CUDA_TRY(emb_malloc_async(&lv.bits, nw * sizeof(uint64_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&lv.wpre, (nw + 1) * sizeof(uint32_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&pc, (nw + 1) * sizeof(uint32_t), s));
        EMB_CUDA_TRY(emb_malloc_async(&tmp, emb_scan_tmp_words(nw) * sizeof(uint64_t), s));
    }
    emb_status rc = emb_enq_level_index(lv, pc, tmp, s);
    if (pc) EMB_CUDA_TRY(cudaFreeAsync(pc, s));
    if (tmp) EMB_CUDA_TRY(cudaFreeAsync(tmp, s));
    return rc;
}

// Ids of the blocks at x - 1, x, x + 1 on row (y, z) of a rank-bitmap level into
// out[0..2] (-1: no block, or outside the level).  The three positions are consecutive
// bits, so they take at most two words and two rank prefixes.
__device__ __forceinline__ void nbr_row3(const EmbLookup &lk, int64_t x, int64_t y, int64_t z, int32_t out[3])
{
    const int64_t nb = lk.nb;
    out[0] = out[1] = out[2] = -1;
    if (y < 0 || z < 0 || y >= nb || z >= nb) return;
    const int64_t row = (z * nb + y) * nb;
    const int64_t lo = x > 0 ? x - 1 : 0, hi = x + 1 < nb ? x + 1 : nb - 1;
    const int64_t la = row + lo, lb = row + hi;
    if (!emb_ck((uint64_t)lb, (uint64_t)nb * nb * nb, lk.st)) return;
    const uint64_t wa = __ldg(lk.bits + (la >> 6)), wb = __ldg(lk.bits + (lb >> 6));
    const uint32_t pa = __ldg(lk.wpre + (la >> 6)), pb = __ldg(lk.wpre + (lb >> 6));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t xx = x - 1 + k;
        if (xx < lo || xx > hi) continue;
        const int64_t l = row + xx;
        const bool first = (l >> 6) == (la >> 6);
        const uint64_t w = first ? wa : wb;
        const int sh = (int)(l & 63);
        if (!((w >> sh) & 1ull)) continue;
        const int32_t id = (int32_t)((first ? pa : pb) + (uint32_t)__popcll(w & ((1ull << sh) - 1ull)));
        out[k] = emb_ck((uint64_t)id, (uint64_t)lk.n, lk.st) ? id : -1;
    }
}

// One thread per block: its 26 neighbours, found row by row (9 rows of 3 positions),
// staged in shared memory so that the CTA writes its blocks' consecutive rows of the
// table with coalesced stores.
#define NBR_BLOCK 128
__global__ void __launch_bounds__(NBR_BLOCK) k_neighbors(const uint64_t *__restrict__ key, int64_t n, int64_t nb,
                                                          EmbLookup lk, int32_t *__restrict__ nbr, const uint32_t *d_n)
{
    __shared__ int32_t stage[NBR_BLOCK * 26];
    const int64_t cnt = emb_count(n, d_n);
    const int64_t b0 = (int64_t)blockIdx.x * NBR_BLOCK;
    if (b0 >= cnt) return;  // the whole CTA
    const int64_t b = b0 + threadIdx.x;
    if (b < cnt) {
        const uint64_t k = key[b];
        const int64_t bx = (int64_t)(k & EMB_KEY_MASK), by = (int64_t)((k >> EMB_KEY_BITS) & EMB_KEY_MASK),
                      bz = (int64_t)(k >> (2 * EMB_KEY_BITS));
        int32_t id[27];  // by offset code (ox + 1) + 3 (oy + 1) + 9 (oz + 1)
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            const int oy = r % 3 - 1, oz = r / 3 - 1;
            if (lk.bits) {
                nbr_row3(lk, bx, by + oy, bz + oz, id + 3 * r);
            } else {
#pragma unroll
                for (int ox = -1; ox <= 1; ++ox) {
                    const int64_t x = bx + ox, y = by + oy, z = bz + oz;
                    id[3 * r + ox + 1] = x >= 0 && y >= 0 && z >= 0 && x < nb && y < nb && z < nb ? emb_lookup(lk, x, y, z) : -1;
                }
            }
        }
#pragma unroll
        for (int d = 1; d < 27; ++d) {
            int cx, cy, cz;
            emb_dir(d, cx, cy, cz);
            stage[threadIdx.x * 26 + d - 1] = id[(cx + 1) + 3 * (cy + 1) + 9 * (cz + 1)];
        }
    }
    __syncthreads();
    const int m = (int)((cnt - b0 < NBR_BLOCK ? cnt - b0 : NBR_BLOCK) * 26);
    for (int j = threadIdx.x; j < m; j += NBR_BLOCK) nbr[b0 * 26 + j] = stage[j];
}

emb_status emb_enq_neighbors(EmbLevel &lv, cudaStream_t s)
{
    if (lv.n > 0)
        EMB_LAUNCH((k_neighbors), emb_grid(lv.n, NBR_BLOCK), NBR_BLOCK, 0, s)(lv.key, lv.n, lv.nb_axis, emb_lookup_of(lv),
                                                                                    lv.nbr, lv.d_n);
    EMB_CUDA_TRY(cudaGetLastError());
    return EMB_OK;
}

emb_status emb_build_neighbors(EmbLevel &lv, cudaStream_t s)
{
    if (lv.nbr) return EMB_OK;
    EMB_CUDA_TRY(emb_malloc_async(&lv.nbr, (lv.n * 26 + 1) * sizeof(int32_t), s));
    return emb_enq_neighbors(lv, s);
}

// ---------------------------------------------------------------------------
// chunk queue of large triangles
// ---------------------------------------------------------------------------
int64_t emb_bigq_capacity(int64_t T)
{
    const int64_t c = 16 * T + 1024;
    return c < (1 << 20) ? c : (1 << 20);
}

emb_status emb_bigq_alloc(EmbBigQ &Q, int64_t T, cudaStream_t s)
{
    Q.q = nullptr;
    Q.n = nullptr;
    Q.cap = (uint32_t)emb_bigq_capacity(T);
    char *p = nullptr;
    EMB_CUDA_TRY(emb_malloc_async((void **)&p, 256 + (size_t)Q.cap * sizeof(uint2), s));
    Q.n = (unsigned long long *)p;
    Q.q = (uint2 *)(p + 256);
    return EMB_OK;
}

void emb_bigq_free(EmbBigQ &Q, cudaStream_t s)
{
    if (Q.n) cudaFreeAsync(Q.n, s);
    Q.q = nullptr;
    Q.n = nullptr;
    Q.cap = 0;
}

// Multiprocessors of the current device (cached per device; persistent grids).
int emb_sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}
