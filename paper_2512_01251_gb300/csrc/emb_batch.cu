// Batched embedding of many meshes (a deployment path; the paper embeds one
// geometry at a time, Sec. 3).
//
// emb_batch_create plans: it embeds every mesh once through the per-call path
// (which synchronises to size its buffers) and records every count (blocks per
// level, filtered triangles per level, flagged blocks, bin entries, blocks with
// links, links).  It then allocates, once, every buffer a replay needs.
//
// emb_batch_run replays the whole batch from those plans with no allocation
// and no host synchronisation: the per-mesh pipelines are enqueued round-robin
// on several streams, every count the device recomputes is checked against the
// plan by a one-thread kernel (EMB_ERR_STATE on any difference, e.g. when the
// geometry moved), and all meshes' cut links are produced by one persistent
// launch of the link kernel over a shared work queue of (mesh, block) items
// once every pipeline is done ("joint" placement), or each mesh's links by a
// launch on its own stream right after its pipeline, with a grid sized to its
// work, so that the link work of early meshes overlaps the pipelines of later
// ones ("per-mesh" placement).
// Because it neither allocates nor synchronises, the replay can be captured in a
// CUDA graph (emb_batch_capture) and relaunched (emb_batch_launch).
// emb_batch_autotune times a small set of launch shapes (stream count, thread
// block size of the triangle-parallel kernels, resident link CTAs per SM) on
// this batch and keeps the fastest; emb_batch_configure sets one directly.
#include <stdio.h>
#include <stdlib.h>

#include <mutex>
#include <vector>

#include "emb_internal.cuh"

#define BATCH_MAX_STREAMS 32

struct BLevel {
    EmbLevel lv;                     // key, hash, bitmap, mask (+ nbr at the finest level)
    uint8_t *flags = nullptr;        // refine flags (levels below the finest)
    uint32_t *flist = nullptr;       // filtered triangles
    int64_t nf = 0, F = 0;           // planned counts
};

struct BMesh {
    emb_mesh m = nullptr;
    int R = 0, Lf = 0, band = 0, lattice = 0;
    emb_forest_s geo;                // frame and level geometry (no buffers)
    BLevel L[EMB_MAX_LEVELS];
    // scratch sized for the largest level / the triangle count
    uint32_t *flag = nullptr, *pos = nullptr;       // T + 1
    unsigned long long *s_acc = nullptr;            // max blocks
    unsigned int *p_acc = nullptr, *t_acc = nullptr;
    uint32_t *cnt = nullptr, *rank = nullptr;       // max blocks + 1
    uint32_t *pc = nullptr;                         // max bitmap words + 1
    uint64_t *tmp = nullptr;                        // scan scratch
    // finest level
    uint32_t *bin_off = nullptr, *bin_ent = nullptr;
    uint2 *list_bs = nullptr;                       // pair list of the binning pass (planned pairs)
    uint32_t *list_tri = nullptr;
    unsigned long long *list_n = nullptr;
    uint64_t *cand = nullptr;
    uint32_t *work_n = nullptr, *work = nullptr, *blk_off = nullptr;
    unsigned int *next = nullptr;                   // queue cursor of a per-mesh link launch
    uint2 *witem = nullptr;                         // link work items
    uint2 *extra = nullptr;                         // extra parts of split blocks
    unsigned long long *extra_n = nullptr;
    EmbBigQ bq = {nullptr, nullptr, 0};             // chunk queue of large triangles
    unsigned long long *fbits = nullptr;            // dense flagged bits (largest refined level)
    int32_t *o_cell = nullptr, *o_tri = nullptr;
    uint8_t *o_dir = nullptr;
    float *o_q = nullptr;
    int64_t pairs = 0, nwork = 0, links = 0;
    uint32_t *d_n = nullptr;                        // with headroom: blocks of each level in this replay
    std::vector<void *> owned;
};

struct emb_batch_s {
    std::vector<BMesh> m;
    cudaStream_t st[BATCH_MAX_STREAMS] = {};   // pipelines (highest priority)
    cudaStream_t lst[BATCH_MAX_STREAMS] = {};  // link launches of placement 2 (lowest priority)
    cudaEvent_t ev_fork = nullptr, ev_join[BATCH_MAX_STREAMS] = {}, ev_ljoin[BATCH_MAX_STREAMS] = {};
    cudaEvent_t ev_mesh[EMB_MAX_BATCH] = {};    // a mesh's pipeline is done
    unsigned int *next = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // launch shape (autotuned): streams, block size of the triangle-parallel
    // kernels, link CTAs per SM (0 = as many as fit), link placement (0 joint, 1 per
    // mesh on its pipeline's stream, 2 per mesh on a low-priority stream of its own)
    int nstreams = 8, tri_block = 256, link_ctas = 0, per_mesh_links = 1;
    int headroom = 0;  // percent of room above the planned counts (0: the counts must match the plan)
    int device = 0;
};

template <class T>
static emb_status balloc(BMesh &B, T **p, size_t count)
{
    void *q = nullptr;
    EMB_CUDA_TRY(cudaMalloc(&q, (count ? count : 1) * sizeof(T)));
    B.owned.push_back(q);
    *p = (T *)q;
    return EMB_OK;
}

#define BTRY(x)                          \
    do {                                 \
        emb_status _r = (x);             \
        if (_r != EMB_OK) return _r;     \
    } while (0)

// Embeds mesh B once through the per-call path, recording every count.
static emb_status plan_mesh(BMesh &B, cudaStream_t s)
{
    emb_forest f = nullptr;
    BTRY(emb_forest_root(B.R, B.Lf, s, &f));
    emb_status rc = EMB_OK;
    uint8_t *fl = nullptr;
    for (int L = 0; L <= B.Lf && rc == EMB_OK; ++L) {
        emb_bins b = nullptr;
        rc = emb_bin(B.m, f, L, B.lattice, s, &b);
        if (rc != EMB_OK) break;
        rc = emb_bins_sync(b);
        if (rc != EMB_OK) {
            emb_bins_destroy(b);
            break;
        }
        B.L[L].nf = b->nf;
        rc = emb_voxelize(f, b, L, nullptr, s);
        if (rc == EMB_OK && L < B.Lf) {
            const int64_t n = f->lv[L].n;
            if (emb_malloc_async(&fl, n + 1, s) != cudaSuccess) rc = EMB_ERR_CUDA;
            if (rc == EMB_OK) rc = emb_refine_flags(f, b, L, B.band, fl, s);
            if (rc == EMB_OK) rc = emb_forest_refine(f, L, fl, s);
            if (rc == EMB_OK) rc = emb_forest_settle(f);
            if (rc == EMB_OK) B.L[L].F = f->lv[L + 1].n / 8;
            cudaFreeAsync(fl, s);
        } else if (rc == EMB_OK) {
            B.pairs = b->npairs;
            int64_t nl = 0;
            rc = emb_cutlinks_count(f, B.lattice, &nl, s);
            B.links = nl;
            if (rc == EMB_OK) {
                uint32_t nw = 0;
                if (cudaMemcpyAsync(&nw, f->work_n + f->lv[L].n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    rc = EMB_ERR_CUDA;
                B.nwork = nw;
            }
        }
        emb_bins_destroy(b);
    }
    if (rc == EMB_OK) {
        B.geo.R = f->R;
        B.geo.r_o = f->r_o;
        B.geo.k = f->k;
        B.geo.max_level = f->max_level;
        B.geo.top = f->top;
        for (int L = 0; L <= B.Lf; ++L) {
            B.L[L].lv.n = f->lv[L].n;
            B.L[L].lv.nb_axis = f->lv[L].nb_axis;
        }
    }
    emb_forest_destroy(f);
    return rc;
}

// With headroom h percent, the planned counts become capacities of count (1 + h / 100)
// plus 64: flagged blocks per refined level (so 8 x that many child blocks), bin
// entries, blocks with links, links.  The replay then reads each level's block count
// on the device (lv.d_n) and checks every count against its capacity.
static void headroom_caps(BMesh &B, int headroom)
{
    auto cap = [&](int64_t x) { return x + (x * headroom + 99) / 100 + 64; };
    for (int L = 0; L < B.Lf; ++L) {
        B.L[L].F = cap(B.L[L].F);
        B.L[L + 1].lv.n = 8 * B.L[L].F;
    }
    B.pairs = cap(B.pairs);
    B.links = cap(B.links);
    B.nwork = cap(B.nwork);
}

// Allocates every buffer of a replay of mesh B.
static emb_status alloc_mesh(BMesh &B, int headroom)
{
    const int64_t T = B.m->T;
    if (headroom > 0) {
        headroom_caps(B, headroom);
        BTRY(balloc(B, &B.d_n, EMB_MAX_LEVELS));
        for (int L = 1; L <= B.Lf; ++L) B.L[L].lv.d_n = B.d_n + L;
    }
    int64_t nmax = 1, wmax = 1;
    for (int L = 0; L <= B.Lf; ++L) {
        EmbLevel &lv = B.L[L].lv;
        nmax = lv.n > nmax ? lv.n : nmax;
        const int64_t nw = emb_bitmap_words(lv.nb_axis);
        wmax = nw > wmax ? nw : wmax;
        BTRY(balloc(B, &lv.key, lv.n + 1));
        if (nw == 0) {  // the level is looked up through its hash
            lv.hcap = emb_hash_capacity(lv.n);
            BTRY(balloc(B, &lv.hkey, lv.hcap));
            BTRY(balloc(B, &lv.hval, lv.hcap));
        } else {
            BTRY(balloc(B, &lv.bits, nw));
            BTRY(balloc(B, &lv.wpre, nw + 1));
        }
        BTRY(balloc(B, &lv.mask, lv.n + 1));
        BTRY(balloc(B, &B.L[L].flist, T + 1));
        if (L < B.Lf) BTRY(balloc(B, &B.L[L].flags, lv.n + 1));
    }
    int64_t fw = 1;
    for (int L = 0; L < B.Lf; ++L) {
        const int64_t nw = emb_bitmap_words(B.L[L].lv.nb_axis);
        fw = nw > fw ? nw : fw;
    }
    BTRY(balloc(B, &B.fbits, fw));
    EmbLevel &fin = B.L[B.Lf].lv;
    BTRY(balloc(B, &fin.nbr, fin.n * 26 + 1));
    BTRY(balloc(B, &B.flag, T + 1));
    BTRY(balloc(B, &B.pos, T + 1));
    BTRY(balloc(B, &B.s_acc, nmax));
    BTRY(balloc(B, &B.p_acc, nmax));
    BTRY(balloc(B, &B.t_acc, nmax));
    BTRY(balloc(B, &B.cnt, nmax + 1));
    BTRY(balloc(B, &B.rank, nmax + 1));
    BTRY(balloc(B, &B.pc, wmax + 1));
    const int64_t sw = emb_scan_tmp_words(T > nmax ? (T > wmax ? T : wmax) : (nmax > wmax ? nmax : wmax));
    BTRY(balloc(B, &B.tmp, sw));
    BTRY(balloc(B, &B.bin_off, fin.n + 1));
    BTRY(balloc(B, &B.bin_ent, B.pairs + 1));
    BTRY(balloc(B, &B.list_bs, B.pairs + 1));
    BTRY(balloc(B, &B.list_tri, B.pairs + 1));
    BTRY(balloc(B, &B.list_n, 1));
    BTRY(balloc(B, &B.cand, fin.n * 26 + 1));
    BTRY(balloc(B, &B.work_n, fin.n + 1));
    BTRY(balloc(B, &B.work, fin.n + 1));
    BTRY(balloc(B, &B.blk_off, fin.n + 1));
    BTRY(balloc(B, &B.next, 1));
    BTRY(balloc(B, &B.witem, fin.n + 1));
    BTRY(balloc(B, &B.extra, (size_t)emb_link_extra_capacity(fin.n)));
    BTRY(balloc(B, &B.extra_n, 1));
    BTRY(balloc(B, &B.bq.n, 1));
    BTRY(balloc(B, &B.bq.q, (size_t)emb_bigq_capacity(T)));
    B.bq.cap = (uint32_t)emb_bigq_capacity(T);
    BTRY(balloc(B, &B.o_cell, B.links + 1));
    BTRY(balloc(B, &B.o_dir, B.links + 1));
    BTRY(balloc(B, &B.o_q, B.links + 1));
    BTRY(balloc(B, &B.o_tri, B.links + 1));
    return EMB_OK;
}

// d_n = 8 x the flagged count of the parent level, capped at the level's capacity
// (EMB_ERR_CAPACITY when the flagged blocks need more).
__global__ void k_level_count(const uint32_t *__restrict__ nflags, int64_t cap, uint32_t *__restrict__ d_n, int *st)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t n = 8ull * *nflags;
    if (n > (uint64_t)cap) emb_set_status(st, EMB_ERR_CAPACITY);
    *d_n = (uint32_t)(n < (uint64_t)cap ? n : (uint64_t)cap);
}

// EMB_ERR_CAPACITY when the pair list asked for more entries than it holds.
__global__ void k_list_check(const unsigned long long *__restrict__ list_n, uint64_t cap, int *st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && *list_n > cap) emb_set_status(st, EMB_ERR_CAPACITY);
}

// Enqueues the pipeline of mesh B up to (not including) the link kernel, on stream s.
static emb_status enqueue_mesh(BMesh &B, int tri_block, cudaStream_t s)
{
    const int4 *rec = B.m->rec;
    const int64_t T = B.m->T;
    const bool hr = B.d_n != nullptr;  // headroom: counts up to capacity, read on the device
    int *st = emb_status_word();
    if (!st) return EMB_ERR_CUDA;
    BTRY(emb_enq_root_keys(B.R, B.L[0].lv.key, s));
    BTRY(emb_enq_level_index(B.L[0].lv, B.pc, B.tmp, s));
    for (int L = 0; L <= B.Lf; ++L) {
        BLevel &BL = B.L[L];
        EmbLevel &lv = BL.lv;
        const LevelGeom g = level_geom(&B.geo, L);
        BTRY(emb_enq_filter(rec, T, g, B.flag, B.pos, BL.flist, B.tmp, tri_block, s, hr ? EMB_NO_EXPECT : (uint64_t)BL.nf));
        BTRY(emb_enq_voxelize(rec, T, BL.flist, hr ? T : BL.nf, B.pos + T, nullptr, g, lv, B.s_acc, B.p_acc, B.t_acc, B.bq,
                              tri_block, s));
        if (L < B.Lf) {
            const long long dil = emb_refine_dilation(&B.geo, L, B.band);
            if (dil < 0) return EMB_ERR_RANGE;
            BTRY(emb_enq_refine(rec, T, g, dil, lv, BL.flags, B.fbits, B.bq, s));
            BTRY(emb_enq_flag_ranks(lv, BL.flags, B.cnt, B.rank, B.tmp, s, hr ? EMB_NO_EXPECT : (uint64_t)BL.F));
            EmbLevel &C = B.L[L + 1].lv;
            if (hr) EMB_LAUNCH((k_level_count), 1, 32, 0, s)(B.rank + lv.n, C.n, B.d_n + L + 1, st);
            BTRY(emb_enq_children(lv, BL.flags, B.rank, C.key, C.n, true, s));
            BTRY(emb_enq_level_index(C, B.pc, B.tmp, s));
        } else {
            BTRY(emb_enq_bin_pairs(rec, T, g, lv, B.cnt, B.bin_off, B.list_bs, B.list_tri, B.list_n, (uint64_t)B.pairs,
                                   B.tmp, B.bq, s, hr ? EMB_NO_EXPECT : (uint64_t)B.pairs));
            if (hr) EMB_LAUNCH((k_list_check), 1, 32, 0, s)(B.list_n, (uint64_t)B.pairs, st);
            BTRY(emb_enq_bin_scatter(B.list_bs, B.list_tri, B.list_n, (uint64_t)B.pairs, B.bin_off, B.bin_ent,
                                     (uint64_t)B.pairs, s));
            BTRY(emb_enq_neighbors(lv, s));
            BTRY(emb_enq_link_prep(lv, B.lattice, B.cand, B.cnt, B.rank, B.work_n, B.work, B.blk_off, B.tmp, s,
                                   hr ? EMB_NO_EXPECT : (uint64_t)B.nwork, hr ? EMB_NO_EXPECT : (uint64_t)B.links));
            BTRY(emb_enq_link_split(lv, B.work, B.work_n + lv.n, B.cand, B.blk_off, B.bin_off, B.witem, B.extra,
                                    B.extra_n, (uint32_t)emb_link_extra_capacity(lv.n), s));
        }
    }
    return EMB_OK;
}

static void free_mesh(BMesh &B)
{
    for (void *p : B.owned) cudaFree(p);
    B.owned.clear();
}

extern "C" void emb_batch_destroy(emb_batch b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (int i = 0; i < BATCH_MAX_STREAMS; ++i) {
        if (b->st[i]) cudaStreamDestroy(b->st[i]);
        if (b->lst[i]) cudaStreamDestroy(b->lst[i]);
        if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
        if (b->ev_ljoin[i]) cudaEventDestroy(b->ev_ljoin[i]);
    }
    for (int j = 0; j < EMB_MAX_BATCH; ++j)
        if (b->ev_mesh[j]) cudaEventDestroy(b->ev_mesh[j]);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->next) cudaFree(b->next);
    for (BMesh &B : b->m) free_mesh(B);
    delete b;
}

extern "C" emb_status emb_batch_create(const emb_mesh *meshes, const int32_t *levels, const int32_t *bands,
                                       const int32_t *lattices, int32_t n, void *stream, emb_batch *out)
{
    return emb_batch_create_ex(meshes, levels, bands, lattices, n, 0, stream, out);
}

extern "C" emb_status emb_batch_create_ex(const emb_mesh *meshes, const int32_t *levels, const int32_t *bands,
                                          const int32_t *lattices, int32_t n, int32_t headroom, void *stream,
                                          emb_batch *out)
{
    if (!out || !meshes || !levels || !bands || !lattices || n < 1 || n > EMB_MAX_BATCH || headroom < 0 ||
        headroom > 1000)
        return EMB_ERR_BAD_INPUT;
    *out = nullptr;
    cudaStream_t s = emb_stream(stream);
    emb_batch b = new emb_batch_s();
    b->headroom = headroom;
    cudaGetDevice(&b->device);
    b->m.resize(n);
    emb_status rc = EMB_OK;
    for (int j = 0; j < n && rc == EMB_OK; ++j) {
        BMesh &B = b->m[j];
        if (!meshes[j] || levels[j] < 0 || levels[j] >= EMB_MAX_LEVELS || bands[j] < 1 ||
            (lattices[j] != 19 && lattices[j] != 27)) {
            rc = EMB_ERR_BAD_INPUT;
            break;
        }
        B.m = meshes[j];
        B.R = meshes[j]->R;
        B.Lf = levels[j];
        B.band = bands[j];
        B.lattice = lattices[j];
        rc = plan_mesh(B, s);
        if (rc == EMB_OK) rc = alloc_mesh(B, b->headroom);
    }
    if (rc == EMB_OK && cudaMalloc(&b->next, sizeof(unsigned int)) != cudaSuccess) rc = EMB_ERR_CUDA;
    if (rc == EMB_OK) rc = emb_link_emit_init();  // kernel attributes are set outside of any capture
    if (rc == EMB_OK && !emb_status_word()) rc = EMB_ERR_CUDA;
    int prio_least = 0, prio_greatest = 0;
    if (rc == EMB_OK && cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) rc = EMB_ERR_CUDA;
    for (int i = 0; i < BATCH_MAX_STREAMS && rc == EMB_OK; ++i) {
        if (cudaStreamCreateWithPriority(&b->st[i], cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&b->lst[i], cudaStreamNonBlocking, prio_least) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_ljoin[i], cudaEventDisableTiming) != cudaSuccess)
            rc = EMB_ERR_CUDA;
    }
    for (int j = 0; j < n && rc == EMB_OK; ++j)
        if (cudaEventCreateWithFlags(&b->ev_mesh[j], cudaEventDisableTiming) != cudaSuccess) rc = EMB_ERR_CUDA;
    if (rc == EMB_OK && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) rc = EMB_ERR_CUDA;
    if (rc == EMB_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = EMB_ERR_CUDA;
    if (rc != EMB_OK) {
        emb_batch_destroy(b);
        return rc;
    }
    *out = b;
    return EMB_OK;
}

// The replay: fork to the worker streams, one pipeline per mesh, join, one link launch.
// Planned work of mesh B in rough units: triangle passes per level, bin entries,
// blocks and links (used only to order and place the meshes).
static double plan_cost(const BMesh &B)
{
    double c = (double)B.m->T * (B.Lf + 1) + 4.0 * (double)B.pairs + 4.0 * (double)B.links;
    for (int L = 0; L <= B.Lf; ++L) c += 8.0 * (double)B.L[L].lv.n;
    return c;
}

// The link-kernel view of mesh B's finest level.
static LinkMesh link_mesh(BMesh &B)
{
    const EmbLevel &fin = B.L[B.Lf].lv;
    LinkMesh M;
    M.key = fin.key;
    M.cand = B.cand;
    M.blk_off = B.blk_off;
    M.bin_off = B.bin_off;
    M.bin_ent = B.bin_ent;
    M.ent_cap = (uint64_t)B.pairs;
    M.rec = B.m->rec;
    M.T = (uint32_t)B.m->T;
    M.work_n = B.work_n + fin.n;
    M.witem = B.witem;
    M.extra = B.extra;
    M.extra_n = B.extra_n;
    M.extra_cap = (uint32_t)emb_link_extra_capacity(fin.n);
    M.o_cell = B.o_cell;
    M.o_dir = B.o_dir;
    M.o_q = B.o_q;
    M.o_tri = B.o_tri;
    M.g = level_geom(&B.geo, B.Lf);
    M.cap = (uint32_t)B.links;
    M.nblk = fin.n;
    return M;
}

static emb_status batch_enqueue(emb_batch b, cudaStream_t s)
{
    const int K = b->nstreams < 1 ? 1 : (b->nstreams > BATCH_MAX_STREAMS ? BATCH_MAX_STREAMS : b->nstreams);
    EMB_CUDA_TRY(cudaEventRecord(b->ev_fork, s));
    for (int i = 0; i < K; ++i) {
        EMB_CUDA_TRY(cudaStreamWaitEvent(b->st[i], b->ev_fork, 0));
        if (b->per_mesh_links == 2) EMB_CUDA_TRY(cudaStreamWaitEvent(b->lst[i], b->ev_fork, 0));
    }
    // meshes by decreasing planned work, each to the stream with the least work so far
    std::vector<int> order(b->m.size());
    for (size_t j = 0; j < order.size(); ++j) order[j] = (int)j;
    for (size_t a = 1; a < order.size(); ++a)
        for (size_t c = a; c > 0 && plan_cost(b->m[order[c]]) > plan_cost(b->m[order[c - 1]]); --c) {
            int t = order[c];
            order[c] = order[c - 1];
            order[c - 1] = t;
        }
    double load[BATCH_MAX_STREAMS] = {0};
    for (size_t q = 0; q < order.size(); ++q) {
        BMesh &B = b->m[order[q]];
        int k = 0;
        for (int i = 1; i < K; ++i)
            if (load[i] < load[k]) k = i;
        load[k] += plan_cost(B);
        BTRY(enqueue_mesh(B, b->tri_block, b->st[k]));
        if (b->per_mesh_links) {
            LinkTable one;
            one.n = 1;
            one.m[0] = link_mesh(B);
            cudaStream_t ls = b->st[k];
            if (b->per_mesh_links == 2) {
                // the link kernel yields SMs to the latency-bound pipelines of other meshes
                ls = b->lst[k];
                EMB_CUDA_TRY(cudaEventRecord(b->ev_mesh[order[q]], b->st[k]));
                EMB_CUDA_TRY(cudaStreamWaitEvent(ls, b->ev_mesh[order[q]], 0));
            }
            BTRY(emb_enq_link_emit(one, B.next, b->link_ctas, ls, B.nwork > 0 ? B.nwork : 1));
        }
    }
    for (int i = 0; i < K; ++i) {
        EMB_CUDA_TRY(cudaEventRecord(b->ev_join[i], b->st[i]));
        EMB_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_join[i], 0));
        if (b->per_mesh_links == 2) {
            EMB_CUDA_TRY(cudaEventRecord(b->ev_ljoin[i], b->lst[i]));
            EMB_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_ljoin[i], 0));
        }
    }
    if (b->per_mesh_links) return EMB_OK;
    LinkTable tab;
    tab.n = (int)b->m.size();
    for (int j = 0; j < tab.n; ++j) tab.m[j] = link_mesh(b->m[j]);
    return emb_enq_link_emit(tab, b->next, b->link_ctas, s, 0);
}

extern "C" emb_status emb_batch_run(emb_batch b, void *stream)
{
    if (!b) return EMB_ERR_BAD_INPUT;
    return batch_enqueue(b, emb_stream(stream));
}

extern "C" emb_status emb_batch_capture(emb_batch b, void *stream)
{
    if (!b) return EMB_ERR_BAD_INPUT;
    cudaStream_t s = emb_stream(stream);
    if (!s) return EMB_ERR_BAD_INPUT;  // the legacy default stream cannot be captured
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    EMB_CUDA_TRY(cudaStreamSynchronize(s));
    EMB_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    emb_status rc = batch_enqueue(b, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc != EMB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return EMB_ERR_CUDA;
    b->graph = g;
    // kernels keep the priority of the stream they were captured from (where the
    // driver takes per-node priorities; otherwise the graph runs at its launch stream's)
    cudaError_t ie = cudaGraphInstantiate(&b->exec, g, cudaGraphInstantiateFlagUseNodePriority);
    if (ie != cudaSuccess) {
        emb_note_cuda_error(ie, "cudaGraphInstantiate(UseNodePriority)", __FILE__, __LINE__);
        (void)cudaGetLastError();
        b->exec = nullptr;
        EMB_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
    }
    return EMB_OK;
}

extern "C" emb_status emb_batch_launch(emb_batch b, void *stream)
{
    if (!b) return EMB_ERR_BAD_INPUT;
    if (!b->exec) return EMB_ERR_STATE;
    EMB_CUDA_TRY(cudaGraphLaunch(b->exec, emb_stream(stream)));
    return EMB_OK;
}

// Cache of tuned shapes keyed by (SM count, log2 of the batch's triangles, log2 of its
// mesh count, largest lattice): a batch of the same kind takes the cached shape without
// timing.  With EMB_TUNE_CACHE set to a file path, the cache is read from that file at
// first use and written back after every timing run (one line per key, plain text).
struct TuneKey {
    int sm, tb, nb, lat;
    bool operator==(const TuneKey &o) const { return sm == o.sm && tb == o.tb && nb == o.nb && lat == o.lat; }
};
struct TuneEntry {
    TuneKey k;
    int v[4];
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;
static bool g_tune_loaded = false;

static int ilog2_64(int64_t x)
{
    int r = 0;
    while (x > 1) {
        x >>= 1;
        ++r;
    }
    return r;
}

static TuneKey tune_key(const emb_batch_s *b)
{
    int64_t T = 0;
    int lat = 0;
    for (const BMesh &B : b->m) {
        T += B.m->T;
        lat = B.lattice > lat ? B.lattice : lat;
    }
    return TuneKey{emb_sm_count(), ilog2_64(T), ilog2_64((int64_t)b->m.size()), lat};
}

// with g_tune_mu held
static void tune_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("EMB_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "r");
    if (!fp) return;
    TuneEntry e;
    while (fscanf(fp, "%d %d %d %d %d %d %d %d", &e.k.sm, &e.k.tb, &e.k.nb, &e.k.lat, &e.v[0], &e.v[1], &e.v[2],
                  &e.v[3]) == 8) {
        if (e.v[0] < 1 || e.v[0] > BATCH_MAX_STREAMS || (e.v[1] != 128 && e.v[1] != 256 && e.v[1] != 512) || e.v[2] < 0 ||
            e.v[2] > 64 || e.v[3] < 0 || e.v[3] > 2)
            continue;  // not a shape this library makes
        g_tune.push_back(e);
    }
    fclose(fp);
}

// with g_tune_mu held
static void tune_store(const TuneKey &k, const int v[4])
{
    bool found = false;
    for (TuneEntry &e : g_tune)
        if (e.k == k) {
            for (int i = 0; i < 4; ++i) e.v[i] = v[i];
            found = true;
        }
    if (!found) {
        TuneEntry e;
        e.k = k;
        for (int i = 0; i < 4; ++i) e.v[i] = v[i];
        g_tune.push_back(e);
    }
    const char *path = getenv("EMB_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *fp = fopen(path, "w");
    if (!fp) return;
    for (const TuneEntry &e : g_tune)
        fprintf(fp, "%d %d %d %d %d %d %d %d\n", e.k.sm, e.k.tb, e.k.nb, e.k.lat, e.v[0], e.v[1], e.v[2], e.v[3]);
    fclose(fp);
}

static void drop_graph(emb_batch b)
{
    if (b->exec) {  // a captured graph no longer matches the chosen shape
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
}

extern "C" emb_status emb_batch_autotune(emb_batch b, void *stream, int32_t *h_choice)
{
    int32_t c[5];
    const emb_status rc = emb_batch_autotune_ex(b, stream, 0, c);
    if (rc == EMB_OK && h_choice)
        for (int i = 0; i < 4; ++i) h_choice[i] = c[i];
    return rc;
}

extern "C" emb_status emb_batch_autotune_ex(emb_batch b, void *stream, int32_t flags, int32_t *h_choice)
{
    if (!b || (flags & ~EMB_TUNE_FORCE)) return EMB_ERR_BAD_INPUT;
    const TuneKey key = tune_key(b);
    if (!(flags & EMB_TUNE_FORCE)) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        for (const TuneEntry &e : g_tune)
            if (e.k == key) {
                b->nstreams = e.v[0];
                b->tri_block = e.v[1];
                b->link_ctas = e.v[2];
                b->per_mesh_links = e.v[3];
                drop_graph(b);
                if (h_choice) {
                    for (int i = 0; i < 4; ++i) h_choice[i] = e.v[i];
                    h_choice[4] = 1;
                }
                return EMB_OK;
            }
    }
    cudaStream_t s = emb_stream(stream);
    struct Cand {
        int nstreams, tri_block, link_ctas, per_mesh;
    };
    const Cand cands[] = {{1, 256, 0, 0},   {16, 256, 0, 0},  {16, 128, 0, 0}, {8, 256, 0, 1},  {16, 256, 0, 1},
                          {16, 256, 2, 1},  {16, 128, 2, 1},  {16, 256, 0, 2}, {16, 256, 1, 2}, {16, 256, 2, 2},
                          {16, 128, 1, 2},  {16, 128, 2, 2},  {8, 256, 2, 2},  {32, 256, 0, 1}, {32, 256, 2, 1},
                          {32, 256, 0, 2},  {32, 256, 2, 2},  {24, 256, 2, 2}};
    // shapes are timed the way they will run: as captured graphs where the stream can be
    // captured, else as stream launches
    const bool graphs = s != nullptr;
    const int nc = (int)(sizeof(cands) / sizeof(cands[0]));
    cudaEvent_t e0, e1;
    EMB_CUDA_TRY(cudaEventCreate(&e0));
    EMB_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_i = 0;
    for (int i = 0; i < nc; ++i) {
        b->nstreams = cands[i].nstreams;
        b->tri_block = cands[i].tri_block;
        b->link_ctas = cands[i].link_ctas;
        b->per_mesh_links = cands[i].per_mesh;
        if (graphs) {
            BTRY(emb_batch_capture(b, s));
            BTRY(emb_batch_launch(b, s));  // warm-up
        } else {
            BTRY(batch_enqueue(b, s));  // warm-up
        }
        float tot = 0;
        for (int r = 0; r < 3; ++r) {
            EMB_CUDA_TRY(cudaEventRecord(e0, s));
            if (graphs) BTRY(emb_batch_launch(b, s));
            else BTRY(batch_enqueue(b, s));
            EMB_CUDA_TRY(cudaEventRecord(e1, s));
            EMB_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0;
            EMB_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            tot += ms;
        }
        if (tot < best) {
            best = tot;
            best_i = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->nstreams = cands[best_i].nstreams;
    b->tri_block = cands[best_i].tri_block;
    b->link_ctas = cands[best_i].link_ctas;
    b->per_mesh_links = cands[best_i].per_mesh;
    drop_graph(b);
    const int v[4] = {b->nstreams, b->tri_block, b->link_ctas, b->per_mesh_links};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        tune_store(key, v);
    }
    if (h_choice) {
        for (int i = 0; i < 4; ++i) h_choice[i] = v[i];
        h_choice[4] = 0;
    }
    return EMB_OK;
}

extern "C" emb_status emb_batch_configure(emb_batch b, const int32_t *h_choice)
{
    if (!b || !h_choice) return EMB_ERR_BAD_INPUT;
    const int ns = h_choice[0], tb = h_choice[1], lc = h_choice[2], pm = h_choice[3];
    if (ns < 1 || ns > BATCH_MAX_STREAMS || (tb != 128 && tb != 256 && tb != 512) || lc < 0 || lc > 64 || pm < 0 ||
        pm > 2)
        return EMB_ERR_BAD_INPUT;
    b->nstreams = ns;
    b->tri_block = tb;
    b->link_ctas = lc;
    b->per_mesh_links = pm;
    if (b->exec) {  // a captured graph no longer matches the shape
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return EMB_OK;
}

extern "C" emb_status emb_batch_info(emb_batch b, int32_t j, int64_t *h_blocks, int64_t *h_links)
{
    if (!b || j < 0 || j >= (int32_t)b->m.size()) return EMB_ERR_BAD_INPUT;
    const BMesh &B = b->m[j];
    if (h_blocks)
        for (int L = 0; L <= B.Lf; ++L) h_blocks[L] = B.L[L].lv.n;
    if (h_links) *h_links = B.links;
    return EMB_OK;
}

// Counts of mesh j in the last replay: blocks per level and links.  With headroom they
// are read from the device (this synchronises `stream`); otherwise they are the plan.
static emb_status replay_counts(const BMesh &B, cudaStream_t s, int64_t *blocks, int64_t *links)
{
    for (int L = 0; L <= B.Lf; ++L) blocks[L] = B.L[L].lv.n;
    *links = B.links;
    if (!B.d_n) return EMB_OK;
    uint32_t h[EMB_MAX_LEVELS + 1];
    const EmbLevel &fin = B.L[B.Lf].lv;
    if (B.Lf > 0) EMB_CUDA_TRY(cudaMemcpyAsync(h + 1, B.d_n + 1, B.Lf * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    EMB_CUDA_TRY(cudaMemcpyAsync(h + EMB_MAX_LEVELS, B.blk_off + fin.n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    EMB_CUDA_TRY(cudaStreamSynchronize(s));
    for (int L = 1; L <= B.Lf; ++L) blocks[L] = h[L] < (uint64_t)B.L[L].lv.n ? h[L] : B.L[L].lv.n;
    *links = h[EMB_MAX_LEVELS] < (uint64_t)B.links ? h[EMB_MAX_LEVELS] : B.links;
    return EMB_OK;
}

extern "C" emb_status emb_batch_counts(emb_batch b, int32_t j, void *stream, int64_t *h_blocks, int64_t *h_links)
{
    if (!b || j < 0 || j >= (int32_t)b->m.size()) return EMB_ERR_BAD_INPUT;
    const BMesh &B = b->m[j];
    int64_t blocks[EMB_MAX_LEVELS], links = 0;
    BTRY(replay_counts(B, emb_stream(stream), blocks, &links));
    if (h_blocks)
        for (int L = 0; L <= B.Lf; ++L) h_blocks[L] = blocks[L];
    if (h_links) *h_links = links;
    return EMB_OK;
}

extern "C" emb_status emb_batch_results(emb_batch b, int32_t j, int32_t level, uint64_t *d_mask, int32_t *d_blocks,
                                        int32_t *d_cell, uint8_t *d_dir, float *d_q, int32_t *d_tri, void *stream)
{
    if (!b || j < 0 || j >= (int32_t)b->m.size()) return EMB_ERR_BAD_INPUT;
    const BMesh &B = b->m[j];
    if (level < 0 || level > B.Lf) return EMB_ERR_BAD_INPUT;
    cudaStream_t s = emb_stream(stream);
    int64_t cnt_blocks[EMB_MAX_LEVELS], cnt_links = 0;
    BTRY(replay_counts(B, s, cnt_blocks, &cnt_links));
    EmbLevel lv = B.L[level].lv;  // a view: n becomes this replay's count
    lv.n = cnt_blocks[level];
    if (d_mask && lv.n)
        EMB_CUDA_TRY(cudaMemcpyAsync(d_mask, lv.mask, lv.n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    if (d_blocks && lv.n) {
        emb_forest_s tmp;
        tmp.R = B.R;
        tmp.top = level;
        tmp.lv[level] = lv;
        emb_status rc = emb_forest_blocks(&tmp, level, d_blocks, stream);
        tmp.lv[level] = EmbLevel();  // not owned
        BTRY(rc);
    }
    const size_t n = (size_t)cnt_links;
    if (d_cell && n) EMB_CUDA_TRY(cudaMemcpyAsync(d_cell, B.o_cell, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (d_dir && n) EMB_CUDA_TRY(cudaMemcpyAsync(d_dir, B.o_dir, n, cudaMemcpyDeviceToDevice, s));
    if (d_q && n) EMB_CUDA_TRY(cudaMemcpyAsync(d_q, B.o_q, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (d_tri && n) EMB_CUDA_TRY(cudaMemcpyAsync(d_tri, B.o_tri, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return EMB_OK;
}
