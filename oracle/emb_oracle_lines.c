/*
 * Tier B of the CPU oracle for the mesh-embedding hot path (arXiv 2512.01251,
 * Sec. 3.3-3.4): the same definitions as emb_oracle.c, evaluated along sorted
 * lattice lines so that meshes of millions of triangles finish in minutes.
 *
 * TEST INFRASTRUCTURE ONLY.  Compiled into liboracle.so beside emb_oracle.c and
 * loaded by the tests and the CPU-baseline leg of bench.py; the product library
 * never links, loads or calls it, and it shares no code, header or table with the
 * CUDA path.  Its results are checked against the brute force of emb_oracle.c on
 * every case both can run (tests/test_oracle_lines.py).
 *
 * Definitions (identical to emb_oracle.c; integer frame, every query point P
 * pushed to P + (e, e^2, e^3), e -> 0+):
 *   - refine flag of a block: some triangle overlaps its closed box dilated by the
 *     near-wall distance (separating axes, orc_sat of emb_oracle.c);
 *   - a cell is solid iff the +x ray from its centre crosses the surface an odd
 *     number of times (Sec. 3.4 "Partial Surface Voxelization": the centre decides;
 *     Sec. 3.3.1: crossing-count parity);
 *   - a cut link is (fluid cell P, direction i) with P + h c_i solid; q is the
 *     smallest crossing parameter t of the segment P -> P + h c_i (Sec. 3.4
 *     "Link-Length Computation"), ties to the lowest triangle id.
 *
 * What differs from the brute force is only the order of evaluation:
 *   - flags: triangle-major; each triangle visits the blocks whose dilated box can
 *     meet its bounding box;
 *   - masks: triangle-major over the +x centre lines in each triangle's y-z
 *     bounding box (a 2-D orientation test per edge); each crossing is stored as
 *     (line, number of cell centres of the line strictly before the crossing),
 *     computed by exact integer division; per line the list is sorted, and cell i
 *     is solid iff an odd number of the line's crossings have more than i centres
 *     before them;
 *   - links: candidates by definition from the masks, crossings triangle-major
 *     over the cell centres whose link can reach the triangle's bounding box, one
 *     direction per thread (so no two threads update one link).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;
typedef __int128 i128;

int orc_sat(const i64 *tri, const i64 *lo, const i64 *hi); /* emb_oracle.c */

/* Lattice vectors in the library's order: 0 rest, 1-6 axes, 7-18 edge diagonals,
 * 19-26 corners, each odd index followed by its opposite. */
static const int LDIR[27][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},  {-1, -1, -1},
    {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1},
};

static int sg(i64 v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }
static int sg128(i128 v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }

/* floor(a / b) and ceil(a / b) for b > 0 */
static i64 fdiv(i64 a, i64 b)
{
    i64 q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}
static i64 cdiv(i64 a, i64 b) { return -fdiv(-a, b); }

static void normal_of(const i64 *t, i64 *n)
{
    const i64 ux = t[3] - t[0], uy = t[4] - t[1], uz = t[5] - t[2];
    const i64 vx = t[6] - t[0], vy = t[7] - t[1], vz = t[8] - t[2];
    n[0] = uy * vz - uz * vy;
    n[1] = uz * vx - ux * vz;
    n[2] = ux * vy - uy * vx;
}

static void bbox_of(const i64 *t, i64 *mn, i64 *mx)
{
    for (int a = 0; a < 3; ++a) {
        mn[a] = mx[a] = t[a];
        for (int k = 1; k < 3; ++k) {
            const i64 v = t[3 * k + a];
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    }
}

/* Index range of the cell centres (2g + 1) half (cell size 2 half) lying in [lo, hi],
 * clamped to [0, ncell). */
static void centre_range(i64 lo, i64 hi, i64 half, i64 ncell, i64 *g0, i64 *g1)
{
    *g0 = cdiv(lo - half, 2 * half);
    *g1 = fdiv(hi - half, 2 * half);
    if (*g0 < 0) *g0 = 0;
    if (*g1 > ncell - 1) *g1 = ncell - 1;
}

/* ------------------------------------------------------------------ */
/* block lookup: keys (bz nb + by) nb + bx, ascending                  */
/* ------------------------------------------------------------------ */
static i64 find_key(const i64 *keys, i64 n, i64 key)
{
    i64 lo = 0, hi = n;
    while (lo < hi) {
        const i64 mid = lo + (hi - lo) / 2;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && keys[lo] == key) ? lo : -1;
}

/* ------------------------------------------------------------------ */
/* refine flags, triangle-major                                        */
/* ------------------------------------------------------------------ */
/* flags[b] = 1 iff some triangle overlaps the closed box [b W - D, (b + 1) W + D]
 * of block b (keys ascending, nb blocks per axis, block width W, dilation D). */
void orc_lines_flags(const i64 *tri, i64 T, const i64 *keys, i64 n, i64 nb, i64 W, i64 D, uint8_t *flags)
{
    memset(flags, 0, (size_t)n);
#pragma omp parallel for schedule(dynamic, 256)
    for (i64 t = 0; t < T; ++t) {
        const i64 *tr = tri + 9 * t;
        i64 mn[3], mx[3], b0[3], b1[3];
        bbox_of(tr, mn, mx);
        for (int a = 0; a < 3; ++a) {
            b0[a] = cdiv(mn[a] - D - W, W); /* (b + 1) W + D >= mn */
            b1[a] = fdiv(mx[a] + D, W);     /* b W - D <= mx */
            if (b0[a] < 0) b0[a] = 0;
            if (b1[a] > nb - 1) b1[a] = nb - 1;
        }
        for (i64 bz = b0[2]; bz <= b1[2]; ++bz)
            for (i64 by = b0[1]; by <= b1[1]; ++by)
                for (i64 bx = b0[0]; bx <= b1[0]; ++bx) {
                    const i64 id = find_key(keys, n, (bz * nb + by) * nb + bx);
                    if (id < 0) continue;
                    uint8_t seen;
#pragma omp atomic read
                    seen = flags[id];
                    if (seen) continue;
                    const i64 lo[3] = {bx * W - D, by * W - D, bz * W - D};
                    const i64 hi[3] = {(bx + 1) * W + D, (by + 1) * W + D, (bz + 1) * W + D};
                    if (orc_sat(tr, lo, hi)) {
#pragma omp atomic write
                        flags[id] = 1;
                    }
                }
    }
}

/* ------------------------------------------------------------------ */
/* +x centre lines and their sorted crossings                          */
/* ------------------------------------------------------------------ */
/* Orientation of the perturbed point (py + e^2, pz + e^3) against the y-z projection
 * of the edge U -> V: (V - U)_y (P - U)_z - (V - U)_z (P - U)_y.  Its e^2 coefficient
 * is -(V - U)_z and its e^3 coefficient (V - U)_y. */
static int orient_yz(const i64 *U, const i64 *V, i64 py, i64 pz)
{
    const i64 ey = V[1] - U[1], ez = V[2] - U[2];
    const i64 o = ey * (pz - U[2]) - ez * (py - U[1]);
    if (o) return sg(o);
    if (ez) return -sg(ez);
    return sg(ey);
}

/* Number of centres (2i + 1) half, 0 <= i < ncell, strictly below the x where the
 * line (py, pz) meets the plane of the triangle (normal n, vertex A).  A centre on
 * the plane is not below it: the perturbed centre lies beyond. */
static i64 centres_before(const i64 *A, const i64 *n, i64 py, i64 pz, i64 half, i64 ncell)
{
    /* x_hit = num / den with num = n . A - n_y py - n_z pz, den = n_x */
    i128 num = (i128)n[0] * A[0] + (i128)n[1] * (A[1] - py) + (i128)n[2] * (A[2] - pz);
    i128 den = n[0];
    if (den < 0) {
        num = -num;
        den = -den;
    }
    /* centre i is below x_hit iff (2i + 1) half den < num, i.e. i < (num - half den) / (2 half den) */
    const i128 r = num - (i128)half * den;
    if (r <= 0) return 0;
    const i128 step = (i128)2 * half * den;
    const i128 c = (r + step - 1) / step;
    return c > ncell ? ncell : (i64)c;
}

typedef struct {
    i64 line; /* k ncell + j for the line through centres (y_j, z_k) */
    i64 before;
} Crossing;

static int cmp_crossing(const void *a, const void *b)
{
    const Crossing *x = (const Crossing *)a, *y = (const Crossing *)b;
    if (x->line != y->line) return x->line < y->line ? -1 : 1;
    return (x->before > y->before) - (x->before < y->before);
}

/* Does the perturbed +x line through (py, pz) cross the triangle?  Needs n_x != 0. */
static int xline_hits(const i64 *tr, i64 nx, i64 py, i64 pz)
{
    const int s = sg(nx);
    return orient_yz(tr, tr + 3, py, pz) == s && orient_yz(tr + 3, tr + 6, py, pz) == s &&
           orient_yz(tr + 6, tr, py, pz) == s;
}

/* Crossings of triangle t with the level's +x centre lines; with out != NULL they
 * are written there.  Returns their number. */
static i64 triangle_crossings(const i64 *tr, i64 half, i64 ncell, Crossing *out)
{
    i64 n[3], mn[3], mx[3], j0, j1, k0, k1, w = 0;
    normal_of(tr, n);
    if (n[0] == 0) return 0; /* parallel to every x-line */
    bbox_of(tr, mn, mx);
    centre_range(mn[1], mx[1], half, ncell, &j0, &j1);
    centre_range(mn[2], mx[2], half, ncell, &k0, &k1);
    for (i64 k = k0; k <= k1; ++k)
        for (i64 j = j0; j <= j1; ++j) {
            const i64 py = (2 * j + 1) * half, pz = (2 * k + 1) * half;
            if (!xline_hits(tr, n[0], py, pz)) continue;
            if (out) {
                out[w].line = k * ncell + j;
                out[w].before = centres_before(tr, n, py, pz, half, ncell);
            }
            ++w;
        }
    return w;
}

/* All crossings of the level's +x centre lines, sorted by (line, before). */
static Crossing *collect_crossings(const i64 *tri, i64 T, i64 half, i64 ncell, i64 *count)
{
    i64 *off = (i64 *)malloc(((size_t)T + 1) * sizeof(i64));
#pragma omp parallel for schedule(dynamic, 1024)
    for (i64 t = 0; t < T; ++t) off[t] = triangle_crossings(tri + 9 * t, half, ncell, NULL);
    i64 acc = 0;
    for (i64 t = 0; t < T; ++t) {
        const i64 c = off[t];
        off[t] = acc;
        acc += c;
    }
    Crossing *out = (Crossing *)malloc(((size_t)acc + 1) * sizeof(Crossing));
#pragma omp parallel for schedule(dynamic, 1024)
    for (i64 t = 0; t < T; ++t) triangle_crossings(tri + 9 * t, half, ncell, out + off[t]);
    free(off);
    qsort(out, (size_t)acc, sizeof(Crossing), cmp_crossing);
    *count = acc;
    return out;
}

/* First index in the sorted crossings at or after (line, before). */
static i64 lower_crossing(const Crossing *c, i64 n, i64 line, i64 before)
{
    i64 lo = 0, hi = n;
    while (lo < hi) {
        const i64 mid = lo + (hi - lo) / 2;
        if (c[mid].line < line || (c[mid].line == line && c[mid].before < before)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* Solid state of the centre (x index i) of line `line`: the parity of the crossings
 * with more than i centres before them. */
static int solid_on_line(const Crossing *c, i64 n, i64 line, i64 i)
{
    const i64 end = lower_crossing(c, n, line + 1, -1);
    const i64 beyond = lower_crossing(c, n, line, i + 1);
    return (int)((end - beyond) & 1);
}

/* Solid mask words of the blocks (n x 3 block coordinates) of one level: bit
 * x + 4 y + 16 z of word b is the state of that cell of block b.  Cell size 2 half,
 * ncell cells per axis. */
void orc_lines_masks(const i64 *tri, i64 T, const i64 *blocks, i64 n, i64 half, i64 ncell, uint64_t *out)
{
    i64 nc = 0;
    Crossing *c = collect_crossings(tri, T, half, ncell, &nc);
#pragma omp parallel for schedule(dynamic, 64)
    for (i64 b = 0; b < n; ++b) {
        uint64_t w = 0;
        for (int z = 0; z < 4; ++z)
            for (int y = 0; y < 4; ++y) {
                const i64 line = (4 * blocks[3 * b + 2] + z) * ncell + 4 * blocks[3 * b + 1] + y;
                const i64 start = lower_crossing(c, nc, line, -1), end = lower_crossing(c, nc, line + 1, -1);
                for (int x = 0; x < 4; ++x) {
                    const i64 i = 4 * blocks[3 * b] + x;
                    i64 beyond = 0;
                    for (i64 e = start; e < end; ++e) beyond += c[e].before > i;
                    if (beyond & 1) w |= 1ull << (x + 4 * y + 16 * z);
                }
            }
        out[b] = w;
    }
    free(c);
}

/* ------------------------------------------------------------------ */
/* cut links                                                           */
/* ------------------------------------------------------------------ */
/* Sign of the perturbed Pluecker product c . ((U - P') x (V - P')), P' = P + e:
 * it equals c . ((U - P) x (V - P)) + e . (c x (V - U)). */
static int pluecker(const i64 *U, const i64 *V, const i64 *P, const int *c)
{
    const i64 u0 = U[0] - P[0], u1 = U[1] - P[1], u2 = U[2] - P[2];
    const i64 v0 = V[0] - P[0], v1 = V[1] - P[1], v2 = V[2] - P[2];
    const i64 s = c[0] * (u1 * v2 - u2 * v1) + c[1] * (u2 * v0 - u0 * v2) + c[2] * (u0 * v1 - u1 * v0);
    if (s) return sg(s);
    const i64 d0 = V[0] - U[0], d1 = V[1] - U[1], d2 = V[2] - U[2];
    const i64 w[3] = {c[1] * d2 - c[2] * d1, c[2] * d0 - c[0] * d2, c[0] * d1 - c[1] * d0};
    for (int a = 0; a < 3; ++a)
        if (w[a]) return sg(w[a]);
    return 0;
}

/* Sign of X - n . e (the plane offset seen from a perturbed point). */
static int offset_sign(i128 X, const i64 *n)
{
    if (X) return sg128(X);
    for (int a = 0; a < 3; ++a)
        if (n[a]) return -sg(n[a]);
    return 0;
}

/* Does the perturbed segment P -> P + h c cross the triangle?  On success, the
 * crossing parameter is t = N / (h M) with N >= 0, M > 0. */
static int segment_crosses(const i64 *tr, const i64 *n, const i64 *P, const int *c, i64 h, i128 *N, i64 *M)
{
    const i64 nc = n[0] * c[0] + n[1] * c[1] + n[2] * c[2];
    if (nc == 0) return 0;
    const int s = sg(nc);
    if (pluecker(tr, tr + 3, P, c) != s || pluecker(tr + 3, tr + 6, P, c) != s || pluecker(tr + 6, tr, P, c) != s)
        return 0;
    const i128 D = (i128)n[0] * (tr[0] - P[0]) + (i128)n[1] * (tr[1] - P[1]) + (i128)n[2] * (tr[2] - P[2]);
    if (offset_sign(D, n) != s) return 0;                   /* the plane is not ahead of P */
    if (offset_sign(D - (i128)h * nc, n) != -s) return 0;   /* nor behind P + h c */
    *N = s > 0 ? D : -D;
    *M = s > 0 ? nc : -nc;
    return 1;
}

typedef struct {
    i64 n;          /* links */
    i64 *cell;
    int32_t *dir;
    double *q;
    i64 *tri;
    int32_t *ncross;
} LinkTable;

static LinkTable g_links;

/* The cut links of the finest level (blocks n x 3 ascending by z, y, x; masks from
 * orc_lines_masks; cell size 2 half; ncell cells per axis; lattice 19 or 27).
 * Returns the number of links; orc_lines_links_take copies them out.  A neighbour
 * centre outside the domain is fluid; one in a block the level lacks takes its state
 * from the level's +x lines.  A candidate that no triangle crosses keeps q = -1. */
i64 orc_lines_links(const i64 *tri, i64 T, const i64 *blocks, i64 n, const uint64_t *mask, i64 half, i64 ncell,
                    int lattice)
{
    const i64 h = 2 * half;
    const i64 nbl = ncell / 4;
    i64 *keys = (i64 *)malloc(((size_t)n + 1) * sizeof(i64));
    for (i64 b = 0; b < n; ++b) keys[b] = (blocks[3 * b + 2] * nbl + blocks[3 * b + 1]) * nbl + blocks[3 * b];
    i64 ncr = 0;
    Crossing *cr = collect_crossings(tri, T, half, ncell, &ncr);
    /* candidate directions per cell: fluid cell whose lattice neighbour is solid */
    uint32_t *cand = (uint32_t *)calloc((size_t)n * 64 + 1, sizeof(uint32_t));
#pragma omp parallel for schedule(dynamic, 64)
    for (i64 b = 0; b < n; ++b) {
        i64 nbr[27];
        for (int o = 0; o < 27; ++o) {
            const i64 ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
            const i64 x = blocks[3 * b] + ox, y = blocks[3 * b + 1] + oy, z = blocks[3 * b + 2] + oz;
            nbr[o] = (x < 0 || y < 0 || z < 0 || x >= nbl || y >= nbl || z >= nbl) ? -2
                                                                                   : find_key(keys, n, (z * nbl + y) * nbl + x);
        }
        for (int t = 0; t < 64; ++t) {
            if ((mask[b] >> t) & 1) continue;
            const i64 g[3] = {4 * blocks[3 * b] + (t & 3), 4 * blocks[3 * b + 1] + ((t >> 2) & 3),
                              4 * blocks[3 * b + 2] + (t >> 4)};
            uint32_t m = 0;
            for (int i = 1; i < lattice; ++i) {
                const i64 q[3] = {g[0] + LDIR[i][0], g[1] + LDIR[i][1], g[2] + LDIR[i][2]};
                if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= ncell || q[1] >= ncell || q[2] >= ncell) continue;
                const i64 qb[3] = {fdiv(q[0], 4), fdiv(q[1], 4), fdiv(q[2], 4)};
                const int o = (int)((qb[0] - blocks[3 * b] + 1) + 3 * (qb[1] - blocks[3 * b + 1] + 1) +
                                    9 * (qb[2] - blocks[3 * b + 2] + 1));
                int solid;
                if (nbr[o] >= 0) {
                    const int tt = (int)((q[0] - 4 * qb[0]) + 4 * (q[1] - 4 * qb[1]) + 16 * (q[2] - 4 * qb[2]));
                    solid = (int)((mask[nbr[o]] >> tt) & 1);
                } else {
                    solid = solid_on_line(cr, ncr, q[2] * ncell + q[1], q[0]);
                }
                if (solid) m |= 1u << i;
            }
            cand[b * 64 + t] = m;
        }
    }
    free(cr);
    /* link offsets in (cell, dir) order */
    i64 *off = (i64 *)malloc(((size_t)n * 64 + 1) * sizeof(i64));
    i64 acc = 0;
    for (i64 k = 0; k < n * 64; ++k) {
        off[k] = acc;
        acc += __builtin_popcount(cand[k]);
    }
    off[n * 64] = acc;
    LinkTable L;
    L.n = acc;
    L.cell = (i64 *)malloc(((size_t)acc + 1) * sizeof(i64));
    L.dir = (int32_t *)malloc(((size_t)acc + 1) * sizeof(int32_t));
    L.q = (double *)malloc(((size_t)acc + 1) * sizeof(double));
    L.tri = (i64 *)malloc(((size_t)acc + 1) * sizeof(i64));
    L.ncross = (int32_t *)calloc((size_t)acc + 1, sizeof(int32_t));
    i128 *bestN = (i128 *)malloc(((size_t)acc + 1) * sizeof(i128));
    i64 *bestM = (i64 *)malloc(((size_t)acc + 1) * sizeof(i64));
    for (i64 k = 0; k < n * 64; ++k) {
        uint32_t m = cand[k];
        i64 o = off[k];
        while (m) {
            const int i = __builtin_ctz(m);
            m &= m - 1;
            L.cell[o] = k;
            L.dir[o] = i;
            L.tri[o] = -1;
            bestN[o] = 0;
            bestM[o] = 1;
            ++o;
        }
    }
    /* crossings, one direction per thread: each link is updated by one thread only */
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 1; i < lattice; ++i) {
        const int *c = LDIR[i];
        for (i64 t = 0; t < T; ++t) {
            const i64 *tr = tri + 9 * t;
            i64 nrm[3], mn[3], mx[3], g0[3], g1[3];
            normal_of(tr, nrm);
            if (nrm[0] * c[0] + nrm[1] * c[1] + nrm[2] * c[2] == 0) continue;
            bbox_of(tr, mn, mx);
            /* the segment P -> P + h c meets the bounding box only if P lies in it
             * moved back by h c (per axis) */
            for (int a = 0; a < 3; ++a)
                centre_range(mn[a] - (c[a] > 0 ? h : 0), mx[a] + (c[a] < 0 ? h : 0), half, ncell, &g0[a], &g1[a]);
            for (i64 gz = g0[2]; gz <= g1[2]; ++gz)
                for (i64 gy = g0[1]; gy <= g1[1]; ++gy)
                    for (i64 gx = g0[0]; gx <= g1[0]; ++gx) {
                        const i64 b = find_key(keys, n, ((gz >> 2) * nbl + (gy >> 2)) * nbl + (gx >> 2));
                        if (b < 0) continue;
                        const i64 k = b * 64 + (gx & 3) + 4 * (gy & 3) + 16 * (gz & 3);
                        if (!((cand[k] >> i) & 1)) continue;
                        const i64 P[3] = {(2 * gx + 1) * half, (2 * gy + 1) * half, (2 * gz + 1) * half};
                        i128 N;
                        i64 M;
                        if (!segment_crosses(tr, nrm, P, c, h, &N, &M)) continue;
                        const i64 o = off[k] + __builtin_popcount(cand[k] & ((1u << i) - 1u));
                        L.ncross[o] += 1;
                        /* exact N / M < bestN / bestM; t <= 1 keeps N <= h M, so both
                         * products stay below 2^18 * 2^53 * 2^53 */
                        const i128 lhs = N * (i128)bestM[o], rhs = bestN[o] * (i128)M;
                        if (L.tri[o] < 0 || lhs < rhs || (lhs == rhs && t < L.tri[o])) {
                            bestN[o] = N;
                            bestM[o] = M;
                            L.tri[o] = t;
                        }
                    }
        }
    }
    for (i64 o = 0; o < acc; ++o)
        L.q[o] = L.tri[o] < 0 ? -1.0 : (double)bestN[o] / ((double)bestM[o] * (double)h);
    free(bestN);
    free(bestM);
    free(off);
    free(cand);
    free(keys);
    free(g_links.cell); /* a table that was never taken */
    free(g_links.dir);
    free(g_links.q);
    free(g_links.tri);
    free(g_links.ncross);
    g_links = L;
    return acc;
}

/* Copies the table of the last orc_lines_links call out and releases it. */
void orc_lines_links_take(i64 *cell, int32_t *dir, double *q, i64 *tri, int32_t *ncross)
{
    const size_t n = (size_t)g_links.n;
    memcpy(cell, g_links.cell, n * sizeof(i64));
    memcpy(dir, g_links.dir, n * sizeof(int32_t));
    memcpy(q, g_links.q, n * sizeof(double));
    memcpy(tri, g_links.tri, n * sizeof(i64));
    memcpy(ncross, g_links.ncross, n * sizeof(int32_t));
    free(g_links.cell);
    free(g_links.dir);
    free(g_links.q);
    free(g_links.tri);
    free(g_links.ncross);
    memset(&g_links, 0, sizeof(g_links));
}
