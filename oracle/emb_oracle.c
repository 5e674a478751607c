/*
 * CPU oracle for the mesh-embedding hot path (arXiv 2512.01251, Sec. 3.3-3.4).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * loaded by the tests, by __graft_entry__.smoke() and by the CPU-baseline leg
 * of bench.py.  The product library never links, loads or calls it, and it
 * shares no code, header or table with the CUDA path.
 *
 * Everything here is the plain definition, evaluated by brute force over every
 * triangle for every query:
 *   - a cell is solid iff its centre lies inside the closed oriented surface
 *     (Sec. 3.4 "Partial Surface Voxelization": the centre decides the cell's
 *     type; Sec. 3.2: solid cells have their centre inside the geometry),
 *     decided by the parity of ray crossings (Sec. 3.3.1 names the crossing-count
 *     parity as the usual inside test);
 *   - a cut link runs from a fluid cell centre P to a solid lattice neighbour
 *     P + h c; its length q is the distance along the link to the nearest face
 *     crossing, divided by the link length (Sec. 3.4 "Link-Length Computation");
 *   - a block is flagged for refinement iff some triangle overlaps its closed
 *     box dilated by the near-wall distance (triangle/box overlap by separating
 *     axes, Appendix A).
 *
 * Arithmetic: vertices and query points are integers (the 2^-20 vertex grid
 * scaled so that every cell centre is an integer).  Signs are exact (int64 and
 * __int128).  Ties are broken by simulation of simplicity: every query point P
 * is replaced by P + (e, e^2, e^3) with e -> 0+, so a point never lies on a
 * plane, edge or vertex of the mesh and every decision is unique.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef int64_t i64;
typedef __int128 i128;

/* Lattice directions: 0 rest, 1-6 axes, 7-18 edge diagonals, 19-26 corners,
 * consecutive odd/even indices are opposite. */
static const i64 DIR[27][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
    {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1},
};

static int sgn64(i64 v) { return (v > 0) - (v < 0); }
static int sgn128(i128 v) { return (v > 0) - (v < 0); }

/* Sign of the Pluecker product c . ((A - P') x (B - P')) with P' = P + (e,e^2,e^3).
 * Expanding in e gives  c.((A-P)x(B-P)) + e.(c x (B-A)), so an exact zero is
 * resolved by the components of c x (B - A) in x, y, z order. */
static int plucker_sos(const i64 *A, const i64 *B, const i64 *P, const i64 *c)
{
    i64 a0 = A[0] - P[0], a1 = A[1] - P[1], a2 = A[2] - P[2];
    i64 b0 = B[0] - P[0], b1 = B[1] - P[1], b2 = B[2] - P[2];
    i64 m0 = a1 * b2 - a2 * b1;
    i64 m1 = a2 * b0 - a0 * b2;
    i64 m2 = a0 * b1 - a1 * b0;
    i64 s = c[0] * m0 + c[1] * m1 + c[2] * m2;
    if (s) return sgn64(s);
    i64 d0 = B[0] - A[0], d1 = B[1] - A[1], d2 = B[2] - A[2];
    i64 w0 = c[1] * d2 - c[2] * d1;
    i64 w1 = c[2] * d0 - c[0] * d2;
    i64 w2 = c[0] * d1 - c[1] * d0;
    if (w0) return sgn64(w0);
    if (w1) return sgn64(w1);
    return sgn64(w2);
}

static void tri_normal(const i64 *A, const i64 *B, const i64 *C, i64 *n)
{
    i64 u0 = B[0] - A[0], u1 = B[1] - A[1], u2 = B[2] - A[2];
    i64 v0 = C[0] - A[0], v1 = C[1] - A[1], v2 = C[2] - A[2];
    n[0] = u1 * v2 - u2 * v1;
    n[1] = u2 * v0 - u0 * v2;
    n[2] = u0 * v1 - u1 * v0;
}

/* Sign of (D - n.e): the exact value when D != 0, else minus the sign of the
 * first non-zero normal component (x, then y, then z). */
static int side_sos(i128 D, const i64 *n)
{
    if (D) return sgn128(D);
    if (n[0]) return -sgn64(n[0]);
    if (n[1]) return -sgn64(n[1]);
    return -sgn64(n[2]);
}

/* Does the perturbed line through P with direction c pass through triangle
 * (A,B,C)?  On success returns 1 and gives the normal n and n.c. */
static int line_hits(const i64 *A, const i64 *B, const i64 *C, const i64 *P, const i64 *c,
                     i64 *n, i64 *nc)
{
    tri_normal(A, B, C, n);
    *nc = n[0] * c[0] + n[1] * c[1] + n[2] * c[2];
    if (*nc == 0) return 0; /* a line parallel to the plane never crosses it */
    int s1 = plucker_sos(A, B, P, c);
    int s2 = plucker_sos(B, C, P, c);
    int s3 = plucker_sos(C, A, P, c);
    return s1 == s2 && s2 == s3;
}

static i128 plane_offset(const i64 *n, const i64 *A, const i64 *P)
{
    return (i128)n[0] * (A[0] - P[0]) + (i128)n[1] * (A[1] - P[1]) + (i128)n[2] * (A[2] - P[2]);
}

/* Parity of the crossings of the perturbed ray {P' + s c : s > 0}. */
static int ray_parity(const i64 *tri, i64 T, const i64 *P, const i64 *c)
{
    int par = 0;
    for (i64 t = 0; t < T; ++t) {
        const i64 *A = tri + 9 * t, *B = A + 3, *C = A + 6;
        i64 n[3], nc;
        if (!line_hits(A, B, C, P, c, n, &nc)) continue;
        i128 D = plane_offset(n, A, P);
        if (side_sos(D, n) == sgn64(nc)) par ^= 1; /* crossing at s > 0 */
    }
    return par;
}

/* Crossing of the perturbed segment P' -> P' + h c with a triangle.
 * Returns 1 and the exact parameter t = N / (h M) with N >= 0, M > 0. */
static int segment_hit(const i64 *A, const i64 *B, const i64 *C, const i64 *P, const i64 *c, i64 h,
                       i128 *N, i128 *M)
{
    i64 n[3], nc;
    if (!line_hits(A, B, C, P, c, n, &nc)) return 0;
    i128 D = plane_offset(n, A, P);
    int snc = sgn64(nc);
    if (side_sos(D, n) != snc) return 0;                       /* t <= 0 */
    if (side_sos(D - (i128)h * nc, n) != -snc) return 0;       /* t >= 1 */
    *N = snc > 0 ? D : -D;
    *M = snc > 0 ? (i128)nc : -(i128)nc;
    return 1;
}

/* ---------------------------------------------------------------------- */
/* triangle / closed axis-aligned box overlap by separating axes           */
/* ---------------------------------------------------------------------- */
static i128 abs128(i128 v) { return v < 0 ? -v : v; }

/* Axis a separates iff the triangle's projection lies strictly outside the
 * box's projection [-r, r] (coordinates relative to the box centre). */
static int axis_separates(const i128 *a, const i128 v[3][3], const i128 *e)
{
    i128 p0 = a[0] * v[0][0] + a[1] * v[0][1] + a[2] * v[0][2];
    i128 p1 = a[0] * v[1][0] + a[1] * v[1][1] + a[2] * v[1][2];
    i128 p2 = a[0] * v[2][0] + a[1] * v[2][1] + a[2] * v[2][2];
    i128 lo = p0, hi = p0;
    if (p1 < lo) lo = p1;
    if (p1 > hi) hi = p1;
    if (p2 < lo) lo = p2;
    if (p2 > hi) hi = p2;
    i128 r = e[0] * abs128(a[0]) + e[1] * abs128(a[1]) + e[2] * abs128(a[2]);
    return lo > r || hi < -r;
}

int orc_sat(const i64 *tri, const i64 *lo, const i64 *hi)
{
    /* doubled coordinates so that the box centre is an integer */
    i128 v[3][3], e[3];
    for (int d = 0; d < 3; ++d) e[d] = (i128)hi[d] - lo[d];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) v[k][d] = 2 * (i128)tri[3 * k + d] - ((i128)lo[d] + hi[d]);
    /* box face normals */
    for (int d = 0; d < 3; ++d) {
        i128 a[3] = {0, 0, 0};
        a[d] = 1;
        if (axis_separates(a, v, e)) return 0;
    }
    i128 f[3][3];
    for (int d = 0; d < 3; ++d) {
        f[0][d] = v[1][d] - v[0][d];
        f[1][d] = v[2][d] - v[1][d];
        f[2][d] = v[0][d] - v[2][d];
    }
    /* triangle normal */
    i128 n[3] = {f[0][1] * f[1][2] - f[0][2] * f[1][1], f[0][2] * f[1][0] - f[0][0] * f[1][2],
                 f[0][0] * f[1][1] - f[0][1] * f[1][0]};
    if (axis_separates(n, v, e)) return 0;
    /* box edge directions crossed with triangle edges */
    for (int d = 0; d < 3; ++d) {
        for (int j = 0; j < 3; ++j) {
            i128 u[3] = {0, 0, 0};
            u[d] = 1;
            i128 a[3] = {u[1] * f[j][2] - u[2] * f[j][1], u[2] * f[j][0] - u[0] * f[j][2],
                         u[0] * f[j][1] - u[1] * f[j][0]};
            if (axis_separates(a, v, e)) return 0;
        }
    }
    return 1;
}

/* ---------------------------------------------------------------------- */
/* exported batch entry points (OpenMP over queries)                       */
/* ---------------------------------------------------------------------- */

void orc_directions(int32_t *out /* 27 x 3 */)
{
    for (int i = 0; i < 27; ++i)
        for (int d = 0; d < 3; ++d) out[3 * i + d] = (int32_t)DIR[i][d];
}

/* out[i] = parity of crossings of the perturbed ray from pts[i] along DIR[dir]. */
void orc_solid(const i64 *tri, i64 T, const i64 *pts, i64 N, int dir, uint8_t *out)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (i64 i = 0; i < N; ++i) out[i] = (uint8_t)ray_parity(tri, T, pts + 3 * i, DIR[dir]);
}

/* For each query (P, dir): the nearest crossing of the segment P -> P + h c.
 * q[i] = t in FP64 (or -1 if no triangle is crossed), arg[i] = triangle id
 * (lowest id among exactly equal t), ncross[i] = number of crossings. */
void orc_links(const i64 *tri, i64 T, const i64 *pts, const int32_t *dirs, i64 N, i64 h, double *q,
               i64 *arg, int32_t *ncross)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (i64 i = 0; i < N; ++i) {
        const i64 *P = pts + 3 * i;
        const i64 *c = DIR[dirs[i]];
        i128 bestN = 0, bestM = 1;
        i64 best = -1;
        int cnt = 0;
        for (i64 t = 0; t < T; ++t) {
            const i64 *A = tri + 9 * t;
            i128 Nn, Mm;
            if (!segment_hit(A, A + 3, A + 6, P, c, h, &Nn, &Mm)) continue;
            ++cnt;
            /* exact comparison of Nn/Mm < bestN/bestM; both products stay below 2^125 */
            if (best < 0 || Nn * bestM < bestN * Mm) {
                bestN = Nn;
                bestM = Mm;
                best = t;
            }
        }
        arg[i] = best;
        ncross[i] = cnt;
        q[i] = best < 0 ? -1.0 : (double)bestN / ((double)bestM * (double)h);
    }
}

/* out[i] = 1 iff some triangle overlaps the closed box [lo_i, hi_i]. */
void orc_boxes_any(const i64 *tri, i64 T, const i64 *lo, const i64 *hi, i64 N, uint8_t *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (i64 i = 0; i < N; ++i) {
        uint8_t any = 0;
        for (i64 t = 0; t < T && !any; ++t) any = (uint8_t)orc_sat(tri + 9 * t, lo + 3 * i, hi + 3 * i);
        out[i] = any;
    }
}

/* Single (triangle, segment) query used by the closed-form checks. */
int orc_segment_hit(const i64 *tri9, const i64 *P, int dir, i64 h, double *t_out)
{
    i128 N, M;
    if (!segment_hit(tri9, tri9 + 3, tri9 + 6, P, DIR[dir], h, &N, &M)) return 0;
    *t_out = (double)N / ((double)M * (double)h);
    return 1;
}

/* Single (triangle, line) query: does the perturbed line through P along DIR[dir] cross it? */
int orc_line_hits(const i64 *tri9, const i64 *P, int dir)
{
    i64 n[3], nc;
    return line_hits(tri9, tri9 + 3, tri9 + 6, P, DIR[dir], n, &nc);
}

/* out[i * T + t] = 1 iff triangle t overlaps the closed box [lo_i, hi_i]: the
 * (box, triangle) incidence of the per-block bins (Alg. 2). */
void orc_box_pairs(const i64 *tri, i64 T, const i64 *lo, const i64 *hi, i64 N, uint8_t *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (i64 i = 0; i < N; ++i)
        for (i64 t = 0; t < T; ++t) out[i * T + t] = (uint8_t)orc_sat(tri + 9 * t, lo + 3 * i, hi + 3 * i);
}

/* ---------------------------------------------------------------------- */
/* The paper's guard-cell voxelizer (Sec. 3.4, "Partial Surface            */
/* Voxelization", Alg. 3): single-precision nearest-hit classification of  */
/* each cell from the faces of its block's bin.  Plain IEEE binary32        */
/* arithmetic, one rounding per operation in the order written (the file is */
/* compiled with -ffp-contract=off, so no multiply-add is fused).           */
/* ---------------------------------------------------------------------- */
#define GUARD_EPS 1.1920928955078125e-7f /* 2^-23, the binary32 machine epsilon */

/* Does the face (yz projection a, b, c) touch the thin box around the x-line
 * through (py, pz)?  The box spans the domain along x, so only the axes of the
 * yz projection can separate: y, z and the three edge normals.  Half-width in y
 * and z: GUARD_EPS.  Touching counts as overlap. */
static int guard_in_face(const float *ty, const float *tz, float py, float pz)
{
    float y[3], z[3];
    for (int i = 0; i < 3; ++i) {
        y[i] = ty[i] - py;
        z[i] = tz[i] - pz;
    }
    float ylo = y[0], yhi = y[0], zlo = z[0], zhi = z[0];
    for (int i = 1; i < 3; ++i) {
        if (y[i] < ylo) ylo = y[i];
        if (y[i] > yhi) yhi = y[i];
        if (z[i] < zlo) zlo = z[i];
        if (z[i] > zhi) zhi = z[i];
    }
    if (ylo > GUARD_EPS || yhi < -GUARD_EPS) return 0;
    if (zlo > GUARD_EPS || zhi < -GUARD_EPS) return 0;
    for (int i = 0; i < 3; ++i) {
        int k = (i + 1) % 3;
        float ey = y[k] - y[i];
        float ez = z[k] - z[i];
        float r = GUARD_EPS * (fabsf(ey) + fabsf(ez));
        float lo = 0.0f, hi = 0.0f;
        for (int m = 0; m < 3; ++m) {
            float p = z[m] * ey - y[m] * ez; /* projection on the edge normal (-ez, ey) */
            if (m == 0 || p < lo) lo = p;
            if (m == 0 || p > hi) hi = p;
        }
        if (lo > r || hi < -r) return 0;
    }
    return 1;
}

/* state[i * 64 + t] for cell t of block i (t = x + 4 y + 16 z): 0 no face hit,
 * 1 solid, 2 guard.  Cell centre (2 g + 1) / (2 n) per axis (n cells per axis,
 * g the global cell index), one division.  Faces in ascending id order from the
 * CSR bins; for each, the unit normal n = (v2 - v1) x (v3 - v1) / |...|, the
 * signed distance d = ((v1 - c) . n) / n_x along x, and the point-in-face test;
 * the nearest accepted face (strictly smaller |d|, starting from 1) decides:
 * solid if n_x d > 0, guard otherwise. */
void orc_guard_surface(const float *verts, const int32_t *tris, const i64 *blocks, i64 N, const i64 *off,
                       const i64 *ent, i64 ncell, uint8_t *state)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (i64 i = 0; i < N; ++i) {
        for (int t = 0; t < 64; ++t) {
            i64 g[3] = {4 * blocks[3 * i] + (t & 3), 4 * blocks[3 * i + 1] + ((t >> 2) & 3),
                        4 * blocks[3 * i + 2] + (t >> 4)};
            float c[3];
            for (int a = 0; a < 3; ++a) c[a] = (float)(2 * g[a] + 1) / (float)(2 * ncell);
            float dmin = 1.0f;
            int st = 0;
            for (i64 e = off[i]; e < off[i + 1]; ++e) {
                const int32_t *tv = tris + 3 * ent[e];
                const float *v1 = verts + 3 * tv[0], *v2 = verts + 3 * tv[1], *v3 = verts + 3 * tv[2];
                float u[3] = {v2[0] - v1[0], v2[1] - v1[1], v2[2] - v1[2]};
                float w[3] = {v3[0] - v1[0], v3[1] - v1[1], v3[2] - v1[2]};
                float n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
                float len = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                for (int a = 0; a < 3; ++a) n[a] = n[a] / len;
                float d = ((v1[0] - c[0]) * n[0] + (v1[1] - c[1]) * n[1] + (v1[2] - c[2]) * n[2]) / n[0];
                if (!(fabsf(d) < dmin)) continue;
                float ty[3] = {v1[1], v2[1], v3[1]}, tz[3] = {v1[2], v2[2], v3[2]};
                if (!guard_in_face(ty, tz, c[1], c[2])) continue;
                dmin = fabsf(d);
                st = n[0] * d > 0.0f ? 1 : 2;
            }
            state[i * 64 + t] = (uint8_t)st;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* one triangle per query (tests of single decisions in bulk)              */
/* ---------------------------------------------------------------------- */
/* out[i] = the perturbed line through pts[i] along DIR[dirs[i]] crosses triangle tri[i]. */
void orc_each_line(const i64 *tri, const i64 *pts, const int32_t *dirs, i64 N, uint8_t *out)
{
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < N; ++i) {
        i64 n[3], nc;
        const i64 *A = tri + 9 * i;
        out[i] = (uint8_t)line_hits(A, A + 3, A + 6, pts + 3 * i, DIR[dirs[i]], n, &nc);
    }
}

/* hit[i] = the perturbed segment pts[i] -> pts[i] + h[i] DIR[dirs[i]] crosses triangle
 * tri[i]; t[i] = its parameter in FP64 (-1 if not). */
void orc_each_segment(const i64 *tri, const i64 *pts, const int32_t *dirs, const i64 *h, i64 N, uint8_t *hit,
                      double *t)
{
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < N; ++i) {
        i128 Nn, Mm;
        const i64 *A = tri + 9 * i;
        hit[i] = (uint8_t)segment_hit(A, A + 3, A + 6, pts + 3 * i, DIR[dirs[i]], h[i], &Nn, &Mm);
        t[i] = hit[i] ? (double)Nn / ((double)Mm * (double)h[i]) : -1.0;
    }
}

/* out[i] = triangle tri[i] overlaps the closed box [lo[i], hi[i]]. */
void orc_each_box(const i64 *tri, const i64 *lo, const i64 *hi, i64 N, uint8_t *out)
{
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < N; ++i) out[i] = (uint8_t)orc_sat(tri + 9 * i, lo + 3 * i, hi + 3 * i);
}
