/*
 * fhv_oracle.c -- plain, slow, sequential CPU oracle for fragment-history
 * volumes (Inacio & Springer, "Fragment-History Volumes", arXiv 2211.15460).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library calls, links or includes
 * this file; it exists so tests, the smoke check and the benchmark's CPU
 * baseline can check the CUDA path. It shares no code, header or table with
 * the CUDA sources.
 *
 * What it computes, step by step, in the paper's order:
 *   - every fragment the rasteriser produces for every triangle (Section 3.2),
 *     by brute force over each triangle's bounding box of samples, in
 *     (triangle, row, column) order;
 *   - per-pixel linked lists (FHV_PPFL, Section 3.1 "Simple Layout", Fig. 3):
 *     a global counter gives the slot, the pixel array keeps the last index,
 *     each record links to the previous one, -1 marks the end;
 *   - per-octant linked lists (FHV_POFL, Section 3.1 "Octree Layout", Fig. 5):
 *     the same insertion keyed by the Morton code of the leaf octant, plus the
 *     coarser levels' child-occupancy masks;
 *   - per-octant arrays (FHV_POFA, Section 3.1 / 3.2, Fig. 6): fragments
 *     grouped by octant in Morton order, with (offset, count) per octant;
 *   - point splatting for a novel viewpoint keeping the fragment nearest to
 *     the viewer, then local illumination (Section 3.3, Section 5);
 *   - ray casting (Section 3.3, Table 3): per pixel, every fragment on the
 *     pixel's ray, nearest first, composited with per-material opacity.
 *
 * Readings where the paper is silent (fixed here and in the CUDA path alike;
 * both are written independently from the same statement):
 *   - positions are stored as 21-bit cube-quantised integers and interpolated
 *     with exact integer barycentrics (round half up);
 *   - the rasteriser snaps vertices to 1/256 pixel (round half to even),
 *     samples at pixel centres and uses a top-left fill rule;
 *   - tangent-space (1-Pass/Normal, Section 3.2, Fig. 8) rasterisation uses a
 *     per-triangle lattice anchored at the triangle's first vertex; the
 *     three-axis capture (3-Pass/1-Way, Fig. 7) a lattice per axis anchored
 *     at the cube corner;
 *   - normals are interpolated in float32 in a fixed order and stored
 *     octahedrally encoded as two snorm16 values;
 *   - the fragment record is 16 bytes: 63-bit Morton code of the quantised
 *     position, triangle id (material and object ids follow from it), normal;
 *   - POFA orders fragments inside an octant by the full record key;
 *   - the splat visibility key is (24-bit quantised depth << 40) | index;
 *   - a fragment lies on a pixel's ray when its projection falls in that
 *     pixel (the k = 1 splat rule); front-to-back order is the key order.
 * Float steps that decide integers run in float32 with every operation
 * rounded separately (compile with -ffp-contract=off); shading runs in fp64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define QBITS 21
#define QMAX ((1u << QBITS) - 1u)
#define IDX_BITS 40
#define QD_MAX ((1u << 24) - 1u)

typedef struct {
    const uint32_t *idx;          /* 3 * n_tri vertex indices */
    const float *pos;             /* 3 * n_vtx */
    const float *nrm;             /* 3 * n_vtx */
    const uint32_t *tri_material; /* n_tri */
    uint32_t n_tri, n_vtx;
    float cube_min[3];
    float cube_side;
} orc_scene;

typedef struct {
    float origin[3], right[3], up[3], fwd[3];
    float pitch;
    int32_t width, height;
    float z0, z1;
} orc_camera;

typedef struct {
    uint64_t key; /* Morton code of the quantised position */
    uint32_t tri;
    uint32_t nrm; /* octahedral snorm16 x | y << 16 */
} orc_record;

/* ------------------------------------------------------------------ helpers */

/* Morton / Z-order code (Section 3.1, Fig. 5): bit k of x, y, z goes to bit
 * 3k+2, 3k+1, 3k of the code, so x is the most significant of each triple. */
uint64_t orc_morton63(uint32_t x, uint32_t y, uint32_t z)
{
    uint64_t m = 0;
    for (int k = 0; k < QBITS; ++k) {
        m |= (uint64_t)((x >> k) & 1u) << (3 * k + 2);
        m |= (uint64_t)((y >> k) & 1u) << (3 * k + 1);
        m |= (uint64_t)((z >> k) & 1u) << (3 * k);
    }
    return m;
}

static int64_t floordiv(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

static int64_t ceildiv(int64_t a, int64_t b) { return -floordiv(-a, b); }

static float dot3f(const float a[3], const float b[3])
{
    float xx = a[0] * b[0];
    float yy = a[1] * b[1];
    float zz = a[2] * b[2];
    float s = xx + yy;
    return s + zz;
}

static void cross3f(const float a[3], const float b[3], float out[3])
{
    float x1 = a[1] * b[2], x2 = a[2] * b[1];
    float y1 = a[2] * b[0], y2 = a[0] * b[2];
    float z1 = a[0] * b[1], z2 = a[1] * b[0];
    out[0] = x1 - x2;
    out[1] = y1 - y2;
    out[2] = z1 - z2;
}

/* Cube quantisation of one coordinate: floor((p - min) * (2^21 / side)),
 * clamped to [0, 2^21 - 1]. */
static uint32_t quantize1(float p, float cmin, float qscale)
{
    float t = p - cmin;
    float u = t * qscale;
    float f = floorf(u);
    if (!(f >= 0.0f)) return 0u;
    if (f >= (float)QMAX) return QMAX;
    return (uint32_t)f;
}

/* Snap a coordinate in pixel units to 1/256 fixed point, guard band +-2^16 px,
 * round half to even. */
static int32_t snap256(float s)
{
    float v = s * 256.0f;
    v = fmaxf(v, -16777216.0f);
    v = fminf(v, 16777216.0f);
    return (int32_t)rintf(v);
}

/* The normal field of the 16-byte record (the fragment normal of Section
 * 3.1, compressed): octahedral mapping of the unit vector to the square
 * (Cigolle et al. 2014, "A Survey of Efficient Representations for
 * Independent Unit Vectors"), each coordinate rounded to snorm16. */
uint32_t orc_oct_encode(float nx, float ny, float nz)
{
    float ax = fabsf(nx), ay = fabsf(ny), az = fabsf(nz);
    float l1 = (ax + ay) + az;
    float px = 0.0f, py = 0.0f;
    if (l1 > 0.0f) {
        px = nx / l1;
        py = ny / l1;
        if (nz < 0.0f) {
            float sx = px >= 0.0f ? 1.0f : -1.0f;
            float sy = py >= 0.0f ? 1.0f : -1.0f;
            float qx = (1.0f - fabsf(py)) * sx;
            float qy = (1.0f - fabsf(px)) * sy;
            px = qx;
            py = qy;
        }
    }
    px = fminf(fmaxf(px, -1.0f), 1.0f);
    py = fminf(fmaxf(py, -1.0f), 1.0f);
    int32_t ex = (int32_t)rintf(px * 32767.0f);
    int32_t ey = (int32_t)rintf(py * 32767.0f);
    return (uint32_t)(uint16_t)(int16_t)ex | ((uint32_t)(uint16_t)(int16_t)ey << 16);
}

/* Inverse of the encoding, in double, normalised. */
void orc_oct_decode(uint32_t code, double out[3])
{
    double x = (double)(int16_t)(uint16_t)(code & 0xFFFFu) / 32767.0;
    double y = (double)(int16_t)(uint16_t)(code >> 16) / 32767.0;
    double z = 1.0 - fabs(x) - fabs(y);
    if (z < 0.0) {
        double qx = (1.0 - fabs(y)) * (x >= 0.0 ? 1.0 : -1.0);
        double qy = (1.0 - fabs(x)) * (y >= 0.0 ? 1.0 : -1.0);
        x = qx;
        y = qy;
    }
    double l = sqrt(x * x + y * y + z * z);
    out[0] = x / l;
    out[1] = y / l;
    out[2] = z / l;
}

/* ------------------------------------------------------------ rasterisation */

enum { ORC_VIEW = 0, ORC_NORMAL = 1, ORC_AXIS3 = 2 };

typedef void (*orc_emit_fn)(void *ctx, const orc_record *r, int64_t i, int64_t j);

/* One triangle in 2-D fixed point with its quantised positions and normals. */
typedef struct {
    int64_t X[3], Y[3];
    uint32_t Q[3][3];
    float N[3][3];
} orc_tri2d;

static int edge_is_top_left(int64_t dx, int64_t dy) { return dy < 0 || (dy == 0 && dx < 0); }

/* Rasterise one triangle: all samples (i + 1/2, j + 1/2) inside it, row by row.
 * Inside: every edge function positive, or zero on a top or left edge. */
static void raster_tri(orc_tri2d t, int clip, int32_t W, int32_t H, uint32_t tri_id, orc_emit_fn emit, void *ctx)
{
    int64_t A = (t.X[1] - t.X[0]) * (t.Y[2] - t.Y[0]) - (t.Y[1] - t.Y[0]) * (t.X[2] - t.X[0]);
    if (A == 0) return;
    if (A < 0) { /* make the winding counter-clockwise (y up) */
        orc_tri2d s = t;
        s.X[1] = t.X[2]; s.Y[1] = t.Y[2];
        s.X[2] = t.X[1]; s.Y[2] = t.Y[1];
        memcpy(s.Q[1], t.Q[2], sizeof s.Q[1]);
        memcpy(s.Q[2], t.Q[1], sizeof s.Q[2]);
        memcpy(s.N[1], t.N[2], sizeof s.N[1]);
        memcpy(s.N[2], t.N[1], sizeof s.N[2]);
        t = s;
        A = -A;
    }
    int64_t minX = t.X[0], maxX = t.X[0], minY = t.Y[0], maxY = t.Y[0];
    for (int v = 1; v < 3; ++v) {
        if (t.X[v] < minX) minX = t.X[v];
        if (t.X[v] > maxX) maxX = t.X[v];
        if (t.Y[v] < minY) minY = t.Y[v];
        if (t.Y[v] > maxY) maxY = t.Y[v];
    }
    int64_t i0 = ceildiv(minX - 128, 256), i1 = floordiv(maxX - 128, 256);
    int64_t j0 = ceildiv(minY - 128, 256), j1 = floordiv(maxY - 128, 256);
    if (clip) {
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > W - 1) i1 = W - 1;
        if (j1 > H - 1) j1 = H - 1;
    }
    /* edge k is opposite vertex k: (1->2), (2->0), (0->1) */
    static const int ea[3] = {1, 2, 0}, eb[3] = {2, 0, 1};
    for (int64_t j = j0; j <= j1; ++j) {
        for (int64_t i = i0; i <= i1; ++i) {
            int64_t sx = 256 * i + 128, sy = 256 * j + 128;
            int64_t w[3];
            int inside = 1;
            for (int k = 0; k < 3; ++k) {
                int64_t dx = t.X[eb[k]] - t.X[ea[k]];
                int64_t dy = t.Y[eb[k]] - t.Y[ea[k]];
                w[k] = dx * (sy - t.Y[ea[k]]) - dy * (sx - t.X[ea[k]]);
                if (!(w[k] > 0 || (w[k] == 0 && edge_is_top_left(dx, dy)))) inside = 0;
            }
            if (!inside) continue;
            /* position: exact barycentric combination, rounded half up */
            uint32_t q[3];
            for (int c = 0; c < 3; ++c) {
                __int128 num = 0;
                for (int k = 0; k < 3; ++k) num += (__int128)w[k] * (__int128)t.Q[k][c];
                q[c] = (uint32_t)((2 * num + A) / (2 * (__int128)A));
            }
            /* normal: float32 weights times vertex normals, fixed order */
            float fw[3] = {(float)w[0], (float)w[1], (float)w[2]};
            float n[3];
            for (int c = 0; c < 3; ++c) {
                float a0 = fw[0] * t.N[0][c];
                float a1 = fw[1] * t.N[1][c];
                float a2 = fw[2] * t.N[2][c];
                float s = a0 + a1;
                n[c] = s + a2;
            }
            orc_record r;
            r.key = orc_morton63(q[0], q[1], q[2]);
            r.tri = tri_id;
            r.nrm = orc_oct_encode(n[0], n[1], n[2]);
            emit(ctx, &r, i, j);
        }
    }
}

/* Vertex stage: quantise, then project with the capture view (1-Pass/View),
 * with the triangle's own tangent frame (1-Pass/Normal), or along one main
 * axis (3-Pass/1-Way, Fig. 7: axis a looks along world axis a; the 2-D
 * coordinates are the other two axes in cyclic order, (a+1)%3 then (a+2)%3,
 * measured from the cube corner in units of pitch). Returns 0 for a
 * triangle with no tangent frame. */
static int setup_tri(const orc_scene *sc, uint32_t t, int mode, int axis, const orc_camera *cam, float pitch,
                     orc_tri2d *out)
{
    float qscale = 2097152.0f / sc->cube_side;
    float p[3][3];
    for (int v = 0; v < 3; ++v) {
        uint32_t vi = sc->idx[3 * (size_t)t + v];
        for (int c = 0; c < 3; ++c) {
            p[v][c] = sc->pos[3 * (size_t)vi + c];
            out->N[v][c] = sc->nrm[3 * (size_t)vi + c];
            out->Q[v][c] = quantize1(p[v][c], sc->cube_min[c], qscale);
        }
    }
    if (mode == ORC_VIEW) {
        float inv_pitch = 1.0f / cam->pitch;
        float hw = 0.5f * (float)cam->width, hh = 0.5f * (float)cam->height;
        for (int v = 0; v < 3; ++v) {
            float d[3] = {p[v][0] - cam->origin[0], p[v][1] - cam->origin[1], p[v][2] - cam->origin[2]};
            float sx = dot3f(d, cam->right) * inv_pitch + hw;
            float sy = dot3f(d, cam->up) * inv_pitch + hh;
            out->X[v] = snap256(sx);
            out->Y[v] = snap256(sy);
        }
        return 1;
    }
    if (mode == ORC_AXIS3) {
        float inv_h = 1.0f / pitch;
        int cu = (axis + 1) % 3, cv = (axis + 2) % 3;
        for (int v = 0; v < 3; ++v) {
            float du = p[v][cu] - sc->cube_min[cu];
            float dv = p[v][cv] - sc->cube_min[cv];
            out->X[v] = snap256(du * inv_h);
            out->Y[v] = snap256(dv * inv_h);
        }
        return 1;
    }
    /* tangent frame: t = e1/|e1|, n = (e1 x e2)/|e1 x e2|, b = n x t */
    float e1[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
    float e2[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
    float n[3];
    cross3f(e1, e2, n);
    float le = sqrtf(dot3f(e1, e1));
    float ln = sqrtf(dot3f(n, n));
    if (!(le > 0.0f) || !(ln > 0.0f)) return 0;
    float tt[3] = {e1[0] / le, e1[1] / le, e1[2] / le};
    float nn[3] = {n[0] / ln, n[1] / ln, n[2] / ln};
    float bb[3];
    cross3f(nn, tt, bb);
    float inv_h = 1.0f / pitch;
    out->X[0] = 0;
    out->Y[0] = 0;
    out->X[1] = snap256(dot3f(e1, tt) * inv_h);
    out->Y[1] = snap256(dot3f(e1, bb) * inv_h);
    out->X[2] = snap256(dot3f(e2, tt) * inv_h);
    out->Y[2] = snap256(dot3f(e2, bb) * inv_h);
    return 1;
}

/* Enumerate all fragments of the scene in (triangle, [axis,] row, column) order. */
static void raster_scene(const orc_scene *sc, int mode, const orc_camera *cam, float pitch, orc_emit_fn emit, void *ctx)
{
    int passes = mode == ORC_AXIS3 ? 3 : 1;
    for (uint32_t t = 0; t < sc->n_tri; ++t) {
        for (int axis = 0; axis < passes; ++axis) {
            orc_tri2d tri;
            if (!setup_tri(sc, t, mode, axis, cam, pitch, &tri)) continue;
            raster_tri(tri, mode == ORC_VIEW, mode == ORC_VIEW ? cam->width : 0, mode == ORC_VIEW ? cam->height : 0,
                       t, emit, ctx);
        }
    }
}

/* ---------------------------------------------------- plain fragment stream */

typedef struct {
    orc_record *rec;
    int64_t *si, *sj;
    uint64_t cap, count;
} stream_ctx;

static void emit_stream(void *vctx, const orc_record *r, int64_t i, int64_t j)
{
    stream_ctx *c = (stream_ctx *)vctx;
    if (c->count < c->cap) {
        if (c->rec) c->rec[c->count] = *r;
        if (c->si) c->si[c->count] = i;
        if (c->sj) c->sj[c->count] = j;
    }
    c->count++;
}

/* All fragments with their sample coordinates; returns the total number
 * (entries beyond `cap` are counted but not written). */
uint64_t orc_fragments(const orc_scene *sc, int mode, const orc_camera *cam, float pitch, orc_record *rec,
                       int64_t *si, int64_t *sj, uint64_t cap)
{
    stream_ctx c = {rec, si, sj, cap, 0};
    raster_scene(sc, mode, cam, pitch, emit_stream, &c);
    return c.count;
}

/* ------------------------------------------------------------ PPFL / POFL */

typedef struct {
    int32_t *head;
    orc_record *rec;
    int32_t *next;
    uint64_t cap, count;
    int keymode; /* 0: pixel, 1: leaf octant */
    int32_t W;
    int depth;
} list_ctx;

/* Insertion of Section 3.2: take the next index from the global counter;
 * if it is below the pre-allocated size, write the record, store the old
 * head as the record's previous index and make the new index the head. */
static void emit_list(void *vctx, const orc_record *r, int64_t i, int64_t j)
{
    list_ctx *c = (list_ctx *)vctx;
    uint64_t slot = c->keymode == 0 ? (uint64_t)(j * c->W + i) : (r->key >> (63 - 3 * c->depth));
    uint64_t n = c->count++;
    if (n < c->cap) {
        c->rec[n] = *r;
        c->next[n] = c->head[slot];
        c->head[slot] = (int32_t)n;
    }
}

/* FHV_PPFL with the capture view. head: W*H, set to -1 here. */
uint64_t orc_ppfl(const orc_scene *sc, const orc_camera *cam, int32_t *head, orc_record *rec, int32_t *next,
                  uint64_t cap)
{
    for (int64_t p = 0; p < (int64_t)cam->width * cam->height; ++p) head[p] = -1;
    list_ctx c = {head, rec, next, cap, 0, 0, cam->width, 0};
    raster_scene(sc, ORC_VIEW, cam, 0.0f, emit_list, &c);
    return c.count;
}

/* Levels of the octree concatenated root first (Section 3.1, Fig. 6): level
 * l starts after the 8^0 + ... + 8^(l-1) octants above it. */
static uint64_t level_base(int l) { return (((uint64_t)1 << (3 * l)) - 1) / 7; }

/* FHV_POFL: leaf heads (8^depth, set to -1 here) and the child-occupancy
 * masks of levels 0..depth-1 (root first), bit c of octant o at level l set
 * when child 8o+c holds a stored fragment. */
uint64_t orc_pofl(const orc_scene *sc, int mode, const orc_camera *cam, float pitch, int depth, int32_t *leaf_head,
                  uint32_t *levels, orc_record *rec, int32_t *next, uint64_t cap)
{
    uint64_t nleaf = (uint64_t)1 << (3 * depth);
    for (uint64_t k = 0; k < nleaf; ++k) leaf_head[k] = -1;
    for (uint64_t k = 0; k < level_base(depth); ++k) levels[k] = 0;
    list_ctx c = {leaf_head, rec, next, cap, 0, 1, 0, depth};
    raster_scene(sc, mode, cam, pitch, emit_list, &c);
    uint64_t stored = c.count < cap ? c.count : cap;
    for (uint64_t f = 0; f < stored; ++f) {
        for (int l = 0; l < depth; ++l) {
            uint64_t child = rec[f].key >> (63 - 3 * (l + 1));
            levels[level_base(l) + (child >> 3)] |= 1u << (child & 7u);
        }
    }
    return c.count;
}

/* --------------------------------------------------------------------- POFA */

static int cmp_record(const void *a, const void *b)
{
    const orc_record *x = (const orc_record *)a, *y = (const orc_record *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->tri != y->tri) return x->tri < y->tri ? -1 : 1;
    if (x->nrm != y->nrm) return x->nrm < y->nrm ? -1 : 1;
    return 0;
}

/* POFA fragment array (Section 3.1 "Octree Layout", Section 3.2 "FHV_POFA";
 * Fig. 6): all records ordered by (Morton code, triangle, normal); octants
 * are then contiguous in Morton order. */
void orc_pofa_sort(const orc_record *in, uint64_t n, orc_record *out)
{
    memcpy(out, in, n * sizeof(orc_record));
    qsort(out, n, sizeof(orc_record), cmp_record);
}

/* Octant (level, o) of sorted records (the per-octant offset and count of
 * Section 3.1, Fig. 6): off = number of records whose level prefix is below
 * o, cnt = number with prefix o. */
void orc_octant_range(const orc_record *sorted, uint64_t n, int level, uint64_t o, uint32_t *off, uint32_t *cnt)
{
    int sh = 63 - 3 * level;
    uint64_t lo = 0, hi = n;
    while (lo < hi) { /* first record with prefix >= o */
        uint64_t mid = lo + (hi - lo) / 2;
        uint64_t pre = level == 0 ? 0 : sorted[mid].key >> sh;
        if (pre < o) lo = mid + 1; else hi = mid;
    }
    uint64_t first = lo;
    hi = n;
    while (lo < hi) { /* first record with prefix > o */
        uint64_t mid = lo + (hi - lo) / 2;
        uint64_t pre = level == 0 ? 0 : sorted[mid].key >> sh;
        if (pre <= o) lo = mid + 1; else hi = mid;
    }
    *off = (uint32_t)first;
    *cnt = (uint32_t)(lo - first);
}

/* Full FHV_POFA: sorted records and dense (offset, count) for every octant of
 * levels 0..depth, root first. Per level: count fragments per octant, then
 * offsets as the running sum in Morton order (Section 3.2). */
void orc_pofa(const orc_record *in, uint64_t n, int depth, orc_record *out, uint32_t *off, uint32_t *cnt)
{
    orc_pofa_sort(in, n, out);
    for (int l = 0; l <= depth; ++l) {
        uint64_t base = level_base(l), m = (uint64_t)1 << (3 * l);
        for (uint64_t o = 0; o < m; ++o) cnt[base + o] = 0;
        for (uint64_t f = 0; f < n; ++f) {
            uint64_t o = l == 0 ? 0 : out[f].key >> (63 - 3 * l);
            cnt[base + o] += 1;
        }
        uint32_t run = 0;
        for (uint64_t o = 0; o < m; ++o) {
            off[base + o] = run;
            run += cnt[base + o];
        }
    }
}

/* ------------------------------------------------------------------- render */

/* Splat one fragment: dequantise the cell centre, project orthographically,
 * quantise the depth to 24 bits, anchor a k x k footprint. */
static void splat_project(const orc_record *r, const float cmin[3], float cell, const orc_camera *cam, int k,
                          int64_t *ax, int64_t *ay, uint32_t *qd)
{
    uint32_t q[3] = {0, 0, 0};
    for (int b = 0; b < QBITS; ++b) {
        q[0] |= (uint32_t)((r->key >> (3 * b + 2)) & 1u) << b;
        q[1] |= (uint32_t)((r->key >> (3 * b + 1)) & 1u) << b;
        q[2] |= (uint32_t)((r->key >> (3 * b)) & 1u) << b;
    }
    float p[3];
    for (int c = 0; c < 3; ++c) {
        float a = (float)q[c] + 0.5f;
        float b = a * cell;
        p[c] = cmin[c] + b;
    }
    float d[3] = {p[0] - cam->origin[0], p[1] - cam->origin[1], p[2] - cam->origin[2]};
    float inv_pitch = 1.0f / cam->pitch;
    float hw = 0.5f * (float)cam->width, hh = 0.5f * (float)cam->height;
    float sx = dot3f(d, cam->right) * inv_pitch + hw;
    float sy = dot3f(d, cam->up) * inv_pitch + hh;
    float z = dot3f(d, cam->fwd);
    float qscale = 16777216.0f / (cam->z1 - cam->z0);
    float tz = (z - cam->z0) * qscale;
    float fz = floorf(tz);
    if (!(fz >= 0.0f)) *qd = 0;
    else if (fz >= 16777215.0f) *qd = QD_MAX;
    else *qd = (uint32_t)fz;
    float half = 0.5f * (float)(k - 1);
    float fx = floorf(sx - half), fy = floorf(sy - half);
    fx = fminf(fmaxf(fx, -1073741824.0f), 1073741824.0f);
    fy = fminf(fmaxf(fy, -1073741824.0f), 1073741824.0f);
    *ax = (int64_t)fx;
    *ay = (int64_t)fy;
}

/* Visibility of a splatted view (Section 3.3): per pixel the minimum of
 * (qdepth << 40 | index) over all fragments whose footprint covers it (the
 * nearest fragment, ties to the lower index); empty pixels keep all ones. */
void orc_splat_visibility(const orc_record *rec, uint64_t n, const orc_scene *sc, const orc_camera *cam, int k,
                          uint64_t *vis)
{
    int64_t W = cam->width, H = cam->height;
    for (int64_t p = 0; p < W * H; ++p) vis[p] = ~(uint64_t)0;
    float cell = sc->cube_side * (1.0f / 2097152.0f);
    for (uint64_t f = 0; f < n; ++f) {
        int64_t ax, ay;
        uint32_t qd;
        splat_project(&rec[f], sc->cube_min, cell, cam, k, &ax, &ay, &qd);
        uint64_t key = ((uint64_t)qd << IDX_BITS) | f;
        for (int b = 0; b < k; ++b) {
            for (int a = 0; a < k; ++a) {
                int64_t x = ax + a, y = ay + b;
                if (x < 0 || y < 0 || x >= W || y >= H) continue;
                if (key < vis[y * W + x]) vis[y * W + x] = key;
            }
        }
    }
}

/* Lambert colour of one fragment (Section 5): albedo of its material times
 * the sum over lights of intensity * max(0, n . l), in double. */
static void frag_colour(const orc_record *r, const orc_scene *sc, const float *albedo, const float *lights,
                        int n_lights, double out[3])
{
    double cell = (double)sc->cube_side / 2097152.0;
    uint32_t q[3] = {0, 0, 0};
    for (int b = 0; b < QBITS; ++b) {
        q[0] |= (uint32_t)((r->key >> (3 * b + 2)) & 1u) << b;
        q[1] |= (uint32_t)((r->key >> (3 * b + 1)) & 1u) << b;
        q[2] |= (uint32_t)((r->key >> (3 * b)) & 1u) << b;
    }
    double pos[3], n[3];
    for (int c = 0; c < 3; ++c) pos[c] = (double)sc->cube_min[c] + ((double)q[c] + 0.5) * cell;
    orc_oct_decode(r->nrm, n);
    const float *alb = albedo + 3 * (size_t)sc->tri_material[r->tri];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int l = 0; l < n_lights; ++l) {
        const float *L = lights + 8 * l;
        double dir[3];
        if (L[0] == 0.0f) {
            dir[0] = L[1]; dir[1] = L[2]; dir[2] = L[3];
        } else {
            dir[0] = L[1] - pos[0]; dir[1] = L[2] - pos[1]; dir[2] = L[3] - pos[2];
        }
        double len = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        if (!(len > 0.0)) continue;
        double ndl = (n[0] * dir[0] + n[1] * dir[1] + n[2] * dir[2]) / len;
        if (ndl < 0.0) ndl = 0.0;
        for (int c = 0; c < 3; ++c) acc[c] += (double)L[4 + c] * ndl;
    }
    for (int c = 0; c < 3; ++c) out[c] = (double)alb[c] * acc[c];
}

/* Shading of the visible fragment (Section 3.3; local illumination as in
 * Section 5): albedo of
 * the triangle's material times the sum over lights of intensity *
 * max(0, n . l). Light = {type, x, y, z, r, g, b, unused}; type 0 is a
 * direction towards the light, type 1 a point light position. Background is
 * (0, 0, 0, 0), a shaded pixel has alpha 1. */
void orc_shade(const uint64_t *vis, const orc_record *rec, const orc_scene *sc, const float *albedo,
               const float *lights, int n_lights, const orc_camera *cam, float *rgba)
{
    int64_t np = (int64_t)cam->width * cam->height;
    for (int64_t p = 0; p < np; ++p) {
        float *o = rgba + 4 * p;
        if (vis[p] == ~(uint64_t)0) {
            o[0] = o[1] = o[2] = o[3] = 0.0f;
            continue;
        }
        const orc_record *r = &rec[vis[p] & (((uint64_t)1 << IDX_BITS) - 1)];
        double col[3];
        frag_colour(r, sc, albedo, lights, n_lights, col);
        for (int c = 0; c < 3; ++c) o[c] = (float)col[c];
        o[3] = 1.0f;
    }
}

uint64_t orc_level_base(int l) { return level_base(l); }

/* ------------------------------------------------------------ ray casting */

typedef struct {
    uint64_t key;
    uint64_t pix;
} orc_hit;

static int cmp_hit(const void *a, const void *b)
{
    const orc_hit *x = (const orc_hit *)a, *y = (const orc_hit *)b;
    if (x->pix != y->pix) return x->pix < y->pix ? -1 : 1;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return 0;
}

/* Ray casting by brute force over every fragment (Section 3.3): a fragment
 * lies on pixel p's ray when it projects into p (k = 1 splat rule). vis[p]
 * = the smallest key (nearest, ties to the lower index) or all ones. With
 * alpha == NULL the pixel is the nearest fragment's colour with alpha 1;
 * otherwise the pixel's fragments are composited front to back in key
 * order, C += T * a * c, T *= 1 - a, and rgba = (C, 1 - T). */
void orc_raycast(const orc_record *rec, uint64_t n, const orc_scene *sc, const float *albedo, const float *alpha,
                 const float *lights, int n_lights, const orc_camera *cam, uint64_t *vis, float *rgba)
{
    int64_t W = cam->width, H = cam->height, np = W * H;
    float cell = sc->cube_side * (1.0f / 2097152.0f);
    orc_hit *hits = (orc_hit *)malloc((n ? n : 1) * sizeof(orc_hit));
    uint64_t nh = 0;
    for (uint64_t f = 0; f < n; ++f) {
        int64_t ax, ay;
        uint32_t qd;
        splat_project(&rec[f], sc->cube_min, cell, cam, 1, &ax, &ay, &qd);
        if (ax < 0 || ay < 0 || ax >= W || ay >= H) continue;
        hits[nh].key = ((uint64_t)qd << IDX_BITS) | f;
        hits[nh].pix = (uint64_t)(ay * W + ax);
        ++nh;
    }
    qsort(hits, nh, sizeof(orc_hit), cmp_hit);
    for (int64_t p = 0; p < np; ++p) {
        vis[p] = ~(uint64_t)0;
        for (int c = 0; c < 4; ++c) rgba[4 * p + c] = 0.0f;
    }
    uint64_t h = 0;
    while (h < nh) {
        uint64_t p = hits[h].pix, e = h;
        while (e < nh && hits[e].pix == p) ++e;
        vis[p] = hits[h].key;
        double C[3] = {0.0, 0.0, 0.0}, T = 1.0;
        for (uint64_t i = h; i < e; ++i) {
            const orc_record *r = &rec[hits[i].key & (((uint64_t)1 << IDX_BITS) - 1)];
            double col[3];
            frag_colour(r, sc, albedo, lights, n_lights, col);
            double a = alpha ? (double)alpha[sc->tri_material[r->tri]] : 1.0;
            for (int c = 0; c < 3; ++c) C[c] += T * a * col[c];
            T *= 1.0 - a;
            if (!alpha) break;
        }
        for (int c = 0; c < 3; ++c) rgba[4 * p + c] = (float)C[c];
        rgba[4 * p + 3] = (float)(1.0 - T);
        h = e;
    }
    free(hits);
}

