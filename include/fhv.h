/*
 * fhv.h -- C ABI of the GB300 fragment-history-volume library (libfhv.so).
 *
 * Fragment-history volumes (Inacio & Springer, arXiv 2211.15460) record every
 * fragment the rasteriser produces for a triangle scene (Section 3), store
 * them in per-pixel lists (FHV_PPFL), per-octant lists (FHV_POFL) or
 * per-octant arrays (FHV_POFA) (Section 3.1), and resample them for novel
 * viewpoints by point splatting (Section 3.3).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* (and the pointers inside fhv_scene / fhv_frag_buf)
 *    are DEVICE pointers on the current CUDA device; everything else is host
 *    memory. The caller owns and allocates all memory, including the
 *    scratch workspace whose size fhv_query_sizes reports; no entry point
 *    allocates. Device arrays must be 16-byte aligned.
 *  - Calls that take a stream only enqueue work on it and return without
 *    waiting, except fhv_get_count and fhv_read_status, which synchronise
 *    the stream. Argument errors are detected on the host before anything
 *    is enqueued and returned as FHV_ERR_INVALID_ARG (nothing is launched).
 *    A failed launch returns FHV_ERR_CUDA.
 *  - Problems found on the device (a bounded wait that ran out, a triangle
 *    whose sample box is too large) set bits of a status word kept in the
 *    call's workspace; fhv_read_status returns it. Kernels never trap.
 *  - The stream type is the CUDA runtime's cudaStream_t (NULL = the legacy
 *    default stream).
 *
 * Arithmetic contract shared with the test oracle (both sides implement it
 * independently; it fixes what the paper leaves to the hardware):
 *  - positions are cube-quantised to 21 bits per axis:
 *    q = clamp(floor((p - cube_min) * (2^21 / cube_side)), 0, 2^21 - 1);
 *  - vertices are projected in float32 with every operation rounded on its
 *    own, snapped to 1/256 pixel (round half to even, guard band 2^16 px);
 *  - samples sit at pixel centres (i + 1/2, j + 1/2), y up, and a sample is
 *    inside when every edge function is positive or zero on a top or left
 *    edge (after making the winding counter-clockwise); triangles of zero
 *    area produce nothing; culling is off (Section 3.2);
 *  - a fragment's position is the exact barycentric combination of the
 *    vertices' quantised positions, rounded half up; its normal is the
 *    float32 combination w0*n0 + w1*n1 + w2*n2 of the edge weights and
 *    vertex normals, octahedrally encoded to two snorm16 values;
 *  - POFA keeps octants contiguous in Morton order and orders the fragments
 *    inside an octant by the full record (key, tri, nrm), so the array is
 *    unique.
 */
#ifndef FHV_H
#define FHV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as the CUDA runtime's cudaStream_t. */
typedef struct CUstream_st *fhv_stream_t;

typedef enum {
    FHV_OK = 0,
    FHV_ERR_INVALID_ARG = 1, /* bad pointer, size, depth or alignment; nothing launched */
    FHV_ERR_OVERFLOW = 2,    /* more fragments than the fragment buffer holds (Section 3.1) */
    FHV_ERR_CUDA = 3,        /* a CUDA launch or copy failed */
    FHV_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out */
    FHV_ERR_UNSUPPORTED = 5  /* input outside the implemented limits */
} fhv_status;

/* Device status bits (fhv_read_status). */
#define FHV_DEV_TIMEOUT 0x1u        /* a look-back or copy wait gave up */
#define FHV_DEV_HUGE_TRIANGLE 0x2u  /* a triangle's sample box exceeded 2^31 samples and was skipped */
#define FHV_DEV_RANGE 0x4u          /* more records than 2^32 - 1 reached compaction */
#define FHV_DEV_INDEX_OVERFLOW 0x10u /* a sparse index needed more entries than its capacity */

/* How triangles are projected for capture (Section 3.2, Table 2). */
typedef enum {
    FHV_CAPTURE_VIEW = 0,   /* 1-Pass/View: orthographic capture camera */
    FHV_CAPTURE_NORMAL = 1, /* 1-Pass/Normal: each triangle in its own tangent frame */
    FHV_CAPTURE_AXIS3 = 2   /* 3-Pass/1-Way (Fig. 7): each triangle along x, y and z */
} fhv_capture_mode;

typedef enum {
    FHV_LAYOUT_PPFL = 0,
    FHV_LAYOUT_POFL = 1,
    FHV_LAYOUT_POFA = 2,
    FHV_LAYOUT_POFA_DIRECT = 3, /* query sizes only: fhv_build_pofa_direct's workspace */
    FHV_LAYOUT_POFA_SPARSE = 4  /* query sizes only: fhv_compact_pofa_sparse's workspace */
} fhv_layout;

/* Indexed triangle scene (device pointers). tri_material[t] indexes the
 * albedo table given to fhv_render_view; the triangle index is the object
 * id stored with each fragment. cube_min / cube_side define the
 * quantisation cube; cube_side must be > 0. tri_base: id of the first
 * triangle, 0 for a whole scene. A slice of a larger scene's triangles
 * (idx advanced by 3 * t0, n_tri = t1 - t0, the scene's cube, tri_base =
 * t0) is captured with the larger scene's triangle ids: the records carry
 * tri_base + local index, so sharded captures (one slice per rank) render
 * with the whole scene. tri_base + n_tri < 2^32. The render entries read
 * materials by the records' ids and ignore tri_base. */
typedef struct {
    const uint32_t *idx;          /* [3 * n_tri] vertex indices, < n_vtx */
    const float *pos;             /* [3 * n_vtx] world positions */
    const float *nrm;             /* [3 * n_vtx] vertex normals */
    const uint32_t *tri_material; /* [n_tri] */
    uint32_t n_tri, n_vtx;
    float cube_min[3];
    float cube_side;
    uint32_t tri_base;
} fhv_scene;

/* Orthographic camera (Section 3.2): a world point p maps to pixel
 * coordinates sx = dot(p - origin, right) / pitch + width/2,
 * sy = dot(p - origin, up) / pitch + height/2, depth z = dot(p - origin, fwd);
 * pixel (i, j) covers [i, i+1) x [j, j+1), row j = 0 at the bottom. Depth
 * [z0, z1] maps to the 24-bit depth code of the splat visibility pass. */
typedef struct {
    float origin[3], right[3], up[3], fwd[3];
    float pitch;
    int32_t width, height;
    float z0, z1;
} fhv_ortho_camera;

/* 16-byte fragment record (Section 3.1 stores position, normal, material and
 * object id; here the position is the 63-bit Morton code of the quantised
 * position, whose top 3d bits are the leaf octant at depth d, and tri
 * yields material and object id). */
typedef struct {
    uint64_t key; /* Morton code: bit 3k+2 / 3k+1 / 3k = bit k of x / y / z */
    uint32_t tri; /* triangle index */
    uint32_t nrm; /* octahedral normal, snorm16 x | (snorm16 y << 16) */
} fhv_record;

/* Global fragment list (Section 3.1): records, previous-index links (-1 ends
 * a list) and the global counter. The counter keeps counting past
 * capacity; fragments whose index is >= capacity are dropped entirely. */
typedef struct {
    fhv_record *rec;   /* [capacity] */
    int32_t *next;     /* [capacity] */
    uint64_t capacity; /* <= 2^31 - 1 */
    uint64_t *d_count; /* one device uint64, reset by each capture */
} fhv_frag_buf;

/* Sizes a call needs. */
typedef struct {
    uint64_t workspace_bytes; /* scratch to pass as (d_ws, ws_bytes) */
    uint64_t index_bytes;     /* pixel array, leaf heads + levels, or off + cnt arrays */
    uint64_t fragment_bytes;  /* records (+ next links for lists) for n_fragments */
    uint64_t n_index_entries; /* entries of the index array(s) */
} fhv_sizes;

/* One occupied octant of a sparse octree index (fhv_compact_pofa_sparse):
 * the octant's Morton prefix at its level, and the offset and count of its
 * range in the POFA, 16 bytes. */
typedef struct {
    uint64_t octant; /* Morton prefix (3 x level bits) */
    uint32_t off;    /* first POFA record of the octant */
    uint32_t cnt;    /* its records */
} fhv_octant_entry;

/* Octree index layout (POFL levels and POFA off/cnt; the per-level octant
 * arrays of Section 3.1, Fig. 6, whose storage order the paper leaves open):
 * levels are stored root first; level 0 (one octant) occupies entries 0..3 (three unused), level
 * l >= 1 starts at entry (8^l - 1)/7 + 3, so every level starts 16-byte
 * aligned. fhv_level_offset(l) returns that start; fhv_level_offset(d + 1)
 * is the number of entries for levels 0..d. Octant o of level l is the
 * Morton prefix o of length 3l. */
uint64_t fhv_level_offset(int level);

/* Table 4 (Section 4) memory model: bytes of one layout for an input of
 * n_pixels, octree depth `depth`, the pre-allocation rule of Section 3.1
 * (n_pixels x avg_depth_complexity list records of list_record_bytes, plus
 * the pixel array or the complete octree) for PPFL/POFL, and the exact
 * n_fragments x array_record_bytes plus 2 x 4 bytes per octant for POFA.
 * Octant counts follow the complete octree of levels 0..depth, i.e.
 * (8^(depth+1) - 1)/7 octants, without the alignment padding above. */
fhv_status fhv_memory_model(fhv_layout layout, uint64_t n_pixels, int depth, double avg_depth_complexity,
                            uint64_t n_fragments, uint32_t list_record_bytes, uint32_t array_record_bytes,
                            uint64_t *bytes);

/* Sizes for one call of the given layout (Section 3.1: storage is
 * allocated up front and re-allocated when a capture overflows): PPFL =
 * fhv_capture_ppfl, POFL = fhv_build_pofl, POFA = fhv_compact_pofa
 * (n_fragments = the maximum number of input records), POFA_DIRECT =
 * fhv_build_pofa_direct (n_fragments = its capacity). Render needs
 * FHV_RENDER_WS_BYTES. */
fhv_status fhv_query_sizes(fhv_layout layout, uint32_t n_tri, int32_t width, int32_t height, int depth,
                           uint64_t n_fragments, fhv_sizes *out);

#define FHV_RENDER_WS_BYTES 256u

/* FHV_PPFL capture (Section 3.2, "FHV_PPFL"; Fig. 3). Rasterises every
 * triangle with the orthographic camera `cam` (culling off) and appends each
 * fragment: index from the global counter; if below capacity the record is
 * written and linked in front of the pixel's list by an atomic exchange of
 * d_head[j * width + i]. d_head [width*height] is reset to -1 and the
 * counter to 0 first. List order inside a pixel follows the device's
 * atomic order. */
fhv_status fhv_capture_ppfl(const fhv_scene *scene, const fhv_ortho_camera *cam, int32_t *d_head,
                            const fhv_frag_buf *frags, void *d_ws, size_t ws_bytes, fhv_stream_t stream);

/* FHV_POFL build (Section 3.2, "FHV_POFL"; Figs. 5, 8). Same insertion keyed
 * by the leaf octant (Morton prefix of length 3*depth) into d_leaf_head
 * [8^depth], reset to -1 first. The first fragment of a leaf marks it in its
 * parent's child-occupancy mask, and so on up while a parent was empty, so
 * d_levels [fhv_level_offset(depth)] (levels 0..depth-1, zeroed first) ends
 * with bit c of octant o set iff child 8o+c holds a stored fragment.
 * mode FHV_CAPTURE_VIEW rasterises with `cam`; FHV_CAPTURE_NORMAL
 * rasterises each triangle in its tangent frame with sample spacing `pitch`
 * (world units) on a lattice anchored at the triangle's first vertex, and
 * ignores `cam`; FHV_CAPTURE_AXIS3 rasterises each triangle three times,
 * looking along world x, y and z, on a lattice of spacing `pitch` anchored
 * at the cube corner (the 2-D coordinates of the pass along axis a are axes
 * (a+1)%3 and (a+2)%3), and ignores `cam`. 1 <= depth <= 11. The POFL
 * workspace size covers every mode. */
fhv_status fhv_build_pofl(const fhv_scene *scene, fhv_capture_mode mode, const fhv_ortho_camera *cam, float pitch,
                          int depth, int32_t *d_leaf_head, uint32_t *d_levels, const fhv_frag_buf *frags,
                          void *d_ws, size_t ws_bytes, fhv_stream_t stream);

/* fhv_build_pofl for a repeated build into the same lists: d_leaf_head
 * must hold the result of the previous fhv_build_pofl or
 * fhv_build_pofl_reuse with the same depth, d_leaf_head and frags (records
 * and counter untouched since, and that call ordered before this one on the
 * GPU). Instead of resetting all 8^depth heads, the build resets the heads
 * of the previous build's stored records -- the only ones that are not -1 --
 * so the reset costs O(fragments) instead of O(octants). The result is the
 * same as fhv_build_pofl's. No paper counterpart (the paper rebuilds its
 * lists from scratch; Section 3.1 keeps them across frames). */
fhv_status fhv_build_pofl_reuse(const fhv_scene *scene, fhv_capture_mode mode, const fhv_ortho_camera *cam,
                                float pitch, int depth, int32_t *d_leaf_head, uint32_t *d_levels,
                                const fhv_frag_buf *frags, void *d_ws, size_t ws_bytes, fhv_stream_t stream);

/* Fragment capture into the global fragment list only (Section 3.1: every
 * FHV layout stores its fragments in one global list; Section 3.2: the
 * FHV_POFA is made from the fragments of a capture). Rasterises every
 * triangle in `mode` exactly as fhv_build_pofl does (camera for
 * FHV_CAPTURE_VIEW, sample pitch for FHV_CAPTURE_NORMAL and
 * FHV_CAPTURE_AXIS3) and appends each fragment's record at the index the
 * global counter gives it, in the order the rasteriser emits them, but
 * builds no per-pixel or per-octant list: no heads, no links, no occupancy.
 * frags->next is not used (may be NULL). The counter is reset to 0 first,
 * keeps counting past capacity, and a fragment whose index is at or above
 * capacity is dropped (fhv_get_count reports FHV_ERR_OVERFLOW). The records
 * are the input of fhv_compact_pofa. Workspace: fhv_query_sizes with
 * FHV_LAYOUT_POFL (covers every mode). */
fhv_status fhv_capture_fragments(const fhv_scene *scene, fhv_capture_mode mode, const fhv_ortho_camera *cam,
                                 float pitch, const fhv_frag_buf *frags, void *d_ws, size_t ws_bytes,
                                 fhv_stream_t stream);

/* FHV_POFA straight from the triangles, without lists (Section 3.2,
 * "FHV_POFA": rasterise to count the fragments of every octant, scan the
 * counts into offsets, rasterise again to write every fragment into its
 * octant's range). The counting takes two raster passes (marking the
 * occupied leaves, then counting), the writing a third; each range is then
 * put in the canonical order, so d_pofa, d_off and d_cnt are byte for byte
 * what fhv_build_pofl followed by fhv_compact_pofa gives for the same scene,
 * mode and depth. Needs no list heads, links or occupancy levels.
 * mode, cam, pitch and depth as for fhv_build_pofl. *d_count (device,
 * 16-byte aligned) receives the number of fragments n, counted in full
 * even past `capacity`. If n <= capacity: d_pofa [capacity] holds the n
 * sorted records and d_off / d_cnt [fhv_level_offset(depth + 1)] the
 * offsets and counts of every octant of levels 0..depth. If n > capacity:
 * d_off / d_cnt are complete but no record is written (a call with
 * capacity 0 and d_pofa NULL learns n and the index). capacity < 2^32 - 1.
 * Workspace: fhv_query_sizes(FHV_LAYOUT_POFA_DIRECT, n_tri, .., depth,
 * capacity).workspace_bytes, 16-byte aligned. */
fhv_status fhv_build_pofa_direct(const fhv_scene *scene, fhv_capture_mode mode, const fhv_ortho_camera *cam,
                                 float pitch, int depth, fhv_record *d_pofa, uint64_t capacity, uint64_t *d_count,
                                 uint32_t *d_off, uint32_t *d_cnt, void *d_ws, size_t ws_bytes, fhv_stream_t stream);

/* FHV_POFA compaction (Section 3.1 "Octree Layout", Section 3.2 "FHV_POFA";
 * Fig. 6): counts fragments per leaf octant, takes offsets by an exclusive
 * scan in Morton order, scatters every record to its octant's range and
 * orders each range by the full record, giving the unique sorted array.
 * Input: records d_in[0..n) with n = min(*d_n, n_max) when d_n is not NULL
 * (a device counter such as fhv_frag_buf.d_count), else n = n_max.
 * Output: d_pofa [n_max] (first n valid), d_off / d_cnt
 * [fhv_level_offset(depth + 1)]: for every octant of every level 0..depth,
 * off = number of records whose prefix is smaller, cnt = number with that
 * prefix. d_in and d_pofa must not overlap. n must be < 2^32. */
fhv_status fhv_compact_pofa(const fhv_record *d_in, uint64_t n_max, const uint64_t *d_n, int depth,
                            fhv_record *d_pofa, uint32_t *d_off, uint32_t *d_cnt, void *d_ws, size_t ws_bytes,
                            fhv_stream_t stream);

/* FHV_POFA compaction with a sparse octree index (Section 3.1 "Octree
 * Layout": per-octant arrays in Morton order, Fig. 6; Section 3.2
 * "FHV_POFA"). The records come out exactly as from fhv_compact_pofa (the
 * unique sorted array, d_pofa [n_max], first n valid), but instead of the
 * complete octree of Table 4 the index holds only the occupied octants:
 * for every level l = 0..depth, entries d_index[d_level_base[l] ..
 * d_level_base[l + 1]) are that level's occupied octants in increasing
 * Morton order, each with the off and cnt fhv_compact_pofa gives it (every
 * octant missing from a level has cnt 0). Nothing of size 8^depth is used,
 * so depth 11 needs no 79 GB index. Input as for fhv_compact_pofa (n =
 * min(*d_n, n_max), n < 2^32, d_in and d_pofa must not overlap).
 * d_level_base: depth + 2 device uint64 (16-byte aligned), written by the
 * call; d_level_base[depth + 1] = the number of entries needed. d_index
 * [index_capacity] (16-byte aligned): entries at or past index_capacity are
 * not written and FHV_DEV_INDEX_OVERFLOW is set; the caller re-allocates
 * from d_level_base[depth + 1] and calls again (Section 3.1's rule for
 * buffers that turn out too small). An upper bound that never overflows is
 * fhv_query_sizes(FHV_LAYOUT_POFA_SPARSE, .., depth, n_max).n_index_entries.
 * Workspace: fhv_query_sizes(FHV_LAYOUT_POFA_SPARSE, 0, 1, 1, depth,
 * n_max).workspace_bytes, 16-byte aligned; its status word
 * (fhv_read_status) reports FHV_DEV_INDEX_OVERFLOW and FHV_DEV_RANGE. */
fhv_status fhv_compact_pofa_sparse(const fhv_record *d_in, uint64_t n_max, const uint64_t *d_n, int depth,
                                   fhv_record *d_pofa, fhv_octant_entry *d_index, uint64_t index_capacity,
                                   uint64_t *d_level_base, void *d_ws, size_t ws_bytes, fhv_stream_t stream);

/* Self-test of failure detection without a fault (no paper counterpart):
 * runs one of the library's bounded device waits on a condition that
 * nothing satisfies -- kind 0: the
 * decoupled look-back of the scans (a predecessor tile that never publishes;
 * its own limit of 2^20 polls), kind 1: the mbarrier wait of the bulk copies,
 * kind 2: the mbarrier wait of the tensor-core kernels (these two bounded to
 * 2^12 polls here). The wait gives up, sets FHV_DEV_TIMEOUT in the workspace
 * status word (fhv_read_status returns FHV_ERR_TIMEOUT) and the kernel
 * returns; nothing traps and the context stays usable. d_ws: 16-byte
 * aligned, FHV_WAIT_PROBE_WS_BYTES bytes (zeroed by the call). */
#define FHV_WAIT_PROBE_WS_BYTES (256u + 16u)
fhv_status fhv_wait_probe(int kind, void *d_ws, size_t ws_bytes, fhv_stream_t stream);

/* Sparse variant of a POFA's octree index (the per-octant arrays of Section
 * 3.1 kept for the occupied leaves only): for the sorted records
 * d_pofa[0..n) of fhv_compact_pofa at `depth` (n = min(*d_n, n_max) when d_n
 * is not NULL, else n_max), writes the distinct leaf octants
 * leaf = key >> (63 - 3 depth) in increasing order to d_leaf[0..m), the index
 * of each leaf's first record to d_off[0..m) and its record count to
 * d_cnt[0..m), and m to *d_m (device memory). The arrays hold up to n_max
 * entries. On every occupied leaf the result equals fhv_compact_pofa's
 * dense offsets and counts. d_m 16-byte aligned; the workspace needs
 * FHV_LEAF_INDEX_WS_BYTES(n_max) bytes, 16-byte aligned. n_max < 2^32,
 * 1 <= depth <= 11. */
#define FHV_LEAF_INDEX_WS_BYTES(n_max) (16u + 12u * (((unsigned long long)(n_max) + 4095u) / 4096u))
fhv_status fhv_pofa_leaf_index(const fhv_record *d_pofa, uint64_t n_max, const uint64_t *d_n, int depth,
                               uint64_t *d_leaf, uint32_t *d_off, uint32_t *d_cnt, uint64_t *d_m, void *d_ws,
                               size_t ws_bytes, fhv_stream_t stream);

/* Novel-view image generation by point splatting (Section 3.3) keeping the
 * fragment nearest to the viewer, then local illumination (Section 5).
 * Fragments d_frag[0..n) (n as in fhv_compact_pofa) from any layout: each
 * one is projected with `cam`, its depth quantised to 24 bits
 * qd = clamp(floor((z - z0) * 2^24 / (z1 - z0)), 0, 2^24 - 1), and
 * (qd << 40 | index) is min-combined into d_vis[width*height] over a
 * footprint_k x footprint_k pixel block anchored at
 * floor(sx - (k-1)/2), floor(sy - (k-1)/2). d_vis is reset to all ones
 * first. Then each covered pixel is shaded with the winner's record:
 * rgba = (albedo[tri_material[tri]] * sum_l I_l * max(0, n . l_l), 1);
 * uncovered pixels get (0, 0, 0, 0). d_albedo is [3 * n_materials];
 * d_lights is [8 * n_lights] float: {type, x, y, z, r, g, b, unused} with
 * type 0 = directional (direction towards the light), 1 = point light
 * (position). d_rgba is [4 * width * height]. n_lights <= 64, 1 <= k <= 16,
 * n < 2^40. */
fhv_status fhv_render_view(const fhv_record *d_frag, uint64_t n_max, const uint64_t *d_n, const fhv_scene *scene,
                           const float *d_albedo, const float *d_lights, int n_lights, const fhv_ortho_camera *cam,
                           int footprint_k, uint64_t *d_vis, float *d_rgba, void *d_ws, size_t ws_bytes,
                           fhv_stream_t stream);

/* The two steps of fhv_render_view on their own, for a list split into
 * slices (for example one per rank, each holding the records
 * [index_base, index_base + n) of the whole sorted list). Both follow
 * Section 3.3 (splatting, nearest fragment kept) and Section 5 (shading).
 *
 * fhv_splat_visibility: resets d_vis[width*height] to all ones, then
 * min-combines (qd << 40 | (index_base + i)) for every record i < n over the
 * footprint, exactly as fhv_render_view does with index_base = 0. The
 * element-wise unsigned minimum of the slices' d_vis is the d_vis of the
 * whole list.
 *
 * fhv_shade_owned: for every pixel of d_vis (read only) whose winner index
 * lies in [index_base, index_base + n), writes the colour fhv_render_view
 * gives it, reading record (index - index_base) of d_frag; every other pixel
 * gets (0, 0, 0, 0). Summing the slices' d_rgba (each pixel owned by one
 * slice, zeros elsewhere) gives the image of the whole list exactly.
 *
 * Arguments as in fhv_render_view; index_base + n <= 2^40; the workspace
 * needs FHV_RENDER_WS_BYTES. */
fhv_status fhv_splat_visibility(const fhv_record *d_frag, uint64_t n_max, const uint64_t *d_n, uint64_t index_base,
                                const fhv_scene *scene, const fhv_ortho_camera *cam, int footprint_k,
                                uint64_t *d_vis, void *d_ws, size_t ws_bytes, fhv_stream_t stream);
fhv_status fhv_shade_owned(const fhv_record *d_frag, uint64_t n_max, const uint64_t *d_n, uint64_t index_base,
                           const fhv_scene *scene, const float *d_albedo, const float *d_lights, int n_lights,
                           const fhv_ortho_camera *cam, const uint64_t *d_vis, float *d_rgba, void *d_ws,
                           size_t ws_bytes, fhv_stream_t stream);

/* Novel-view image generation by ray casting through a FHV_POFA (Section
 * 3.3, the second evaluation method; Table 3 "R" and "R/T"). One ray per
 * pixel of `cam` walks the octree given by d_off / d_cnt (the output of
 * fhv_compact_pofa at the same depth, [fhv_level_offset(depth + 1)] each)
 * from the root, visiting children that hold fragments nearest first, and
 * tests the records of each leaf it reaches (d_pofa[0..n_max)). A record
 * lies on the pixel's ray when its projection falls in that pixel, with the
 * projection and 24-bit depth key of fhv_render_view (footprint 1), and the
 * ray's records are taken in increasing (qd << 40 | index) order.
 * d_vis[p] = the first key (all ones when the ray meets nothing), exactly the
 * visibility of fhv_render_view with footprint_k = 1.
 * d_alpha = NULL ("R", opaque): rgba = the first record's colour as in
 * fhv_render_view, alpha 1.
 * d_alpha = per-material opacity [n_materials] ("R/T"): colours are
 * composited front to back, C += T * a * c, T *= 1 - a from T = 1, and
 * rgba = (C, 1 - T); the ray stops once T <= t_stop (0 <= t_stop < 1), so
 * a pixel differs from the full composite by at most t_stop times the
 * largest colour. Empty pixels get (0, 0, 0, 0). Arguments as in
 * fhv_render_view; 1 <= depth <= 11, n_max < 2^40; d_off / d_cnt
 * 16-byte aligned. Offsets that point past n_max raise FHV_DEV_RANGE and are
 * clipped. The workspace needs FHV_RENDER_WS_BYTES; bytes beyond those serve
 * as up to 256 overflow buffers of 256 KiB for pixel tiles whose set of
 * octants on the way down does not fit on chip (FHV_RAYCAST_WS_BYTES gives
 * all 256; with fewer, such tiles may take a slower per-pixel traversal,
 * with the same result). Concurrent calls need separate workspaces. */
#define FHV_RAYCAST_WS_BYTES (256u + 256u * 262144u)
fhv_status fhv_raycast_pofa(const fhv_record *d_pofa, uint64_t n_max, const uint32_t *d_off, const uint32_t *d_cnt,
                            int depth, const fhv_scene *scene, const float *d_albedo, const float *d_alpha,
                            float t_stop, const float *d_lights, int n_lights, const fhv_ortho_camera *cam,
                            uint64_t *d_vis, float *d_rgba, void *d_ws, size_t ws_bytes, fhv_stream_t stream);

/* POFA compaction for callers that cannot allocate device memory: plug-ins
 * and interop layers that only receive device pointers from a host
 * application that owns the allocator, and real-time loops that must not call
 * cudaMalloc because it can synchronise the device. Same contract and result
 * as fhv_compact_pofa, but the scratch workspace is a fixed array inside the
 * library (FHV_STATIC_WS_BYTES, held on every GPU that loads the library until
 * the process exits), so no workspace is passed. n_max above
 * FHV_STATIC_MAX_RECORDS returns FHV_ERR_UNSUPPORTED before anything is
 * enqueued. The first call on a device looks up the array's device address
 * (set-up once per device, with that device current), so make it before any
 * stream capture; a call that finds another CUDA context current on the
 * device (after a device reset) looks the address up again. All calls share
 * the array: each call clears what must start at zero, and calls that
 * overlap on the GPU race, so serialise them. The device status word of the
 * last call lives in the array too: read it with fhv_read_static_status.
 * The paper has no counterpart. */
#define FHV_STATIC_MAX_RECORDS (1u << 20)
#define FHV_STATIC_WS_BYTES ((16u << 20) + (64u << 10))
fhv_status fhv_compact_pofa_static(const fhv_record *d_in, uint64_t n_max, const uint64_t *d_n, int depth,
                                   fhv_record *d_pofa, uint32_t *d_off, uint32_t *d_cnt, fhv_stream_t stream);

/* Synchronises `stream` and returns in *host_status the device status word
 * (FHV_DEV_* bits) of the last fhv_compact_pofa_static call on the current
 * device, the counterpart of fhv_read_status for the library-held scratch:
 * FHV_ERR_TIMEOUT if a bounded wait of that call ran out (its POFA is then
 * not valid), FHV_ERR_INVALID_ARG for a NULL host_status. The paper has no
 * counterpart. */
fhv_status fhv_read_static_status(uint32_t *host_status, fhv_stream_t stream);

/* A built FHV_POFA saved to and loaded from a file, from and into HOST
 * buffers (no device calls). The paper keeps an FHV across frames and
 * re-creates it only when the scene changes (Section 4); a saved one lets a
 * later run skip its creation. File: the 8 bytes "FHVPOFA1", this header
 * (little-endian), the n_records 16-byte records, then either the dense
 * index (off, then cnt: fhv_level_offset(depth + 1) uint32 each) or the
 * sparse one (depth + 2 level bases as uint64, then the entries). */
typedef struct {
    int32_t depth;             /* 1..11 */
    int32_t index_kind;        /* 0: complete octree (off, cnt); 1: sparse (fhv_compact_pofa_sparse) */
    uint64_t n_records;        /* < 2^32 - 1 */
    uint64_t n_index_entries;  /* dense: fhv_level_offset(depth + 1); sparse: level_base[depth + 1] */
    uint64_t reserved[5];
} fhv_pofa_header;

/* Writes the POFA h_pofa[0, n) with exactly one index: the dense arrays
 * (h_off, h_cnt not NULL; h_index and h_level_base NULL) or the sparse one
 * (h_index, h_level_base not NULL; h_off and h_cnt NULL). FHV_ERR_INVALID_ARG
 * for bad arguments or a failed write. */
fhv_status fhv_pofa_save(const char *path, int depth, const fhv_record *h_pofa, uint64_t n, const uint32_t *h_off,
                         const uint32_t *h_cnt, const fhv_octant_entry *h_index, const uint64_t *h_level_base);

/* Reads a saved POFA's header (sizes to allocate); FHV_ERR_INVALID_ARG for
 * a file that is missing or not a saved POFA. */
fhv_status fhv_pofa_load_header(const char *path, fhv_pofa_header *out);

/* Reads a saved POFA into host buffers: h_pofa [record_capacity], and the
 * dense index into h_off / h_cnt [n_index_entries each] or the sparse one
 * into h_level_base [depth + 2] and h_index [index_capacity], as the header
 * says. FHV_ERR_OVERFLOW when a capacity is too small (nothing read),
 * FHV_ERR_INVALID_ARG for a missing buffer or a truncated or inconsistent
 * file. */
fhv_status fhv_pofa_load(const char *path, fhv_record *h_pofa, uint64_t record_capacity, uint32_t *h_off,
                         uint32_t *h_cnt, fhv_octant_entry *h_index, uint64_t index_capacity,
                         uint64_t *h_level_base);

/* ---------------------------------------------------------------------------
 * Batched novel views: many viewpoints of many fragment sets in one call
 * (Section 5 suggests submitting the view-port quads of several viewpoints
 * together for better GPU occupancy). Every view gets exactly the visibility
 * and colours fhv_render_view would give it.
 * ------------------------------------------------------------------------- */

/* One fragment set to splat, e.g. the POFA of one scene (device pointers). */
typedef struct {
    const fhv_record *d_frag;     /* [n_max] */
    uint64_t n_max;
    const uint64_t *d_n;          /* optional device count: n = min(*d_n, n_max); NULL: n = n_max */
    const uint32_t *tri_material; /* [n_tri] */
    const float *albedo;          /* [3 * n_materials] */
    float cube_min[3];
    float cube_side;
} fhv_splat_source;

/* One view of one source. */
typedef struct {
    fhv_ortho_camera cam;
    uint32_t source;  /* index into the source array */
    uint64_t *d_vis;  /* [cam.width * cam.height] */
    float *d_rgba;    /* [4 * cam.width * cam.height] */
} fhv_view;

/* Work decomposition (an autotuner picks these per workload). */
typedef struct {
    uint32_t views_per_item; /* views splatted from one staged fragment chunk, 1..32 */
    uint32_t frags_per_item; /* fragments per chunk, a multiple of 32 in 32..2048 */
    uint32_t pixels_per_item;/* pixels per shading work item, a multiple of 256 */
    uint32_t ctas_per_sm;    /* persistent CTAs per SM, 0 = as many as fit */
    uint32_t splat_mode;     /* k = 1 splat: 0 one fragment per thread; 1 each chunk's footprints
                                min-combined in a shared-memory tile of 2048 pixels before probing the
                                view; 2 / 3 four / eight consecutive fragments per thread, one probe
                                per run of one pixel (views whose pixels hold many fragments); 4 as
                                0, and of the lanes whose probe passes on one pixel only the nearest
                                fragment's takes the atomic; 5 as 4, and each chunk first skips the
                                views where a conservative test of its bounding box against the
                                pixels' depths shows that none of its fragments can win. In modes 0,
                                2, 3, 4 and 5 a thread probes eight views at once. k > 1 ignores the
                                mode (one fragment per thread, view by view). */
} fhv_batch_config;

/* Workspace bytes of fhv_render_views (several viewpoints submitted
 * together, Section 5) for n_views views. */
fhv_status fhv_batch_workspace_size(int n_views, size_t *bytes);

/* Renders n_views views (d_views, device array) of n_sources fragment sets
 * (d_sources, device array) with shared lights and footprint: clears every
 * view's visibility, plans the work (views of the same source that are
 * consecutive in d_views are grouped views_per_item at a time), splats
 * every (view group, fragment chunk) item from a persistent work queue --
 * each chunk's records are staged in shared memory by a bulk copy and their
 * positions decoded once for all views of the group -- then shades every
 * (view, pixel block) item. Sort views by source for the best grouping.
 * Views with a bad source index or size are skipped and raise
 * FHV_DEV_BAD_VIEW. The call launches kernels only, so it can be captured
 * in a CUDA graph. No paper counterpart beyond the remark cited above. */
#define FHV_DEV_BAD_VIEW 0x8u
fhv_status fhv_render_views(const fhv_splat_source *d_sources, int n_sources, const fhv_view *d_views, int n_views,
                            const float *d_lights, int n_lights, int footprint_k, const fhv_batch_config *cfg,
                            void *d_ws, size_t ws_bytes, fhv_stream_t stream);

/* ---------------------------------------------------------------------------
 * Learned gap-filler (no counterpart in the paper: a small convolutional
 * network that fills the holes and undersampled gaps of a sparse 1 x 1 splat,
 * trained on pairs the method itself produces -- splat of the FHV versus a
 * direct capture from the new viewpoint; plain splatting stays the
 * reference it is compared with). Activations are NHWC BF16 with 8, 16 or
 * 32 channels, 16-byte aligned; weights [cout][3][3][cin] BF16; tensor-core
 * (tcgen05) kernels accumulate in FP32. d_ws: a 16-byte aligned workspace of
 * at least FHV_RENDER_WS_BYTES whose status word collects FHV_DEV_* bits
 * across calls (clear it to reuse).
 * ------------------------------------------------------------------------- */

/* y = act(conv3x3(x, weight) + bias) with zero padding, act = ReLU if relu,
 * then y *= 1[mask > 0] channelwise if d_mask (NHWC, cout channels) is given.
 * cin in {8, 16, 32}, cout in {16, 32}; d_bias [cout] FP32 or NULL. */
fhv_status fhv_conv3x3_bf16(const void *d_x, int n, int h, int w, int cin, const void *d_weight, const float *d_bias,
                            int cout, int relu, const void *d_mask, void *d_y, void *d_ws, fhv_stream_t stream);

/* Weight and bias gradients of the convolution above (before activation):
 * d_dweight[co][ky][kx][ci] += sum over pixels p of dy[p][co] *
 * x[p + (ky - 1, kx - 1)][ci] (zero outside), d_dbias[co] += sum of dy[p][co]
 * (if not NULL). Both FP32, accumulated with atomics: clear them first;
 * d_dweight 16-byte aligned (it takes 16-byte vector reductions). d_dy is
 * NHWC BF16 with cout channels. Returns FHV_ERR_CUDA if the driver cannot
 * describe the activations to the tensor-copy unit. */
fhv_status fhv_conv3x3_wgrad_bf16(const void *d_x, const void *d_dy, int n, int h, int w, int cin, int cout,
                                  float *d_dweight, float *d_dbias, void *d_ws, fhv_stream_t stream);

/* d_flipped[ci][ky][kx][co] = d_weight[co][2 - ky][2 - kx][ci]: the weights
 * of the input gradient, which is fhv_conv3x3_bf16(dy, flipped, cin' = cout,
 * cout' = cin, mask = the layer's input activation). */
fhv_status fhv_conv3x3_flip_bf16(const void *d_weight, int cin, int cout, void *d_flipped, fhv_stream_t stream);

/* Network input from a 1 x 1 splat (fhv_render_view with footprint 1 of
 * d_frag): per pixel of cam, 8 BF16 channels {r, g, b, qd / 2^24, covered,
 * n . right, n . up, 0} with n the visible record's normal; all 0 where the
 * pixel is empty. */
fhv_status fhv_splat_features(const uint64_t *d_vis, const float *d_rgba, const fhv_record *d_frag,
                              const fhv_ortho_camera *cam, void *d_feat, fhv_stream_t stream);

/* Squared error of RGB = channels 0..2 of d_out (NHWC BF16, 16 channels)
 * plus, if d_base is given, channels 0..2 of d_base (BF16, 8 channels: the
 * splat features, so that the network predicts a residual) against d_target
 * rgb (FP32 rgba per pixel): *d_loss_sum += sum (double); if d_grad (BF16,
 * 16 channels) is given, grad = grad_scale * (out + base - target) on
 * channels 0..2 and 0 elsewhere. */
fhv_status fhv_gapfill_loss(const void *d_out, const void *d_base, const float *d_target, uint64_t pixels,
                            float grad_scale, double *d_loss_sum, void *d_grad, fhv_stream_t stream);

/* The gap-filled image: d_rgba[p] = (out rgb + base rgb, 1), d_base as in
 * fhv_gapfill_loss (or NULL). */
fhv_status fhv_gapfill_compose(const void *d_out, const void *d_base, uint64_t pixels, float *d_rgba,
                               fhv_stream_t stream);

/* One Adam step (bias-corrected; step >= 1) on n FP32 parameters; clears
 * d_grad and writes the BF16 copy to d_out_bf16 if not NULL. */
fhv_status fhv_adam_bf16(float *d_param, float *d_grad, float *d_m, float *d_v, uint64_t n, float lr, float beta1,
                         float beta2, float eps, int step, void *d_out_bf16, fhv_stream_t stream);

/* Microbenchmark of L2 atomic throughput (no paper counterpart): a fixed
 * grid applies ops_per_thread 64-bit atomic minimums per thread to words of
 * d_buf[n_words] (the largest power of two <= n_words of them, one word per
 * 32-byte sector; size the buffer to stay in L2), spread by a hash like a
 * splat's; returning = 0 leaves the results unused (reductions), 1 uses
 * them, 2 only reads the words (volatile loads, like the splat's
 * read-first probes). *ops_total (host, if not NULL) receives the number of operations
 * the launch performs; time it with events on `stream` for atomics/s. */
fhv_status fhv_atomic_probe(uint64_t *d_buf, uint64_t n_words, int ops_per_thread, int returning,
                            uint64_t *ops_total, fhv_stream_t stream);

/* Reads the fragment counter after synchronising `stream`. Returns
 * FHV_ERR_OVERFLOW when it exceeds the buffer's capacity: the caller
 * re-allocates and captures again (Section 3.1). */
fhv_status fhv_get_count(const fhv_frag_buf *frags, uint64_t *host_count, fhv_stream_t stream);

/* Reads the device status word of the last call that used this workspace
 * (FHV_DEV_* bits) after synchronising `stream`. No paper counterpart: the
 * word reports bounded waits that gave up and inputs past the library's
 * ranges, so that no kernel has to trap. */
fhv_status fhv_read_status(const void *d_ws, uint32_t *host_status, fhv_stream_t stream);

/* Kernel timing hook for measurement: while set, the first n launches of the
 * kernel named `kernel` ("fill", "setup_scan", "tile_scan", "raster", "link", "bitmap_clear",
 * "mark", "count", "level_scan", "leaf_scan", "reduce_levels", "scatter",
 * "seg_sort", "huge_sort", "raster_mark", "raster_count", "raster_scatter",
 * "leaf_index", "splat", "shade", "raycast", "batch_clear", "batch_plan",
 * "batch_splat", "batch_shade", "conv_fwd", "conv_wgrad", "gapfill_loss",
 * "atomic_probe" or "wait_probe") record start_events[i] before and stop_events[i] after
 * launch i, on the stream the kernel is launched on. The events are
 * cudaEvent_t handles owned by the caller. kernel = NULL (or n = 0) clears
 * the hook. Process-wide state; not thread-safe. No paper counterpart. */
fhv_status fhv_set_kernel_events(const char *kernel, void *const *start_events, void *const *stop_events, int n);

/* Launches recorded since the hook was last set (measurement; no paper
 * counterpart). */
int fhv_kernel_events_recorded(void);

/* Number of kernels the library has launched in this process (every launch
 * of every entry point, host-side count). No paper counterpart: a benchmark
 * reads it before and after a timed region. */
uint64_t fhv_launch_count(void);

/* Static description of a status code. */
const char *fhv_status_str(fhv_status status);

#ifdef __cplusplus
}
#endif

#endif /* FHV_H */
