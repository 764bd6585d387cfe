// kernels.h -- host-side launchers of the FHV kernels (internal; the public
// interface is include/fhv.h). Every launcher only enqueues work on `stream`
// and returns the launch error, if any.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/fhv.h"
#include "fhv_device.cuh"

namespace fhv {

// Per-triangle raster setup, 160 bytes: the three integer edge functions of
// the counter-clockwise oriented triangle (1/256 fixed-point vertices)
// evaluated at the first sample of the bounding box, lowered by one where
// the edge is not a top or left edge (so a sample is covered iff all three
// are >= 0), their change per sample step in x and y, the twice-area
// (their constant sum) and its reciprocal, the quantised position of
// vertex 0 with the other two as differences, and the vertex normals.
struct __align__(16) TriSetup {
  long long c[3];       // edge k at sample (i0, j0), minus 1 unless top-left
  long long A;          // w0 + w1 + w2 (exact edge values)
  int ea[3], eb[3];     // edge k changes by 256 ea[k] per +1 sample in x, 256 eb[k] per +1 in y
  uint32_t q0[3];       // quantised position of vertex 0 per axis
  int d1[3], d2[3];     // vertices 1 and 2 minus vertex 0 per axis
  float N[9];           // vertex normals 0, 1, 2 (same order)
  int i0, j0;           // bounding box origin sample
  uint32_t bw;          // bounding box width in samples
  float inv_bw;         // 1 / bw (estimate of the row of a sample)
  float inv_den;        // 1 / (2 A), rounded (estimate for the exact division)
  uint32_t bias;        // bit k set: edge k's exact value is one above the stored one
  uint32_t tri;         // triangle index of the records (tri_base + triangle)
  float qerr;           // bound on the float estimate of a quantised coordinate (see eval_sample)
};
static_assert(sizeof(TriSetup) == 160, "TriSetup layout");

struct RangeFill {
  void* ptr;
  unsigned long long n;  // elements
  unsigned long long value;
  int width;             // 4 or 8 bytes
};

struct CaptureArgs {
  // scene
  const uint32_t* idx;
  const float* pos;
  const float* nrm;
  uint32_t n_tri, n_vtx;
  uint32_t tri_base;  // id of the scene's first triangle (a slice of a larger scene)
  float cube_min[3];
  float cube_side;
  // projection
  int mode;          // FHV_CAPTURE_VIEW / FHV_CAPTURE_NORMAL / FHV_CAPTURE_AXIS3
  int passes;        // setups per triangle: 3 for FHV_CAPTURE_AXIS3, else 1
  uint32_t n_setup;  // n_tri * passes
  float origin[3], right[3], up[3];
  float pitch;
  int32_t width, height;
  // storage
  int keymode;  // 0 pixel, 1 leaf octant, 2 none (records only: no lists, no link pass)
  int depth;
  int sparse_reset;  // reset only the heads of the previous build's records (leaf keys)
  int32_t* head;
  uint32_t* levels;  // POFL occupancy (levels 0..depth-1) or null
  Rec* rec;
  int32_t* next;
  unsigned long long capacity;
  unsigned long long* count;
  // workspace
  WsHeader* hdr;
  TriSetup* big_setup;            // [n_setup] setups of the triangles above the warp-batch sample limit
  unsigned long long* big_meta;   // [n_setup] their (samples << 32 | setup entry)
  unsigned long long* big_pref;   // [n_setup + 1] exclusive prefix of their samples
  unsigned long long* big_chunk;  // [n_setup / 4096 + 1] per-chunk sums of the prefix scan
};

struct CompactArgs {
  const Rec* in;
  unsigned long long n_max;
  const unsigned long long* d_n;
  int depth;
  Rec* out;
  uint32_t* off;  // all levels
  uint32_t* cnt;
  WsHeader* hdr;
  unsigned long long* tile_state;
  unsigned long long* huge_list;
  unsigned long long huge_max;
  Rec* scratch;  // [n_max]
};

struct RenderArgs {
  const Rec* rec;
  unsigned long long n_max;
  const unsigned long long* d_n;
  const uint32_t* tri_material;
  const float* albedo;
  const float* lights;
  int n_lights;
  float cube_min[3];
  float cube_side;
  float origin[3], right[3], up[3], fwd[3];
  float pitch;
  int32_t width, height;
  float z0, z1;
  int k;
  unsigned long long* vis;
  float* rgba;
  WsHeader* hdr;
  unsigned long long index_base;  // records are numbered index_base + i in the visibility words
};

// Ray casting through a POFA (raycast.cu). Box bounds of the octants are
// affine in the octant centre, so the host precomputes, per level, the
// screen (s, t) and quantised-depth (q) offsets of a child centre from its
// parent's centre and each level's half extents (margins included).
constexpr int kRayMaxDepth = 11;
struct RayArgs {
  const Rec* pofa;
  unsigned long long n_max;  // records in pofa
  const uint32_t* off;
  const uint32_t* cnt;
  int depth;
  const uint32_t* tri_material;
  const float* albedo;
  const float* alpha;  // per material; NULL = opaque
  float t_stop;
  const float* lights;
  int n_lights;
  float cube_min[3];
  float cube_side;
  float origin[3], right[3], up[3], fwd[3];
  float pitch;
  int32_t width, height;
  float z0, z1;
  float root[3];                         // root centre: s, t, q
  float corner[3];                       // cube_min corner: s, t, q
  float child[kRayMaxDepth][9];          // children of level l: s, t, q offsets of +x, +y, +z halves
  float step[kRayMaxDepth + 1][9];       // level l: s, t, q change per octant along x, y, z
  float ext[kRayMaxDepth + 1][3];        // half extent of a level-l octant in s, t, q (+ half a pixel in s, t), margins added
  unsigned long long* vis;
  float* rgba;
  WsHeader* hdr;
  unsigned char* slabs;  // overflow frontier slabs (after the header)
  uint32_t n_slabs;
};
constexpr unsigned long long kRaySlabBytes = 2ull * 16384ull * 8ull;

// 3x3 convolutions of the gap-filler (conv.cu), NHWC BF16.
struct ConvArgs {
  const __nv_bfloat16* x;       // [n][h][w][cin]
  const __nv_bfloat16* weight;  // [cout][3][3][cin]
  const float* bias;            // [cout] or NULL
  const __nv_bfloat16* mask;    // [n][h][w][cout] or NULL: y *= (mask > 0)
  __nv_bfloat16* y;             // [n][h][w][cout]
  const __nv_bfloat16* dy;      // weight gradient: [n][h][w][cout]
  float* dweight;               // weight gradient, accumulated: [cout][3][3][cin]
  float* dbias;                 // bias gradient, accumulated: [cout] or NULL
  int n, h, w, cin, cout, relu;
  long long pixels_per_cta;     // weight gradient: pixels reduced per CTA
  int rows_per_item;            // forward: output rows per work item of a CTA
  WsHeader* hdr;
};
cudaError_t launch_conv_fwd(const ConvArgs& a, cudaStream_t s);
cudaError_t launch_conv_wgrad(const ConvArgs& a, cudaStream_t s);
cudaError_t launch_conv_flip(const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* out, cudaStream_t s);

// gap-filler inputs, loss and optimiser (gapfill.cu)
cudaError_t launch_splat_features(const unsigned long long* vis, const float4* rgba, const Rec* rec,
                                  const float* right, const float* up, long long pixels, __nv_bfloat16* feat,
                                  cudaStream_t s);
cudaError_t launch_gapfill_loss(const __nv_bfloat16* out, const __nv_bfloat16* base, const float4* target,
                                long long pixels, float grad_scale, double* loss_sum, __nv_bfloat16* grad,
                                cudaStream_t s);
cudaError_t launch_gapfill_compose(const __nv_bfloat16* out, const __nv_bfloat16* base, long long pixels,
                                   float4* rgba, cudaStream_t s);
cudaError_t launch_adam(float* param, float* grad, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, int step, __nv_bfloat16* out_bf16, cudaStream_t s);

cudaError_t launch_atomic_probe(unsigned long long* buf, unsigned long long n_words, int ops, int returning,
                                cudaStream_t s);

int sm_count();

// per-kernel event hook (timing.cu)
void timing_begin(const char* kernel, cudaStream_t s);
void timing_end(const char* kernel, cudaStream_t s);

// NVTX range over an entry point (host side; shows in profiler timelines,
// costs nothing when no tool is attached)
struct ApiRange {
  explicit ApiRange(const char* name);
  ~ApiRange();
};

cudaError_t launch_fill(const RangeFill* ranges, int n_ranges, cudaStream_t s);
// fills[0..n_first) are small resets done first; the rest are list arrays.
cudaError_t launch_capture(const CaptureArgs& a, const RangeFill* fills, int n_first, int n_fills, cudaStream_t s);
cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s);
// Stages of the compaction, shared with the direct POFA build (pofa.cu).
cudaError_t compact_clear_bitmap(const CompactArgs& a, cudaStream_t s);
cudaError_t compact_scan(const CompactArgs& a, cudaStream_t s);
cudaError_t compact_order(const CompactArgs& a, cudaStream_t s);
// FHV_POFA straight from the triangles by rasterising three times (mark,
// count, scatter) around the compaction's scan and order stages (capture.cu).
// `c.d_n` must point at a.hdr->n_kept, and c.n_max is the record capacity.
cudaError_t launch_pofa_direct(const CaptureArgs& a, const CompactArgs& c, const RangeFill* fills, int n_first,
                               int n_fills, cudaStream_t s);
cudaError_t launch_render(const RenderArgs& a, cudaStream_t s);

// Sparse leaf index of a POFA (leaf_index.cu): the occupied leaves in
// increasing order with the offset and count of each.
struct LeafIndexArgs {
  const Rec* pofa;
  unsigned long long n_max;
  const unsigned long long* d_n;
  int depth;
  unsigned long long* leaf;  // [n_max]
  uint32_t* off;             // [n_max]
  uint32_t* cnt;             // [n_max]
  unsigned long long* d_m;   // number of occupied leaves
  uint32_t* tile_sum;        // workspace: per-tile run counts
  unsigned long long* tile_off;  // workspace: per-tile offsets
};
unsigned long long leaf_index_tiles(unsigned long long n_max);

// FHV_POFA with a sparse index (sparse.cu): records ordered through buckets
// of level B = depth - 3 (0 for depth <= 3), then every occupied octant of
// every level as a 16-byte (octant, off, cnt) entry, levels root first.
struct SparseArgs {
  const Rec* in;
  unsigned long long n_max;
  const unsigned long long* d_n;
  int depth;
  int B;          // bucket level
  int leaf_bits;  // 3 (depth - B) <= 9: leaf bits below a bucket
  Rec* out;
  Rec* scratch;   // [n_max] records in bucket order, then merge scratch
  unsigned long long n_buckets;  // 8^B
  uint32_t* bcnt;   // [n_buckets] records per bucket
  uint32_t* boff;   // [n_buckets] first record of each bucket
  uint32_t* bcur;   // [n_buckets] scatter cursors
  uint32_t* blist;  // [n_buckets] buckets too large for a tile sort
  uint32_t* chunk_sum;  // [n_chunks] records per 4096-bucket chunk, then their prefix
  unsigned long long* level_total;  // [depth + 1] occupied octants per level
  unsigned long long n_tiles;  // 4096-record tiles of the index passes
  uint32_t* tile_lvl;          // [depth + 1][n_tiles] octant starts per level and tile, then their prefix
  fhv_octant_entry* index;
  unsigned long long index_capacity;
  unsigned long long* level_base;  // [depth + 2]
  unsigned long long* huge;        // [2 huge_max] (start, length) of leaf ranges longer than kSortCap
  unsigned long long huge_max;
  WsHeader* hdr;
};
struct SparseWs {
  int B;
  unsigned long long n_buckets, n_chunks, n_tiles, huge_max;
  unsigned long long off_bcnt, off_boff, off_bcur, off_blist, off_chunk, off_tiles, off_huge, off_scratch, total;
};
SparseWs sparse_ws(int depth, unsigned long long n_max);
cudaError_t launch_compact_sparse(const SparseArgs& a, cudaStream_t s);
// Bounded device waits on conditions nothing satisfies (selftest.cu).
cudaError_t launch_wait_probe(void* ws, int kind, cudaStream_t s);
cudaError_t launch_leaf_index(const LeafIndexArgs& a, cudaStream_t s);
// The two steps of launch_render on their own: the splat (visibility words
// only) and the shading of the pixels whose winner is one of the records
// [index_base, index_base + n), every other pixel (0, 0, 0, 0).
cudaError_t launch_splat(const RenderArgs& a, cudaStream_t s);
cudaError_t launch_shade_owned(const RenderArgs& a, cudaStream_t s);
cudaError_t launch_raycast(const RayArgs& a, cudaStream_t s);

// Workspace layout helpers (bytes), shared by fhv_query_sizes and the calls.
constexpr unsigned long long kHeaderBytes = 256;
// Setups with more bounding-box samples than these take the flattened path:
// view and normal captures, and the three-axis capture (whose triangles are
// small along every axis, so longer warp batches stay balanced).
constexpr uint32_t kSmallSamples = 128;
constexpr uint32_t kSmallSamplesAxis3 = 256;
constexpr int kLeafTile = 4096;     // leaves per compaction scan CTA (8^4)
constexpr int kSortCap = 4096;      // largest range sorted in shared memory
constexpr int kOrderSmem = 2048;    // records of the in-leaf order's shared-memory tile: longer ranges are listed

// Occupancy bitmap of the leaves during a compaction, kept inside each
// 4096-leaf tile's own stretch of the leaf offset array (offsets are written
// only later, by the CTA that owns the tile, after it has read its bitmap):
// bit (leaf & 31) of word (leaf & ~4095) + ((leaf & 4095) >> 5).
__device__ __forceinline__ uint32_t* bitmap_word(uint32_t* off_leaf, unsigned long long leaf) {
  return off_leaf + ((leaf >> 12) << 12) + ((leaf & 4095ull) >> 5);
}

inline unsigned long long round256(unsigned long long b) { return (b + 255ull) & ~255ull; }

struct CaptureWs {
  unsigned long long off_setup, off_meta, off_pref, off_chunk, total;
};
inline CaptureWs capture_ws(uint32_t n_setup) {
  CaptureWs w;
  w.off_setup = kHeaderBytes;
  w.off_meta = w.off_setup + round256((unsigned long long)n_setup * sizeof(TriSetup));
  w.off_pref = w.off_meta + round256((unsigned long long)n_setup * 8ull);
  w.off_chunk = w.off_pref + round256(((unsigned long long)n_setup + 1ull) * 8ull);
  w.total = w.off_chunk + round256(((unsigned long long)n_setup / 4096ull + 1ull) * 8ull);
  return w;
}

struct CompactWs {
  unsigned long long tiles, huge_max, off_state, off_huge, off_scratch, total;
};
inline CompactWs compact_ws(int depth, unsigned long long n_max) {
  CompactWs w;
  // look-back tiles of the scan over level T = depth - 4 (the leaf tiles' parents)
  const int T = depth > 4 ? depth - 4 : 0;
  const unsigned long long nT = 1ull << (3 * T);
  w.tiles = (nT + kLeafTile - 1) / kLeafTile;
  w.huge_max = n_max / (kOrderSmem + 1) + 1;  // ranges above the order stage's shared-memory sort
  w.off_state = kHeaderBytes;
  w.off_huge = w.off_state + round256(w.tiles * 8ull);
  w.off_scratch = w.off_huge + round256(w.huge_max * 8ull);
  w.total = w.off_scratch + round256(n_max * 16ull);
  return w;
}

}  // namespace fhv
