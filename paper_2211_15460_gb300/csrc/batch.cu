// batch.cu -- many novel views of many fragment sets in one call
// (fhv_render_views). Section 5 of the paper suggests submitting the
// view-port quads of several viewpoints together to keep the GPU busy; here
// the views share persistent kernels and work queues:
//  * batch_clear: every view's visibility to all ones (one grid row per view).
//  * batch_plan: one CTA groups consecutive views of the same source
//    (views_per_item at a time) and reserves each group's run of
//    (group, fragment chunk) work items with a single packed 64-bit atomic,
//    so the group table comes out ordered by first item.
//  * batch_splat: persistent CTAs take items from a queue; an item's records
//    (frags_per_item x 16 bytes) come into shared memory with one bulk copy,
//    their positions are decoded once, in place, and every view of the group
//    splats them with the single-view arithmetic (splat.cuh), so each view's
//    visibility is bit-identical to fhv_render_view's. k = 1 modes: runs of
//    one / four / eight consecutive records per thread (splat_mode 0 / 2 /
//    3), min-combined per pixel run, each thread probing a batch of views
//    with all their loads in flight at once (splat_mode 4: one record per
//    thread, and of the lanes whose probe passes on one pixel only the
//    nearest record's takes the atomic; splat_mode 5: as 4, after a
//    conservative per-chunk depth pre-test per view that skips the views
//    the chunk cannot change); and a tile (splat_mode 1),
//    where each view's fragments of the chunk are min-combined in a
//    shared-memory tile over their pixels' bounding box first, and only the
//    tile's covered pixels probe the view's buffer. The autotuner picks the
//    mode per workload. Items are handed out group by group, so the
//    visibility buffers being written at a time stay few.
//  * batch_shade: persistent CTAs shade (view, pixel block) items.
#include "kernels.h"
#include "splat.cuh"

namespace fhv {

struct BatchHeader {
  uint32_t status;
  uint32_t n_groups;
  unsigned long long splat_queue, shade_queue;
  unsigned long long packed;  // groups << 40 | items, for the planner
  unsigned long long max_pixels;
};
static_assert(sizeof(BatchHeader) <= kHeaderBytes, "batch header");

struct BatchGroup {
  uint32_t source, first_view, n_views, n_chunks;
  unsigned long long item_base;
  unsigned long long pad;
};

struct BatchArgs {
  const fhv_splat_source* src;
  int n_sources;
  const fhv_view* views;
  int n_views;
  const float* lights;
  int n_lights;
  int k;
  uint32_t G, C, P;
  uint32_t mode;  // k = 1 splat: 0 one record per thread, 1 shared-memory tile, 2 / 3 runs of 4 / 8 records
  BatchHeader* hdr;
  BatchGroup* groups;
};

__device__ __forceinline__ unsigned long long source_n(const fhv_splat_source& s) {
  unsigned long long n = s.n_max;
  if (s.d_n) {
    const unsigned long long c = *s.d_n;
    n = c < n ? c : n;
  }
  return n;
}

// A source is usable when its buffers exist and the records are 16-byte
// aligned (they are staged with bulk copies).
__device__ __forceinline__ bool source_ok(const fhv_splat_source& s) {
  return (s.n_max == 0 || (s.d_frag && ((uintptr_t)s.d_frag & 15u) == 0)) && s.tri_material && s.albedo &&
         s.cube_side > 0.0f;
}

// A view is usable when its source is, its size is positive and its
// visibility / colour buffers are 16-byte aligned (16-byte stores).
__device__ __forceinline__ bool view_ok(const BatchArgs& a, const fhv_view& v) {
  return v.source < (uint32_t)a.n_sources && v.cam.width > 0 && v.cam.height > 0 && v.d_vis && v.d_rgba &&
         ((uintptr_t)v.d_vis & 15u) == 0 && ((uintptr_t)v.d_rgba & 15u) == 0 && source_ok(a.src[v.source]);
}

__global__ void __launch_bounds__(256) batch_clear_kernel(BatchArgs a) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    a.hdr->status = 0;
    a.hdr->n_groups = 0;
    a.hdr->splat_queue = 0;
    a.hdr->shade_queue = 0;
    a.hdr->packed = 0;
    a.hdr->max_pixels = 0;
  }
  const fhv_view v = a.views[blockIdx.y];
  if (!view_ok(a, v)) return;
  const unsigned long long np = (unsigned long long)v.cam.width * v.cam.height;
  ulonglong2* q = reinterpret_cast<ulonglong2*>(v.d_vis);
  const unsigned long long nv = np / 2;
  const ulonglong2 e = make_ulonglong2(kVisEmpty, kVisEmpty);
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += step) q[i] = e;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (np & 1ull)) v.d_vis[np - 1] = kVisEmpty;
}

__global__ void __launch_bounds__(256) batch_plan_kernel(BatchArgs a) {
  for (int i = threadIdx.x; i < a.n_views; i += blockDim.x) {
    const fhv_view v = a.views[i];
    const bool ok = view_ok(a, v);
    if (!ok) {
      atomicOr(&a.hdr->status, FHV_DEV_BAD_VIEW);
      continue;
    }
    atomicMax(&a.hdr->max_pixels, (unsigned long long)v.cam.width * v.cam.height);
    const bool start = i == 0 || a.views[i - 1].source != v.source || !view_ok(a, a.views[i - 1]);
    if (!start) continue;
    int e = i + 1;  // end of this run of views of the same source
    while (e < a.n_views && a.views[e].source == v.source && view_ok(a, a.views[e])) ++e;
    const unsigned long long n = source_n(a.src[v.source]);
    const uint32_t chunks = (uint32_t)((n + a.C - 1) / a.C);
    for (int f = i; f < e; f += (int)a.G) {
      const uint32_t nv = (uint32_t)min((int)a.G, e - f);
      const unsigned long long p = atomicAdd(&a.hdr->packed, (1ull << 40) | (unsigned long long)chunks);
      BatchGroup g;
      g.source = v.source;
      g.first_view = (uint32_t)f;
      g.n_views = nv;
      g.n_chunks = chunks;
      g.item_base = p & ((1ull << 40) - 1ull);
      g.pad = 0;
      a.groups[p >> 40] = g;
    }
  }
}

constexpr int kMaxViewsPerItem = 32;
constexpr int kMaxFragsPerItem = 2048;
constexpr int kTilePixels = 2048;  // shared-memory visibility tile of one chunk's footprints in one view

// k = 1 splat of a staged chunk into the views v0 .. v0 + kViews - 1 of
// the group, kRun consecutive records per thread (kRun = 1: one record per
// thread). Neighbours in Morton order often share a pixel, so runs of one
// pixel are min-combined in registers first. The last run of each view is
// probed together with the other views': the batch's visibility loads are
// all issued before the first compare, so a thread has up to kViews reads
// in flight where a view-by-view loop has one. Earlier runs (a pixel change
// inside the kRun records) probe at once. With kElect, of the lanes whose
// probe passes on one pixel only the nearest record's takes the atomic
// (worth its match when pixels hold many fragments).
template <uint32_t kRun, uint32_t kViews, bool kElect>
__device__ __forceinline__ void splat_runs(const float4* s_pos, uint32_t cnt, unsigned long long lo,
                                           const SplatView* s_view, uint32_t v0, uint32_t n_views, uint32_t need) {
  const uint32_t lane = threadIdx.x & 31u;
  // the loop runs on the warp's first lane, so every lane of the warp takes
  // every iteration (the probe step below is warp-collective); lanes past
  // the chunk's end hold no records
  for (uint32_t w0 = (threadIdx.x - lane) * kRun; w0 < cnt; w0 += blockDim.x * kRun) {
    const uint32_t i0 = w0 + lane * kRun;
    const uint32_t m = i0 < cnt ? min(kRun, cnt - i0) : 0u;  // records of this thread's run
    float4 q[kRun];
#pragma unroll
    for (uint32_t j = 0; j < kRun; ++j) q[j] = s_pos[m ? i0 + (j < m ? j : 0u) : 0u];
    unsigned long long* ptr[kViews];
    unsigned long long key[kViews];
#pragma unroll
    for (uint32_t b = 0; b < kViews; ++b) {
      ptr[b] = nullptr;
      key[b] = kVisEmpty;
      if (v0 + b >= n_views || !((need >> (v0 + b)) & 1u)) continue;  // past the group, or culled
      const SplatView sv = load_view(&s_view[v0 + b]);
      unsigned long long run_pix = ~0ull, run_key = kVisEmpty;
#pragma unroll
      for (uint32_t j = 0; j < kRun; ++j) {
        if (j >= m) break;
        const float p[3] = {q[j].x, q[j].y, q[j].z};
        uint32_t ax, ay, qd;
        if (!project_k1(p, sv, ax, ay, qd)) continue;
        const unsigned long long pix = (unsigned long long)ay * (unsigned)sv.W + ax;
        const unsigned long long k = ((unsigned long long)qd << kIdxBits) | (lo + i0 + j);
        if (pix == run_pix) {
          run_key = k < run_key ? k : run_key;
        } else {
          if (run_pix != ~0ull && ld_vis(sv.vis + run_pix) > run_key) atomicMin(sv.vis + run_pix, run_key);
          run_pix = pix;
          run_key = k;
        }
      }
      if (run_pix != ~0ull) {
        ptr[b] = sv.vis + run_pix;
        key[b] = run_key;
      }
    }
    unsigned long long cur[kViews];
#pragma unroll
    for (uint32_t b = 0; b < kViews; ++b) cur[b] = ptr[b] ? ld_vis(ptr[b]) : 0ull;
    // lanes whose probe passed and that hit one pixel: only the nearest
    // record's lane (the lowest lane on a depth tie: lanes hold increasing
    // record indices) takes the atomic
#pragma unroll
    for (uint32_t b = 0; b < kViews; ++b) {
      const bool pass = ptr[b] && cur[b] > key[b];
      if (kElect) {
        const uint32_t pm = __ballot_sync(0xffffffffu, pass);
        if (!pass) continue;
        const uint32_t peers = __match_any_sync(pm, (uint32_t)(reinterpret_cast<uintptr_t>(ptr[b]) >> 3));
        bool lead = true;
        if (peers & (peers - 1u)) {
          const uint32_t code = ((uint32_t)(key[b] >> kIdxBits) << 5) | lane;
          lead = (__reduce_min_sync(peers, code) & 31u) == lane;
        }
        if (lead) atomicMin(ptr[b], key[b]);
      } else if (pass) {
        atomicMin(ptr[b], key[b]);
      }
    }
  }
}

// k = 1 splat of a staged chunk into one view through a shared-memory tile:
// the chunk's records are projected once, the bounding box of their pixels
// is reduced over the CTA, every fragment min-combines its key into the
// tile, and only the tile's covered pixels go to the view's visibility
// buffer (load first, then atomicMin), one global probe per pixel instead
// of one per fragment. Min is associative, so the result is the same as
// splat_point's. A box larger than the tile falls back to splat_point.
__device__ __forceinline__ void splat_chunk_tiled(const float4* s_pos, uint32_t cnt, unsigned long long lo,
                                                  const SplatView& sv, unsigned long long* s_tile, int* s_box) {
  constexpr int kPer = kMaxFragsPerItem / 256;
  const int tid = threadIdx.x;
  int px[kPer], py[kPer];
  uint32_t qd[kPer];
  int x0 = 0x7fffffff, y0 = 0x7fffffff, x1 = -1, y1 = -1;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const uint32_t i = (uint32_t)(j * 256 + tid);
    px[j] = -1;
    if (i < cnt) {
      const float4 q = s_pos[i];
      const float p[3] = {q.x, q.y, q.z};
      const Projected pr = project_point(p, sv);
      if (pr.ax >= 0 && pr.ax < sv.W && pr.ay >= 0 && pr.ay < sv.H) {
        px[j] = pr.ax;
        py[j] = pr.ay;
        qd[j] = pr.qd;
        x0 = min(x0, pr.ax);
        y0 = min(y0, pr.ay);
        x1 = max(x1, pr.ax);
        y1 = max(y1, pr.ay);
      }
    }
  }
  x0 = __reduce_min_sync(0xffffffffu, x0);
  y0 = __reduce_min_sync(0xffffffffu, y0);
  x1 = __reduce_max_sync(0xffffffffu, x1);
  y1 = __reduce_max_sync(0xffffffffu, y1);
  if ((tid & 31) == 0) {
    atomicMin(&s_box[0], x0);
    atomicMin(&s_box[1], y0);
    atomicMax(&s_box[2], x1);
    atomicMax(&s_box[3], y1);
  }
  __syncthreads();  // the box is complete
  const bool empty = s_box[2] < 0;
  const int bx = s_box[0], by = s_box[1];
  const long long bw = empty ? 0 : (long long)s_box[2] - bx + 1, bh = empty ? 0 : (long long)s_box[3] - by + 1;
  const bool tiled = !empty && bw * bh <= kTilePixels;
  __syncthreads();  // read by every thread: reset it for the next view
  if (tid == 0) {
    s_box[0] = 0x7fffffff;
    s_box[1] = 0x7fffffff;
    s_box[2] = -1;
    s_box[3] = -1;
  }
  if (!tiled) {  // CTA-uniform: nothing in view, or a box larger than the tile
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (px[j] < 0) continue;
      const unsigned long long key = ((unsigned long long)qd[j] << kIdxBits) | (lo + (unsigned long long)(j * 256 + tid));
      unsigned long long* g = sv.vis + (unsigned long long)py[j] * sv.W + px[j];
      if (ld_vis(g) > key) atomicMin(g, key);
    }
    __syncthreads();  // the reset is seen before the next view's box
    return;
  }
  const int area = (int)(bw * bh);
  for (int p = tid; p < area; p += blockDim.x) s_tile[p] = kVisEmpty;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    if (px[j] < 0) continue;
    const unsigned long long key = ((unsigned long long)qd[j] << kIdxBits) | (lo + (unsigned long long)(j * 256 + tid));
    atomicMin(&s_tile[(py[j] - by) * (int)bw + (px[j] - bx)], key);
  }
  __syncthreads();
  for (int p = tid; p < area; p += blockDim.x) {
    const unsigned long long key = s_tile[p];
    if (key == kVisEmpty) continue;
    unsigned long long* g = sv.vis + (unsigned long long)(by + p / (int)bw) * sv.W + (bx + p % (int)bw);
    if (ld_vis(g) > key) atomicMin(g, key);
  }
  __syncthreads();  // tile free for the next view
}

// Per-chunk depth pre-test (splat mode 5). The chunk's records lie in the
// box bb (min x, y, z, max x, y, z) of their decoded positions. Projected
// with the splat's own float32 steps, a position's screen coordinate and
// depth differ from their exact (affine) values by a few roundings of terms
// bounded by ext = |dx| + |dy| + |dz| (d = position - view origin): below
// 8u ext inv_pitch + u |sx| pixels and 8u ext in depth (u = 2^-24). The
// exact values of an inner point lie between the corners' exact values, so
// every record's pixel lies within 2 pixels of the corners' pixel range
// while ext inv_pitch and |sx| stay below 2^19, and its depth code is at
// least the corners' smallest minus M = 2^-18 ext qscale + 8 (monotone
// rounding of the code's steps, four codes per rounding, doubled). If every
// pixel of that rectangle already holds a depth code below the bound, no
// record of the chunk can win a pixel in this view; a rectangle wholly off
// the screen means none lands on it. Values only decrease, so a stale
// read only makes the test fail. One warp per view.
constexpr uint32_t kCullArea = 4096;  // larger rectangles are not tested

__device__ __forceinline__ void chunk_bounds(const float4* s_pos, uint32_t cnt, float* s_red, float bb[6]) {
  float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const float4 q = s_pos[i];
    v[0] = fminf(v[0], q.x), v[1] = fminf(v[1], q.y), v[2] = fminf(v[2], q.z);
    v[3] = fmaxf(v[3], q.x), v[4] = fmaxf(v[4], q.y), v[5] = fmaxf(v[5], q.z);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float w = __shfl_xor_sync(0xffffffffu, v[k], o);
      v[k] = k < 3 ? fminf(v[k], w) : fmaxf(v[k], w);
    }
  const uint32_t warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31u) == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) s_red[6 * warp + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 6; ++k) bb[k] = s_red[k];
  for (uint32_t w = 1; w < nw; ++w)
#pragma unroll
    for (int k = 0; k < 6; ++k) bb[k] = k < 3 ? fminf(bb[k], s_red[6 * w + k]) : fmaxf(bb[k], s_red[6 * w + k]);
}

// True when the chunk in box bb may still change view sv (called by a whole
// warp; every lane gets the answer).
__device__ __forceinline__ bool chunk_may_splat(const SplatView& sv, const float bb[6]) {
  const uint32_t lane = threadIdx.x & 31u, c = lane & 7u;
  const float p[3] = {(c & 1u) ? bb[3] : bb[0], (c & 2u) ? bb[4] : bb[1], (c & 4u) ? bb[5] : bb[2]};
  const Projected pr = project_point(p, sv);
  float ext = fabsf(fsub(p[0], sv.o[0])) + fabsf(fsub(p[1], sv.o[1])) + fabsf(fsub(p[2], sv.o[2]));
  int x0 = pr.ax, x1 = pr.ax, y0 = pr.ay, y1 = pr.ay, mag = max(abs(pr.ax), abs(pr.ay));
  uint32_t qmin = pr.qd;
#pragma unroll
  for (int o = 4; o >= 1; o >>= 1) {  // over the eight corners (lanes repeat them by eights)
    x0 = min(x0, __shfl_xor_sync(0xffffffffu, x0, o));
    x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, o));
    y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, o));
    y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    mag = max(mag, __shfl_xor_sync(0xffffffffu, mag, o));
    qmin = min(qmin, __shfl_xor_sync(0xffffffffu, qmin, o));
    ext = fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, o));
  }
  if (!(ext * sv.inv_pitch < 524288.0f) || mag >= (1 << 19)) return true;  // bounds not established
  const int X0 = max(x0 - 2, 0), X1 = min(x1 + 2, sv.W - 1), Y0 = max(y0 - 2, 0), Y1 = min(y1 + 2, sv.H - 1);
  if (X0 > X1 || Y0 > Y1) return false;  // every record off the screen
  const float m = ext * sv.qscale * (1.0f / 262144.0f) + 8.0f;
  if (!(m < 16777216.0f) || (float)qmin <= m) return true;
  const uint32_t qlim = qmin - (uint32_t)ceilf(m);
  const uint32_t bw = (uint32_t)(X1 - X0 + 1), area = bw * (uint32_t)(Y1 - Y0 + 1);
  if (area > kCullArea) return true;
  for (uint32_t base = 0; base < area; base += 32) {  // warp-uniform trip count
    const uint32_t k = base + lane;
    bool open = false;
    if (k < area) {
      const uint32_t py = (uint32_t)Y0 + k / bw, px = (uint32_t)X0 + k % bw;
      open = (uint32_t)(ld_vis(sv.vis + (unsigned long long)py * (unsigned)sv.W + px) >> kIdxBits) >= qlim;
    }
    if (__any_sync(0xffffffffu, open)) return true;
  }
  return false;
}

// Splat kernel of one mode (each mode its own kernel, so each is register-
// allocated for its own loop): 0 / 2 / 3 runs of 1 / 4 / 8 records with the
// probes of kViewBatch views at a time, 4 runs of 1 with the pixel election,
// 5 as 4 after the per-chunk depth pre-test, 1 the shared-memory tile, 6 any
// footprint k (one record per thread, view by view; not a splat_mode).
constexpr uint32_t kViewBatch = 8;
enum SplatKernel : int {
  kSplatRuns1 = 0, kSplatTile = 1, kSplatRuns4 = 2, kSplatRuns8 = 3, kSplatElect1 = 4, kSplatCull1 = 5,
  kSplatFootprint = 6
};

template <int kMode>
__global__ void __launch_bounds__(256, kMode == kSplatRuns4 || kMode == kSplatRuns8 ? 2 : 4)
    batch_splat_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint4* s_rec = reinterpret_cast<uint4*>(smem);                         // [C] staged records
  float4* s_pos = reinterpret_cast<float4*>(smem);                       // [C] their positions, decoded in place
  SplatView* s_view = reinterpret_cast<SplatView*>(smem + 16 * a.C);     // [G]
  unsigned long long* s_tile =                                             // [kTilePixels] in mode 1
      reinterpret_cast<unsigned long long*>(smem + 16 * a.C + sizeof(SplatView) * a.G);
  __shared__ int s_box[4];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ unsigned long long s_item;
  __shared__ int s_group;
  __shared__ float s_red[6 * 8];  // mode 5: per-warp bounds of the chunk
  __shared__ uint32_t s_need;     // mode 5: views of the group the chunk may change (bit v)
  const int tid = threadIdx.x;
  const unsigned long long packed = a.hdr->packed;
  const uint32_t n_groups = (uint32_t)(packed >> 40);
  const unsigned long long n_items = packed & ((1ull << 40) - 1ull);
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
    s_box[0] = 0x7fffffff;
    s_box[1] = 0x7fffffff;
    s_box[2] = -1;
    s_box[3] = -1;
  }
  __syncthreads();
  uint32_t phase = 0;
  while (true) {
    if (tid == 0) {
      const unsigned long long it = atomicAdd(&a.hdr->splat_queue, 1ull);
      s_item = it;
      s_need = 0u;
      int g = -1;
      if (it < n_items) {  // last group whose first item <= it
        int lo = 0, hi = (int)n_groups;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (a.groups[mid].item_base <= it) lo = mid + 1;
          else hi = mid;
        }
        g = lo - 1;
      }
      s_group = g;
    }
    __syncthreads();
    const unsigned long long item = s_item;
    if (item >= n_items) break;
    const BatchGroup grp = a.groups[s_group];
    const fhv_splat_source src = a.src[grp.source];
    const unsigned long long n = source_n(src);
    const unsigned long long lo = (item - grp.item_base) * a.C;
    const uint32_t cnt = lo < n ? (uint32_t)min((unsigned long long)a.C, n - lo) : 0u;
    if (tid == 0 && cnt) {
      fence_proxy_async_smem();  // earlier generic reads of s_rec before the async write
      mbar_arrive_expect_tx(&s_bar, cnt * 16u);
      bulk_g2s(s_rec, src.d_frag + lo, cnt * 16u, &s_bar);
    }
    if ((uint32_t)tid < grp.n_views) {
      const fhv_view v = a.views[grp.first_view + tid];
      s_view[tid] = make_splat_view(src.cube_min, src.cube_side, v.cam.origin, v.cam.right, v.cam.up, v.cam.fwd,
                                    v.cam.pitch, v.cam.width, v.cam.height, v.cam.z0, v.cam.z1, a.k,
                                    reinterpret_cast<unsigned long long*>(v.d_vis));
    }
    if (cnt) {
      if (!mbar_wait_bounded(&s_bar, phase)) {
        if (tid == 0) set_status(&a.hdr->status, FHV_DEV_TIMEOUT);
        mbar_wait_bounded(&s_bar, phase);
      }
      phase ^= 1u;
    }
    __syncthreads();  // views ready
    const SplatView s0 = load_view(&s_view[0]);  // the source's cube, shared by the group's views
    for (uint32_t i = tid; i < cnt; i += blockDim.x) {  // in place: each thread reads and writes its own slot
      const uint4 r = s_rec[i];
      float p[3];
      dequantize((unsigned long long)r.x | ((unsigned long long)r.y << 32), s0, p);
      s_pos[i] = make_float4(p[0], p[1], p[2], 0.0f);
    }
    __syncthreads();
    if (kMode == kSplatTile) {
      for (uint32_t v = 0; v < grp.n_views; ++v)
        splat_chunk_tiled(s_pos, cnt, lo, load_view(&s_view[v]), s_tile, s_box);
    } else if (kMode == kSplatFootprint) {
      for (uint32_t v = 0; v < grp.n_views; ++v) {
        const SplatView sv = load_view(&s_view[v]);
        for (uint32_t i = tid; i < cnt; i += blockDim.x) {
          const float4 q = s_pos[i];
          const float p[3] = {q.x, q.y, q.z};
          splat_point(p, lo + i, sv);
        }
      }
    } else {
      constexpr bool kOne = kMode == kSplatRuns1 || kMode == kSplatElect1 || kMode == kSplatCull1;
      constexpr uint32_t kRun = kOne ? 1u : kMode == kSplatRuns4 ? 4u : 8u;
      uint32_t need = 0xffffffffu;
      if (kMode == kSplatCull1 && cnt) {  // CTA-uniform
        float bb[6];
        chunk_bounds(s_pos, cnt, s_red, bb);
        for (uint32_t v = (uint32_t)tid >> 5; v < grp.n_views; v += blockDim.x >> 5)  // warp-uniform
          if (chunk_may_splat(load_view(&s_view[v]), bb) && (tid & 31) == 0) atomicOr(&s_need, 1u << v);
        __syncthreads();
        need = s_need;
      }
      for (uint32_t v0 = 0; v0 < grp.n_views; v0 += kViewBatch)
        splat_runs<kRun, kViewBatch, kMode == kSplatElect1 || kMode == kSplatCull1>(s_pos, cnt, lo, s_view, v0,
                                                                                   grp.n_views, need);
    }
    __syncthreads();  // shared buffers free for the next item
  }
}

__global__ void __launch_bounds__(256) batch_shade_kernel(BatchArgs a) {
  __shared__ float s_l[64 * 8];
  __shared__ unsigned long long s_item;
  for (int i = threadIdx.x; i < a.n_lights * 8; i += blockDim.x) s_l[i] = a.lights[i];
  const unsigned long long tiles = (a.hdr->max_pixels + a.P - 1) / a.P;
  const unsigned long long n_items = tiles * (unsigned long long)a.n_views;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(&a.hdr->shade_queue, 1ull);
    __syncthreads();
    const unsigned long long item = s_item;
    if (item >= n_items) break;
    const fhv_view v = a.views[item / tiles];
    if (!view_ok(a, v)) continue;
    const fhv_splat_source src = a.src[v.source];
    const unsigned long long np = (unsigned long long)v.cam.width * v.cam.height;
    const unsigned long long p0 = (item % tiles) * a.P, p1 = min(np, p0 + a.P);
    for (unsigned long long p = p0 + threadIdx.x; p < p1; p += blockDim.x)
      reinterpret_cast<float4*>(v.d_rgba)[p] = shade_pixel(v.d_vis[p], reinterpret_cast<const Rec*>(src.d_frag),
                                                          src.tri_material, src.albedo, src.cube_min, src.cube_side,
                                                          s_l, a.n_lights);
  }
}

static int blocks_per_sm(const void* fn, size_t smem) {
  int v = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, 256, smem);
  return v > 0 ? v : 1;
}

}  // namespace fhv

using namespace fhv;

extern "C" fhv_status fhv_batch_workspace_size(int n_views, size_t* bytes) {
  if (!bytes || n_views < 0) return FHV_ERR_INVALID_ARG;
  *bytes = kHeaderBytes + round256((unsigned long long)n_views * sizeof(BatchGroup));
  return FHV_OK;
}

extern "C" fhv_status fhv_render_views(const fhv_splat_source* d_sources, int n_sources, const fhv_view* d_views,
                                       int n_views, const float* d_lights, int n_lights, int footprint_k,
                                       const fhv_batch_config* cfg, void* d_ws, size_t ws_bytes,
                                       fhv_stream_t stream) {
  ApiRange range_("fhv_render_views");
  if (!d_sources || n_sources < 1 || !d_views || n_views < 1 || n_views > 65535) return FHV_ERR_INVALID_ARG;
  if (n_lights < 0 || n_lights > 64 || (n_lights > 0 && !d_lights) || footprint_k < 1 || footprint_k > 16)
    return FHV_ERR_INVALID_ARG;
  if (((uintptr_t)d_sources & 15u) || ((uintptr_t)d_views & 15u) || ((uintptr_t)d_ws & 15u)) return FHV_ERR_INVALID_ARG;
  fhv_batch_config c = cfg ? *cfg : fhv_batch_config{8u, 2048u, 4096u, 0u, 0u};
  if (c.views_per_item < 1 || c.views_per_item > (uint32_t)kMaxViewsPerItem) return FHV_ERR_INVALID_ARG;
  if (c.frags_per_item < 32 || c.frags_per_item > (uint32_t)kMaxFragsPerItem || c.frags_per_item % 32)
    return FHV_ERR_INVALID_ARG;
  if (c.pixels_per_item < 256 || c.pixels_per_item % 256 || c.ctas_per_sm > 8 || c.splat_mode > 5)
    return FHV_ERR_INVALID_ARG;
  size_t need = 0;
  fhv_batch_workspace_size(n_views, &need);
  if (!d_ws || ws_bytes < need) return FHV_ERR_INVALID_ARG;
  BatchArgs a;
  a.src = d_sources;
  a.n_sources = n_sources;
  a.views = d_views;
  a.n_views = n_views;
  a.lights = d_lights;
  a.n_lights = n_lights;
  a.k = footprint_k;
  a.G = c.views_per_item;
  a.C = c.frags_per_item;
  a.P = c.pixels_per_item;
  a.mode = c.splat_mode;
  a.hdr = reinterpret_cast<BatchHeader*>(d_ws);
  a.groups = reinterpret_cast<BatchGroup*>((char*)d_ws + kHeaderBytes);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int km = a.k != 1 ? kSplatFootprint : (int)c.splat_mode;
  const void* fn = km == kSplatRuns1   ? (const void*)batch_splat_kernel<kSplatRuns1>
                   : km == kSplatTile  ? (const void*)batch_splat_kernel<kSplatTile>
                   : km == kSplatRuns4 ? (const void*)batch_splat_kernel<kSplatRuns4>
                   : km == kSplatRuns8 ? (const void*)batch_splat_kernel<kSplatRuns8>
                   : km == kSplatElect1 ? (const void*)batch_splat_kernel<kSplatElect1>
                   : km == kSplatCull1  ? (const void*)batch_splat_kernel<kSplatCull1>
                                        : (const void*)batch_splat_kernel<kSplatFootprint>;
  const size_t smem = (size_t)a.C * 16 + sizeof(SplatView) * a.G + (km == kSplatTile ? kTilePixels * 8 : 0);
  static bool attr = false;
  if (!attr) {
    const int most = kMaxFragsPerItem * 16 + (int)sizeof(SplatView) * kMaxViewsPerItem + kTilePixels * 8;
    cudaFuncSetAttribute(batch_splat_kernel<kSplatRuns1>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(batch_splat_kernel<kSplatTile>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(batch_splat_kernel<kSplatRuns4>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(batch_splat_kernel<kSplatRuns8>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(batch_splat_kernel<kSplatElect1>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(batch_splat_kernel<kSplatCull1>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(batch_splat_kernel<kSplatFootprint>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    attr = true;
  }
  const int sms = sm_count();
  timing_begin("batch_clear", s);
  batch_clear_kernel<<<dim3(16, n_views), 256, 0, s>>>(a);
  timing_end("batch_clear", s);
  timing_begin("batch_plan", s);
  batch_plan_kernel<<<1, 256, 0, s>>>(a);
  timing_end("batch_plan", s);
  const int bs = c.ctas_per_sm ? (int)c.ctas_per_sm : blocks_per_sm(fn, smem);
  void* args[] = {&a};
  timing_begin("batch_splat", s);
  cudaLaunchKernel(fn, dim3(sms * bs), dim3(256), args, smem, s);
  timing_end("batch_splat", s);
  const int bh = c.ctas_per_sm ? (int)c.ctas_per_sm : blocks_per_sm((const void*)batch_shade_kernel, 0);
  timing_begin("batch_shade", s);
  batch_shade_kernel<<<sms * bh, 256, 0, s>>>(a);
  timing_end("batch_shade", s);
  return cudaGetLastError() == cudaSuccess ? FHV_OK : FHV_ERR_CUDA;
}
