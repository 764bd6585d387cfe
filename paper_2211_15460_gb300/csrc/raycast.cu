// raycast.cu -- image generation by ray casting through the octree of a
// FHV_POFA (Section 3.3; Table 3 "R" and "R/T").
//
// What is computed. A fragment lies on a pixel's ray when its projection
// falls in the pixel (the rule of a 1 x 1 splat: same float32 arithmetic, so
// membership and the depth key (qdepth << 40 | index) are bit-equal to the
// splat's). A ray takes its fragments in increasing key order and composites
// them front to back, C += T a c, T *= 1 - a, stopping once T <= t_stop (the
// paper's early-out on accumulated transparency; opaque casting R has a = 1).
//
// Exact order. Appending whole octants in visiting order is not exact: two
// fragments of one pixel in different octants can swap depth order near an
// octant face. So a fragment is composited only once its depth lies below
// the smallest depth bound of the octants still to visit; until then it
// waits in a buffer of the K nearest pending keys. When the buffer is full,
// a key or octant beyond its largest key is dropped and the drop lowers
// `bhi`, the key below which the pass has seen everything; the ray then runs
// another pass over what lies behind its last composited key. R uses K = 1.
//
// GB300 layout. One warp casts the 32 rays of an 8 x 4 pixel tile together:
//  * breadth-first descent of the octree over the tile's beam: every child
//    (node, c) of the current level is one lane's work item, so each level's
//    count loads are issued together (32 bytes per node, coalesced), and the
//    survivors -- children that hold fragments and whose projected box
//    reaches the tile -- are appended with a ballot to a per-warp frontier in
//    shared memory;
//  * the leaves reached are bucket-sorted by depth lower bound and a suffix
//    minimum of those bounds gives, after each batch, the exact release bound
//    of the leaves not yet processed;
//  * leaves are processed 32 at a time: their records are loaded coalesced,
//    one per lane, projected, and each hit is handed through shared memory to
//    the lane that owns its pixel (a per-lane inbox mask built with a match
//    on the destination), which inserts it into its register buffer;
//  * the warp stops when every lane is done.
// A tile whose frontier outgrows the shared buffer moves it to an overflow
// slab of the workspace (claimed from a bitmap, never waited for); only if
// no slab is free or it outgrows that too does the tile fall back to one
// depth-first traversal per pixel (nearest child first, with the depth bound
// of everything still on the stack kept as a prefix minimum per level).
// Later passes skip leaf batches that lie wholly in front of every lane's
// lower key bound.
//
// Octant bounds are affine in the octant centre: the host precomputes, in
// (s, t, q) = (screen x, screen y, quantised depth), the projection of the
// cube corner, per-level steps and child offsets, and per-level half extents
// widened by a margin that covers the float32 rounding of both the bounds
// and the fragment projection.
#include "kernels.h"
#include "splat.cuh"

namespace fhv {

namespace {

constexpr uint32_t kNoQ = 0xFFFFFFFFu;
constexpr unsigned long long kNoKey = ~0ull;
constexpr int kTileW = 8, kTileH = 4;
constexpr int kRayWarps = 4;      // warps (tiles) per CTA
constexpr int kFrontCap = 768;    // frontier entries per warp and buffer, shared memory (4 CTAs per SM)
constexpr int kSlabCap = 16384;   // the same in an overflow slab (global memory)
constexpr int kBuckets = 32;

__device__ __forceinline__ uint32_t q_floor(float v) {
  const float f = floorf(v);
  if (!(f >= 0.0f)) return 0u;
  if (f >= 16777215.0f) return (1u << 24) - 1u;
  return (uint32_t)f;
}

__device__ __forceinline__ uint32_t q_ceil(float v) {
  const float f = ceilf(v);
  if (!(f >= 0.0f)) return 0u;
  if (f >= 16777215.0f) return (1u << 24) - 1u;
  return (uint32_t)f;
}

// Centre of child k (bit 2 = +x half, bit 1 = +y, bit 0 = +z) from its
// parent's centre; d holds the (s, t, q) offsets of the +x, +y, +z halves.
__device__ __forceinline__ void child_centre(float s, float t, float q, const float* d, int k, float& cs, float& ct,
                                             float& cq) {
  cs = s + ((k & 4) ? d[0] : -d[0]) + ((k & 2) ? d[3] : -d[3]) + ((k & 1) ? d[6] : -d[6]);
  ct = t + ((k & 4) ? d[1] : -d[1]) + ((k & 2) ? d[4] : -d[4]) + ((k & 1) ? d[7] : -d[7]);
  cq = q + ((k & 4) ? d[2] : -d[2]) + ((k & 2) ? d[5] : -d[5]) + ((k & 1) ? d[8] : -d[8]);
}

// Centre of octant `node` (Morton index) of a level from its coordinates:
// corner + (coordinate + 1/2) * step per axis.
__device__ __forceinline__ void node_centre(unsigned long long node, const float* corner, const float* st, float& s,
                                            float& t, float& q) {
  const float i = (float)compact3(node >> 2) + 0.5f, j = (float)compact3(node >> 1) + 0.5f,
              k = (float)compact3(node) + 0.5f;
  s = corner[0] + i * st[0] + j * st[3] + k * st[6];
  t = corner[1] + i * st[1] + j * st[4] + k * st[7];
  q = corner[2] + i * st[2] + j * st[5] + k * st[8];
}

__device__ __forceinline__ void cswap(uint32_t& a, uint32_t& b) {
  const uint32_t lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// Batcher's odd-even merge network for 8 keys (19 comparators).
__device__ __forceinline__ void sort8(uint32_t v[8]) {
  cswap(v[0], v[1]); cswap(v[2], v[3]); cswap(v[4], v[5]); cswap(v[6], v[7]);
  cswap(v[0], v[2]); cswap(v[1], v[3]); cswap(v[4], v[6]); cswap(v[5], v[7]);
  cswap(v[1], v[2]); cswap(v[5], v[6]);
  cswap(v[0], v[4]); cswap(v[1], v[5]); cswap(v[2], v[6]); cswap(v[3], v[7]);
  cswap(v[2], v[4]); cswap(v[3], v[5]);
  cswap(v[1], v[2]); cswap(v[3], v[4]); cswap(v[5], v[6]);
}

// Shading inputs shared by every ray of a CTA.
struct ShadeCtx {
  const RayArgs* a;
  const float* lights;  // shared-memory copy
};

// One ray's compositing state: the K nearest pending keys (sorted, in
// registers), the composited colour and the pass bounds.
template <int K>
struct RayState {
  unsigned long long buf[K];
  int nb;
  unsigned long long lmin;   // keys below lmin are composited
  unsigned long long bhi;    // this pass has seen every key below bhi
  unsigned long long last;   // last composited key
  unsigned long long first;  // nearest key (the visibility word)
  float cr, cg, cb, T;
  bool fin;                  // nothing more to do for this ray

  __device__ __forceinline__ void init(bool active) {
#pragma unroll
    for (int j = 0; j < K; ++j) buf[j] = kNoKey;
    nb = 0;
    lmin = 0;
    bhi = kNoKey;
    last = kNoKey;
    first = kVisEmpty;
    cr = cg = cb = 0.0f;
    T = 1.0f;
    fin = !active;
  }

  __device__ __forceinline__ void insert(unsigned long long key) {
    if (key < lmin || key >= bhi) return;
    if (nb == K) {
      if (key > buf[K - 1]) {
        bhi = min(bhi, key);
        return;
      }
      bhi = min(bhi, buf[K - 1]);
      --nb;
    }
    unsigned long long v = key;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (j < nb) {
        const unsigned long long b = buf[j];
        if (v < b) {
          buf[j] = v;
          v = b;
        }
      } else if (j == nb) {
        buf[j] = v;
      }
    }
    ++nb;
  }

  __device__ __forceinline__ void composite(unsigned long long key, const ShadeCtx& cx) {
    const RayArgs& a = *cx.a;
    const uint4 r = __ldg(reinterpret_cast<const uint4*>(a.pofa) + (key & kIdxMask));
    const float4 c = shade_pixel(key, a.pofa, a.tri_material, a.albedo, a.cube_min, a.cube_side, cx.lights, a.n_lights);
    const float al = a.alpha ? __ldg(a.alpha + __ldg(a.tri_material + r.z)) : 1.0f;
    const float w = T * al;
    cr += w * c.x;
    cg += w * c.y;
    cb += w * c.z;
    T *= 1.0f - al;
    if (first == kVisEmpty) first = key;
    last = key;
    if (T <= a.t_stop) fin = true;
  }

  // Composite, in order, the pending keys whose depth lies below lim.
  __device__ __forceinline__ void release(uint32_t lim, const ShadeCtx& cx) {
    while (nb > 0 && !fin && (uint32_t)(buf[0] >> kIdxBits) < lim) {
      composite(buf[0], cx);
#pragma unroll
      for (int j = 0; j + 1 < K; ++j) buf[j] = buf[j + 1];
      buf[K - 1] = kNoKey;
      --nb;
    }
  }

  // End of a pass: composite what is left; another pass is needed only if
  // something was dropped and the ray is not done.
  __device__ __forceinline__ bool end_pass(const ShadeCtx& cx) {
    release(kNoQ, cx);
    if (fin || bhi == kNoKey || last == kNoKey) {
      fin = true;
      return false;
    }
    lmin = last + 1;
    bhi = kNoKey;
    return true;
  }
};

// Depth-first cast of one ray (the fallback for tiles whose frontier does
// not fit in shared memory).
template <int K>
__device__ void dfs_ray(const RayArgs& a, const ShadeCtx& cx, const float (*s_child)[9], const float (*s_ext)[3], int x,
                        int y, const SplatView& sv, RayState<K>& st) {
  const float pcx = (float)x + 0.5f, pcy = (float)y + 0.5f;
  const int depth = a.depth;
  const uint4* recs = reinterpret_cast<const uint4*>(a.pofa);
  // par[top]: index of the octant whose children stack level top holds (at
  // levels <= 10 an index fits in 30 bits; a child's index, up to 8^11, is
  // formed in 64 bits)
  uint32_t par[kRayMaxDepth + 1], ord[kRayMaxDepth + 1], pm[kRayMaxDepth + 1];
  float cs[kRayMaxDepth + 1], ct[kRayMaxDepth + 1], cq[kRayMaxDepth + 1];
  const bool root_ok =
      __ldg(a.cnt) > 0u && fabsf(a.root[0] - pcx) <= s_ext[0][0] && fabsf(a.root[1] - pcy) <= s_ext[0][1];
  if (!root_ok) st.fin = true;
  while (!st.fin) {
    const uint32_t lmin_q = (uint32_t)(st.lmin >> kIdxBits);
    int top = 0;
    par[0] = 0;
    ord[0] = 1u << 24;  // one entry (child id 0): the root
    pm[0] = 0;
    while (top >= 0 && !st.fin) {
      const uint32_t o = ord[top];
      uint32_t n = o >> 24;
      if (n == 0) {
        --top;
        continue;
      }
      const int c = (int)(o & 7u);
      --n;
      ord[top] = (n << 24) | ((o & 0xFFFFFFu) >> 3);
      const unsigned long long node = top ? ((unsigned long long)par[top] << 3) + (unsigned long long)c : 0ull;
      const float* d = top ? s_child[top - 1] : nullptr;
      float s, t, q;
      if (top == 0) {
        s = a.root[0];
        t = a.root[1];
        q = a.root[2];
      } else {
        child_centre(cs[top], ct[top], cq[top], d, c, s, t, q);
      }
      const float eq = s_ext[top][2];
      // depth bound of everything still on the stack after this pop
      const uint32_t below = top ? pm[top - 1] : kNoQ;
      uint32_t nxt = kNoQ;
      if (n) {
        float s2, t2, q2;
        child_centre(cs[top], ct[top], cq[top], d, (int)(ord[top] & 7u), s2, t2, q2);
        nxt = q_floor(q2 - eq);
      }
      pm[top] = min(below, nxt);
      const uint32_t qlo = q_floor(q - eq);
      const unsigned long long lo_key = (unsigned long long)qlo << kIdxBits;
      // Siblings are ordered by qlo, so a bound that drops this octant drops
      // the rest of the level too.
      if (lo_key >= st.bhi) {
        ord[top] = 0;
        pm[top] = below;
        continue;
      }
      if (st.nb == K && lo_key > st.buf[K - 1]) {
        st.bhi = min(st.bhi, lo_key);
        ord[top] = 0;
        pm[top] = below;
        continue;
      }
      if (q_ceil(q + eq) < lmin_q) continue;  // composited in an earlier pass

      if (top == depth) {
        const unsigned long long e = level_offset(depth) + node;
        const unsigned long long beg = __ldg(a.off + e);
        unsigned long long end = beg + __ldg(a.cnt + e);
        if (end > a.n_max) {  // inconsistent offsets: stay inside the record array
          set_status(&a.hdr->status, FHV_DEV_RANGE);
          end = a.n_max;
        }
        for (unsigned long long i = beg; i < end; ++i) {
          const uint4 r = __ldg(recs + i);
          float p[3];
          dequantize((unsigned long long)r.x | ((unsigned long long)r.y << 32), sv, p);
          const Projected pr = project_point(p, sv);
          if (pr.ax == x && pr.ay == y) st.insert(((unsigned long long)pr.qd << kIdxBits) | i);
        }
        st.release(pm[top], cx);
        continue;
      }

      // Expand: children at level top + 1 that hold fragments and reach the pixel.
      const uint32_t* cp = a.cnt + level_offset(top + 1) + 8ull * node;
      const uint4 c0 = __ldg(reinterpret_cast<const uint4*>(cp)), c1 = __ldg(reinterpret_cast<const uint4*>(cp) + 1);
      const uint32_t cc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
      const float* dc = s_child[top];
      const float es = s_ext[top + 1][0], et = s_ext[top + 1][1], eqc = s_ext[top + 1][2];
      uint32_t v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        v[k] = kNoQ;
        if (cc[k] == 0u) continue;
        float s2, t2, q2;
        child_centre(s, t, q, dc, k, s2, t2, q2);
        if (fabsf(s2 - pcx) > es || fabsf(t2 - pcy) > et) continue;
        if (q_ceil(q2 + eqc) < lmin_q) continue;
        const uint32_t lo = q_floor(q2 - eqc);
        const unsigned long long lk = (unsigned long long)lo << kIdxBits;
        if (lk >= st.bhi) continue;
        if (st.nb == K && lk > st.buf[K - 1]) {
          st.bhi = min(st.bhi, lk);
          continue;
        }
        v[k] = (lo << 3) | (uint32_t)k;
      }
      sort8(v);
      uint32_t cnt = 0, ids = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (v[k] != kNoQ) {
          ids |= (v[k] & 7u) << (3 * cnt);
          ++cnt;
        }
      if (cnt == 0) continue;
      ++top;
      par[top] = (uint32_t)node;
      cs[top] = s;
      ct[top] = t;
      cq[top] = q;
      ord[top] = (cnt << 24) | ids;
      pm[top] = min(pm[top - 1], v[0] >> 3);
    }
    if (st.fin) break;
    st.end_pass(cx);
  }
}

// Claims a free overflow slab (a 256-bit map in the workspace header), or
// -1. Never waits: a bounded number of attempts, then the caller falls back.
__device__ int claim_slab(const RayArgs& a, int start) {
  for (int w = 0; w < 4; ++w) {
    const int word = (start + w) & 3;
    const int lo = word * 64;
    if ((int)a.n_slabs <= lo) continue;
    const unsigned long long all = (int)a.n_slabs >= lo + 64 ? ~0ull : ((1ull << (a.n_slabs - lo)) - 1ull);
    unsigned long long* bm = &a.hdr->ticket[word];
    for (int tries = 0; tries < 16; ++tries) {
      const unsigned long long free = ~(*(volatile unsigned long long*)bm) & all;
      if (!free) break;
      const int b = __ffsll((long long)free) - 1;
      if (!(atomicOr(bm, 1ull << b) & (1ull << b))) return lo + b;
    }
  }
  return -1;
}

struct __align__(16) WarpSmem {
  unsigned long long front[2][kFrontCap];  // frontier entries: (qlo << 40) | node
  unsigned long long slot_key[32];         // hits handed to their pixel's lane
  uint32_t inbox[32];                      // per pixel lane: mask of the slots holding its hits
  uint32_t pre[32];                        // inclusive prefix of the batch's record counts
  uint32_t off[32];
  uint32_t hist[kBuckets];
};

}  // namespace

template <int K>
__global__ void __launch_bounds__(kRayWarps * 32) raycast_kernel(const __grid_constant__ RayArgs a) {
  extern __shared__ __align__(16) unsigned char ray_smem[];
  __shared__ float s_child[kRayMaxDepth][9];
  __shared__ float s_ext[kRayMaxDepth + 1][3];
  __shared__ float s_step[kRayMaxDepth + 1][9];
  __shared__ float s_l[64 * 8];
  for (int i = threadIdx.x; i < kRayMaxDepth * 9; i += blockDim.x) (&s_child[0][0])[i] = (&a.child[0][0])[i];
  for (int i = threadIdx.x; i < (kRayMaxDepth + 1) * 3; i += blockDim.x) (&s_ext[0][0])[i] = (&a.ext[0][0])[i];
  for (int i = threadIdx.x; i < (kRayMaxDepth + 1) * 9; i += blockDim.x) (&s_step[0][0])[i] = (&a.step[0][0])[i];
  for (int i = threadIdx.x; i < a.n_lights * 8; i += blockDim.x) s_l[i] = a.lights[i];
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpSmem& ws = reinterpret_cast<WarpSmem*>(ray_smem)[warp];
  const int tiles_x = (a.width + kTileW - 1) / kTileW;
  const int tiles = tiles_x * ((a.height + kTileH - 1) / kTileH);
  const int tile = blockIdx.x * kRayWarps + warp;
  if (tile >= tiles) return;  // whole warp
  const int x0 = (tile % tiles_x) * kTileW, y0 = (tile / tiles_x) * kTileH;
  const int x = x0 + (lane & 7), y = y0 + (lane >> 3);
  const bool active = x < a.width && y < a.height;
  const SplatView sv = make_splat_view(a.cube_min, a.cube_side, a.origin, a.right, a.up, a.fwd, a.pitch, a.width,
                                       a.height, a.z0, a.z1, 1, nullptr);
  const ShadeCtx cx{&a, s_l};
  const int depth = a.depth;
  const float tcx = (float)x0 + 0.5f * kTileW, tcy = (float)y0 + 0.5f * kTileH;
  const float thx = 0.5f * kTileW - 0.5f, thy = 0.5f * kTileH - 0.5f;  // tile half size minus the pixel's
  const unsigned lt_mask = (1u << lane) - 1u;

  RayState<K> st;
  st.init(active);

  // ---- breadth-first descent over the tile's beam (frontier in shared
  // memory, moved to an overflow slab if it outgrows it)
  unsigned long long* fr[2] = {ws.front[0], ws.front[1]};
  int cap = kFrontCap, slab = -1;
  int n = 0, cur = 0;
  bool overflow = false;
  {
    float s, t, q;
    node_centre(0, a.corner, s_step[0], s, t, q);
    const bool ok = __ldg(a.cnt) > 0u && fabsf(s - tcx) <= s_ext[0][0] + thx && fabsf(t - tcy) <= s_ext[0][1] + thy;
    if (ok && lane == 0) fr[0][0] = (unsigned long long)q_floor(q - s_ext[0][2]) << kIdxBits;
    n = ok ? 1 : 0;
  }
  __syncwarp();
  for (int l = 0; l < depth && n > 0; ++l) {
    const unsigned long long lbase = level_offset(l + 1);
    const float* stp = s_step[l + 1];
    const float es = s_ext[l + 1][0] + thx, et = s_ext[l + 1][1] + thy, eq = s_ext[l + 1][2];
    const unsigned long long* src = fr[cur];
    unsigned long long* dst = fr[cur ^ 1];
    int m = 0;
    for (int base = 0; base < n * 8; base += 32) {
      const int item = base + lane;
      bool keep = false;
      unsigned long long ent = 0;
      if (item < n * 8) {
        const unsigned long long node = (src[item >> 3] & kIdxMask) * 8ull + (unsigned)(item & 7);
        if (__ldg(a.cnt + lbase + node) > 0u) {
          float s, t, q;
          node_centre(node, a.corner, stp, s, t, q);
          if (fabsf(s - tcx) <= es && fabsf(t - tcy) <= et) {
            keep = true;
            ent = ((unsigned long long)q_floor(q - eq) << kIdxBits) | node;
          }
        }
      }
      const unsigned mk = __ballot_sync(~0u, keep);
      const int pos = m + __popc(mk & lt_mask);
      if (keep && pos < cap) dst[pos] = ent;
      m += __popc(mk);
    }
    __syncwarp();
    if (m > cap) {
      if (slab < 0) {
        int sl = lane == 0 ? claim_slab(a, tile) : -1;
        sl = __shfl_sync(~0u, sl, 0);
        if (sl >= 0) {
          // move the current level to the slab and expand it again there
          slab = sl;
          unsigned long long* sb = reinterpret_cast<unsigned long long*>(a.slabs) + (size_t)slab * 2 * kSlabCap;
          for (int i = lane; i < n; i += 32) sb[(size_t)cur * kSlabCap + i] = src[i];
          fr[0] = sb;
          fr[1] = sb + kSlabCap;
          cap = kSlabCap;
          __syncwarp();
          --l;
          continue;
        }
      }
      overflow = true;
      break;
    }
    cur ^= 1;
    n = m;
  }

  if (overflow) {
    if (lane == 0) atomicAdd(&a.hdr->huge_count, 1u);
    if (active) dfs_ray<K>(a, cx, s_child, s_ext, x, y, sv, st);
  } else if (n > 0) {
    // ---- bucket sort of the leaves by depth lower bound (into front[cur ^ 1])
    const unsigned long long* src = fr[cur];
    unsigned long long* lst = fr[cur ^ 1];
    uint32_t qmin = kNoQ, qmax = 0;
    for (int i = lane; i < n; i += 32) {
      const uint32_t q = (uint32_t)(src[i] >> kIdxBits);
      qmin = min(qmin, q);
      qmax = max(qmax, q);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      qmin = min(qmin, __shfl_xor_sync(~0u, qmin, o));
      qmax = max(qmax, __shfl_xor_sync(~0u, qmax, o));
    }
    const unsigned long long span = (unsigned long long)(qmax - qmin) + 1ull;
    ws.hist[lane] = 0u;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const uint32_t b = (uint32_t)(((unsigned long long)((uint32_t)(src[i] >> kIdxBits) - qmin) * kBuckets) / span);
      atomicAdd(&ws.hist[b], 1u);
    }
    __syncwarp();
    const uint32_t h = ws.hist[lane];
    uint32_t inc = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(~0u, inc, o);
      if (lane >= o) inc += v;
    }
    ws.hist[lane] = inc - h;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const unsigned long long e = src[i];
      const uint32_t b = (uint32_t)(((unsigned long long)((uint32_t)(e >> kIdxBits) - qmin) * kBuckets) / span);
      lst[atomicAdd(&ws.hist[b], 1u)] = e;
    }
    __syncwarp();
    // suffix minimum of the bounds: suf[i] = min over lst[i..n) (front[cur] reused)
    uint32_t* suf = reinterpret_cast<uint32_t*>(fr[cur]);
    uint32_t carry = kNoQ;
    for (int cb = ((n - 1) >> 5) << 5; cb >= 0; cb -= 32) {
      const int i = cb + lane;
      uint32_t v = i < n ? (uint32_t)(lst[i] >> kIdxBits) : kNoQ;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t w2 = __shfl_down_sync(~0u, v, o);
        if (lane + o < 32) v = min(v, w2);
      }
      v = min(v, carry);
      if (i < n) suf[i] = v;
      carry = __shfl_sync(~0u, v, 0);
    }
    if (lane == 0) suf[n] = kNoQ;
    __syncwarp();

    // ---- front-to-back leaf batches, as many passes as some lane needs
    const unsigned long long lleaf = level_offset(depth);
    const uint4* recs = reinterpret_cast<const uint4*>(a.pofa);
    const uint32_t lspan = (uint32_t)(2.0f * s_ext[depth][2]) + 3u;  // >= qhi - qlo of a leaf
    for (int pass = 0;; ++pass) {
      // later passes skip batches that lie wholly in front of every lane's lmin
      uint32_t need = st.fin ? kNoQ : (uint32_t)(st.lmin >> kIdxBits);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) need = min(need, __shfl_xor_sync(~0u, need, o));
      for (int b = 0; b < n; b += 32) {
        const int nl = min(32, n - b);
        if (pass > 0) {
          uint32_t bq = lane < nl ? (uint32_t)(lst[b + lane] >> kIdxBits) : 0u;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) bq = max(bq, __shfl_xor_sync(~0u, bq, o));
          if (bq + lspan < need) continue;
        }
        uint32_t o = 0, c = 0;
        if (lane < nl) {
          const unsigned long long e = lleaf + (lst[b + lane] & kIdxMask);
          o = __ldg(a.off + e);
          c = __ldg(a.cnt + e);
        }
        uint32_t pre = c;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
          const uint32_t v = __shfl_up_sync(~0u, pre, s);
          if (lane >= s) pre += v;
        }
        ws.pre[lane] = pre;
        ws.off[lane] = o;
        const uint32_t total = __shfl_sync(~0u, pre, 31);
        __syncwarp();
        for (uint32_t r0 = 0; r0 < total; r0 += 32) {
          const uint32_t r = r0 + lane;
          int dst = -1;
          unsigned long long key = kNoKey;
          if (r < total) {
            int j = 0;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1)
              if (ws.pre[j + s - 1] <= r) j += s;
            const unsigned long long ri = (unsigned long long)ws.off[j] + (r - (j ? ws.pre[j - 1] : 0u));
            if (ri < a.n_max) {
              const uint4 rc = __ldg(recs + ri);
              float p[3];
              dequantize((unsigned long long)rc.x | ((unsigned long long)rc.y << 32), sv, p);
              const Projected pr = project_point(p, sv);
              if (pr.ax >= x0 && pr.ax < x0 + kTileW && pr.ay >= y0 && pr.ay < y0 + kTileH) {
                dst = (pr.ax - x0) + kTileW * (pr.ay - y0);
                key = ((unsigned long long)pr.qd << kIdxBits) | ri;
              }
            } else {
              set_status(&a.hdr->status, FHV_DEV_RANGE);
            }
          }
          // hand each hit to the lane of its pixel: the first lane of every
          // group with the same destination posts the group's mask there
          const unsigned grp = __match_any_sync(~0u, dst);
          ws.inbox[lane] = 0u;
          ws.slot_key[lane] = key;
          __syncwarp();
          if (dst >= 0 && lane == __ffs(grp) - 1) ws.inbox[dst] = grp;
          __syncwarp();
          unsigned mine = ws.inbox[lane];
          while (mine) {
            const int s = __ffs(mine) - 1;
            mine &= mine - 1;
            if (!st.fin) st.insert(ws.slot_key[s]);
          }
          __syncwarp();
        }
        // every leaf not yet processed has a depth bound >= suf[b + nl]
        if (!st.fin) st.release(suf[b + nl], cx);
        if (__all_sync(~0u, st.fin)) break;
      }
      bool again = false;
      if (!st.fin) again = st.end_pass(cx);
      if (!__any_sync(~0u, again)) break;
    }
  }

  if (slab >= 0) {
    __syncwarp();
    __threadfence();
    if (lane == 0) atomicAnd(&a.hdr->ticket[slab >> 6], ~(1ull << (slab & 63)));
  }
  if (active) {
    const unsigned long long p = (unsigned long long)y * a.width + x;
    a.vis[p] = st.first;
    reinterpret_cast<float4*>(a.rgba)[p] =
        st.first == kVisEmpty ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : make_float4(st.cr, st.cg, st.cb, 1.0f - st.T);
  }
}

cudaError_t launch_raycast(const RayArgs& a, cudaStream_t s) {
  const long long tiles = (long long)((a.width + kTileW - 1) / kTileW) * ((a.height + kTileH - 1) / kTileH);
  const unsigned grid = (unsigned)((tiles + kRayWarps - 1) / kRayWarps);
  const size_t smem = sizeof(WarpSmem) * kRayWarps;
  // per launch: cheap, and correct whichever device is current
  if (cudaFuncSetAttribute(raycast_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(raycast_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return cudaGetLastError();
  timing_begin("raycast", s);
  if (a.alpha)
    raycast_kernel<8><<<grid, kRayWarps * 32, smem, s>>>(a);
  else
    raycast_kernel<1><<<grid, kRayWarps * 32, smem, s>>>(a);
  timing_end("raycast", s);
  return cudaGetLastError();
}

}  // namespace fhv
