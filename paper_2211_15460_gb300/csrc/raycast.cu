// raycast.cu -- image generation by ray casting through the octree of a
// FHV_POFA (Section 3.3; Table 3 "R" and "R/T").
//
// One thread per output pixel walks the octree from the root. The children
// of an octant that hold fragments (cnt > 0) and whose box can project into
// the pixel are visited nearest first (ordered by the lower bound of their
// quantised depth along the view direction); a leaf's records are tested
// against the ray and kept in a small sorted buffer (the in-octant sort).
//
// A fragment lies on the pixel's ray when its projection falls in the pixel
// (the rule of a 1 x 1 splat), and the composite takes the ray's fragments
// in increasing (qdepth << 40 | index) order. That order is exact here,
// whereas appending whole octants in visiting order is not: two fragments in
// the same pixel but in different octants can swap depth order near an
// octant face. So the stack carries, per level, the smallest depth bound of
// the octants still to visit (a prefix minimum), and a buffered fragment is
// composited only once its depth lies below that bound -- after which no
// unvisited fragment can precede it. Compositing is front to back,
// C += T a c, T *= 1 - a, and the ray stops as soon as T <= t_stop (the
// per-octant early-out of the paper; t_stop = 0 with opaque materials gives
// the exact result).
//
// The buffer holds K keys. When it is full, an octant or record beyond its
// largest key is dropped and the drop lowers `bhi`, the bound below which
// the pass has seen every fragment. A pass ends when the stack is empty;
// if anything was dropped and the ray is not done, another pass starts
// after the last composited key. Opaque casting (R) uses K = 1, for which
// the first pass always finishes the ray.
//
// Octant bounds are affine in the octant centre: the host precomputes the
// root centre in (s, t, q) = (screen x, screen y, quantised depth) and, per
// level, the offsets of a child centre and the half extents, widened by a
// margin that covers the float32 rounding of both the bounds and the
// fragment projection (every fragment is projected with the exact
// arithmetic of the splat, so pixel membership and depth keys are bit-equal
// to the splat's).
#include "kernels.h"
#include "splat.cuh"

namespace fhv {

namespace {

constexpr uint32_t kNoQ = 0xFFFFFFFFu;
constexpr unsigned long long kNoKey = ~0ull;

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

}  // namespace

template <int K>
__global__ void __launch_bounds__(128) raycast_kernel(const __grid_constant__ RayArgs a) {
  __shared__ float s_child[kRayMaxDepth][9];
  __shared__ float s_ext[kRayMaxDepth + 1][3];
  __shared__ float s_l[64 * 8];
  for (int i = threadIdx.x; i < kRayMaxDepth * 9; i += blockDim.x) (&s_child[0][0])[i] = (&a.child[0][0])[i];
  for (int i = threadIdx.x; i < (kRayMaxDepth + 1) * 3; i += blockDim.x) (&s_ext[0][0])[i] = (&a.ext[0][0])[i];
  for (int i = threadIdx.x; i < a.n_lights * 8; i += blockDim.x) s_l[i] = a.lights[i];
  __syncthreads();

  // 16 x 8 pixels per CTA, 8 x 4 per warp, so that a warp's rays are close.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
  const int y = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
  if (x >= a.width || y >= a.height) return;

  const SplatView sv = make_splat_view(a.cube_min, a.cube_side, a.origin, a.right, a.up, a.fwd, a.pitch, a.width,
                                       a.height, a.z0, a.z1, 1, nullptr);
  const float pcx = (float)x + 0.5f, pcy = (float)y + 0.5f;
  const int depth = a.depth;
  const uint4* recs = reinterpret_cast<const uint4*>(a.pofa);

  unsigned long long buf[K];
#pragma unroll
  for (int i = 0; i < K; ++i) buf[i] = kNoKey;
  int nb = 0;
  unsigned long long lmin = 0;        // keys below lmin are composited
  unsigned long long last = kNoKey;   // last composited key
  unsigned long long first = kVisEmpty;
  float cr = 0.0f, cg = 0.0f, cb = 0.0f, T = 1.0f;
  bool done = false;

  auto composite = [&](unsigned long long key) {
    const uint4 r = __ldg(recs + (key & kIdxMask));
    const float4 c = shade_pixel(key, a.pofa, a.tri_material, a.albedo, a.cube_min, a.cube_side, s_l, a.n_lights);
    const float al = a.alpha ? __ldg(a.alpha + __ldg(a.tri_material + r.z)) : 1.0f;
    const float w = T * al;
    cr += w * c.x;
    cg += w * c.y;
    cb += w * c.z;
    T *= 1.0f - al;
    if (first == kVisEmpty) first = key;
    last = key;
    if (T <= a.t_stop) done = true;
  };
  // Composite, in order, the buffered keys whose depth lies below lim.
  auto release = [&](uint32_t lim) {
    int r = 0;
    while (r < nb && !done && (uint32_t)(buf[r] >> kIdxBits) < lim) composite(buf[r++]);
    if (r) {
      for (int i = r; i < nb; ++i) buf[i - r] = buf[i];
      nb -= r;
    }
  };

  uint32_t grp[kRayMaxDepth + 1], ord[kRayMaxDepth + 1], pm[kRayMaxDepth + 1];
  float cs[kRayMaxDepth + 1], ct[kRayMaxDepth + 1], cq[kRayMaxDepth + 1];

  // The root, if it holds fragments and can reach this pixel.
  bool root_ok = __ldg(a.cnt) > 0u && fabsf(a.root[0] - pcx) <= s_ext[0][0] && fabsf(a.root[1] - pcy) <= s_ext[0][1];

  while (root_ok && !done) {
    unsigned long long bhi = kNoKey;  // every fragment with key < bhi has been seen in this pass
    const uint32_t lmin_q = (uint32_t)(lmin >> kIdxBits);
    nb = 0;
    int top = 0;
    grp[0] = 0;
    ord[0] = 1u << 24;  // one entry (child id 0): the root
    pm[0] = 0;
    while (top >= 0 && !done) {
      const uint32_t o = ord[top];
      uint32_t n = o >> 24;
      if (n == 0) {
        --top;
        continue;
      }
      const int c = (int)(o & 7u);
      --n;
      ord[top] = (n << 24) | ((o & 0xFFFFFFu) >> 3);
      const uint32_t node = grp[top] + (uint32_t)c;
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
      if (lo_key >= bhi) {
        ord[top] = 0;
        pm[top] = below;
        continue;
      }
      if (nb == K && lo_key > buf[K - 1]) {
        bhi = min(bhi, lo_key);
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
          const unsigned long long mk = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
          float p[3];
          dequantize(mk, sv, p);
          const Projected pr = project_point(p, sv);
          if (pr.ax != x || pr.ay != y) continue;
          const unsigned long long key = ((unsigned long long)pr.qd << kIdxBits) | i;
          if (key < lmin || key >= bhi) continue;
          if (nb == K) {
            if (key > buf[K - 1]) {
              bhi = min(bhi, key);
              continue;
            }
            bhi = min(bhi, buf[K - 1]);
            --nb;
          }
          int j = nb;
          while (j > 0 && buf[j - 1] > key) {
            buf[j] = buf[j - 1];
            --j;
          }
          buf[j] = key;
          ++nb;
        }
        release(pm[top]);
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
        if (lk >= bhi) continue;
        if (nb == K && lk > buf[K - 1]) {
          bhi = min(bhi, lk);
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
      grp[top] = node * 8u;
      cs[top] = s;
      ct[top] = t;
      cq[top] = q;
      ord[top] = (cnt << 24) | ids;
      pm[top] = min(pm[top - 1], v[0] >> 3);
    }
    if (done) break;
    release(kNoQ);
    if (done || bhi == kNoKey || last == kNoKey) break;
    lmin = last + 1;  // next pass: what lies behind the last composited key
  }

  const unsigned long long p = (unsigned long long)y * a.width + x;
  a.vis[p] = first;
  reinterpret_cast<float4*>(a.rgba)[p] =
      first == kVisEmpty ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : make_float4(cr, cg, cb, 1.0f - T);
}

cudaError_t launch_raycast(const RayArgs& a, cudaStream_t s) {
  const dim3 grid((unsigned)((a.width + 15) / 16), (unsigned)((a.height + 7) / 8));
  timing_begin("raycast", s);
  if (a.alpha)
    raycast_kernel<8><<<grid, 128, 0, s>>>(a);
  else
    raycast_kernel<1><<<grid, 128, 0, s>>>(a);
  timing_end("raycast", s);
  return cudaGetLastError();
}

}  // namespace fhv
