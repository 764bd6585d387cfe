// capture.cu -- FHV creation (Section 3.2): triangle setup, sample-range
// scan, rasterisation and fragment insertion into per-pixel lists (PPFL) or
// per-octant lists (POFL), plus the multi-range fill used to reset arrays.
//
// GB300 layout of the work:
//  * setup_scan: one thread per triangle projects, snaps and orients it and
//    builds a 96-byte TriSetup, staged in shared memory so the CTA stores
//    its 256 setups with coalesced 16-byte writes; the CTA scans its
//    triangles' bounding-box sample counts (no cross-CTA wait). Extra CTAs
//    of the same launch reset the list heads (and POFL occupancy levels), so
//    the bandwidth-bound reset overlaps the latency-bound setup.
//  * tile_scan: one CTA scans the per-tile sample totals; the flattened
//    sample space [0, total) is then tile_off[t / 256] + samp_rel[t].
//  * raster: a persistent kernel (SM count x resident CTAs). Each warp owns
//    an equal, contiguous share of the flattened sample space, so tiny
//    heightfield triangles and large box faces balance alike. Per step a
//    warp takes 32 consecutive samples, finds each lane's triangle in a
//    32-wide window of the offset array (shuffle binary search), evaluates
//    the three integer edge functions with the top-left rule, and appends
//    covered samples with one counter atomic per warp and coalesced 16-byte
//    record stores.
//  * link: one thread per stored record exchanges it into its slot's list
//    head and stores the old head as its link (plus POFL occupancy). The
//    exchanges hit a multi-GB head array at random; issued from a kernel
//    that does nothing else, their DRAM latency is hidden by occupancy
//    instead of stalling the raster's warps.
//  * raster_pofa (direct POFA build): the same sample walk three times, its
//    fragments handed to the compaction's per-record steps (mark, count,
//    scatter) around the compaction's scan, then its in-octant order; no
//    lists are built.
#include "kernels.h"
#include "lookback.cuh"

namespace fhv {

// ------------------------------------------------------------------- fill

struct FillSet {
  RangeFill r[6];
  int n;
};

// Stores of every range, by `nthreads` threads numbered from t0.
__device__ void fill_ranges(const FillSet& fs, unsigned long long t0, unsigned long long stride) {
  for (int k = 0; k < fs.n; ++k) {
    const RangeFill r = fs.r[k];
    if (r.width == 4) {
      uint32_t* p = (uint32_t*)r.ptr;
      uint32_t v = (uint32_t)r.value;
      // scalar head up to 16-byte alignment, vector body, scalar tail
      unsigned long long head = ((16ull - ((uintptr_t)p & 15ull)) & 15ull) / 4ull;
      if (head > r.n) head = r.n;
      for (unsigned long long i = t0; i < head; i += stride) p[i] = v;
      unsigned long long nv = (r.n - head) / 4ull;
      uint4* q = (uint4*)(p + head);
      uint4 vv = make_uint4(v, v, v, v);
      for (unsigned long long i = t0; i < nv; i += stride) q[i] = vv;
      for (unsigned long long i = head + nv * 4ull + t0; i < r.n; i += stride) p[i] = v;
    } else {
      unsigned long long* p = (unsigned long long*)r.ptr;
      unsigned long long v = r.value;
      unsigned long long head = ((16ull - ((uintptr_t)p & 15ull)) & 15ull) / 8ull;
      if (head > r.n) head = r.n;
      for (unsigned long long i = t0; i < head; i += stride) p[i] = v;
      unsigned long long nv = (r.n - head) / 2ull;
      ulonglong2* q = (ulonglong2*)(p + head);
      ulonglong2 vv = make_ulonglong2(v, v);
      for (unsigned long long i = t0; i < nv; i += stride) q[i] = vv;
      for (unsigned long long i = head + nv * 2ull + t0; i < r.n; i += stride) p[i] = v;
    }
  }
}

__global__ void fill_kernel(FillSet fs) {
  fill_ranges(fs, (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x, (unsigned long long)gridDim.x * blockDim.x);
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

cudaError_t launch_fill(const RangeFill* ranges, int n_ranges, cudaStream_t s) {
  unsigned long long total = 0;
  for (int i = 0; i < n_ranges; ++i) total += ranges[i].n;
  if (total == 0) return cudaSuccess;
  for (int base = 0; base < n_ranges; base += 6) {
    FillSet fs;
    fs.n = 0;
    unsigned long long biggest = 0;
    for (int i = base; i < n_ranges && i < base + 6; ++i) {
      if (ranges[i].n == 0) continue;
      fs.r[fs.n++] = ranges[i];
      unsigned long long vecs = ranges[i].n / (ranges[i].width == 4 ? 4ull : 2ull) + 4;
      if (vecs > biggest) biggest = vecs;
    }
    if (fs.n == 0) continue;
    unsigned long long blocks = (biggest + 255) / 256;
    unsigned long long cap = (unsigned long long)sm_count() * 32ull;  // 32 CTAs/SM: ~7.2 TB/s of stores
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    timing_begin("fill", s);
    fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(fs);
    timing_end("fill", s);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ setup

__device__ __forceinline__ long long floordiv256(long long a) {
  return a >= 0 ? a / 256 : -((-a + 255) / 256);
}
__device__ __forceinline__ long long ceildiv256(long long a) { return -floordiv256(-a); }

__device__ __forceinline__ void cross3(const float* a, const float* b, float* o) {
  o[0] = fsub(fmul(a[1], b[2]), fmul(a[2], b[1]));
  o[1] = fsub(fmul(a[2], b[0]), fmul(a[0], b[2]));
  o[2] = fsub(fmul(a[0], b[1]), fmul(a[1], b[0]));
}

// Returns the triangle's bounding-box sample count (0: no fragments). For
// FHV_CAPTURE_AXIS3, setup entry e is triangle e / 3 seen along axis e % 3.
__device__ unsigned long long setup_triangle(const CaptureArgs& a, uint32_t e, TriSetup& ts) {
  const uint32_t t = e / (uint32_t)a.passes;
  const int axis = (int)(e % (uint32_t)a.passes);
  uint32_t vi[3];
  for (int v = 0; v < 3; ++v) vi[v] = a.idx[3ull * t + v];
  if (vi[0] >= a.n_vtx || vi[1] >= a.n_vtx || vi[2] >= a.n_vtx) return 0ull;
  float p[3][3], N[3][3];
  uint32_t Q[3][3];
  const float qscale = fdiv(2097152.0f, a.cube_side);
  for (int v = 0; v < 3; ++v)
    for (int c = 0; c < 3; ++c) {
      p[v][c] = a.pos[3ull * vi[v] + c];
      N[v][c] = a.nrm[3ull * vi[v] + c];
      Q[v][c] = quantize1(p[v][c], a.cube_min[c], qscale);
    }
  long long X[3], Y[3];
  if (a.mode == FHV_CAPTURE_VIEW) {
    const float inv_pitch = fdiv(1.0f, a.pitch);
    const float hw = fmul(0.5f, (float)a.width), hh = fmul(0.5f, (float)a.height);
    for (int v = 0; v < 3; ++v) {
      float dx = fsub(p[v][0], a.origin[0]), dy = fsub(p[v][1], a.origin[1]), dz = fsub(p[v][2], a.origin[2]);
      float sx = fadd(fmul(dot3(dx, dy, dz, a.right[0], a.right[1], a.right[2]), inv_pitch), hw);
      float sy = fadd(fmul(dot3(dx, dy, dz, a.up[0], a.up[1], a.up[2]), inv_pitch), hh);
      X[v] = snap256(sx);
      Y[v] = snap256(sy);
    }
  } else if (a.mode == FHV_CAPTURE_AXIS3) {
    const float inv_h = fdiv(1.0f, a.pitch);
    const int cu = (axis + 1) % 3, cv = (axis + 2) % 3;
    for (int v = 0; v < 3; ++v) {
      X[v] = snap256(fmul(fsub(p[v][cu], a.cube_min[cu]), inv_h));
      Y[v] = snap256(fmul(fsub(p[v][cv], a.cube_min[cv]), inv_h));
    }
  } else {
    // tangent frame: t = e1/|e1|, n = (e1 x e2)/|e1 x e2|, b = n x t
    float e1[3], e2[3], n[3], tt[3], nn[3], bb[3];
    for (int c = 0; c < 3; ++c) {
      e1[c] = fsub(p[1][c], p[0][c]);
      e2[c] = fsub(p[2][c], p[0][c]);
    }
    cross3(e1, e2, n);
    float le = __fsqrt_rn(dot3(e1[0], e1[1], e1[2], e1[0], e1[1], e1[2]));
    float ln = __fsqrt_rn(dot3(n[0], n[1], n[2], n[0], n[1], n[2]));
    if (!(le > 0.0f) || !(ln > 0.0f)) return 0ull;
    for (int c = 0; c < 3; ++c) {
      tt[c] = fdiv(e1[c], le);
      nn[c] = fdiv(n[c], ln);
    }
    cross3(nn, tt, bb);
    const float inv_h = fdiv(1.0f, a.pitch);
    X[0] = 0;
    Y[0] = 0;
    X[1] = snap256(fmul(dot3(e1[0], e1[1], e1[2], tt[0], tt[1], tt[2]), inv_h));
    Y[1] = snap256(fmul(dot3(e1[0], e1[1], e1[2], bb[0], bb[1], bb[2]), inv_h));
    X[2] = snap256(fmul(dot3(e2[0], e2[1], e2[2], tt[0], tt[1], tt[2]), inv_h));
    Y[2] = snap256(fmul(dot3(e2[0], e2[1], e2[2], bb[0], bb[1], bb[2]), inv_h));
  }
  long long A = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
  if (A == 0) return 0ull;
  const int v1 = A < 0 ? 2 : 1, v2 = A < 0 ? 1 : 2;  // counter-clockwise winding (y up)
  const int vo[3] = {0, v1, v2};
  long long minX = X[0], maxX = X[0], minY = Y[0], maxY = Y[0];
  for (int k = 1; k < 3; ++k) {
    minX = min(minX, X[k]);
    maxX = max(maxX, X[k]);
    minY = min(minY, Y[k]);
    maxY = max(maxY, Y[k]);
  }
  long long i0 = ceildiv256(minX - 128), i1 = floordiv256(maxX - 128);
  long long j0 = ceildiv256(minY - 128), j1 = floordiv256(maxY - 128);
  if (a.mode == FHV_CAPTURE_VIEW) {
    i0 = max(i0, 0ll);
    j0 = max(j0, 0ll);
    i1 = min(i1, (long long)a.width - 1);
    j1 = min(j1, (long long)a.height - 1);
  }
  if (i1 < i0 || j1 < j0) return 0ull;
  const unsigned long long bw = (unsigned long long)(i1 - i0 + 1), bh = (unsigned long long)(j1 - j0 + 1);
  const unsigned long long ns = bw * bh;
  if (ns > (1ull << 31)) {
    set_status(&a.hdr->status, FHV_DEV_HUGE_TRIANGLE);
    return 0ull;
  }
  for (int k = 0; k < 3; ++k) {
    const int v = vo[k];
    ts.X[k] = (int)X[v];
    ts.Y[k] = (int)Y[v];
    ts.Q[k] = (unsigned long long)Q[v][0] | ((unsigned long long)Q[v][1] << 21) | ((unsigned long long)Q[v][2] << 42);
    ts.N[3 * k] = N[v][0];
    ts.N[3 * k + 1] = N[v][1];
    ts.N[3 * k + 2] = N[v][2];
  }
  ts.i0 = (int)i0;
  ts.j0 = (int)j0;
  ts.bw = (uint32_t)bw;
  return ns;
}

// CTAs [0, tiles) set up kSetupTile triangles each; CTAs [tiles, gridDim)
// store the fill ranges (list heads, occupancy levels).
__global__ void __launch_bounds__(kSetupTile) setup_scan_kernel(CaptureArgs a, FillSet fs, unsigned tiles) {
  __shared__ __align__(16) TriSetup s_ts[kSetupTile];
  __shared__ unsigned long long s_warp[kSetupTile / 32];
  const int tid = threadIdx.x;
  if (blockIdx.x >= tiles) {
    const unsigned long long t0 = (unsigned long long)(blockIdx.x - tiles) * blockDim.x + tid;
    const unsigned long long stride = (unsigned long long)(gridDim.x - tiles) * blockDim.x;
    fill_ranges(fs, t0, stride);
    if (a.sparse_reset) {
      // every head is -1 except those of the previous build's stored records:
      // reset exactly those (the counter is cleared later, by tile_scan)
      const unsigned long long prev = *a.count < a.capacity ? *a.count : a.capacity;
      const int sh = 63 - 3 * a.depth;
      for (unsigned long long i = t0; i < prev; i += stride) {
        const unsigned long long key = reinterpret_cast<const unsigned long long*>(a.rec)[2 * i];
        a.head[key >> sh] = -1;
      }
    }
    return;
  }
  const unsigned long long tile = blockIdx.x;
  const unsigned long long t = tile * kSetupTile + tid;  // setup entry
  unsigned long long ns = 0;
  if (t < a.n_setup) ns = setup_triangle(a, (uint32_t)t, s_ts[tid]);
  // block exclusive scan of the sample counts
  const uint32_t lane = tid & 31, warp = tid >> 5;
  unsigned long long incl = ns;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < kSetupTile / 32 ? s_warp[lane] : 0ull;
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long v = __shfl_up_sync(0xffffffffu, wi, o);
      if ((int)lane >= o) wi += v;
    }
    if (lane < kSetupTile / 32) s_warp[lane] = wi - w;
    if (lane == kSetupTile / 32 - 1) a.tile_sum[tile] = wi;
  }
  __syncthreads();
  if (t < a.n_setup) a.samp_rel[t] = s_warp[warp] + (incl - ns);
  // coalesced copy of the tile's setups
  const unsigned long long n_here = min((unsigned long long)kSetupTile, (unsigned long long)a.n_setup - tile * kSetupTile);
  const uint4* src = reinterpret_cast<const uint4*>(s_ts);
  uint4* dst = reinterpret_cast<uint4*>(a.setup + tile * kSetupTile);
  const uint32_t nvec = (uint32_t)(n_here * sizeof(TriSetup) / 16);
  for (uint32_t i = tid; i < nvec; i += kSetupTile) dst[i] = src[i];
}

// One CTA: exclusive scan of the tile totals; tile_off[tiles] = total.
__global__ void __launch_bounds__(1024) tile_scan_kernel(CaptureArgs a, unsigned tiles) {
  __shared__ unsigned long long s_warp[32];
  const int tid = threadIdx.x;
  const uint32_t lane = tid & 31, warp = tid >> 5;
  const unsigned per = (tiles + blockDim.x - 1) / blockDim.x;
  const unsigned b = tid * per, e = min(tiles, b + per);
  unsigned long long sum = 0;
  for (unsigned i = b; i < e; ++i) sum += a.tile_sum[i];
  unsigned long long incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = s_warp[lane], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long v = __shfl_up_sync(0xffffffffu, wi, o);
      if ((int)lane >= o) wi += v;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) {
      if (a.sparse_reset) *a.count = 0;  // read by setup_scan's reset, which has finished
      a.tile_off[tiles] = wi;
      a.hdr->total = wi;
    }
  }
  __syncthreads();
  unsigned long long run = s_warp[warp] + (incl - sum);
  for (unsigned i = b; i < e; ++i) {
    a.tile_off[i] = run;
    run += a.tile_sum[i];
  }
}

// ----------------------------------------------------------------- raster

// floor(num / den) for den > 0 with a float estimate and exact correction.
__device__ __forceinline__ long long floordiv_est(long long num, long long den, float inv_den) {
  long long q = (long long)floorf(__fmul_rn(__ll2float_rn(num), inv_den));
  long long r = num - q * den;
  for (int it = 0; it < 8 && r < 0; ++it) {
    q -= 1;
    r += den;
  }
  for (int it = 0; it < 8 && r >= den; ++it) {
    q += 1;
    r -= den;
  }
  if (r < 0 || r >= den) {  // estimate far off: exact division
    q = num / den;
    if ((num % den) != 0 && num < 0) q -= 1;
  }
  return q;
}

struct Frag {
  bool covered;
  unsigned long long slot;
  Rec r;
};

__device__ __forceinline__ uint32_t qcomp(unsigned long long q, int c) { return (uint32_t)(q >> (21 * c)) & kQMax; }

__device__ __forceinline__ void eval_sample(const CaptureArgs& a, const TriSetup* __restrict__ setup, uint32_t tri,
                                            uint32_t l, Frag& f) {
  const TriSetup& ts = setup[tri];
  const uint32_t bw = ts.bw;
  const uint32_t jj = l / bw, ii = l - jj * bw;
  const long long sx = 256ll * (ts.i0 + (int)ii) + 128, sy = 256ll * (ts.j0 + (int)jj) + 128;
  const long long X0 = ts.X[0], X1 = ts.X[1], X2 = ts.X[2], Y0 = ts.Y[0], Y1 = ts.Y[1], Y2 = ts.Y[2];
  // edge k runs from vertex (k+1)%3 to (k+2)%3; w_k = its edge function
  const long long dx0 = X2 - X1, dy0 = Y2 - Y1, dx1 = X0 - X2, dy1 = Y0 - Y2, dx2 = X1 - X0, dy2 = Y1 - Y0;
  long long w[3];
  w[0] = dx0 * (sy - Y1) - dy0 * (sx - X1);
  w[1] = dx1 * (sy - Y2) - dy1 * (sx - X2);
  w[2] = dx2 * (sy - Y0) - dy2 * (sx - X0);
  const bool tl0 = dy0 < 0 || (dy0 == 0 && dx0 < 0);
  const bool tl1 = dy1 < 0 || (dy1 == 0 && dx1 < 0);
  const bool tl2 = dy2 < 0 || (dy2 == 0 && dx2 < 0);
  const bool in = (w[0] > 0 || (w[0] == 0 && tl0)) && (w[1] > 0 || (w[1] == 0 && tl1)) &&
                  (w[2] > 0 || (w[2] == 0 && tl2));
  f.covered = in;
  if (!in) return;
  const long long A = w[0] + w[1] + w[2];
  uint32_t q[3];
  if (A < (1ll << 40)) {
    const float inv_den = __frcp_rn(__ll2float_rn(2 * A));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long q0 = qcomp(ts.Q[0], c), d1 = (long long)qcomp(ts.Q[1], c) - q0,
                      d2 = (long long)qcomp(ts.Q[2], c) - q0;
      const long long num = 2 * (w[1] * d1 + w[2] * d2) + A;
      q[c] = (uint32_t)(q0 + floordiv_est(num, 2 * A, inv_den));
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const unsigned __int128 num = (unsigned __int128)w[0] * qcomp(ts.Q[0], c) +
                                    (unsigned __int128)w[1] * qcomp(ts.Q[1], c) +
                                    (unsigned __int128)w[2] * qcomp(ts.Q[2], c);
      q[c] = (uint32_t)((2 * num + (unsigned __int128)A) / (2 * (unsigned __int128)A));
    }
  }
  const float fw0 = __ll2float_rn(w[0]), fw1 = __ll2float_rn(w[1]), fw2 = __ll2float_rn(w[2]);
  float n[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) n[c] = fadd(fadd(fmul(fw0, ts.N[c]), fmul(fw1, ts.N[3 + c])), fmul(fw2, ts.N[6 + c]));
  f.r.key = morton63(q[0], q[1], q[2]);
  f.r.tri = a.tri_base + tri / (uint32_t)a.passes;
  f.r.nrm = oct_encode(n[0], n[1], n[2]);
  if (a.keymode == 0) {
    f.slot = (unsigned long long)(ts.j0 + (int)jj) * (unsigned long long)a.width + (unsigned long long)(ts.i0 + (int)ii);
  } else {
    f.slot = f.r.key >> (63 - 3 * a.depth);
  }
}

// Start of setup entry k's samples in the flattened sample space (k <= n_setup).
__device__ __forceinline__ unsigned long long samp_start(const CaptureArgs& a, unsigned long long k) {
  return k < a.n_setup ? a.tile_off[k / kSetupTile] + a.samp_rel[k]
                       : a.tile_off[(a.n_setup + kSetupTile - 1) / kSetupTile];
}

// Link a stored record into its list and, for the first fragment of a POFL
// leaf, mark the leaf in its parent's occupancy mask and so on up while the
// parent was empty.
__device__ __forceinline__ void finish_insert(const CaptureArgs& a, unsigned long long idx, int32_t prev,
                                              unsigned long long slot) {
  a.next[idx] = prev;
  if (a.levels && prev == -1) {
    unsigned long long child = slot;
    for (int l = a.depth - 1; l >= 0; --l) {
      const unsigned long long parent = child >> 3;
      const uint32_t old = atomicOr(&a.levels[level_offset(l) + parent], 1u << (uint32_t)(child & 7ull));
      if (old != 0u) break;
      child = parent;
    }
  }
}

// The covered samples of one warp step appended to the fragment buffer: one
// counter atomic per warp, 16-byte record stores.
struct AppendSink {
  __device__ __forceinline__ void operator()(const CaptureArgs& a, const Frag& f, uint32_t lane) const {
    const uint32_t mask = __ballot_sync(0xffffffffu, f.covered);
    unsigned long long idx = ~0ull;
    if (mask) {
      const uint32_t leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(a.count, (unsigned long long)__popc(mask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (f.covered) idx = base + __popc(mask & lanemask_lt());
    }
    if (idx < a.capacity) {
      reinterpret_cast<uint4*>(a.rec)[idx] = make_uint4((uint32_t)f.r.key, (uint32_t)(f.r.key >> 32), f.r.tri, f.r.nrm);
      if (a.keymode == 0) a.next[idx] = (int32_t)f.slot;  // pixel, until link_kernel links the record
    }
  }
};

// Every warp walks its share of the flattened sample space 32 samples at a
// time and hands each step's fragments to `sink` (called by all 32 lanes).
template <class Sink>
__device__ __forceinline__ void raster_samples(const CaptureArgs& a, const Sink& sink) {
  const unsigned long long total = a.hdr->total;
  if (total == 0) return;
  const uint32_t lane = lane_id();
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x / 32);
  const unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const unsigned long long chunks = (total + 31) / 32;
  const unsigned long long c0 = chunks * w / nwarps, c1 = chunks * (w + 1) / nwarps;
  if (c0 >= c1) return;
  const uint32_t T = a.n_setup;
  // setup entry containing sample 32*c0: last t with start(t) <= s
  unsigned long long t;
  {
    const unsigned long long s = c0 * 32;
    uint32_t lo = 0, hi = T;
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (samp_start(a, mid) <= s) lo = mid + 1;
      else hi = mid;
    }
    t = lo - 1;
  }
  unsigned long long t_start = samp_start(a, t);
  for (unsigned long long c = c0; c < c1; ++c) {
    const unsigned long long s = c * 32 + lane;
    const bool valid = s < total;
    // find this lane's triangle: windows of 32 offsets starting after t
    bool found = !valid;
    uint32_t my_tri = 0;
    unsigned long long my_start = 0;
    unsigned long long wbase = t, wstart = t_start;
    while (true) {
      const unsigned long long k = wbase + 1 + lane;
      const unsigned long long o = k <= T ? samp_start(a, k) : ~0ull;
      uint32_t cnt = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        unsigned long long v = __shfl_sync(0xffffffffu, o, cnt + step - 1);
        if (v <= s) cnt += step;
      }
      const unsigned long long last = __shfl_sync(0xffffffffu, o, 31);
      const unsigned long long prev = __shfl_sync(0xffffffffu, o, cnt > 0 ? cnt - 1 : 0);
      if (!found && last > s) {
        found = true;
        my_tri = (uint32_t)(wbase + cnt);
        my_start = cnt > 0 ? prev : wstart;
      }
      if (__all_sync(0xffffffffu, found)) break;
      wbase += 32;
      wstart = last;
    }
    Frag f;
    f.covered = false;
    if (valid) eval_sample(a, a.setup, my_tri, (uint32_t)(s - my_start), f);
    sink(a, f, lane);
    const uint32_t lt = __shfl_sync(0xffffffffu, my_tri, 31);
    const unsigned long long ls = __shfl_sync(0xffffffffu, my_start, 31);
    const bool lvalid = __shfl_sync(0xffffffffu, valid ? 1 : 0, 31) != 0;
    if (lvalid) {
      t = lt;
      t_start = ls;
    }
  }
}

__global__ void __launch_bounds__(256, 5) raster_kernel(CaptureArgs a) { raster_samples(a, AppendSink{}); }

// ------------------------------------------------ direct POFA build passes

// Section 3.2 creates the FHV_POFA by rasterising twice: once to count the
// fragments of every octant, then, after a scan, again to write each at its
// octant's offset. Here the counting takes two passes (the first marks the
// occupied leaves and zeroes their counters, so the dense counter array is
// never cleared; the second counts), and the third scatters. The covered
// samples of a warp step are grouped by leaf (__match_any_sync) so one
// atomic serves each group, as in the compaction's per-record steps.
enum { kPassMark = 0, kPassCount = 1, kPassScatter = 2 };

template <int kPass>
struct PofaSink {
  CompactArgs c;
  int T;  // level of the leaf tiles' parents (0: none)
  __device__ __forceinline__ void operator()(const CaptureArgs& a, const Frag& f, uint32_t lane) const {
    const uint32_t mask = __ballot_sync(0xffffffffu, f.covered);
    if (!mask) return;
    uint32_t* off_leaf = c.off + level_offset(c.depth);
    uint32_t* cnt_leaf = c.cnt + level_offset(c.depth);
    if (kPass == kPassMark && lane == (uint32_t)(__ffs(mask) - 1))
      atomicAdd(a.count, (unsigned long long)__popc(mask));
    if (!f.covered) return;
    const unsigned long long leaf = f.slot;
    const uint32_t peers = __match_any_sync(mask, leaf);
    const uint32_t leader = __ffs(peers) - 1;
    if (kPass == kPassMark) {
      if (lane == leader) {
        const uint32_t bit = 1u << (uint32_t)(leaf & 31ull);
        const uint32_t old = atomicOr(bitmap_word(off_leaf, leaf), bit);
        if (!(old & bit)) cnt_leaf[leaf] = 0u;
      }
    } else if (kPass == kPassCount) {
      if (lane == leader) atomicAdd(&cnt_leaf[leaf], (uint32_t)__popc(peers));
      if (T >= 1) {
        const unsigned long long oT = f.r.key >> (63 - 3 * T);
        const uint32_t pT = __match_any_sync(mask, oT);
        if (lane == (uint32_t)(__ffs(pT) - 1)) atomicAdd(&c.cnt[level_offset(T) + oT], (uint32_t)__popc(pT));
      }
    } else {
      uint32_t pos = 0;
      if (lane == leader) pos = atomicAdd(&off_leaf[leaf], (uint32_t)__popc(peers));
      pos = __shfl_sync(peers, pos, leader) + __popc(peers & lanemask_lt());
      if (pos < c.n_max)
        reinterpret_cast<uint4*>(c.out)[pos] = make_uint4((uint32_t)f.r.key, (uint32_t)(f.r.key >> 32), f.r.tri, f.r.nrm);
    }
  }
};

template <int kPass>
__global__ void __launch_bounds__(256, 5) raster_pofa_kernel(CaptureArgs a, CompactArgs c, int T) {
  if (kPass == kPassCount && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long n = *a.count;  // final: the mark pass has counted every fragment
    a.hdr->n_kept = n <= c.n_max ? n : 0ull;
  }
  if (kPass == kPassScatter && *a.count > c.n_max) return;  // over capacity: nothing is stored
  raster_samples(a, PofaSink<kPass>{c, T});
}

// Insertion into the lists, one stored record per thread: the previous head
// of the record's slot becomes its link (Section 3.2). The slot is the pixel
// parked in next[] by the raster (PPFL) or the record's leaf octant (POFL).
__global__ void __launch_bounds__(256) link_kernel(CaptureArgs a) {
  const unsigned long long c = *a.count;
  const unsigned long long n = c < a.capacity ? c : a.capacity;
  const int sh = 63 - 3 * a.depth;
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    const unsigned long long slot =
        a.keymode == 0 ? (unsigned long long)(uint32_t)a.next[i] : (a.rec[i].key >> sh);
    const int32_t prev = atomicExch(&a.head[slot], (int32_t)i);
    finish_insert(a, i, prev, slot);
  }
}

template <class K>
static int blocks_per_sm(K kernel) {
  int v = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, 256, 0);
  return v > 0 ? v : 1;
}

static int raster_blocks_per_sm() {
  static int cached = 0;
  if (cached == 0) cached = blocks_per_sm(raster_kernel);
  return cached;
}

// fills[0] is the small header/counter reset (launched alone, first); the
// other ranges are stored by the setup launch's extra CTAs.
// Resets, triangle setup and the sample-space scan shared by every capture.
static cudaError_t launch_setup(const CaptureArgs& a, const RangeFill* fills, int n_fills, cudaStream_t s) {
  cudaError_t e = launch_fill(fills, 1, s);
  if (e != cudaSuccess) return e;
  if (a.n_setup == 0) return launch_fill(fills + 1, n_fills - 1, s);
  FillSet fs;
  fs.n = 0;
  for (int i = 1; i < n_fills && fs.n < 6; ++i)
    if (fills[i].n) fs.r[fs.n++] = fills[i];
  const unsigned tiles = (a.n_setup + kSetupTile - 1) / kSetupTile;
  const unsigned fill_ctas = fs.n ? (unsigned)sm_count() * 8u : 0u;
  timing_begin("setup_scan", s);
  setup_scan_kernel<<<tiles + fill_ctas, kSetupTile, 0, s>>>(a, fs, tiles);
  timing_end("setup_scan", s);
  timing_begin("tile_scan", s);
  tile_scan_kernel<<<1, 1024, 0, s>>>(a, tiles);
  timing_end("tile_scan", s);
  return cudaGetLastError();
}

cudaError_t launch_capture(const CaptureArgs& a, const RangeFill* fills, int n_fills, cudaStream_t s) {
  cudaError_t e = launch_setup(a, fills, n_fills, s);
  if (e != cudaSuccess || a.n_setup == 0) return e;
  timing_begin("raster", s);
  raster_kernel<<<sm_count() * raster_blocks_per_sm(), 256, 0, s>>>(a);
  timing_end("raster", s);
  timing_begin("link", s);
  link_kernel<<<sm_count() * 16, 256, 0, s>>>(a);
  timing_end("link", s);
  return cudaGetLastError();
}

cudaError_t launch_pofa_direct(const CaptureArgs& a, const CompactArgs& c, const RangeFill* fills, int n_fills,
                               cudaStream_t s) {
  static int per_sm[3] = {0, 0, 0};
  if (per_sm[0] == 0) {
    per_sm[0] = blocks_per_sm(raster_pofa_kernel<kPassMark>);
    per_sm[1] = blocks_per_sm(raster_pofa_kernel<kPassCount>);
    per_sm[2] = blocks_per_sm(raster_pofa_kernel<kPassScatter>);
  }
  const int T = c.depth > 4 ? c.depth - 4 : 0;
  cudaError_t e = launch_setup(a, fills, n_fills, s);
  if (e == cudaSuccess) e = compact_clear_bitmap(c, s);
  if (e != cudaSuccess) return e;
  timing_begin("raster_mark", s);
  raster_pofa_kernel<kPassMark><<<sm_count() * per_sm[0], 256, 0, s>>>(a, c, T);
  timing_end("raster_mark", s);
  timing_begin("raster_count", s);
  raster_pofa_kernel<kPassCount><<<sm_count() * per_sm[1], 256, 0, s>>>(a, c, T);
  timing_end("raster_count", s);
  e = compact_scan(c, s);
  if (e != cudaSuccess || c.n_max == 0) return e;
  timing_begin("raster_scatter", s);
  raster_pofa_kernel<kPassScatter><<<sm_count() * per_sm[2], 256, 0, s>>>(a, c, T);
  timing_end("raster_scatter", s);
  return compact_order(c, s);
}

}  // namespace fhv
