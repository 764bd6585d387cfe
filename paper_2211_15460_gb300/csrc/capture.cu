// capture.cu -- FHV creation (Section 3.2): triangle setup, sample-range
// scan, rasterisation and fragment insertion into per-pixel lists (PPFL) or
// per-octant lists (POFL), plus the multi-range fill used to reset arrays.
//
// GB300 layout of the work:
//  * setup_scan: one thread per triangle projects, snaps and orients it and
//    writes a 160-byte TriSetup; the CTA then scans the triangles'
//    bounding-box sample counts and chains tiles with decoupled look-back,
//    so the flattened sample space [0, total) is known in one pass.
//  * raster: a persistent kernel (SM count x resident CTAs). Each warp owns
//    an equal, contiguous share of the flattened sample space, so tiny
//    heightfield triangles and large box faces balance alike. Per step a
//    warp takes 32 consecutive samples, finds each lane's triangle in a
//    32-wide window of the offset array (shuffle binary search), evaluates
//    the three integer edge functions with the top-left rule, and appends
//    covered samples with one counter atomic per warp, coalesced 16-byte
//    record stores and an atomic exchange on the list head.
#include "kernels.h"
#include "lookback.cuh"

namespace fhv {

// ------------------------------------------------------------------- fill

struct FillSet {
  RangeFill r[6];
  int n;
};

__global__ void fill_kernel(FillSet fs) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
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

// Returns the triangle's bounding-box sample count (0: no fragments).
__device__ unsigned long long setup_triangle(const CaptureArgs& a, uint32_t t, TriSetup& ts) {
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
  int v1 = 1, v2 = 2;
  if (A < 0) {  // counter-clockwise winding (y up)
    v1 = 2;
    v2 = 1;
    A = -A;
  }
  const int vo[3] = {0, v1, v2};
  long long Xo[3], Yo[3];
  for (int k = 0; k < 3; ++k) {
    Xo[k] = X[vo[k]];
    Yo[k] = Y[vo[k]];
  }
  long long minX = min(Xo[0], min(Xo[1], Xo[2])), maxX = max(Xo[0], max(Xo[1], Xo[2]));
  long long minY = min(Yo[0], min(Yo[1], Yo[2])), maxY = max(Yo[0], max(Yo[1], Yo[2]));
  long long i0 = ceildiv256(minX - 128), i1 = floordiv256(maxX - 128);
  long long j0 = ceildiv256(minY - 128), j1 = floordiv256(maxY - 128);
  if (a.mode == FHV_CAPTURE_VIEW) {
    i0 = max(i0, 0ll);
    j0 = max(j0, 0ll);
    i1 = min(i1, (long long)a.width - 1);
    j1 = min(j1, (long long)a.height - 1);
  }
  if (i1 < i0 || j1 < j0) return 0ull;
  unsigned long long bw = (unsigned long long)(i1 - i0 + 1), bh = (unsigned long long)(j1 - j0 + 1);
  unsigned long long ns = bw * bh;
  if (ns > (1ull << 31)) {
    set_status(&a.hdr->status, FHV_DEV_HUGE_TRIANGLE);
    return 0ull;
  }
  const long long sx0 = 256 * i0 + 128, sy0 = 256 * j0 + 128;
  uint32_t tl = 0;
  for (int k = 0; k < 3; ++k) {
    int ea = (k + 1) % 3, eb = (k + 2) % 3;
    long long dx = Xo[eb] - Xo[ea], dy = Yo[eb] - Yo[ea];
    ts.dx[k] = (int)dx;
    ts.dy[k] = (int)dy;
    ts.E0[k] = dx * (sy0 - Yo[ea]) - dy * (sx0 - Xo[ea]);
    if (dy < 0 || (dy == 0 && dx < 0)) tl |= 1u << k;
  }
  ts.i0 = (int)i0;
  ts.j0 = (int)j0;
  ts.bw = (uint32_t)bw;
  ts.tl = tl;
  ts.A = A;
  for (int c = 0; c < 3; ++c) {
    ts.Q0[c] = Q[0][c];
    ts.dQ1[c] = (int)Q[v1][c] - (int)Q[0][c];
    ts.dQ2[c] = (int)Q[v2][c] - (int)Q[0][c];
    ts.N[c] = N[0][c];
    ts.N[3 + c] = N[v1][c];
    ts.N[6 + c] = N[v2][c];
  }
  ts.inv_den = 1.0f / (float)(2 * A);
  return ns;
}

__global__ void __launch_bounds__(kSetupTile) setup_scan_kernel(CaptureArgs a) {
  __shared__ unsigned long long s_tile, s_prefix;
  __shared__ unsigned long long s_warp[kSetupTile / 32];
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(&a.hdr->ticket[0], 1ull);
  __syncthreads();
  const unsigned long long tile = s_tile;
  const unsigned long long t = tile * kSetupTile + tid;
  unsigned long long ns = 0;
  if (t < a.n_tri) {
    TriSetup ts;
    ns = setup_triangle(a, (uint32_t)t, ts);
    if (ns) a.setup[t] = ts;
  }
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
    unsigned long long total = __shfl_sync(0xffffffffu, wi, 31);
    if (lane < kSetupTile / 32) s_warp[lane] = wi - w;  // exclusive warp offsets
    unsigned long long pre = lookback_exclusive(a.tile_state, tile, total, &a.hdr->status);
    if (lane == 0) s_prefix = pre;
  }
  __syncthreads();
  const unsigned long long off = s_prefix + s_warp[warp] + (incl - ns);
  if (t < a.n_tri) {
    a.samp_off[t] = off;
    if (t == (unsigned long long)a.n_tri - 1ull) {
      a.samp_off[a.n_tri] = off + ns;
      a.hdr->total = off + ns;
    }
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

__device__ __forceinline__ void eval_sample(const CaptureArgs& a, const TriSetup* __restrict__ setup, uint32_t tri,
                                            uint32_t l, Frag& f) {
  const TriSetup& ts = setup[tri];
  const uint32_t bw = ts.bw;
  const uint32_t jj = l / bw, ii = l - jj * bw;
  long long w[3];
  bool in = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    w[k] = ts.E0[k] + (long long)ts.dx[k] * (256ll * jj) - (long long)ts.dy[k] * (256ll * ii);
    in = in && (w[k] > 0 || (w[k] == 0 && ((ts.tl >> k) & 1u)));
  }
  f.covered = in;
  if (!in) return;
  const long long A = ts.A;
  uint32_t q[3];
  if (A < (1ll << 40)) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      long long num = 2 * (w[1] * (long long)ts.dQ1[c] + w[2] * (long long)ts.dQ2[c]) + A;
      q[c] = (uint32_t)((long long)ts.Q0[c] + floordiv_est(num, 2 * A, ts.inv_den));
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      unsigned __int128 q0 = ts.Q0[c];
      unsigned __int128 num = (unsigned __int128)w[0] * q0 +
                              (unsigned __int128)w[1] * (unsigned __int128)(long long)(ts.Q0[c] + ts.dQ1[c]) +
                              (unsigned __int128)w[2] * (unsigned __int128)(long long)(ts.Q0[c] + ts.dQ2[c]);
      q[c] = (uint32_t)((2 * num + (unsigned __int128)A) / (2 * (unsigned __int128)A));
    }
  }
  const float fw0 = __ll2float_rn(w[0]), fw1 = __ll2float_rn(w[1]), fw2 = __ll2float_rn(w[2]);
  float n[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) n[c] = fadd(fadd(fmul(fw0, ts.N[c]), fmul(fw1, ts.N[3 + c])), fmul(fw2, ts.N[6 + c]));
  f.r.key = morton63(q[0], q[1], q[2]);
  f.r.tri = tri;
  f.r.nrm = oct_encode(n[0], n[1], n[2]);
  if (a.keymode == 0) {
    f.slot = (unsigned long long)(ts.j0 + (int)jj) * (unsigned long long)a.width + (unsigned long long)(ts.i0 + (int)ii);
  } else {
    f.slot = f.r.key >> (63 - 3 * a.depth);
  }
}

__global__ void __launch_bounds__(256) raster_kernel(CaptureArgs a) {
  const unsigned long long total = a.hdr->total;
  if (total == 0) return;
  const uint32_t lane = lane_id();
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x / 32);
  const unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const unsigned long long chunks = (total + 31) / 32;
  const unsigned long long c0 = chunks * w / nwarps, c1 = chunks * (w + 1) / nwarps;
  if (c0 >= c1) return;
  const unsigned long long* __restrict__ off = a.samp_off;
  const uint32_t T = a.n_tri;
  // triangle containing sample 32*c0: last t with off[t] <= s
  unsigned long long t;
  {
    const unsigned long long s = c0 * 32;
    uint32_t lo = 0, hi = T;  // search in off[0..T]: first index with off > s, minus one
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (off[mid] <= s) lo = mid + 1;
      else hi = mid;
    }
    t = lo - 1;
  }
  unsigned long long t_start = off[t];
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
      const unsigned long long o = k <= T ? off[k] : ~0ull;
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
    // append: one counter atomic per warp
    const uint32_t mask = __ballot_sync(0xffffffffu, f.covered);
    if (mask) {
      const uint32_t leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(a.count, (unsigned long long)__popc(mask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (f.covered) {
        const unsigned long long idx = base + __popc(mask & lanemask_lt());
        if (idx < a.capacity) {
          reinterpret_cast<uint4*>(a.rec)[idx] =
              make_uint4((uint32_t)f.r.key, (uint32_t)(f.r.key >> 32), f.r.tri, f.r.nrm);
          const int32_t prev = atomicExch(&a.head[f.slot], (int32_t)idx);
          a.next[idx] = prev;
          if (a.levels && prev == -1) {
            // first fragment of this leaf: mark it in the parent, and so on
            // up while the parent was empty before
            unsigned long long child = f.slot;
            for (int l = a.depth - 1; l >= 0; --l) {
              const unsigned long long parent = child >> 3;
              const uint32_t old = atomicOr(&a.levels[level_offset(l) + parent], 1u << (uint32_t)(child & 7ull));
              if (old != 0u) break;
              child = parent;
            }
          }
        }
      }
    }
    const uint32_t lt = __shfl_sync(0xffffffffu, my_tri, 31);
    const unsigned long long ls = __shfl_sync(0xffffffffu, my_start, 31);
    const bool lvalid = __shfl_sync(0xffffffffu, valid ? 1 : 0, 31) != 0;
    if (lvalid) {
      t = lt;
      t_start = ls;
    }
  }
}

static int raster_blocks_per_sm() {
  static int cached = 0;
  if (cached == 0) {
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, raster_kernel, 256, 0);
    cached = v > 0 ? v : 1;
  }
  return cached;
}

cudaError_t launch_capture(const CaptureArgs& a, cudaStream_t s) {
  if (a.n_tri > 0) {
    const unsigned tiles = (a.n_tri + kSetupTile - 1) / kSetupTile;
    timing_begin("setup_scan", s);
    setup_scan_kernel<<<tiles, kSetupTile, 0, s>>>(a);
    timing_end("setup_scan", s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    timing_begin("raster", s);
    raster_kernel<<<sm_count() * raster_blocks_per_sm(), 256, 0, s>>>(a);
    timing_end("raster", s);
  }
  return cudaGetLastError();
}

}  // namespace fhv
