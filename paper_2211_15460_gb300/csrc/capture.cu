// capture.cu -- FHV creation (Section 3.2): triangle setup, sample-range
// scan, rasterisation and fragment insertion into per-pixel lists (PPFL) or
// per-octant lists (POFL), plus the multi-range fill used to reset arrays.
//
// GB300 layout of the work:
//  * raster (setup fused in): persistent warps take batches of 32 triangles
//    (setup entries) by ticket. Each lane projects, snaps and orients one
//    triangle into the warp's shared-memory slots (160-byte setups that
//    never go to HBM: edge functions at the box origin with the top-left
//    rule folded in, their per-sample steps, the twice-area and its
//    reciprocal), the warp scans their bounding-box sample counts in
//    registers, and walks the batch's samples 32 at a time: each lane finds
//    its triangle by a five-step shuffle search of that scan, evaluates the
//    three integer edge functions with the top-left rule, and the covered
//    samples are appended through a per-warp staging buffer (one counter
//    atomic per run of about a hundred records, coalesced 16-byte record
//    stores; per warp step for the PPFL, whose records carry their pixel). Triangles with more samples than the mode's limit
//    are listed instead (their setups written out), so that no warp is left
//    walking a long batch while the others idle.
//  * big_scan + raster_big: the listed triangles' samples are flattened
//    (prefix of their counts) and every warp walks an equal contiguous share,
//    finding each lane's triangle in a 32-wide window of the prefix.
//  * reset (list captures): list heads and POFL occupancy levels are reset
//    before the raster; a rebuild into lists that hold the previous build
//    resets only that build's heads.
//  * link: one thread per stored record exchanges it into its slot's list
//    head and stores the old head as its link (plus POFL occupancy); a
//    records-only capture (the global fragment list a compaction reads)
//    stops before it. The exchanges hit a multi-GB head array at random;
//    issued from a kernel that does nothing else, their DRAM latency is
//    hidden by occupancy instead of stalling the raster's warps.
//  * raster_pofa (direct POFA build): the same walk three times, its
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
    // the two axes across the projection direction (selects, no indexed local arrays)
    const float mu = axis == 0 ? a.cube_min[1] : (axis == 1 ? a.cube_min[2] : a.cube_min[0]);
    const float mv = axis == 0 ? a.cube_min[2] : (axis == 1 ? a.cube_min[0] : a.cube_min[1]);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const float pu = axis == 0 ? p[v][1] : (axis == 1 ? p[v][2] : p[v][0]);
      const float pv = axis == 0 ? p[v][2] : (axis == 1 ? p[v][0] : p[v][1]);
      X[v] = snap256(fmul(fsub(pu, mu), inv_h));
      Y[v] = snap256(fmul(fsub(pv, mv), inv_h));
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
  const bool flip = A < 0;  // counter-clockwise winding (y up): vertices 1 and 2 swapped
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
  // oriented vertices (selects, no indexed local arrays)
  const long long OX[3] = {X[0], flip ? X[2] : X[1], flip ? X[1] : X[2]};
  const long long OY[3] = {Y[0], flip ? Y[2] : Y[1], flip ? Y[1] : Y[2]};
  int dmax = 0;  // largest |d1| + |d2| over the axes
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float n1 = flip ? N[2][c] : N[1][c], n2 = flip ? N[1][c] : N[2][c];
    const uint32_t q1 = flip ? Q[2][c] : Q[1][c], q2 = flip ? Q[1][c] : Q[2][c];
    ts.N[c] = N[0][c];
    ts.N[3 + c] = n1;
    ts.N[6 + c] = n2;
    ts.q0[c] = Q[0][c];
    ts.d1[c] = (int)q1 - (int)Q[0][c];
    ts.d2[c] = (int)q2 - (int)Q[0][c];
    dmax = max(dmax, abs(ts.d1[c]) + abs(ts.d2[c]));
  }
  ts.tri = a.tri_base + t;
  ts.qerr = __fmul_ru(__int2float_ru(dmax + 1), 1.0f / 2097152.0f);  // 2^-21 (D + 1), rounded up
  // edge k runs from vertex (k+1)%3 to (k+2)%3; at sample (i0 + i, j0 + j)
  // w_k = dx_k (sy - Y_{k+1}) - dy_k (sx - X_{k+1}), sx = 256 (i0 + i) + 128
  const long long sx0 = 256ll * i0 + 128, sy0 = 256ll * j0 + 128;
  long long sum = 0;
  uint32_t bias = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    const long long dx = OX[k2] - OX[k1], dy = OY[k2] - OY[k1];
    const long long w = dx * (sy0 - OY[k1]) - dy * (sx0 - OX[k1]);
    const bool tl = dy < 0 || (dy == 0 && dx < 0);  // top-left: a zero edge value still covers
    sum += w;
    ts.c[k] = tl ? w : w - 1;
    bias |= (tl ? 0u : 1u) << k;
    ts.ea[k] = (int)(-dy);
    ts.eb[k] = (int)dx;
  }
  ts.A = sum;
  ts.bias = bias;
  ts.inv_den = __frcp_rn(__ll2float_rn(2 * sum));
  ts.i0 = (int)i0;
  ts.j0 = (int)j0;
  ts.bw = (uint32_t)bw;
  ts.inv_bw = __frcp_rn((float)(uint32_t)bw);
  return ns;
}

// List heads (and POFL occupancy) reset before a list capture: the fill
// ranges, or, when the lists hold the previous build (reuse), exactly the
// heads of its stored records.
__global__ void __launch_bounds__(256) reset_kernel(CaptureArgs a, FillSet fs) {
  const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  fill_ranges(fs, t0, stride);
  if (a.sparse_reset) {
    const unsigned long long prev = *a.count < a.capacity ? *a.count : a.capacity;
    const int sh = 63 - 3 * a.depth;
    for (unsigned long long i = t0; i < prev; i += stride) {
      const unsigned long long key = reinterpret_cast<const unsigned long long*>(a.rec)[2 * i];
      a.head[key >> sh] = -1;
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

// Sample l (row-major in the bounding box) of the setup ts.
__device__ __forceinline__ void eval_sample(const CaptureArgs& a, const TriSetup& ts, uint32_t l,
                                            Frag& f) {
  const uint32_t bw = ts.bw;
  uint32_t jj = (uint32_t)__fmul_rz(__uint2float_rz(l), ts.inv_bw);  // row estimate, then exact
  long long r = (long long)l - (long long)jj * bw;
  if (r < 0 || r >= (long long)bw) {
    jj = l / bw;
    r = (long long)(l - jj * bw);
  }
  const uint32_t ii = (uint32_t)r;
  long long w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    w[k] = ts.c[k] + 256ll * ((long long)ts.ea[k] * (long long)ii + (long long)ts.eb[k] * (long long)jj);
  const bool in = (w[0] | w[1] | w[2]) >= 0;  // every edge covers (top-left rule folded into c)
  f.covered = in;
  if (!in) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) w[k] += (long long)((ts.bias >> k) & 1u);  // exact edge values
  const long long A = ts.A;
  const float fw0 = __ll2float_rn(w[0]), fw1 = __ll2float_rn(w[1]), fw2 = __ll2float_rn(w[2]);
  uint32_t q[3];
  if (A < (1ll << 40)) {
    // q = q0 + floor(x / A + 1/2), x = w1 d1 + w2 d2, 0 <= w1, w2 <= A. The
    // float estimate t of x / A + 1/2 (six roundings of relative size u =
    // 2^-24 on terms bounded by D = |d1| + |d2|, one on t itself) is within
    // 7u (D + 1) of it, below qerr = 8u (D + 1): when t's fraction is more
    // than qerr from an integer its floor is exact, else the exact division.
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float s = fadd(fmul(fw1, (float)ts.d1[c]), fmul(fw2, (float)ts.d2[c]));
      const float t = fadd(fmul(fadd(s, s), ts.inv_den), 0.5f);
      const float fl = floorf(t);
      const float fr = fsub(t, fl);
      if (fr > ts.qerr && fr < fsub(1.0f, ts.qerr)) {
        q[c] = (uint32_t)((int)ts.q0[c] + (int)fl);
      } else {
        const long long num = 2 * (w[1] * (long long)ts.d1[c] + w[2] * (long long)ts.d2[c]) + A;
        q[c] = (uint32_t)((long long)ts.q0[c] + floordiv_est(num, 2 * A, ts.inv_den));
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const unsigned long long q0 = ts.q0[c];
      const unsigned __int128 num = (unsigned __int128)w[0] * q0 +
                                    (unsigned __int128)w[1] * (unsigned long long)((long long)q0 + ts.d1[c]) +
                                    (unsigned __int128)w[2] * (unsigned long long)((long long)q0 + ts.d2[c]);
      q[c] = (uint32_t)((2 * num + (unsigned __int128)A) / (2 * (unsigned __int128)A));
    }
  }
  float n[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) n[c] = fadd(fadd(fmul(fw0, ts.N[c]), fmul(fw1, ts.N[3 + c])), fmul(fw2, ts.N[6 + c]));
  f.r.key = morton63(q[0], q[1], q[2]);
  f.r.tri = ts.tri;
  f.r.nrm = oct_encode(n[0], n[1], n[2]);
  if (a.keymode == 0) {
    f.slot = (unsigned long long)(ts.j0 + (int)jj) * (unsigned long long)a.width + (unsigned long long)(ts.i0 + (int)ii);
  } else if (a.keymode == 1) {
    f.slot = f.r.key >> (63 - 3 * a.depth);
  } else {
    f.slot = 0;
  }
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
  __device__ __forceinline__ void flush(const CaptureArgs&, uint32_t) const {}
};

// The covered samples appended through a per-warp staging buffer in shared
// memory: a warp reserves its staged run with one counter atomic once the
// buffer is nearly full (and when it is done), then stores the run with
// coalesced 16-byte stores. The counter is a single word that every warp of
// the grid adds to, so one atomic per about a hundred records instead of
// one per warp step keeps it from serialising the raster. Used where the
// records carry no slot (keymodes 1 and 2); the order of the appended
// records is arbitrary either way.
constexpr uint32_t kStage = 120;  // records staged per warp (1920 bytes)

struct StagedSink {
  uint4* buf;     // this warp's kStage records
  uint32_t fill;  // staged records (warp-uniform)
  __device__ __forceinline__ void operator()(const CaptureArgs& a, const Frag& f, uint32_t lane) {
    const uint32_t mask = __ballot_sync(0xffffffffu, f.covered);
    if (f.covered)
      buf[fill + __popc(mask & lanemask_lt())] =
          make_uint4((uint32_t)f.r.key, (uint32_t)(f.r.key >> 32), f.r.tri, f.r.nrm);
    fill += __popc(mask);
    if (fill > kStage - 32) flush(a, lane);
  }
  __device__ __forceinline__ void flush(const CaptureArgs& a, uint32_t lane) {
    if (fill == 0) return;
    __syncwarp();  // the staged records are visible to the whole warp
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.count, (unsigned long long)fill);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t i = lane; i < fill; i += 32)
      if (base + i < a.capacity) reinterpret_cast<uint4*>(a.rec)[base + i] = buf[i];
    __syncwarp();  // read out before the buffer fills again
    fill = 0;
  }
};

// Every warp takes batches of 32 setup entries by ticket: each lane sets up
// one triangle into the warp's shared-memory slots, the warp scans the
// bounding-box sample counts, and walks the batch's samples 32 at a time,
// each lane finding its triangle by a binary search over the scan held in
// registers. Setups with more samples than the mode's limit (kSmallSamples,
// kSmallSamplesAxis3) go to the chunked
// path (the first pass lists them; later passes of the direct POFA build
// skip them). `sink` takes each step's fragments (called by all 32 lanes).
constexpr int kRasterThreads = 256;

template <class Sink>
__device__ __forceinline__ void raster_small(const CaptureArgs& a, Sink& sink, int pass) {
  __shared__ __align__(16) TriSetup s_ts[kRasterThreads / 32][32];
  const uint32_t lane = lane_id();
  TriSetup* my = s_ts[threadIdx.x >> 5];
  const unsigned long long n_batches = ((unsigned long long)a.n_setup + 31ull) / 32ull;
  unsigned long long* ticket = &a.hdr->raster_ticket[pass][0];
  while (true) {
    unsigned long long batch = 0;
    if (lane == 0) batch = atomicAdd(ticket, 1ull);
    batch = __shfl_sync(0xffffffffu, batch, 0);
    if (batch >= n_batches) break;
    const uint32_t e0 = (uint32_t)(batch * 32ull);
    const uint32_t e = e0 + lane;
    unsigned long long ns = 0;
    if (e < a.n_setup) ns = setup_triangle(a, e, my[lane]);
    if (ns > (a.mode == FHV_CAPTURE_AXIS3 ? kSmallSamplesAxis3 : kSmallSamples)) {
      if (pass == 0) {
        const unsigned long long k = atomicAdd(&a.hdr->n_big, 1ull);
        a.big_setup[k] = my[lane];
        a.big_meta[k] = (ns << 32) | e;
      }
      ns = 0;
    }
    uint32_t incl = (uint32_t)ns;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)lane >= o) incl += v;
    }
    const uint32_t excl = incl - (uint32_t)ns;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();  // the batch's setups are in shared memory
    for (uint32_t s0 = 0; s0 < total; s0 += 32) {
      const uint32_t smp = s0 + lane;
      const bool valid = smp < total;
      uint32_t t = 0;  // first lane whose inclusive count exceeds smp
#pragma unroll
      for (uint32_t step = 16; step >= 1; step >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, incl, t + step - 1);
        if (v <= smp) t += step;
      }
      t = min(t, 31u);
      const uint32_t start = __shfl_sync(0xffffffffu, excl, t);
      Frag f;
      f.covered = false;
      if (valid) eval_sample(a, my[t], smp - start, f);
      sink(a, f, lane);
    }
    __syncwarp();  // done with the slots before the next batch
  }
}

// Exclusive prefix of the listed setups' sample counts (big_pref[0..n_big],
// big_pref[n_big] = their total, also in hdr->big_total), in three steps:
// per-4096-entry chunk sums, one CTA over the chunks, then each chunk's
// entries. The grids cover every setup entry; chunks past n_big idle.
constexpr uint32_t kBigScanChunk = 4096;

__device__ __forceinline__ unsigned long long big_samples(const CaptureArgs& a, unsigned long long k) {
  return a.big_meta[k] >> 32;
}

__global__ void __launch_bounds__(256) big_chunk_kernel(CaptureArgs a) {
  __shared__ unsigned long long s_w[8];
  const unsigned long long nb = a.hdr->n_big;
  const unsigned long long k0 = (unsigned long long)blockIdx.x * kBigScanChunk;
  unsigned long long sum = 0;
  for (unsigned long long k = k0 + threadIdx.x; k < min(nb, k0 + kBigScanChunk); k += blockDim.x)
    sum += big_samples(a, k);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    a.big_chunk[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) big_chunk_scan_kernel(CaptureArgs a, unsigned n_chunks) {
  __shared__ unsigned long long s_w[32];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned per = (n_chunks + blockDim.x - 1) / blockDim.x;
  const unsigned b = threadIdx.x * per, e = min(n_chunks, b + per);
  unsigned long long sum = 0;
  for (unsigned i = b; i < e; ++i) sum += a.big_chunk[i];
  unsigned long long incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += v;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long w = s_w[lane];
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, wi, o);
      if ((int)lane >= o) wi += v;
    }
    s_w[lane] = wi - w;
    if (lane == 31) {
      a.hdr->big_total = wi;
      a.big_pref[a.hdr->n_big] = wi;
    }
  }
  __syncthreads();
  unsigned long long run = s_w[warp] + (incl - sum);
  for (unsigned i = b; i < e; ++i) {
    const unsigned long long c = a.big_chunk[i];
    a.big_chunk[i] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(256) big_pref_kernel(CaptureArgs a) {
  __shared__ unsigned long long s_w[9];
  const unsigned long long nb = a.hdr->n_big;
  const unsigned long long k0 = (unsigned long long)blockIdx.x * kBigScanChunk;
  if (k0 >= nb) return;
  constexpr uint32_t per = kBigScanChunk / 256;  // 16 consecutive entries per thread
  const unsigned long long kb = k0 + (unsigned long long)threadIdx.x * per;
  unsigned long long sum = 0;
  for (uint32_t j = 0; j < per; ++j)
    if (kb + j < nb) sum += big_samples(a, kb + j);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += v;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long r = 0;
    for (int w = 0; w < 8; ++w) {
      const unsigned long long x = s_w[w];
      s_w[w] = r;
      r += x;
    }
  }
  __syncthreads();
  unsigned long long run = a.big_chunk[blockIdx.x] + s_w[warp] + (incl - sum);
  for (uint32_t j = 0; j < per; ++j) {
    if (kb + j < nb) {
      a.big_pref[kb + j] = run;
      run += big_samples(a, kb + j);
    }
  }
}

// The listed setups' samples, flattened: every warp walks an equal
// contiguous share 32 samples at a time, finding each lane's setup in a
// 32-wide window of the prefix array (shuffle search), so large and tiny
// triangles balance alike; the setups are read from the list (L1-resident).
template <class Sink>
__device__ __forceinline__ void raster_big(const CaptureArgs& a, Sink& sink) {
  const unsigned long long total = a.hdr->big_total;
  const unsigned long long nb = a.hdr->n_big;
  if (total == 0 || nb == 0) return;
  const uint32_t lane = lane_id();
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x / 32);
  const unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const unsigned long long chunks = (total + 31) / 32;
  const unsigned long long c0 = chunks * w / nwarps, c1 = chunks * (w + 1) / nwarps;
  if (c0 >= c1) return;
  unsigned long long t;  // listed setup containing sample 32 c0: last t with start(t) <= s
  {
    const unsigned long long s = c0 * 32;
    unsigned long long lo = 0, hi = nb;
    while (lo < hi) {
      const unsigned long long mid = (lo + hi) >> 1;
      if (a.big_pref[mid] <= s) lo = mid + 1;
      else hi = mid;
    }
    t = lo - 1;
  }
  unsigned long long t_start = a.big_pref[t];
  for (unsigned long long c = c0; c < c1; ++c) {
    const unsigned long long s = c * 32 + lane;
    const bool valid = s < total;
    bool found = !valid;
    unsigned long long my_k = 0, my_start = 0;
    unsigned long long wbase = t, wstart = t_start;
    while (true) {  // windows of 32 starts after t; big_pref[nb] = total ends the search
      const unsigned long long k = wbase + 1 + lane;
      const unsigned long long o = k <= nb ? a.big_pref[k] : ~0ull;
      uint32_t cnt = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const unsigned long long v = __shfl_sync(0xffffffffu, o, cnt + step - 1);
        if (v <= s) cnt += step;
      }
      const unsigned long long last = __shfl_sync(0xffffffffu, o, 31);
      const unsigned long long prev = __shfl_sync(0xffffffffu, o, cnt > 0 ? cnt - 1 : 0);
      if (!found && last > s) {
        found = true;
        my_k = wbase + cnt;
        my_start = cnt > 0 ? prev : wstart;
      }
      if (__all_sync(0xffffffffu, found)) break;
      wbase += 32;
      wstart = last;
    }
    Frag f;
    f.covered = false;
    if (valid) eval_sample(a, a.big_setup[my_k], (uint32_t)(s - my_start), f);
    sink(a, f, lane);
    const unsigned long long lt = __shfl_sync(0xffffffffu, my_k, 31);
    const unsigned long long ls = __shfl_sync(0xffffffffu, my_start, 31);
    const bool lvalid = __shfl_sync(0xffffffffu, valid ? 1 : 0, 31) != 0;
    if (lvalid) {
      t = lt;
      t_start = ls;
    }
  }
}

// Dynamic shared memory of the staged capture kernels (keymodes 1 and 2):
// the warps' staging buffers.
constexpr uint32_t kStageBytes = (kRasterThreads / 32) * kStage * 16;

template <bool kStaged>
__global__ void __launch_bounds__(kRasterThreads, 4) raster_kernel(CaptureArgs a) {
  if (!kStaged) {
    AppendSink sink{};
    raster_small(a, sink, 0);
  } else {
    extern __shared__ __align__(16) uint4 s_stage[];
    StagedSink sink{s_stage + (threadIdx.x >> 5) * kStage, 0u};
    raster_small(a, sink, 0);
    sink.flush(a, lane_id());
  }
}
template <bool kStaged>
__global__ void __launch_bounds__(kRasterThreads, 4) raster_big_kernel(CaptureArgs a) {
  if (!kStaged) {
    AppendSink sink{};
    raster_big(a, sink);
  } else {
    extern __shared__ __align__(16) uint4 s_stage[];
    StagedSink sink{s_stage + (threadIdx.x >> 5) * kStage, 0u};
    raster_big(a, sink);
    sink.flush(a, lane_id());
  }
}

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
  int T;             // level of the leaf tiles' parents (0: none)
  uint32_t counted;  // mark pass: covered samples of this warp not yet added to the count (warp-uniform)
  __device__ __forceinline__ void operator()(const CaptureArgs& a, const Frag& f, uint32_t lane) {
    const uint32_t mask = __ballot_sync(0xffffffffu, f.covered);
    if (!mask) return;
    uint32_t* off_leaf = c.off + level_offset(c.depth);
    uint32_t* cnt_leaf = c.cnt + level_offset(c.depth);
    if (kPass == kPassMark) {  // one count atomic per warp and 2^30 samples, not per step
      counted += __popc(mask);
      if (counted >= (1u << 30)) flush(a, lane);
    }
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
  __device__ __forceinline__ void flush(const CaptureArgs& a, uint32_t lane) {
    if (kPass == kPassMark && counted) {
      if (lane == 0) atomicAdd(a.count, (unsigned long long)counted);
      counted = 0;
    }
  }
};

template <int kPass>
__global__ void __launch_bounds__(kRasterThreads, 4) raster_pofa_kernel(CaptureArgs a, CompactArgs c, int T) {
  if (kPass == kPassCount && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long n = *a.count;  // final: the mark pass has counted every fragment
    a.hdr->n_kept = n <= c.n_max ? n : 0ull;
  }
  if (kPass == kPassScatter && *a.count > c.n_max) return;  // over capacity: nothing is stored
  PofaSink<kPass> sink{c, T, 0u};
  raster_small(a, sink, kPass);
  sink.flush(a, lane_id());
}

template <int kPass>
__global__ void __launch_bounds__(kRasterThreads, 4) raster_pofa_big_kernel(CaptureArgs a, CompactArgs c, int T) {
  if (kPass == kPassScatter && *a.count > c.n_max) return;
  PofaSink<kPass> sink{c, T, 0u};
  raster_big(a, sink);
  sink.flush(a, lane_id());
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
static int blocks_per_sm(K kernel, size_t smem = 0) {
  int v = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, kRasterThreads, smem);
  return v > 0 ? v : 1;
}

// fills[0..n_first) are the small resets (header, counter), launched first
// as one fill; the other ranges (list heads, occupancy levels) are stored
// by reset_kernel, which also does the reuse mode's sparse head reset
// before the counter is cleared.
static cudaError_t launch_resets(const CaptureArgs& a, const RangeFill* fills, int n_first, int n_fills,
                                 cudaStream_t s) {
  cudaError_t e = launch_fill(fills, n_first, s);
  if (e != cudaSuccess) return e;
  FillSet fs;
  fs.n = 0;
  for (int i = n_first; i < n_fills && fs.n < 6; ++i)
    if (fills[i].n) fs.r[fs.n++] = fills[i];
  if (fs.n == 0 && !a.sparse_reset) return cudaSuccess;
  timing_begin("reset", s);
  reset_kernel<<<sm_count() * 8, 256, 0, s>>>(a, fs);
  timing_end("reset", s);
  if (a.sparse_reset) {  // the previous count was read by the reset
    RangeFill c{a.count, 1ull, 0ull, 8};
    e = launch_fill(&c, 1, s);
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// The listed setups' sample prefix (three launches).
static void launch_big_scan(const CaptureArgs& a, cudaStream_t s) {
  const unsigned chunks = a.n_setup ? (a.n_setup + kBigScanChunk - 1) / kBigScanChunk : 1u;  // >= 1 launchable
  timing_begin("big_scan", s);
  big_chunk_kernel<<<chunks, 256, 0, s>>>(a);
  timing_end("big_scan", s);
  timing_begin("big_scan", s);
  big_chunk_scan_kernel<<<1, 1024, 0, s>>>(a, chunks);
  timing_end("big_scan", s);
  timing_begin("big_scan", s);
  big_pref_kernel<<<chunks, 256, 0, s>>>(a);
  timing_end("big_scan", s);
}

cudaError_t launch_capture(const CaptureArgs& a, const RangeFill* fills, int n_first, int n_fills, cudaStream_t s) {
  static int per_sm[2][2] = {{0, 0}, {0, 0}};  // [staged][small, big]
  if (per_sm[0][0] == 0) {
    cudaFuncSetAttribute(raster_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes);
    cudaFuncSetAttribute(raster_big_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes);
    per_sm[0][0] = blocks_per_sm(raster_kernel<false>);
    per_sm[0][1] = blocks_per_sm(raster_big_kernel<false>);
    per_sm[1][0] = blocks_per_sm(raster_kernel<true>, kStageBytes);
    per_sm[1][1] = blocks_per_sm(raster_big_kernel<true>, kStageBytes);
  }
  cudaError_t e = launch_resets(a, fills, n_first, n_fills, s);
  if (e != cudaSuccess || a.n_setup == 0) return e;
  const bool staged = a.keymode != 0;  // keymode 0 parks each record's pixel in next[]
  const int sms = sm_count();
  timing_begin("raster", s);
  if (staged) raster_kernel<true><<<sms * per_sm[1][0], kRasterThreads, kStageBytes, s>>>(a);
  else raster_kernel<false><<<sms * per_sm[0][0], kRasterThreads, 0, s>>>(a);
  timing_end("raster", s);
  launch_big_scan(a, s);
  timing_begin("raster_big", s);
  if (staged) raster_big_kernel<true><<<sms * per_sm[1][1], kRasterThreads, kStageBytes, s>>>(a);
  else raster_big_kernel<false><<<sms * per_sm[0][1], kRasterThreads, 0, s>>>(a);
  timing_end("raster_big", s);
  if (a.keymode == 2) return cudaGetLastError();  // records only: nothing to link
  timing_begin("link", s);
  link_kernel<<<sm_count() * 16, 256, 0, s>>>(a);
  timing_end("link", s);
  return cudaGetLastError();
}

cudaError_t launch_pofa_direct(const CaptureArgs& a, const CompactArgs& c, const RangeFill* fills, int n_first,
                               int n_fills, cudaStream_t s) {
  static int per_sm[6] = {0, 0, 0, 0, 0, 0};
  if (per_sm[0] == 0) {
    per_sm[0] = blocks_per_sm(raster_pofa_kernel<kPassMark>);
    per_sm[1] = blocks_per_sm(raster_pofa_kernel<kPassCount>);
    per_sm[2] = blocks_per_sm(raster_pofa_kernel<kPassScatter>);
    per_sm[3] = blocks_per_sm(raster_pofa_big_kernel<kPassMark>);
    per_sm[4] = blocks_per_sm(raster_pofa_big_kernel<kPassCount>);
    per_sm[5] = blocks_per_sm(raster_pofa_big_kernel<kPassScatter>);
  }
  const int T = c.depth > 4 ? c.depth - 4 : 0;
  const int sms = sm_count();
  cudaError_t e = launch_resets(a, fills, n_first, n_fills, s);
  if (e == cudaSuccess) e = compact_clear_bitmap(c, s);
  if (e != cudaSuccess) return e;
  timing_begin("raster_mark", s);
  raster_pofa_kernel<kPassMark><<<sms * per_sm[0], kRasterThreads, 0, s>>>(a, c, T);
  timing_end("raster_mark", s);
  launch_big_scan(a, s);
  timing_begin("raster_mark", s);
  raster_pofa_big_kernel<kPassMark><<<sms * per_sm[3], kRasterThreads, 0, s>>>(a, c, T);
  timing_end("raster_mark", s);
  timing_begin("raster_count", s);
  raster_pofa_kernel<kPassCount><<<sms * per_sm[1], kRasterThreads, 0, s>>>(a, c, T);
  timing_end("raster_count", s);
  timing_begin("raster_count", s);
  raster_pofa_big_kernel<kPassCount><<<sms * per_sm[4], kRasterThreads, 0, s>>>(a, c, T);
  timing_end("raster_count", s);
  e = compact_scan(c, s);
  if (e != cudaSuccess || c.n_max == 0) return e;
  timing_begin("raster_scatter", s);
  raster_pofa_kernel<kPassScatter><<<sms * per_sm[2], kRasterThreads, 0, s>>>(a, c, T);
  timing_end("raster_scatter", s);
  timing_begin("raster_scatter", s);
  raster_pofa_big_kernel<kPassScatter><<<sms * per_sm[5], kRasterThreads, 0, s>>>(a, c, T);
  timing_end("raster_scatter", s);
  return compact_order(c, s);
}

}  // namespace fhv
