// sort.cuh -- ordering of 16-byte fragment records by their whole 128-bit
// key (Morton code, triangle, normal): the canonical POFA order inside an
// octant. Shared by the dense compaction (pofa.cu) and the sparse one
// (sparse.cu).
#pragma once

#include "kernels.h"

namespace fhv {

static __device__ __forceinline__ bool rec_less(const uint4& x, const uint4& y) {
  const unsigned long long kx = (unsigned long long)x.x | ((unsigned long long)x.y << 32);
  const unsigned long long ky = (unsigned long long)y.x | ((unsigned long long)y.y << 32);
  if (kx != ky) return kx < ky;
  if (x.z != y.z) return x.z < y.z;
  return x.w < y.w;
}

// Bitonic sort of s[0..P) (P a power of two) by the whole CTA.
static __device__ void bitonic_smem(uint4* s, uint32_t P) {
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint4 x = s[i], y = s[ixj];
          const bool up = (i & k) == 0;
          if (up ? rec_less(y, x) : rec_less(x, y)) {
            s[i] = y;
            s[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Sort pofa[lo, hi) (hi - lo <= kSortCap) in shared memory.
static __device__ void sort_range_smem(uint4* g, unsigned long long lo, unsigned long long hi, uint4* s) {
  const uint32_t len = (uint32_t)(hi - lo);
  if (len <= 1) return;
  uint32_t P = 2;
  while (P < len) P <<= 1;
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
    s[i] = i < len ? g[lo + i] : make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
  __syncthreads();
  bitonic_smem(s, P);
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) g[lo + i] = s[i];
  __syncthreads();
}

// Sort src[lo, hi) (hi - lo <= kSortCap) in shared memory into dst[lo, hi).
static __device__ void sort_range_smem_to(const uint4* src, uint4* dst, unsigned long long lo, unsigned long long hi,
                                          uint4* s) {
  const uint32_t len = (uint32_t)(hi - lo);
  if (len == 0) return;
  uint32_t P = 1;
  while (P < len) P <<= 1;
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
    s[i] = i < len ? src[lo + i] : make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
  __syncthreads();
  if (P > 1) bitonic_smem(s, P);
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) dst[lo + i] = s[i];
  __syncthreads();
}

static __device__ __forceinline__ uint4 shfl_xor_rec(const uint4& x, int m) {
  return make_uint4(__shfl_xor_sync(0xffffffffu, x.x, m), __shfl_xor_sync(0xffffffffu, x.y, m),
                    __shfl_xor_sync(0xffffffffu, x.z, m), __shfl_xor_sync(0xffffffffu, x.w, m));
}

// Bitonic sort of 32 records, one per lane, in registers: lane i ends with
// the i-th smallest.
static __device__ __forceinline__ uint4 warp_sort32(uint4 x) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const uint4 y = shfl_xor_rec(x, (int)j);
      const bool up = (lane & k) == 0;     // this 2k-block ascends
      const bool lower = (lane & j) == 0;  // lower index of the pair: keeps the min when ascending
      if ((lower == up) ? rec_less(y, x) : rec_less(x, y)) x = y;
    }
  }
  return x;
}

// One merge pass over s_src[0, len), sorted runs of `width`: pairs of runs
// merged into s_dst (stable: on ties the left run first). Each thread makes
// a contiguous slice of the output, locating it by a merge-path search.
static __device__ void merge_pass_smem(const uint4* s_src, uint4* s_dst, uint32_t len, uint32_t width) {
  const uint32_t per = (len + blockDim.x - 1) / blockDim.x;
  uint32_t o = threadIdx.x * per;
  const uint32_t o1 = min(len, o + per);
  while (o < o1) {
    const uint32_t a0 = (o / (2 * width)) * (2 * width);
    const uint32_t la = min(width, len - a0);
    const uint32_t b0 = a0 + la;
    const uint32_t lb = b0 < len ? min(width, len - b0) : 0u;
    const uint32_t end = min(o1, a0 + la + lb);
    const uint4* A = s_src + a0;
    const uint4* B = s_src + b0;
    const uint32_t d = o - a0;
    uint32_t lo = d > lb ? d - lb : 0u, hi = min(d, la);
    while (lo < hi) {  // i = number of A elements among the first d outputs
      const uint32_t mid = (lo + hi) >> 1;
      if (!rec_less(B[d - mid - 1], A[mid])) lo = mid + 1;
      else hi = mid;
    }
    uint32_t i = lo, j = d - lo;
    for (; o < end; ++o) {
      const bool take_a = j >= lb || (i < la && !rec_less(B[j], A[i]));
      s_dst[a0 + (o - a0)] = take_a ? A[i++] : B[j++];
    }
  }
}

// Sort src[lo, hi) (hi - lo <= kSortCap) into dst[lo, hi) by the whole CTA:
// 32-record warp sorts in registers, then merge passes between two shared
// buffers s_a, s_b (kSortCap records each). Ends with a barrier.
static __device__ void merge_sort_smem_to(const uint4* src, uint4* dst, unsigned long long lo, unsigned long long hi,
                                          uint4* s_a, uint4* s_b) {
  const uint32_t len = (uint32_t)(hi - lo);
  if (len == 0) return;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint4 big = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
  for (uint32_t c = warp; c * 32 < len; c += nwarps) {
    const uint32_t i = c * 32 + lane;
    uint4 x = i < len ? src[lo + i] : big;
    x = warp_sort32(x);
    if (i < len) s_a[i] = x;  // the padding sorts to the chunk's end
  }
  __syncthreads();
  uint4* s = s_a;
  uint4* t = s_b;
  for (uint32_t width = 32; width < len; width <<= 1) {
    merge_pass_smem(s, t, len, width);
    __syncthreads();
    uint4* tmp = s;
    s = t;
    t = tmp;
  }
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) dst[lo + i] = s[i];
  __syncthreads();
}

// Merge sort of s[0, len) in shared memory with t[0, len) as scratch, by
// the whole CTA (warp sorts of 32, then merge passes); the result ends in s.
// Ends with a barrier.
static __device__ void merge_sort_smem_inplace(uint4* s, uint4* t, uint32_t len) {
  if (len <= 1) {
    __syncthreads();
    return;
  }
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint4 big = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
  for (uint32_t c = warp; c * 32 < len; c += nwarps) {
    const uint32_t i = c * 32 + lane;
    uint4 x = i < len ? s[i] : big;
    x = warp_sort32(x);
    if (i < len) s[i] = x;
  }
  __syncthreads();
  uint4* a = s;
  uint4* b = t;
  for (uint32_t width = 32; width < len; width <<= 1) {
    merge_pass_smem(a, b, len, width);
    __syncthreads();
    uint4* tmp = a;
    a = b;
    b = tmp;
  }
  if (a != s) {
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) s[i] = a[i];
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned long long rec_key(const uint4& r) {
  return (unsigned long long)r.x | ((unsigned long long)r.y << 32);
}

constexpr uint32_t kRankRange = 64;    // groups this short are ranked record by record
// ---- sorts of packed 64-bit values (unique, so no tie rule)

// Bitonic sort of one value per lane, ascending with the lane.
static __device__ __forceinline__ unsigned long long warp_sort32_u64(unsigned long long x) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (uint32_t k = 2; k <= 32; k <<= 1)
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, j);
      const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);  // lower lane of an ascending pair, or upper of a descending one
      x = keep_min ? (y < x ? y : x) : (y > x ? y : x);
    }
  return x;
}

// One merge pass over src[0, len), sorted runs of `width`, into dst: each
// thread makes a contiguous slice of the output, found by a merge-path
// search, holding the two run heads in registers.
static __device__ void merge_pass_u64(const unsigned long long* src, unsigned long long* dst, uint32_t len,
                                      uint32_t width) {
  const uint32_t per = (len + blockDim.x - 1) / blockDim.x;
  uint32_t o = threadIdx.x * per;
  const uint32_t o1 = min(len, o + per);
  while (o < o1) {
    const uint32_t a0 = (o / (2 * width)) * (2 * width);
    const uint32_t la = min(width, len - a0);
    const uint32_t b0 = a0 + la;
    const uint32_t lb = b0 < len ? min(width, len - b0) : 0u;
    const uint32_t end = min(o1, a0 + la + lb);
    const unsigned long long* A = src + a0;
    const unsigned long long* B = src + b0;
    const uint32_t d = o - a0;
    uint32_t lo = d > lb ? d - lb : 0u, hi = min(d, la);
    while (lo < hi) {  // i = number of A elements among the first d outputs
      const uint32_t mid = (lo + hi) >> 1;
      if (!(B[d - mid - 1] < A[mid])) lo = mid + 1;
      else hi = mid;
    }
    uint32_t i = lo, j = d - lo;
    unsigned long long ai = i < la ? A[i] : ~0ull, bj = j < lb ? B[j] : ~0ull;
    for (; o < end; ++o) {
      if (j >= lb || (i < la && !(bj < ai))) {
        dst[o] = ai;
        ++i;
        ai = i < la ? A[i] : ~0ull;
      } else {
        dst[o] = bj;
        ++j;
        bj = j < lb ? B[j] : ~0ull;
      }
    }
  }
}

// Merge sort of s[0, len) with t[0, len) as scratch, by the whole CTA; the
// result ends in s. Ends with a barrier.
static __device__ void merge_sort_u64(unsigned long long* s, unsigned long long* t, uint32_t len) {
  if (len > 1) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint32_t c = warp; c * 32 < len; c += nwarps) {  // warp-uniform: the shuffles see every lane
      const uint32_t i = c * 32 + lane;
      const unsigned long long x = warp_sort32_u64(i < len ? s[i] : ~0ull);
      if (i < len) s[i] = x;
    }
    __syncthreads();
    unsigned long long* a = s;
    unsigned long long* b = t;
    for (uint32_t width = 32; width < len; width <<= 1) {
      merge_pass_u64(a, b, len, width);
      __syncthreads();
      unsigned long long* tmp = a;
      a = b;
      b = tmp;
    }
    if (a != s)
      for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) s[i] = a[i];
  }
  __syncthreads();
}

constexpr uint32_t kTileGroups = 4096;  // group starts a tile can hold
constexpr uint32_t kLargeList = 64;     // groups above kRankRange in one tile: at most 63
constexpr uint32_t kMiscWords = 48;

// The whole range s_a[0, len) (len <= 2048, groups in s_gid) ordered into
// s_b through packed keys: (group << (gsh + 11)) | (key bits below gsh << 11)
// | position, so one 64-bit sort orders by the whole Morton key (groups
// share the bits from gsh up, which the group index orders) and the records
// move once. Equal keys (rare) are then ordered by triangle, normal and
// position. Needs gsh <= 42. s_tmp (len values) may alias s_b. Ends with a
// barrier.
static __device__ void packed_order(const uint4* s_a, uint4* s_b, uint32_t len, int gsh, const uint32_t* s_gid,
                                    unsigned long long* s_key, unsigned long long* s_tmp) {
  const unsigned long long low = (1ull << gsh) - 1ull;
  for (uint32_t p = threadIdx.x; p < len; p += blockDim.x)
    s_key[p] = ((unsigned long long)s_gid[p] << (gsh + 11)) | ((rec_key(s_a[p]) & low) << 11) | p;
  __syncthreads();
  merge_sort_u64(s_key, s_tmp, len);
  for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) {
    const unsigned long long k = s_key[q] >> 11;
    const uint32_t p = (uint32_t)(s_key[q] & 2047u);
    const uint4 x = s_a[p];
    uint32_t dst = q;
    if ((q > 0 && (s_key[q - 1] >> 11) == k) || (q + 1 < len && (s_key[q + 1] >> 11) == k)) {
      uint32_t rs = q, re = q + 1;  // the run of equal keys around q
      while (rs > 0 && (s_key[rs - 1] >> 11) == k) --rs;
      while (re < len && (s_key[re] >> 11) == k) ++re;
      dst = rs;
      for (uint32_t j = rs; j < re; ++j) {
        const uint32_t pj = (uint32_t)(s_key[j] & 2047u);
        if (pj == p) continue;
        const uint4 y = s_a[pj];
        if (y.z != x.z ? y.z < x.z : y.w != x.w ? y.w < x.w : pj < p) ++dst;
      }
    }
    s_b[dst] = x;
  }
  __syncthreads();
}

// Orders a tile range held in s_a[0, len) (len <= kSortCap) by the whole
// record into s_b[0, len). The range is made of whole groups (records with
// equal key >> gsh, contiguous and in increasing order: octree leaves after
// the dense scatter, buckets after the sparse one); inside a group the
// order is arbitrary. Every record of a group of at most kRankRange records
// is placed at its rank among the group (records smaller, or equal and
// earlier), all groups at once; a larger group is merge-sorted by the whole
// CTA, or, with merge_whole, the whole range is sorted instead as soon as
// one group is large (fewer passes when large groups are the rule): through
// packed 64-bit keys (packed_order) when s_key [len] is given and gsh <= 42,
// else merge-sorted record by record. s_gstart [len + 1], s_gid [len],
// s_list [kLargeList] and s_misc [kMiscWords] are shared scratch. Ends with
// a barrier.
static __device__ void tile_order_smem(uint4* s_a, uint4* s_b, uint32_t len, int gsh, bool merge_whole,
                                       uint32_t* s_gstart, uint32_t* s_gid, uint32_t* s_list, uint32_t* s_misc,
                                       unsigned long long* s_key = nullptr) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x;
  const uint32_t lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  // 1. group starts: one flag per record, compacted in order by a block scan
  const uint32_t per = (len + nt - 1) / nt;  // consecutive records per thread
  const uint32_t p0 = tid * per, p1 = min(len, p0 + per);
  uint32_t flags = 0, cnt = 0;
  for (uint32_t p = p0; p < p1; ++p) {
    const bool st = p == 0 || (rec_key(s_a[p]) >> gsh) != (rec_key(s_a[p - 1]) >> gsh);
    flags |= (st ? 1u : 0u) << (p - p0);
    cnt += st ? 1u : 0u;
  }
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += v;
  }
  if (lane == 31) s_misc[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < nw ? s_misc[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, wi, o);
      if ((int)lane >= o) wi += v;
    }
    if (lane < nw) s_misc[lane] = wi - w;
    if (lane == 31) s_misc[32] = wi;  // groups in the range
  }
  __syncthreads();
  const uint32_t n_groups = s_misc[32];
  {
    uint32_t g = s_misc[warp] + incl - cnt;  // groups before this thread's first record
    for (uint32_t p = p0; p < p1; ++p) {
      if (flags & (1u << (p - p0))) s_gstart[g++] = p;
      s_gid[p] = g - 1;
    }
  }
  if (tid == 0) {
    s_gstart[n_groups] = len;
    s_misc[33] = 0u;  // large groups listed
    s_misc[34] = 0u;  // some group is large
  }
  __syncthreads();
  if (merge_whole) {  // one large group: merge-sort the whole range, skip the ranking
    for (uint32_t g = tid; g < n_groups; g += nt)
      if (s_gstart[g + 1] - s_gstart[g] > kRankRange) s_misc[34] = 1u;
    __syncthreads();
    if (s_misc[34]) {
      if (s_key && gsh <= 42 && len <= 2048u) {  // packed keys (s_b is the sort's scratch until the records move)
        packed_order(s_a, s_b, len, gsh, s_gid, s_key, reinterpret_cast<unsigned long long*>(s_b));
        return;
      }
      merge_sort_smem_inplace(s_a, s_b, len);
      for (uint32_t i = tid; i < len; i += nt) s_b[i] = s_a[i];
      __syncthreads();
      return;
    }
  }
  // 2. short groups: every record at its rank; large groups listed
  for (uint32_t p = tid; p < len; p += nt) {
    const uint32_t g = s_gid[p];
    const uint32_t gs = s_gstart[g], ge = s_gstart[g + 1];
    if (ge - gs <= kRankRange) {
      // rank = records smaller than x, or equal and earlier. Keys of one
      // group agree on every bit from gsh up, so with gsh <= 32 the low key
      // word alone orders them, else the 64-bit key; the rest of a record
      // is read only on a key tie.
      const uint4 x = s_a[p];
      uint32_t r = 0;
      if (gsh <= 32) {
        for (uint32_t j = gs; j < ge; ++j) {
          const uint32_t ky = s_a[j].x;
          bool lt = ky < x.x;
          if (ky == x.x) {
            const uint4 y = s_a[j];
            lt = y.z != x.z ? y.z < x.z : y.w != x.w ? y.w < x.w : j < p;
          }
          r += lt ? 1u : 0u;
        }
      } else {
        const unsigned long long kx = rec_key(x);
        for (uint32_t j = gs; j < ge; ++j) {
          const unsigned long long ky = *reinterpret_cast<const unsigned long long*>(&s_a[j]);
          bool lt = ky < kx;
          if (ky == kx) {
            const uint4 y = s_a[j];
            lt = y.z != x.z ? y.z < x.z : y.w != x.w ? y.w < x.w : j < p;
          }
          r += lt ? 1u : 0u;
        }
      }
      s_b[gs + r] = x;
    } else if (p == gs) {
      s_list[atomicAdd(&s_misc[33], 1u)] = g;
    }
  }
  __syncthreads();
  // 3. large groups, one after the other by the whole CTA
  const uint32_t n_large = s_misc[33];
  for (uint32_t k = 0; k < n_large; ++k) {
    const uint32_t g = s_list[k];
    const uint32_t gs = s_gstart[g], c = s_gstart[g + 1] - gs;
    uint4* A = s_a + gs;
    uint4* B = s_b + gs;
    merge_sort_smem_inplace(A, B, c);  // scratch B, result in A, then into B
    for (uint32_t i = tid; i < c; i += nt) B[i] = A[i];
    __syncthreads();
  }
}

constexpr uint32_t kWarpRange = 64;  // ranges this short are sorted by one warp (two records per lane)
constexpr uint32_t kMaxLong = 40;    // ranges longer than kWarpRange starting in one chunk: at most 32

static __device__ __forceinline__ uint4 shfl_rec(const uint4& x, int src) {
  return make_uint4(__shfl_sync(0xffffffffu, x.x, src), __shfl_sync(0xffffffffu, x.y, src),
                    __shfl_sync(0xffffffffu, x.z, src), __shfl_sync(0xffffffffu, x.w, src));
}

// Rank of record x (position px) among the range: how many records are
// smaller, or equal with a smaller position. Warp-uniform loop over the
// range's records held by the lanes (positions j and j + 32).
static __device__ __forceinline__ void warp_rank_sort(uint4* g, unsigned long long s, uint32_t len) {
  const uint32_t lane = lane_id();
  const uint4 big = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
  const uint4 x0 = lane < len ? g[s + lane] : big;
  const uint4 x1 = lane + 32 < len ? g[s + lane + 32] : big;
  uint32_t r0 = 0, r1 = 0;
  const uint32_t m = len < 32 ? len : 32;
  for (uint32_t j = 0; j < m; ++j) {
    const uint4 y0 = shfl_rec(x0, (int)j);
    r0 += (rec_less(y0, x0) || (!rec_less(x0, y0) && j < lane)) ? 1u : 0u;
    r1 += (rec_less(y0, x1) || !rec_less(x1, y0)) ? 1u : 0u;  // position j < lane + 32 always
    if (j + 32 < len) {
      const uint4 y1 = shfl_rec(x1, (int)j);
      r0 += rec_less(y1, x0) ? 1u : 0u;  // position j + 32 > lane
      r1 += (rec_less(y1, x1) || (!rec_less(x1, y1) && j < lane)) ? 1u : 0u;
    }
  }
  // every lane holds its records in registers: the warp may overwrite the range
  __syncwarp();
  if (lane < len) g[s + r0] = x0;
  if (lane + 32 < len) g[s + r1] = x1;
}

// Merge sorted runs x[0, la) and y[0, lb) into out[0, la + lb) by the CTA.
static __device__ void merge_runs(const uint4* x, unsigned long long la, const uint4* y, unsigned long long lb, uint4* out) {
  const unsigned long long total = la + lb;
  const unsigned long long per = (total + blockDim.x - 1) / blockDim.x;
  const unsigned long long d0 = min(total, per * threadIdx.x);
  const unsigned long long d1 = min(total, d0 + per);
  if (d0 >= d1) return;
  // merge path: number of x elements among the first d0 outputs
  unsigned long long l = d0 > lb ? d0 - lb : 0, h = min(d0, la);
  while (l < h) {
    const unsigned long long m = (l + h) >> 1;
    if (!rec_less(y[d0 - m - 1], x[m])) l = m + 1;
    else h = m;
  }
  unsigned long long i = l, j = d0 - l;
  for (unsigned long long o = d0; o < d1; ++o) {
    const bool take_x = j >= lb || (i < la && !rec_less(y[j], x[i]));
    out[o] = take_x ? x[i++] : y[j++];
  }
}

}  // namespace fhv
