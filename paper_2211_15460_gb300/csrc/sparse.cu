// sparse.cu -- FHV_POFA with a sparse octree index (Section 3.1 "Octree
// Layout": per-octant arrays in Morton order; Section 3.2 "FHV_POFA"). The
// records come out in exactly the order of the dense compaction (pofa.cu),
// but the index holds only the occupied octants of every level, so no array
// of 8^depth entries is ever touched.
//
// GB300 layout of the work:
//  * buckets: the octants of level B = depth - 2 when 8^B is at most half
//    the records, else of level depth - 3 (level 0 for depth <= 3), are
//    counted per record (aggregated atomics into an 8^B counter array, at
//    most 537 MB at depth 11 and never above 4 bytes per two records of the
//    finer level), scanned in 4096-bucket chunks (chunk sums, one CTA over
//    the chunks, then the per-chunk offsets), and the records scattered into
//    bucket order. Two levels above the leaves a bucket of the stress scenes
//    holds about 60 records (about 230 one level further up).
//  * tile_sort: one CTA per 512 records of the bucket-ordered array orders,
//    in shared memory and by the whole record, exactly the buckets that
//    start in its tile: the range between the first bucket boundary at or
//    after each end of the tile (found from the record there and its
//    bucket's offset), so the tiles' ranges partition the array. A bucket
//    of at most 64 records is ordered by ranking every record among its
//    bucket, all such buckets at once; when a larger one is present the
//    whole range is sorted through packed 64-bit keys (bucket rank, key
//    bits below the bucket, position; warp sorts of 32 in registers, then
//    merge-path passes) and the records moved once. Ranges above 1024
//    records are cut into runs of whole buckets; buckets above 1024
//    records are listed.
//  * bucket_sort: for the listed buckets only, persistent CTAs histogram
//    the bucket's records by leaf (up to 512 bins in shared memory), scan,
//    scatter them into leaf order straight into the output, then sort each
//    leaf's range (one warp per range of up to 64 records, the CTA in
//    shared memory up to 4096, longer ranges listed for a merge kernel).
//  * index: one pass over 4096-record tiles counts, for every level, the
//    records that start a new octant (the first level whose Morton prefix
//    differs from the previous record's); one CTA per level scans those
//    counts, one thread turns the level totals into level bases; a second
//    pass writes (octant, offset) at each start, and a last pass sets each
//    entry's count from the next entry's offset.
#include "kernels.h"
#include "sort.cuh"

namespace fhv {

namespace {

constexpr int kBucketChunk = 4096;   // buckets per offset-scan CTA
constexpr uint32_t kTileRecords = 512;  // records per tile_sort CTA
constexpr uint32_t kTileCap = 2 * kTileRecords;  // largest run of whole buckets a tile sorts at once
constexpr uint32_t kBucketLeaves = 512;  // bins of a listed bucket's leaf histogram (8^(depth - B) <= 64 used)
constexpr int kIndexTile = 4096;     // records per index CTA (256 threads x 16)
constexpr int kIndexThreads = 256;
constexpr int kSortThreads = 512;
constexpr int kMaxLevels = 12;       // levels 0..11
constexpr uint32_t kLongList = 256;  // leaf ranges longer than a warp's listed per bucket

__device__ __forceinline__ unsigned long long n_records(const SparseArgs& a) {
  unsigned long long n = a.n_max;
  if (a.d_n) {
    const unsigned long long c = *a.d_n;
    n = c < n ? c : n;
  }
  return n;
}

__device__ __forceinline__ unsigned long long bucket_of(const SparseArgs& a, unsigned long long key) {
  return a.B == 0 ? 0ull : key >> (63 - 3 * a.B);
}

// ------------------------------------------------------------- buckets

__global__ void __launch_bounds__(256) bucket_count_kernel(SparseArgs a) {
  const unsigned long long n = n_records(a);
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n; base += step) {
    const unsigned long long i = base + threadIdx.x;
    const bool valid = i < n;
    const uint32_t active = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const unsigned long long b = bucket_of(a, a.in[i].key);
      const uint32_t peers = __match_any_sync(active, b);
      if (lane_id() == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&a.bcnt[b], (uint32_t)__popc(peers));
    }
  }
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024);
// returns the prefix, *total gets the block's sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp, T* total) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T x = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += x;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const T w = lane < nw ? s_warp[lane] : (T)0;
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T x = __shfl_up_sync(0xffffffffu, wi, o);
      if ((int)lane >= o) wi += x;
    }
    if (lane < nw) s_warp[lane] = wi - w;
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  const T out = s_warp[warp] + (incl - v);
  *total = s_warp[32];
  __syncthreads();
  return out;
}

// Per chunk of 4096 buckets: the sum of their counts.
__global__ void __launch_bounds__(256) bucket_chunk_kernel(SparseArgs a) {
  __shared__ uint32_t s_a[33];
  const unsigned long long c0 = (unsigned long long)blockIdx.x * kBucketChunk;
  uint32_t sum = 0;
  for (uint32_t k = threadIdx.x; k < kBucketChunk; k += blockDim.x) {
    const unsigned long long b = c0 + k;
    if (b < a.n_buckets) sum += a.bcnt[b];
  }
  uint32_t ts;
  block_exclusive_scan(sum, s_a, &ts);
  if (threadIdx.x == 0) a.chunk_sum[blockIdx.x] = ts;
}

// One CTA: exclusive scan of the chunk sums (in place).
__global__ void __launch_bounds__(1024) bucket_chunk_scan_kernel(SparseArgs a, unsigned n_chunks) {
  __shared__ unsigned long long s_a[33];
  const unsigned per = (n_chunks + blockDim.x - 1) / blockDim.x;
  const unsigned b = threadIdx.x * per, e = min(n_chunks, b + per);
  unsigned long long sum = 0;
  for (unsigned i = b; i < e; ++i) sum += a.chunk_sum[i];
  unsigned long long ts;
  unsigned long long ps = block_exclusive_scan(sum, s_a, &ts);
  for (unsigned i = b; i < e; ++i) {
    const uint32_t cs = a.chunk_sum[i];
    a.chunk_sum[i] = (uint32_t)ps;
    ps += cs;
  }
}

// Per chunk: bucket offsets and scatter cursors.
__global__ void __launch_bounds__(256) bucket_offsets_kernel(SparseArgs a) {
  __shared__ uint32_t s_a[33];
  const unsigned long long c0 = (unsigned long long)blockIdx.x * kBucketChunk;
  constexpr int per = kBucketChunk / 256;  // 16 consecutive buckets per thread
  const unsigned long long b0 = c0 + (unsigned long long)threadIdx.x * per;
  uint32_t c[per];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    c[k] = b0 + k < a.n_buckets ? a.bcnt[b0 + k] : 0u;
    sum += c[k];
  }
  uint32_t ts;
  uint32_t ps = block_exclusive_scan(sum, s_a, &ts) + a.chunk_sum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < per; ++k) {
    if (b0 + k < a.n_buckets) {
      a.boff[b0 + k] = ps;
      a.bcur[b0 + k] = ps;
      ps += c[k];
    }
  }
}

__global__ void __launch_bounds__(256) bucket_scatter_kernel(SparseArgs a) {
  const unsigned long long n = n_records(a);
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n; base += step) {
    const unsigned long long i = base + threadIdx.x;
    const bool valid = i < n;
    const uint32_t active = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const uint4 r = reinterpret_cast<const uint4*>(a.in)[i];
      const unsigned long long key = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
      const unsigned long long b = bucket_of(a, key);
      const uint32_t peers = __match_any_sync(active, b);
      const uint32_t leader = __ffs(peers) - 1;
      uint32_t pos = 0;
      if (lane_id() == leader) pos = atomicAdd(&a.bcur[b], (uint32_t)__popc(peers));
      pos = __shfl_sync(peers, pos, leader) + __popc(peers & lanemask_lt());
      reinterpret_cast<uint4*>(a.scratch)[pos] = r;
    }
  }
}

// ------------------------------------------------------ order inside a bucket

__device__ __forceinline__ unsigned long long scratch_key(const SparseArgs& a, unsigned long long i) {
  return reinterpret_cast<const unsigned long long*>(a.scratch)[2 * i];
}

// First bucket boundary at or after record x of the bucket-ordered array (n if none).
__device__ __forceinline__ unsigned long long next_boundary(const SparseArgs& a, unsigned long long x,
                                                            unsigned long long n) {
  if (x >= n) return n;
  const unsigned long long b = bucket_of(a, scratch_key(a, x));
  const unsigned long long start = a.boff[b];
  return start == x ? x : start + a.bcnt[b];
}

// One CTA per tile of kTileRecords bucket-ordered records: the buckets that
// start in the tile, sorted by the whole record into the output.
constexpr int kTileThreads = 256;
constexpr int kTileCtas = 4;  // CTAs per SM the shared memory allows
constexpr int kTileDyn = kTileCap * (2 * 16 + 8);  // records in and out, packed keys (bytes)

// Whole buckets src[lo, hi) (at most kTileCap records) ordered into dst
// through shared memory (tile_order_smem with buckets as groups: small ones
// ranked; with a large one, the range merge-sorted). Ends with a barrier.
__device__ __forceinline__ void order_buckets(const SparseArgs& a, const uint4* src, uint4* dst, unsigned long long lo,
                                              unsigned long long hi, uint4* s_a, uint4* s_b, uint32_t* s_gstart,
                                              uint32_t* s_gid, uint32_t* s_list, uint32_t* s_misc,
                                              unsigned long long* s_key) {
  const uint32_t len = (uint32_t)(hi - lo);
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) s_a[i] = src[lo + i];
  __syncthreads();
  // with a large bucket the whole range is sorted, through packed 64-bit
  // keys at depth 10 and deeper (per large bucket, whether by leaf counts or
  // by merges, was slower at depth 11: 41.8 and 43.4 against 34.3 ms)
  tile_order_smem(s_a, s_b, len, a.B == 0 ? 63 : 63 - 3 * a.B, true, s_gstart, s_gid, s_list, s_misc, s_key);
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) dst[lo + i] = s_b[i];
  __syncthreads();
}

__global__ void __launch_bounds__(kTileThreads, kTileCtas) tile_sort_kernel(SparseArgs a) {
  extern __shared__ __align__(16) uint4 s_rec[];  // 2 x kTileCap records, then kTileCap packed keys
  uint4* s_alt = s_rec + kTileCap;
  unsigned long long* s_key = reinterpret_cast<unsigned long long*>(s_rec + 2 * kTileCap);
  __shared__ uint32_t s_start[kTileRecords + 1];  // bucket starts in the tile, relative to R0, then R1 - R0
  __shared__ uint32_t s_run[2 * kTileRecords];    // runs: [first, end) indices into s_start
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_nruns;
  __shared__ uint32_t s_gstart[kTileCap + 1], s_gid[kTileCap];
  __shared__ uint32_t s_list[kLargeList], s_misc[kMiscWords];
  const unsigned long long n = n_records(a);
  const unsigned long long r0 = (unsigned long long)blockIdx.x * kTileRecords;
  if (r0 >= n) return;
  const unsigned long long r1 = min(n, r0 + kTileRecords);
  const unsigned long long R0 = next_boundary(a, r0, n);
  const unsigned long long R1 = next_boundary(a, r1, n);
  if (R0 >= R1) return;  // no bucket starts in this tile
  const uint4* in = reinterpret_cast<const uint4*>(a.scratch);
  uint4* out = reinterpret_cast<uint4*>(a.out);
  if (R1 - R0 <= (unsigned long long)kTileCap) {
    order_buckets(a, in, out, R0, R1, s_rec, s_alt, s_gstart, s_gid, s_list, s_misc, s_key);
    return;
  }
  // Longer: a bucket above kTileCap records starts here, or small buckets
  // plus a long last one. Find every bucket start in [R0, r1) in parallel
  // (record x starts its bucket when the bucket's offset is x), then cut
  // runs of whole buckets of at most kTileCap records; larger buckets are
  // listed for bucket_sort.
  constexpr uint32_t per = kTileRecords / kTileThreads;  // consecutive records per thread
  const unsigned long long x0 = R0 + (unsigned long long)threadIdx.x * per;
  uint32_t flags = 0, cnt = 0;
  for (uint32_t j = 0; j < per; ++j) {
    const unsigned long long x = x0 + j;
    if (x < r1 && a.boff[bucket_of(a, scratch_key(a, x))] == x) {
      flags |= 1u << j;
      ++cnt;
    }
  }
  uint32_t tot;
  uint32_t pos = block_exclusive_scan(cnt, s_warp, &tot);
  for (uint32_t j = 0; j < per; ++j)
    if (flags & (1u << j)) s_start[pos++] = (uint32_t)(x0 + j - R0);
  if (threadIdx.x == 0) s_start[tot] = (uint32_t)(R1 - R0);
  __syncthreads();
  if (threadIdx.x == 0) {  // runs, from shared memory only
    uint32_t nr = 0, k = 0;
    while (k < tot) {
      const uint32_t size = s_start[k + 1] - s_start[k];
      if (size > kTileCap) {  // a large bucket alone: listed
        const unsigned long long b = bucket_of(a, scratch_key(a, R0 + s_start[k]));
        const unsigned long long slot = atomicAdd(&a.hdr->n_huge_buckets, 1ull);
        a.blist[slot] = (uint32_t)b;
        ++k;
        continue;
      }
      uint32_t e = k + 1;
      while (e < tot && s_start[e + 1] - s_start[k] <= kTileCap) ++e;
      s_run[2 * nr] = k;
      s_run[2 * nr + 1] = e;
      ++nr;
      k = e;
    }
    s_nruns = nr;
  }
  __syncthreads();
  const uint32_t nr = s_nruns;
  for (uint32_t r = 0; r < nr; ++r)
    order_buckets(a, in, out, R0 + s_start[s_run[2 * r]], R0 + s_start[s_run[2 * r + 1]], s_rec, s_alt, s_gstart,
                  s_gid, s_list, s_misc, s_key);
}

// Persistent: each CTA takes listed (large) buckets by ticket and leaves
// every record of the bucket at its final position in the output.
__global__ void __launch_bounds__(kSortThreads) bucket_sort_kernel(SparseArgs a) {
  extern __shared__ __align__(16) uint4 s_rec[];  // kSortCap records
  __shared__ uint32_t s_hist[kBucketLeaves];      // per-leaf counts, then cursors
  __shared__ uint32_t s_start[kBucketLeaves + 1]; // leaf range starts, relative to the bucket
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_long[kLongList];  // leaves whose range exceeds a warp's
  __shared__ uint32_t s_nlong;
  __shared__ unsigned long long s_ticket;
  const uint32_t n_huge = (uint32_t)a.hdr->n_huge_buckets;  // listed by tile_sort
  const uint32_t nl = 1u << a.leaf_bits;
  const int sh = 63 - 3 * a.depth;
  const uint4* in = reinterpret_cast<const uint4*>(a.scratch);
  uint4* out = reinterpret_cast<uint4*>(a.out);
  const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  constexpr uint32_t per = kBucketLeaves / kSortThreads > 0 ? kBucketLeaves / kSortThreads : 1;  // bins per thread
  while (true) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(&a.hdr->ticket[1], 1ull);
    __syncthreads();
    const unsigned long long t = s_ticket;
    if (t >= n_huge) break;
    const uint32_t b = a.blist[t];
    const unsigned long long lo = a.boff[b];
    const uint32_t len = a.bcnt[b];
    for (uint32_t k = threadIdx.x; k < nl; k += blockDim.x) s_hist[k] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
      const unsigned long long key = (unsigned long long)in[lo + i].x | ((unsigned long long)in[lo + i].y << 32);
      atomicAdd(&s_hist[(uint32_t)(key >> sh) & (nl - 1u)], 1u);
    }
    __syncthreads();
    // exclusive scan of the bins: thread t owns bins [per t, per t + per)
    uint32_t v[per], sum = 0;
#pragma unroll
    for (uint32_t k = 0; k < per; ++k) {
      const uint32_t bin = threadIdx.x * per + k;
      v[k] = bin < nl ? s_hist[bin] : 0u;
      sum += v[k];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(sum, s_warp, &tot);
#pragma unroll
    for (uint32_t k = 0; k < per; ++k) {
      const uint32_t bin = threadIdx.x * per + k;
      if (bin < nl) {
        s_start[bin] = run;
        s_hist[bin] = run;
      }
      run += v[k];
    }
    if (threadIdx.x == 0) {
      s_start[nl] = len;
      s_nlong = 0u;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
      const uint4 r = in[lo + i];
      const unsigned long long key = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
      const uint32_t pos = atomicAdd(&s_hist[(uint32_t)(key >> sh) & (nl - 1u)], 1u);
      out[lo + pos] = r;
    }
    __syncthreads();  // the scattered records are visible to the whole CTA
    for (uint32_t l = warp; l < nl; l += nwarps) {
      const uint32_t c = s_start[l + 1] - s_start[l];
      if (c >= 2u && c <= kWarpRange) warp_rank_sort(out, lo + s_start[l], c);
      if (c > kWarpRange && lane_id() == 0) {
        const uint32_t k = atomicAdd(&s_nlong, 1u);
        if (k < kLongList) s_long[k] = l;
      }
    }
    __syncthreads();
    // longer ranges one after the other by the whole CTA: from the list, or
    // (list overflowed) by a CTA-uniform walk over every leaf
    const uint32_t nlong = s_nlong;
    const uint32_t walk = nlong <= kLongList ? nlong : nl;
    for (uint32_t k = 0; k < walk; ++k) {
      const uint32_t l = nlong <= kLongList ? s_long[k] : k;
      const uint32_t c = s_start[l + 1] - s_start[l];
      if (c <= kWarpRange) continue;
      if (c <= (uint32_t)kSortCap) {
        sort_range_smem(out, lo + s_start[l], lo + s_start[l] + c, s_rec);
      } else if (threadIdx.x == 0) {
        const uint32_t slot = atomicAdd(&a.hdr->huge_count, 1u);
        if (slot < a.huge_max) {
          a.huge[2 * slot] = lo + s_start[l];
          a.huge[2 * slot + 1] = c;
        } else {
          set_status(&a.hdr->status, FHV_DEV_RANGE);
        }
      }
    }
    __syncthreads();
  }
}

// Leaf ranges longer than kSortCap: one CTA each, tiles sorted in shared
// memory, then pairwise merges between the range and its scratch copy.
__global__ void __launch_bounds__(kSortThreads) huge_range_sort_kernel(SparseArgs a) {
  extern __shared__ __align__(16) uint4 s_rec[];
  const uint32_t count = min((unsigned long long)a.hdr->huge_count, a.huge_max);
  uint4* g = reinterpret_cast<uint4*>(a.out);
  uint4* scratch = reinterpret_cast<uint4*>(a.scratch);  // the bucket order is no longer needed
  for (uint32_t slot = blockIdx.x; slot < count; slot += gridDim.x) {
    const unsigned long long s = a.huge[2 * slot], len = a.huge[2 * slot + 1];
    for (unsigned long long b = 0; b < len; b += kSortCap) sort_range_smem(g, s + b, s + min(len, b + kSortCap), s_rec);
    uint4* src = g + s;
    uint4* dst = scratch + s;
    for (unsigned long long width = kSortCap; width < len; width <<= 1) {
      for (unsigned long long p = 0; p < len; p += 2 * width) {
        const unsigned long long la = min(width, len - p);
        const unsigned long long lb = p + width < len ? min(width, len - p - width) : 0ull;
        merge_runs(src + p, la, src + p + la, lb, dst + p);
      }
      __syncthreads();
      uint4* tmp = src;
      src = dst;
      dst = tmp;
    }
    if (src != g + s) {
      for (unsigned long long i = threadIdx.x; i < len; i += blockDim.x) g[s + i] = src[i];
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------- index

// The coarsest level at which record i starts a new octant: 0 for the
// first record; else the first level whose Morton prefix (the top 3l bits
// of the 63-bit code) differs from the previous record's; depth + 1 when
// the two share their leaf.
__device__ __forceinline__ int start_level(unsigned long long key, unsigned long long prev, bool first, int depth) {
  if (first) return 0;
  const unsigned long long x = key ^ prev;
  if (x == 0ull) return depth + 1;
  const int h = 63 - __clzll(x);  // highest differing bit, 0..62
  const int l = (65 - h) / 3;     // bit h lies in the prefix of levels >= l
  return l <= depth ? l : depth + 1;
}

// Per thread: records [16 t, 16 t + 16) of the tile; per level, how many of
// them start an octant.
__device__ __forceinline__ void tile_level_counts(const SparseArgs& a, unsigned long long n, unsigned long long r0,
                                                  uint32_t* cnt, int* lv) {
  const unsigned long long* keys = reinterpret_cast<const unsigned long long*>(a.out);
  for (int l = 0; l < kMaxLevels; ++l) cnt[l] = 0u;
  unsigned long long prev = r0 > 0 && r0 < n ? keys[2 * (r0 - 1)] : 0ull;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const unsigned long long i = r0 + k;
    int s = a.depth + 1;
    if (i < n) {
      const unsigned long long key = keys[2 * i];
      s = start_level(key, prev, i == 0, a.depth);
      prev = key;
    }
    lv[k] = s;
#pragma unroll
    for (int l = 0; l < kMaxLevels; ++l) cnt[l] += (s <= l) ? 1u : 0u;
  }
}

__global__ void __launch_bounds__(kIndexThreads) index_count_kernel(SparseArgs a) {
  __shared__ uint32_t s_tot[kIndexThreads / 32][kMaxLevels];
  const unsigned long long n = n_records(a);
  const unsigned long long tile = blockIdx.x;
  const unsigned long long r0 = tile * kIndexTile + 16ull * threadIdx.x;
  uint32_t cnt[kMaxLevels];
  int lv[16];
  tile_level_counts(a, n, r0, cnt, lv);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l) {
    uint32_t x = cnt[l];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_tot[warp][l] = x;
  }
  __syncthreads();
  if (threadIdx.x <= (unsigned)a.depth) {
    uint32_t t = 0;
    for (int w = 0; w < kIndexThreads / 32; ++w) t += s_tot[w][threadIdx.x];
    a.tile_lvl[(unsigned long long)threadIdx.x * a.n_tiles + tile] = t;
  }
}

// One CTA per level: exclusive scan of that level's tile counts (in place)
// and the level's total.
__global__ void __launch_bounds__(1024) index_scan_kernel(SparseArgs a) {
  __shared__ unsigned long long s_w[33];
  const int l = blockIdx.x;
  const unsigned long long nt = a.n_tiles;
  const unsigned long long per = (nt + blockDim.x - 1) / blockDim.x;
  uint32_t* t = a.tile_lvl + (unsigned long long)l * nt;
  const unsigned long long b = threadIdx.x * per, e = min(nt, b + per);
  unsigned long long sum = 0;
  for (unsigned long long i = b; i < e; ++i) sum += t[i];
  unsigned long long tot;
  unsigned long long run = block_exclusive_scan(sum, s_w, &tot);
  for (unsigned long long i = b; i < e; ++i) {
    const uint32_t c = t[i];
    t[i] = (uint32_t)run;
    run += c;
  }
  if (threadIdx.x == 0) a.level_total[l] = tot;
}

// Level bases from the level totals; the index overflow check.
__global__ void index_base_kernel(SparseArgs a) {
  unsigned long long base = 0;
  for (int l = 0; l <= a.depth; ++l) {
    a.level_base[l] = base;
    base += a.level_total[l];
  }
  a.level_base[a.depth + 1] = base;
  if (base > a.index_capacity) set_status(&a.hdr->status, FHV_DEV_INDEX_OVERFLOW);
}

__global__ void __launch_bounds__(kIndexThreads) index_write_kernel(SparseArgs a) {
  __shared__ uint32_t s_w[kMaxLevels][kIndexThreads / 32];
  const unsigned long long n = n_records(a);
  const unsigned long long tile = blockIdx.x;
  const unsigned long long r0 = tile * kIndexTile + 16ull * threadIdx.x;
  const unsigned long long* keys = reinterpret_cast<const unsigned long long*>(a.out);
  uint32_t cnt[kMaxLevels];
  int lv[16];
  tile_level_counts(a, n, r0, cnt, lv);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t excl[kMaxLevels];
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l) {
    uint32_t incl = cnt[l];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)lane >= o) incl += x;
    }
    excl[l] = incl - cnt[l];
    if (lane == 31) s_w[l][warp] = incl;
  }
  __syncthreads();
  unsigned long long pos[kMaxLevels];
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l) {
    uint32_t before = 0;
    for (uint32_t w = 0; w < warp; ++w) before += s_w[l][w];
    pos[l] = l <= a.depth ? a.level_base[l] + a.tile_lvl[(unsigned long long)l * a.n_tiles + tile] + before + excl[l]
                          : 0ull;
  }
  fhv_octant_entry* idx = a.index;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const unsigned long long i = r0 + k;
    if (lv[k] > a.depth) continue;
    const unsigned long long key = keys[2 * i];
#pragma unroll
    for (int l = 0; l < kMaxLevels; ++l) {
      if (l < lv[k] || l > a.depth) continue;
      const unsigned long long p = pos[l]++;
      if (p < a.index_capacity) {
        const unsigned long long oct = l == 0 ? 0ull : key >> (63 - 3 * l);
        *reinterpret_cast<uint4*>(idx + p) = make_uint4((uint32_t)oct, (uint32_t)(oct >> 32), (uint32_t)i, 0u);
      }
    }
  }
}

// cnt of entry k = the next entry's offset (same level) - its own; the
// last entry of a level ends at n.
__global__ void __launch_bounds__(256) index_cnt_kernel(SparseArgs a) {
  __shared__ unsigned long long s_base[kMaxLevels + 1];
  const unsigned long long n = n_records(a);
  if (threadIdx.x <= (unsigned)a.depth + 1) s_base[threadIdx.x] = a.level_base[threadIdx.x];
  __syncthreads();
  const unsigned long long total = min(s_base[a.depth + 1], a.index_capacity);
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += step) {
    int l = 0;
    while (l < a.depth && s_base[l + 1] <= k) ++l;
    uint32_t next = (uint32_t)n;
    if (k + 1 < s_base[l + 1]) {
      if (k + 1 >= a.index_capacity) continue;  // its successor was not written
      next = a.index[k + 1].off;
    }
    a.index[k].cnt = next - a.index[k].off;
  }
}

}  // namespace

SparseWs sparse_ws(int depth, unsigned long long n_max) {
  SparseWs w;
  // buckets two levels above the leaves when that level has no more than
  // one bucket per two records (else its scans outweigh the shorter sorts),
  // three levels above otherwise
  w.B = depth > 3 ? depth - 3 : 0;
  if (depth > 2 && (1ull << (3 * (depth - 2))) * 2ull <= n_max) w.B = depth - 2;
  w.n_buckets = 1ull << (3 * w.B);
  w.n_chunks = (w.n_buckets + kBucketChunk - 1) / kBucketChunk;
  w.n_tiles = (n_max + kIndexTile - 1) / kIndexTile;
  if (w.n_tiles == 0) w.n_tiles = 1;
  w.huge_max = n_max / (kSortCap + 1) + 1;
  unsigned long long o = kHeaderBytes;
  w.off_bcnt = o;
  o += round256(w.n_buckets * 4ull);
  w.off_boff = o;
  o += round256(w.n_buckets * 4ull);
  w.off_bcur = o;
  o += round256(w.n_buckets * 4ull);
  w.off_blist = o;
  o += round256(w.n_buckets * 4ull);
  w.off_chunk = o;  // chunk sums, then the level totals
  o += round256(w.n_chunks * 4ull) + round256(16ull * 8ull);
  w.off_tiles = o;
  o += round256(w.n_tiles * (unsigned long long)(depth + 1) * 4ull);
  w.off_huge = o;
  o += round256(w.huge_max * 16ull);
  w.off_scratch = o;
  o += round256(n_max * 16ull);
  w.total = o;
  return w;
}

cudaError_t launch_compact_sparse(const SparseArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(bucket_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortCap * 16);
    cudaFuncSetAttribute(tile_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileDyn);
    cudaFuncSetAttribute(huge_range_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortCap * 16);
    attr = true;
  }
  const int grid_rec = sm_count() * 8;
  if (a.n_max > 0) {
    timing_begin("bucket_count", s);
    bucket_count_kernel<<<grid_rec, 256, 0, s>>>(a);
    timing_end("bucket_count", s);
  }
  const unsigned n_chunks = (unsigned)((a.n_buckets + kBucketChunk - 1) / kBucketChunk);
  timing_begin("bucket_chunk", s);
  bucket_chunk_kernel<<<n_chunks, 256, 0, s>>>(a);
  timing_end("bucket_chunk", s);
  timing_begin("bucket_chunk_scan", s);
  bucket_chunk_scan_kernel<<<1, 1024, 0, s>>>(a, n_chunks);
  timing_end("bucket_chunk_scan", s);
  timing_begin("bucket_offsets", s);
  bucket_offsets_kernel<<<n_chunks, 256, 0, s>>>(a);
  timing_end("bucket_offsets", s);
  if (a.n_max > 0) {
    timing_begin("bucket_scatter", s);
    bucket_scatter_kernel<<<grid_rec, 256, 0, s>>>(a);
    timing_end("bucket_scatter", s);
    timing_begin("tile_sort", s);
    tile_sort_kernel<<<(unsigned)((a.n_max + kTileRecords - 1) / kTileRecords), kTileThreads, kTileDyn, s>>>(a);
    timing_end("tile_sort", s);
    timing_begin("bucket_sort", s);
    bucket_sort_kernel<<<sm_count() * 2, kSortThreads, kSortCap * 16, s>>>(a);
    timing_end("bucket_sort", s);
    const unsigned long long hg = a.huge_max < 1024ull ? a.huge_max : 1024ull;
    timing_begin("huge_range_sort", s);
    huge_range_sort_kernel<<<(unsigned)hg, kSortThreads, kSortCap * 16, s>>>(a);
    timing_end("huge_range_sort", s);
  }
  timing_begin("index_count", s);
  index_count_kernel<<<(unsigned)a.n_tiles, kIndexThreads, 0, s>>>(a);
  timing_end("index_count", s);
  timing_begin("index_scan", s);
  index_scan_kernel<<<a.depth + 1, 1024, 0, s>>>(a);
  timing_end("index_scan", s);
  timing_begin("index_base", s);
  index_base_kernel<<<1, 1, 0, s>>>(a);
  timing_end("index_base", s);
  timing_begin("index_write", s);
  index_write_kernel<<<(unsigned)a.n_tiles, kIndexThreads, 0, s>>>(a);
  timing_end("index_write", s);
  timing_begin("index_cnt", s);
  index_cnt_kernel<<<sm_count() * 8, 256, 0, s>>>(a);
  timing_end("index_cnt", s);
  return cudaGetLastError();
}

}  // namespace fhv
