// leaf_index.cu -- the sparse variant of a POFA's octree index: the leaf
// octants that hold records, each with its offset and count (Section 3.1's
// per-octant arrays, kept for the occupied leaves only).
//
// The records are sorted by key, so a leaf's records are one run and a run
// starts where the leaf (key >> (63 - 3 depth)) differs from the previous
// record's. Four streaming passes over the keys:
//  * tile_count: per tile of 4096 records, the number of run starts;
//  * tile_scan: one CTA turns the tile counts into exclusive offsets and
//    writes the total m;
//  * starts: each tile writes its runs' leaf ids and start offsets at its
//    offset, in order (block scan of the start flags);
//  * counts: cnt[j] = off[j + 1] - off[j], with off[m] = n.
#include "kernels.h"

namespace fhv {

namespace {

constexpr int kLeafIdxTile = 4096;
constexpr int kLeafIdxThreads = 256;  // 16 records per thread

__device__ __forceinline__ unsigned long long leaf_n(const LeafIndexArgs& a) {
  unsigned long long n = a.n_max;
  if (a.d_n) {
    const unsigned long long c = *a.d_n;
    n = c < n ? c : n;
  }
  return n;
}

__device__ __forceinline__ bool run_start(const LeafIndexArgs& a, unsigned long long i, int sh) {
  const unsigned long long* keys = reinterpret_cast<const unsigned long long*>(a.pofa);
  return i == 0 || (keys[2 * i] >> sh) != (keys[2 * (i - 1)] >> sh);
}

// Block-wide exclusive scan of one value per thread; returns the total.
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t& excl, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t before = 0, total = 0;
  for (int w = 0; w < kLeafIdxThreads / 32; ++w) {
    if (w < warp) before += s_warp[w];
    total += s_warp[w];
  }
  excl = before + incl - v;
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kLeafIdxThreads) leaf_tile_count_kernel(LeafIndexArgs a) {
  __shared__ uint32_t s_warp[kLeafIdxThreads / 32];
  const unsigned long long n = leaf_n(a);
  const int sh = 63 - 3 * a.depth;
  const unsigned long long lo = (unsigned long long)blockIdx.x * kLeafIdxTile;
  uint32_t c = 0;
  for (int k = 0; k < kLeafIdxTile / kLeafIdxThreads; ++k) {
    const unsigned long long i = lo + (unsigned long long)k * kLeafIdxThreads + threadIdx.x;
    if (i < n && run_start(a, i, sh)) ++c;
  }
  uint32_t excl;
  const uint32_t total = block_scan(c, excl, s_warp);
  if (threadIdx.x == 0) a.tile_sum[blockIdx.x] = total;
}

// One CTA of 1024 threads: exclusive offsets of the tile counts, total m.
__global__ void __launch_bounds__(1024) leaf_tile_scan_kernel(LeafIndexArgs a, unsigned long long tiles) {
  __shared__ unsigned long long s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long per = (tiles + blockDim.x - 1) / blockDim.x;
  const unsigned long long b = (unsigned long long)tid * per, e = min(tiles, b + per);
  unsigned long long sum = 0;
  for (unsigned long long i = b; i < e; ++i) sum += a.tile_sum[i];
  unsigned long long incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long w = s_warp[lane];
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) *a.d_m = wi;
  }
  __syncthreads();
  unsigned long long run = s_warp[warp] + (incl - sum);
  for (unsigned long long i = b; i < e; ++i) {
    const unsigned long long t = a.tile_sum[i];
    a.tile_off[i] = run;
    run += t;
  }
}

// Thread t owns records lo + 16 t .. lo + 16 t + 15, so that the block scan
// of per-thread start counts keeps the runs in record order.
__global__ void __launch_bounds__(kLeafIdxThreads) leaf_starts_kernel(LeafIndexArgs a) {
  __shared__ uint32_t s_warp[kLeafIdxThreads / 32];
  constexpr int kPer = kLeafIdxTile / kLeafIdxThreads;
  const unsigned long long n = leaf_n(a);
  const int sh = 63 - 3 * a.depth;
  const unsigned long long lo = (unsigned long long)blockIdx.x * kLeafIdxTile + (unsigned long long)threadIdx.x * kPer;
  uint32_t c = 0;
  for (int k = 0; k < kPer; ++k)
    if (lo + k < n && run_start(a, lo + k, sh)) ++c;
  uint32_t excl;
  block_scan(c, excl, s_warp);
  unsigned long long j = a.tile_off[blockIdx.x] + excl;
  const unsigned long long* keys = reinterpret_cast<const unsigned long long*>(a.pofa);
  for (int k = 0; k < kPer; ++k) {
    const unsigned long long i = lo + k;
    if (i < n && run_start(a, i, sh)) {
      a.leaf[j] = keys[2 * i] >> sh;
      a.off[j] = (uint32_t)i;
      ++j;
    }
  }
}

__global__ void __launch_bounds__(256) leaf_counts_kernel(LeafIndexArgs a) {
  const unsigned long long n = leaf_n(a);
  const unsigned long long m = *a.d_m;
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += step)
    a.cnt[j] = (uint32_t)((j + 1 < m ? (unsigned long long)a.off[j + 1] : n) - a.off[j]);
}

}  // namespace

unsigned long long leaf_index_tiles(unsigned long long n_max) {
  return (n_max + kLeafIdxTile - 1) / kLeafIdxTile;
}

cudaError_t launch_leaf_index(const LeafIndexArgs& a, cudaStream_t s) {
  const unsigned long long tiles = leaf_index_tiles(a.n_max);
  if (tiles == 0) {
    // no records: m = 0
    return cudaMemsetAsync(a.d_m, 0, sizeof(unsigned long long), s);
  }
  timing_begin("leaf_index", s);
  leaf_tile_count_kernel<<<(unsigned)tiles, kLeafIdxThreads, 0, s>>>(a);
  leaf_tile_scan_kernel<<<1, 1024, 0, s>>>(a, tiles);
  leaf_starts_kernel<<<(unsigned)tiles, kLeafIdxThreads, 0, s>>>(a);
  leaf_counts_kernel<<<sm_count() * 8, 256, 0, s>>>(a);
  timing_end("leaf_index", s);
  return cudaGetLastError();
}

}  // namespace fhv
