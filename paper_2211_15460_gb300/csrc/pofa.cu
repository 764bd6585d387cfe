// pofa.cu -- FHV_POFA compaction (Section 3.1 "Octree Layout", Section 3.2
// "FHV_POFA", Fig. 6): per-leaf fragment counts, offsets by an exclusive
// scan in Morton order, scatter into per-octant ranges, and the canonical
// order inside each octant.
//
// GB300 layout of the work:
//  * mark / count / scatter: grid-stride over the 16-byte records; lanes
//    holding the same leaf are grouped with __match_any_sync so one atomic
//    per group sets the leaf's occupancy bit (mark; the first setter zeroes
//    the leaf's counter, so the dense counter array is never cleared),
//    updates the counter (count), or reserves the group's slots (scatter,
//    using the leaf offsets themselves as cursors).
//  * offsets: count also counts per level-T octant (T = depth - 4, the
//    parents of 4096-leaf tiles). level_scan turns level T's counts into
//    offsets (bulk copies in and out, tiles chained by decoupled look-back)
//    and writes levels T-1..T-4; reduce_levels continues above. leaf_scan
//    then handles every 4096-leaf tile independently from its parent's
//    offset: it reads the tile's occupancy bitmap, gathers the occupied
//    leaves' counts, and writes every leaf's offset and count with 16-byte
//    stores (each thread its own 64 bytes), plus levels depth-1..T+1. No
//    leaf tile waits for another; the dense leaf arrays are written once
//    and never read.
//  * seg_sort: one CTA per 1024 records (two per SM) restores the offsets
//    used as cursors and orders every octant range that starts in its
//    chunk. When those ranges fit in shared memory together (up to 2048
//    records: the
//    common case in deep octrees) they are loaded once, every record of a
//    range of up to 64 is ranked against its range and stored at its rank,
//    longer ranges are merge-sorted, and the chunk is stored once.
//    Otherwise: ranges of up to 64 records one warp each (rank sort through
//    shuffles), longer ones one at a time by the CTA in shared memory
//    (bitonic network on 128-bit keys); ranges longer than the
//    shared-memory tile go to a list that huge_sort merges in global memory.
// The bitmap clear, the scan and the order stages are also driven by the
// direct POFA build (capture.cu), whose raster passes replace the
// record-reading mark / count / scatter.
#include "kernels.h"
#include "lookback.cuh"
#include "sort.cuh"

namespace fhv {

__device__ __forceinline__ unsigned long long n_records(const CompactArgs& a) {
  unsigned long long n = a.n_max;
  if (a.d_n) {
    unsigned long long c = *a.d_n;
    n = c < n ? c : n;
  }
  return n;
}

// ------------------------------------------------------------ count / scatter

// The leaves' occupancy bitmap (bitmap_word) lives in the leaf offset array
// until the scan. The first lane group to set a leaf's bit zeroes that
// leaf's counter, so only touched counters are reset.

__global__ void __launch_bounds__(256) bitmap_clear_kernel(CompactArgs a, unsigned long long tl,
                                                           unsigned long long tiles) {
  uint32_t* off_leaf = a.off + level_offset(a.depth);
  const unsigned long long words = (tl + 31) / 32;
  const unsigned long long total = tiles * words;
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step)
    off_leaf[(i / words) * tl + (i % words)] = 0u;
}

__global__ void __launch_bounds__(256) mark_kernel(CompactArgs a) {
  const unsigned long long n = n_records(a);
  const int sh = 63 - 3 * a.depth;
  uint32_t* off_leaf = a.off + level_offset(a.depth);
  uint32_t* cnt_leaf = a.cnt + level_offset(a.depth);
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n; base += step) {
    const unsigned long long i = base + threadIdx.x;
    const bool valid = i < n;
    const uint32_t active = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const unsigned long long leaf = a.in[i].key >> sh;
      const uint32_t peers = __match_any_sync(active, leaf);
      if (lane_id() == (uint32_t)(__ffs(peers) - 1)) {
        const uint32_t bit = 1u << (uint32_t)(leaf & 31ull);
        const uint32_t old = atomicOr(bitmap_word(off_leaf, leaf), bit);
        if (!(old & bit)) cnt_leaf[leaf] = 0u;
      }
    }
  }
}

// Counts per leaf and, when the tile level T = depth - 4 is >= 1, per
// level-T octant (the parents of the 4096-leaf tiles).
__global__ void __launch_bounds__(256) count_kernel(CompactArgs a, int T) {
  const unsigned long long n = n_records(a);
  const int sh = 63 - 3 * a.depth;
  const int shT = 63 - 3 * T;
  uint32_t* cnt_leaf = a.cnt + level_offset(a.depth);
  uint32_t* cnt_T = a.cnt + level_offset(T);
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n; base += step) {
    const unsigned long long i = base + threadIdx.x;
    const bool valid = i < n;
    const uint32_t active = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const unsigned long long key = a.in[i].key;
      const unsigned long long leaf = key >> sh;
      const uint32_t peers = __match_any_sync(active, leaf);
      if (lane_id() == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&cnt_leaf[leaf], (uint32_t)__popc(peers));
      if (T >= 1) {
        const unsigned long long oT = key >> shT;
        const uint32_t pT = __match_any_sync(active, oT);
        if (lane_id() == (uint32_t)(__ffs(pT) - 1)) atomicAdd(&cnt_T[oT], (uint32_t)__popc(pT));
      }
    }
  }
}

__global__ void __launch_bounds__(256) scatter_kernel(CompactArgs a) {
  const unsigned long long n = n_records(a);
  const int sh = 63 - 3 * a.depth;
  uint32_t* off_leaf = a.off + level_offset(a.depth);
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n; base += step) {
    const unsigned long long i = base + threadIdx.x;
    const bool valid = i < n;
    const uint32_t active = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const uint4 r = reinterpret_cast<const uint4*>(a.in)[i];
      const unsigned long long key = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
      const unsigned long long leaf = key >> sh;
      const uint32_t peers = __match_any_sync(active, leaf);
      const uint32_t leader = __ffs(peers) - 1;
      uint32_t pos = 0;
      if (lane_id() == leader) pos = atomicAdd(&off_leaf[leaf], (uint32_t)__popc(peers));
      pos = __shfl_sync(peers, pos, leader) + __popc(peers & lanemask_lt());
      reinterpret_cast<uint4*>(a.out)[pos] = r;
    }
  }
}

// ------------------------------------------------------- scan and levels

// Writes (off, cnt) of the coarser levels whose octants lie inside a tile.
// Thread tid holds one octant of level L-1 (its 8 children at level L):
// `toff` = its offset, `tsum` = its count. Levels L-2.. use groups of 8, 64
// and 512 threads. `first` = index of this tile's first level-(L-1) octant.
__device__ __forceinline__ void write_coarse(const CompactArgs& a, int L, unsigned long long first, uint32_t toff,
                                             uint32_t tsum, uint32_t n_in_tile, uint32_t* s_wsum, uint32_t* s_woff) {
  const bool has = threadIdx.x < n_in_tile;
  const int tid = threadIdx.x;
  const uint32_t lane = tid & 31, warp = tid >> 5;
  if (L - 1 >= 0 && has) {
    a.off[level_offset(L - 1) + first + tid] = toff;
    a.cnt[level_offset(L - 1) + first + tid] = tsum;
  }
  if (L - 2 < 0) return;
  uint32_t g = tsum;  // groups of 8 lanes
  g += __shfl_xor_sync(0xffffffffu, g, 1);
  g += __shfl_xor_sync(0xffffffffu, g, 2);
  g += __shfl_xor_sync(0xffffffffu, g, 4);
  if ((tid & 7) == 0 && has) {
    a.off[level_offset(L - 2) + first / 8 + tid / 8] = toff;
    a.cnt[level_offset(L - 2) + first / 8 + tid / 8] = g;
  }
  if (L - 3 < 0) return;
  uint32_t wsum = g + __shfl_xor_sync(0xffffffffu, g, 8);
  wsum += __shfl_xor_sync(0xffffffffu, wsum, 16);
  if (lane == 0) {
    s_wsum[warp] = wsum;
    s_woff[warp] = toff;
  }
  __syncthreads();
  // level L-3: groups of 64 threads = warps (2m, 2m+1)
  if (tid < 8 && (uint32_t)tid * 64 < n_in_tile) {
    const uint32_t off3 = s_woff[2 * tid];
    const uint32_t cnt3 = s_wsum[2 * tid] + s_wsum[2 * tid + 1];
    a.off[level_offset(L - 3) + first / 64 + tid] = off3;
    a.cnt[level_offset(L - 3) + first / 64 + tid] = cnt3;
  }
  if (L - 4 >= 0 && tid == 0 && n_in_tile == 512) {
    uint32_t c4 = 0;
    for (int k = 0; k < 16; ++k) c4 += s_wsum[k];
    a.off[level_offset(L - 4) + first / 512] = s_woff[0];
    a.cnt[level_offset(L - 4) + first / 512] = c4;
  }
}

// Exclusive scan of the counts of level L (8^L octants, already counted)
// into its offsets, plus (off, cnt) of levels L-1..L-4 inside each tile.
// One CTA (256 threads) per tile of tl = min(4096, 8^L) octants, taken in
// ticket order and chained by decoupled look-back. Thread t owns octants
// 16t..16t+15 of the tile, i.e. level-(L-1) octants 2t and 2t+1; four
// threads form a level-(L-2) octant, a warp a level-(L-3) octant and the
// CTA the level-(L-4) octant.
constexpr int kScanThreads = 256;
__global__ void __launch_bounds__(kScanThreads, 5) level_scan_kernel(CompactArgs a, int L, unsigned long long tl) {
  __shared__ __align__(128) uint32_t s_buf[kLeafTile];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ unsigned long long s_tile, s_prefix;
  __shared__ uint32_t s_wtot[kScanThreads / 32], s_total;
  const int tid = threadIdx.x;
  const uint32_t lane = tid & 31, warp = tid >> 5;
  const int d = L;
  const uint32_t* cnt_leaf = a.cnt + level_offset(d);
  uint32_t* off_leaf = a.off + level_offset(d);
  if (tid == 0) {
    s_tile = atomicAdd(&a.hdr->ticket[0], 1ull);
    mbar_init(&s_bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const unsigned long long tile = s_tile;
  const unsigned long long leaf0 = tile * tl;
  const uint32_t bytes = (uint32_t)(tl * 4ull);
  if (tid == 0) {
    mbar_arrive_expect_tx(&s_bar, bytes);
    bulk_g2s(s_buf, cnt_leaf + leaf0, bytes, &s_bar);
  }
  if (!mbar_wait_bounded(&s_bar, 0)) {
    if (tid == 0) set_status(&a.hdr->status, FHV_DEV_TIMEOUT);
    mbar_wait_bounded(&s_bar, 0);  // give the copy a second chance before reuse
  }
  // per-thread sums of its two level-(d-1) octants
  const bool has0 = (unsigned long long)tid * 16ull < tl;
  const bool has1 = (unsigned long long)tid * 16ull + 8ull < tl;
  uint4 q[4] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
  const uint4* b4 = reinterpret_cast<const uint4*>(s_buf) + 4 * tid;
  if (has0) {
    q[0] = b4[0];
    q[1] = b4[1];
  }
  if (has1) {
    q[2] = b4[2];
    q[3] = b4[3];
  }
  const uint32_t c0 = q[0].x + q[0].y + q[0].z + q[0].w + q[1].x + q[1].y + q[1].z + q[1].w;
  const uint32_t c1 = q[2].x + q[2].y + q[2].z + q[2].w + q[3].x + q[3].y + q[3].z + q[3].w;
  const uint32_t tsum = c0 + c1;
  // block exclusive scan of the thread sums; warp 0 chains the tiles
  uint32_t incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += v;
  }
  if (lane == 31) s_wtot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kScanThreads / 32 ? s_wtot[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < kScanThreads / 32; o <<= 1) {
      uint32_t v = __shfl_up_sync(0xffffffffu, wi, o);
      if ((int)lane >= o) wi += v;
    }
    const uint32_t tile_total = __shfl_sync(0xffffffffu, wi, kScanThreads / 32 - 1);
    if (lane < kScanThreads / 32) s_wtot[lane] = wi - w;
    const unsigned long long pre = lookback_exclusive(a.tile_state, tile, tile_total, &a.hdr->status);
    if (lane == 0) {
      s_prefix = pre;
      s_total = tile_total;
    }
  }
  __syncthreads();
  const uint32_t toff = (uint32_t)s_prefix + s_wtot[warp] + (incl - tsum);
  // leaf offsets back into shared memory (counts re-read rather than kept
  // live across the look-back), out with one bulk copy
  {
    uint32_t run = toff;
    uint4* o4 = reinterpret_cast<uint4*>(s_buf) + 4 * tid;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if ((j < 2 && has0) || (j >= 2 && has1)) q[j] = o4[j];
      uint4 o;
      o.x = run; run += q[j].x;
      o.y = run; run += q[j].y;
      o.z = run; run += q[j].z;
      o.w = run; run += q[j].w;
      if ((j < 2 && has0) || (j >= 2 && has1)) o4[j] = o;
    }
  }
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0) {
    bulk_s2g(off_leaf + leaf0, s_buf, bytes);
    bulk_commit();
  }
  // coarse levels inside the tile
  const unsigned long long first = leaf0 / 8;  // level d-1 index of this tile's first octant
  if (d - 1 >= 0) {
    const uint64_t b = level_offset(d - 1) + first + 2ull * tid;
    if (has1) {
      *reinterpret_cast<uint2*>(a.off + b) = make_uint2(toff, toff + c0);
      *reinterpret_cast<uint2*>(a.cnt + b) = make_uint2(c0, c1);
    } else if (has0) {
      a.off[b] = toff;
      a.cnt[b] = c0;
    }
  }
  if (d - 2 >= 0) {
    uint32_t g = tsum;
    g += __shfl_xor_sync(0xffffffffu, g, 1);
    g += __shfl_xor_sync(0xffffffffu, g, 2);
    if ((tid & 3) == 0 && (unsigned long long)tid * 16ull < tl) {
      const uint64_t b = level_offset(d - 2) + first / 8 + tid / 4;
      a.off[b] = toff;
      a.cnt[b] = g;
    }
    if (d - 3 >= 0) {
      uint32_t wsum = g + __shfl_xor_sync(0xffffffffu, g, 4);
      wsum += __shfl_xor_sync(0xffffffffu, wsum, 8);
      wsum += __shfl_xor_sync(0xffffffffu, wsum, 16);
      if (lane == 0 && (unsigned long long)warp * 512ull < tl) {
        const uint64_t b = level_offset(d - 3) + first / 64 + warp;
        a.off[b] = toff;
        a.cnt[b] = wsum;
      }
      if (d - 4 >= 0 && tid == 0 && tl == (unsigned long long)kLeafTile) {
        const uint64_t b = level_offset(d - 4) + first / 512;
        a.off[b] = toff;
        a.cnt[b] = s_total;
      }
    }
  }
  if (tid == 0) bulk_wait_read0();
}

// Leaf offsets and counts: one CTA (256 threads) per tile of
// tl = 8^(depth - T) leaves (4096 when depth >= 4), i.e. per level-T octant,
// whose offset is already known (0 when T = 0). No tile waits for another.
// The tile is 1024 chunks of 4 leaves; thread t owns chunks v = 256j + t,
// j = 0..3, so every 16-byte store instruction of a warp covers 512
// contiguous bytes. The CTA reads the tile's occupancy bitmap (512 bytes),
// gathers the counts of occupied leaves only, scans in leaf order (four
// interleaved block scans, one per j), and writes every leaf's offset and
// count. Chunk pairs form level-(depth-1) octants, 16-lane groups level
// depth-2, 4-warp groups level depth-3; those inside the tile are written
// here, and level 0 too when T = 0.
__global__ void __launch_bounds__(kScanThreads, 6) leaf_scan_kernel(CompactArgs a, int T, unsigned long long tl) {
  __shared__ uint32_t s_bits[kLeafTile / 32];
  __shared__ uint32_t s_w[4][kScanThreads / 32];    // per-slice warp totals
  __shared__ uint32_t s_pre[4][kScanThreads / 32];  // exclusive prefix of (slice, warp) in leaf order
  const int tid = threadIdx.x;
  const uint32_t lane = tid & 31, warp = tid >> 5;
  const int d = a.depth;
  const unsigned long long tile = blockIdx.x;
  const unsigned long long leaf0 = tile * tl;
  uint32_t* off_tile = a.off + level_offset(d) + leaf0;
  const uint32_t* cnt_tile = a.cnt + level_offset(d) + leaf0;
  uint4* off4 = reinterpret_cast<uint4*>(off_tile);
  uint4* cnt4 = reinterpret_cast<uint4*>(a.cnt + level_offset(d) + leaf0);
  const uint32_t nvec = (uint32_t)(tl / 4);  // chunks in this tile (<= 1024)
  const uint32_t words = (uint32_t)((tl + 31) / 32);
  if ((uint32_t)tid < words) s_bits[tid] = off_tile[tid];
  const uint32_t P = T >= 1 ? a.off[level_offset(T) + tile] : 0u;
  __syncthreads();
  // counts of this thread's chunks (only occupied leaves are read)
  uint4 q[4];
  uint32_t c[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t v = j * kScanThreads + tid;
    uint32_t e[4] = {0u, 0u, 0u, 0u};
    if (v < nvec) {
      uint32_t bits = (s_bits[v >> 3] >> (4 * (v & 7))) & 0xfu;
      while (bits) {
        const int k = __ffs(bits) - 1;
        bits &= bits - 1;
        const uint32_t x = __ldcg(cnt_tile + 4 * v + k);
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (m == k) e[m] = x;
      }
    }
    q[j] = make_uint4(e[0], e[1], e[2], e[3]);
    c[j] = e[0] + e[1] + e[2] + e[3];
  }
  // four interleaved warp scans, then the (slice, warp) prefixes
  uint32_t incl[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    incl[j] = c[j];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl[j], o);
      if ((int)lane >= o) incl[j] += x;
    }
    if (lane == 31) s_w[j][warp] = incl[j];
  }
  __syncthreads();
  if (warp == 0) {  // 32 lanes = 4 slices x 8 warps, in leaf order
    const uint32_t w = s_w[lane >> 3][lane & 7];
    uint32_t x = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if ((int)lane >= o) x += y;
    }
    s_pre[lane >> 3][lane & 7] = x - w;
  }
  __syncthreads();
  const unsigned long long first = leaf0 / 8;  // level d-1 index of the tile's first octant
  const bool lvl1 = d - 1 > T || (d - 1 == 0 && T == 0);
  const bool lvl2 = d - 2 >= 0 && (d - 2 > T || T == 0);
  const bool lvl3 = d - 3 >= 0 && (d - 3 > T || T == 0);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t v = j * kScanThreads + tid;
    const bool has = v < nvec;
    const uint32_t base = P + s_pre[j][warp] + (incl[j] - c[j]);
    if (has) {
      uint4 o;
      o.x = base;
      o.y = o.x + q[j].x;
      o.z = o.y + q[j].y;
      o.w = o.z + q[j].z;
      __stcs(off4 + v, o);
      __stcs(cnt4 + v, q[j]);
    }
    // level d-1: chunk pairs
    const uint32_t c2 = c[j] + __shfl_xor_sync(0xffffffffu, c[j], 1);
    if (lvl1 && has && (v & 1u) == 0u) {
      const uint64_t b = level_offset(d - 1) + first + (v >> 1);
      a.off[b] = base;
      a.cnt[b] = c2;
    }
    // level d-2: 16-chunk groups
    uint32_t c16 = c2 + __shfl_xor_sync(0xffffffffu, c2, 2);
    c16 += __shfl_xor_sync(0xffffffffu, c16, 4);
    c16 += __shfl_xor_sync(0xffffffffu, c16, 8);
    if (lvl2 && has && (v & 15u) == 0u) {
      const uint64_t b = level_offset(d - 2) + first / 8 + (v >> 4);
      a.off[b] = base;
      a.cnt[b] = c16;
    }
  }
  // level d-3: 128-chunk groups = 4 warps of one slice
  if (lvl3 && tid < 8) {
    const int j = tid >> 1, g = tid & 1;
    const uint32_t v = j * kScanThreads + g * 128;
    if (v < nvec) {
      const uint64_t b = level_offset(d - 3) + first / 64 + (v >> 7);
      a.off[b] = P + s_pre[j][4 * g];
      a.cnt[b] = s_w[j][4 * g] + s_w[j][4 * g + 1] + s_w[j][4 * g + 2] + s_w[j][4 * g + 3];
    }
  }
  if (T == 0 && d >= 4 && tid == 0) {  // level 0 = the whole (single) tile
    uint32_t tot = 0;
    for (int j = 0; j < 4; ++j)
      for (int w = 0; w < kScanThreads / 32; ++w) tot += s_w[j][w];
    a.off[0] = 0u;
    a.cnt[0] = tot;
  }
}

// Levels above the scan tiles: level L is final; write L-1..L-4 from it.
__global__ void __launch_bounds__(512) reduce_levels_kernel(CompactArgs a, int L) {
  __shared__ uint32_t s_wsum[16], s_woff[16];
  const int tid = threadIdx.x;
  const unsigned long long n_child = 1ull << (3 * L);
  const unsigned long long first = (unsigned long long)blockIdx.x * 512ull;  // first level-(L-1) octant
  const unsigned long long n_parent = n_child / 8ull;
  const uint32_t n_in_tile = (uint32_t)min(512ull, n_parent - first);
  const bool has = (uint32_t)tid < n_in_tile;
  uint32_t tsum = 0, toff = 0;
  if (has) {
    const unsigned long long c0 = (first + tid) * 8ull;
    const uint4* cp = reinterpret_cast<const uint4*>(a.cnt + level_offset(L) + c0);
    uint4 x = cp[0], y = cp[1];
    tsum = x.x + x.y + x.z + x.w + y.x + y.y + y.z + y.w;
    toff = a.off[level_offset(L) + c0];
  }
  write_coarse(a, L, first, toff, tsum, n_in_tile, s_wsum, s_woff);
}

// --------------------------------------------------- in-octant canonical order

// The per-range order of the records of one chunk [lo, hi): every octant
// range that starts in the chunk is put into (key, tri, nrm) order -- ranges
// of up to kWarpRange records one warp each (rank sort through shuffles),
// longer ones one after the other in shared memory by the whole CTA, and
// ranges longer than kOrderSmem are left to huge_sort_kernel. The scatter used
// the leaf offsets as cursors; the first pass restores them.
constexpr int kOrderCap = kOrderSmem / 2;    // largest run of whole leaves ordered in shared memory at once
constexpr int kOrderChunk = kOrderSmem / 4;  // records per in-leaf order CTA

__device__ void seg_sort_chunk(const CompactArgs& a, unsigned long long n, unsigned long long lo, uint4* s_rec) {
  __shared__ uint32_t s_start[kOrderChunk];  // starts of the short ranges, relative to lo
  __shared__ unsigned long long s_long[kMaxLong];
  __shared__ uint32_t s_nshort, s_nlong;
  const unsigned long long hi = min(n, lo + (unsigned long long)kOrderChunk);
  const int sh = 63 - 3 * a.depth;
  uint32_t* off_leaf = a.off + level_offset(a.depth);
  const uint32_t* cnt_leaf = a.cnt + level_offset(a.depth);
  const unsigned long long* keys = reinterpret_cast<const unsigned long long*>(a.out);
  if (threadIdx.x == 0) {
    s_nshort = 0;
    s_nlong = 0;
  }
  __syncthreads();
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const unsigned long long leaf = keys[2 * i] >> sh;
    const bool start = i == 0 || (keys[2 * (i - 1)] >> sh) != leaf;
    if (start) {
      off_leaf[leaf] = (uint32_t)i;
      const uint32_t len = cnt_leaf[leaf];
      if (len <= kWarpRange) {
        if (len > 1) s_start[atomicAdd(&s_nshort, 1u)] = (uint32_t)(i - lo);
      } else {
        const uint32_t k = atomicAdd(&s_nlong, 1u);
        if (k < kMaxLong) s_long[k] = i;
      }
    }
  }
  __syncthreads();
  uint4* g = reinterpret_cast<uint4*>(a.out);
  const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (uint32_t k = warp; k < s_nshort; k += nwarps) {
    const unsigned long long st = lo + s_start[k];
    warp_rank_sort(g, st, cnt_leaf[keys[2 * st] >> sh]);
  }
  const uint32_t nlong = min(s_nlong, kMaxLong);
  for (uint32_t k = 0; k < nlong; ++k) {
    const unsigned long long st = s_long[k];
    const uint32_t len = cnt_leaf[keys[2 * st] >> sh];
    if (len <= (uint32_t)kOrderSmem) {
      sort_range_smem(g, st, st + len, s_rec);  // CTA-wide, ends with a barrier
    } else if (threadIdx.x == 0) {
      const uint32_t slot = atomicAdd(&a.hdr->huge_count, 1u);
      if (slot < a.huge_max) a.huge_list[slot] = st;
    }
  }
  if (s_nlong > kMaxLong && threadIdx.x == 0) set_status(&a.hdr->status, FHV_DEV_RANGE);
}

// One CTA per chunk of kOrderChunk scattered records: the octant ranges that
// start in the chunk get their canonical order. Usually they fit in shared
// memory together (the range from the first leaf start at or after lo to
// the first at or after hi, at most kSortCap records): one coalesced load,
// every record ranked within its leaf (tile_order_smem), one coalesced
// store, and the offsets used as cursors by the scatter restored from the
// leaf starts. Otherwise the per-range path above.
constexpr int kOrderThreads = 256;
__global__ void __launch_bounds__(kOrderThreads, 4) seg_sort_kernel(CompactArgs a) {
  extern __shared__ __align__(16) uint4 s_rec[];  // kOrderSmem records: 2 x kOrderCap, or the per-range sorts' tile
  uint4* s_alt = s_rec + kOrderCap;
  __shared__ uint32_t s_gstart[kOrderCap + 1], s_gid[kOrderCap];
  __shared__ uint32_t s_list[kLargeList], s_misc[kMiscWords];
  __shared__ unsigned long long s_R[2];
  const unsigned long long n = n_records(a);
  const unsigned long long lo = (unsigned long long)blockIdx.x * kOrderChunk;
  if (lo >= n) return;
  const unsigned long long hi = min(n, lo + (unsigned long long)kOrderChunk);
  const int sh = 63 - 3 * a.depth;
  const unsigned long long* keys = reinterpret_cast<const unsigned long long*>(a.out);
  if (threadIdx.x < 32) {  // first leaf start in [lo, hi), first at or after hi (within lo + kOrderCap)
    const uint32_t lane = threadIdx.x;
    unsigned long long r0 = hi;
    for (unsigned long long x0 = lo; x0 < hi; x0 += 32) {
      const unsigned long long x = x0 + lane;
      const bool st = x < hi && (x == 0 || (keys[2 * x] >> sh) != (keys[2 * (x - 1)] >> sh));
      const uint32_t m = __ballot_sync(0xffffffffu, st);
      if (m) {
        r0 = x0 + (__ffs(m) - 1);
        break;
      }
    }
    const unsigned long long limit = min(n, lo + (unsigned long long)kOrderCap + 1ull);
    unsigned long long r1 = ~0ull;  // not found within the limit: the range is too long
    if (hi >= n) {
      r1 = n;
    } else {
      for (unsigned long long x0 = hi; x0 < limit; x0 += 32) {
        const unsigned long long x = x0 + lane;
        const bool st = x < limit && (keys[2 * x] >> sh) != (keys[2 * (x - 1)] >> sh);
        const uint32_t m = __ballot_sync(0xffffffffu, st);
        if (m) {
          r1 = x0 + (__ffs(m) - 1);
          break;
        }
      }
      if (r1 == ~0ull && limit == n) r1 = n;
    }
    if (lane == 0) {
      s_R[0] = r0;
      s_R[1] = r1;
    }
  }
  __syncthreads();
  const unsigned long long R0 = s_R[0], R1 = s_R[1];
  if (R0 >= hi) return;  // no octant range starts in this chunk
  if (R1 == ~0ull || R1 - R0 > (unsigned long long)kOrderCap) {
    seg_sort_chunk(a, n, lo, s_rec);
    return;
  }
  const uint32_t len = (uint32_t)(R1 - R0);
  uint4* g = reinterpret_cast<uint4*>(a.out);
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) s_rec[i] = g[R0 + i];
  __syncthreads();
  tile_order_smem(s_rec, s_alt, len, sh, false, s_gstart, s_gid, s_list, s_misc);
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) g[R0 + i] = s_alt[i];
  uint32_t* off_leaf = a.off + level_offset(a.depth);
  const uint32_t n_groups = s_misc[32];
  for (uint32_t k = threadIdx.x; k < n_groups; k += blockDim.x)
    off_leaf[rec_key(s_alt[s_gstart[k]]) >> sh] = (uint32_t)(R0 + s_gstart[k]);
}

// Octant ranges longer than kSortCap: one CTA each, tiles sorted in shared
// memory, then pairwise merges between the range and its scratch copy.
__global__ void __launch_bounds__(512) huge_sort_kernel(CompactArgs a) {
  extern __shared__ __align__(16) uint4 s_rec[];
  const uint32_t count = min((unsigned long long)a.hdr->huge_count, a.huge_max);
  const int sh = 63 - 3 * a.depth;
  const uint32_t* cnt_leaf = a.cnt + level_offset(a.depth);
  uint4* g = reinterpret_cast<uint4*>(a.out);
  uint4* scratch = reinterpret_cast<uint4*>(a.scratch);
  for (uint32_t slot = blockIdx.x; slot < count; slot += gridDim.x) {
    const unsigned long long s = a.huge_list[slot];
    const unsigned long long len = cnt_leaf[a.out[s].key >> sh];
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
      uint4* t = src;
      src = dst;
      dst = t;
    }
    if (src != g + s) {
      for (unsigned long long i = threadIdx.x; i < len; i += blockDim.x) g[s + i] = src[i];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ driver

static int compact_tile_level(int d) { return d > 4 ? d - 4 : 0; }  // level of the leaf tiles' parents

// Clears the leaves' occupancy bitmap (before marking).
cudaError_t compact_clear_bitmap(const CompactArgs& a, cudaStream_t s) {
  const unsigned long long leaves = 1ull << (3 * a.depth);
  const unsigned long long tl = leaves < (unsigned long long)kLeafTile ? leaves : (unsigned long long)kLeafTile;
  const unsigned long long words = (leaves / tl) * ((tl + 31) / 32);
  unsigned long long blocks = (words + 255) / 256;
  if (blocks > (unsigned long long)sm_count() * 32ull) blocks = (unsigned long long)sm_count() * 32ull;
  timing_begin("bitmap_clear", s);
  bitmap_clear_kernel<<<(unsigned)blocks, 256, 0, s>>>(a, tl, leaves / tl);
  timing_end("bitmap_clear", s);
  return cudaGetLastError();
}

// Offsets and counts of every level from the counted leaves (and level-T octants).
cudaError_t compact_scan(const CompactArgs& a, cudaStream_t s) {
  const unsigned long long leaves = 1ull << (3 * a.depth);
  const unsigned long long tl = leaves < (unsigned long long)kLeafTile ? leaves : (unsigned long long)kLeafTile;
  const int T = compact_tile_level(a.depth);
  if (T >= 1) {
    // offsets of level T by look-back scan, levels T-1.. by reduction
    const unsigned long long nT = 1ull << (3 * T);
    const unsigned long long tlT = nT < (unsigned long long)kLeafTile ? nT : (unsigned long long)kLeafTile;
    timing_begin("level_scan", s);
    level_scan_kernel<<<(unsigned)(nT / tlT), kScanThreads, 0, s>>>(a, T, tlT);
    timing_end("level_scan", s);
    for (int L = T - 4; L > 0; L -= 4) {
      const unsigned long long parents = 1ull << (3 * (L - 1));
      timing_begin("reduce_levels", s);
      reduce_levels_kernel<<<(unsigned)((parents + 511) / 512), 512, 0, s>>>(a, L);
      timing_end("reduce_levels", s);
    }
  }
  timing_begin("leaf_scan", s);
  leaf_scan_kernel<<<(unsigned)(leaves / tl), kScanThreads, 0, s>>>(a, T, tl);
  timing_end("leaf_scan", s);
  return cudaGetLastError();
}

// Canonical order inside every octant range of the scattered records (and
// the offsets, used as cursors by the scatter, restored).
cudaError_t compact_order(const CompactArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(seg_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kOrderSmem * 16);
    cudaFuncSetAttribute(huge_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortCap * 16);
    attr = true;
  }
  const unsigned long long chunks = (a.n_max + kOrderChunk - 1) / kOrderChunk;
  timing_begin("seg_sort", s);
  seg_sort_kernel<<<(unsigned)chunks, kOrderThreads, kOrderSmem * 16, s>>>(a);
  timing_end("seg_sort", s);
  unsigned long long hg = a.huge_max < 1024ull ? a.huge_max : 1024ull;
  timing_begin("huge_sort", s);
  huge_sort_kernel<<<(unsigned)hg, 512, kSortCap * 16, s>>>(a);
  timing_end("huge_sort", s);
  return cudaGetLastError();
}

cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s) {
  const int grid_rec = sm_count() * 8;
  const int T = compact_tile_level(a.depth);
  cudaError_t e = compact_clear_bitmap(a, s);
  if (e != cudaSuccess) return e;
  if (a.n_max > 0) {
    timing_begin("mark", s);
    mark_kernel<<<grid_rec, 256, 0, s>>>(a);
    timing_end("mark", s);
    timing_begin("count", s);
    count_kernel<<<grid_rec, 256, 0, s>>>(a, T);
    timing_end("count", s);
  }
  e = compact_scan(a, s);
  if (e != cudaSuccess || a.n_max == 0) return e;
  timing_begin("scatter", s);
  scatter_kernel<<<grid_rec, 256, 0, s>>>(a);
  timing_end("scatter", s);
  return compact_order(a, s);
}

}  // namespace fhv
