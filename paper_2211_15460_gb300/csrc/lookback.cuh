// lookback.cuh -- single-pass exclusive scan across CTAs by decoupled
// look-back (Merrill & Garland, "Single-pass Parallel Prefix Scan with
// Decoupled Look-back", NVIDIA tech report NVR-2016-002).
//
// Tile state word: bits 62..63 = flag (0 nothing yet, 1 tile aggregate,
// 2 inclusive prefix), bits 0..61 = value. Tiles are numbered by a ticket
// taken when a CTA starts, so every tile a CTA waits for belongs to a CTA
// that is already running. Every wait is bounded; on expiry the tile is
// treated as contributing 0 and FHV_DEV_TIMEOUT is raised.
#pragma once

#include "fhv_device.cuh"

namespace fhv {

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1ull;
constexpr uint32_t kLookbackSpin = 1u << 20;

// Called by all 32 lanes of one warp of the CTA that owns `tile`, once the
// tile's aggregate is known. Returns the exclusive prefix to every lane.
__device__ inline unsigned long long lookback_exclusive(unsigned long long* state, unsigned long long tile,
                                                        unsigned long long aggregate, uint32_t* status) {
  const uint32_t lane = lane_id();
  if (tile == 0) {
    if (lane == 0) st_release_u64(&state[0], kFlagInc | (aggregate & kValMask));
    return 0ull;
  }
  if (lane == 0) st_release_u64(&state[tile], kFlagAgg | (aggregate & kValMask));
  unsigned long long excl = 0;
  long long win_hi = (long long)tile - 1;  // lane 31 reads win_hi, lane 0 reads win_hi - 31
  bool timed_out = false;
  while (true) {
    long long idx = win_hi - (31 - (long long)lane);
    unsigned long long v = kFlagInc;  // before tile 0: inclusive 0
    if (idx >= 0) {
      uint32_t it = 0;
      while (true) {
        v = ld_acquire_u64(&state[idx]);
        if ((v >> 62) != 0ull) break;
        if (++it > kLookbackSpin) {
          timed_out = true;
          v = kFlagInc;
          break;
        }
        if (it > 16) __nanosleep(32);
      }
    }
    uint32_t inc = __ballot_sync(0xffffffffu, (v >> 62) == 2ull);
    int hi = inc ? 31 - __clz(inc) : -1;
    unsigned long long c = ((int)lane >= hi) ? (v & kValMask) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    excl += c;
    if (hi >= 0) break;
    win_hi -= 32;
  }
  if (__any_sync(0xffffffffu, timed_out) && lane == 0) set_status(status, FHV_DEV_TIMEOUT);
  if (lane == 0) st_release_u64(&state[tile], kFlagInc | ((excl + aggregate) & kValMask));
  return excl;
}

}  // namespace fhv
