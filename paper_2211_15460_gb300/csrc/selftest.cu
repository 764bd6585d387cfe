// selftest.cu -- failure detection without a fault: the library's bounded
// device waits, run on conditions that nothing satisfies, give up and report
// FHV_DEV_TIMEOUT in the workspace status word. Nothing traps, and the
// context stays usable for the next call.
#include "kernels.h"
#include "lookback.cuh"
#include "tc.cuh"

namespace fhv {

namespace {

// kind 0: the scans' decoupled look-back, for tile 1 whose predecessor never
//         publishes (state[0] stays 0), bounded by its spin limit;
// kind 1: the bulk copies' mbarrier wait on a barrier no one arrives at;
// kind 2: the tensor-core kernels' mbarrier wait, likewise.
// The mbarrier waits poll 2^12 times here (their polls may suspend for a
// hardware-defined time); the look-back keeps its own limit.
__global__ void __launch_bounds__(32) wait_probe_kernel(WsHeader* hdr, unsigned long long* state, int kind) {
  if (kind == 0) {
    lookback_exclusive(state, 1ull, 0ull, &hdr->status);
    return;
  }
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (threadIdx.x == 0) {
    const bool done = kind == 1 ? mbar_wait_bounded(&bar, 0u, 1u << 12) : tc::mbar_wait(&bar, 0u, 1 << 12);
    if (!done) set_status(&hdr->status, FHV_DEV_TIMEOUT);
  }
}

}  // namespace

cudaError_t launch_wait_probe(void* ws, int kind, cudaStream_t s) {
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  unsigned long long* state = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ws) + kHeaderBytes);
  timing_begin("wait_probe", s);
  wait_probe_kernel<<<1, 32, 0, s>>>(hdr, state, kind);
  timing_end("wait_probe", s);
  return cudaGetLastError();
}

}  // namespace fhv
