// atomics.cu -- microbenchmark of L2 atomic throughput, the second ceiling of
// the visibility pass (64-bit atomicMin per splatted fragment) and of list
// insertion (atomicExch on the heads). No paper counterpart.
//
// Every thread applies `ops` 64-bit atomic minimums to words spread over a
// buffer small enough to stay in L2 (the caller sizes it): word index =
// a multiplicative hash of (thread, op) so that consecutive operations of a
// warp hit different 32-byte sectors, as a splat's do. With returning = 0
// the result is unused (reductions, like the splat); with returning = 1 the
// old value feeds a dependent sum (atomics that return, like list insertion);
// with returning = 2 the words are only read, by volatile loads (the
// splat's read-first probes), their sum kept live.
#include "kernels.h"

namespace fhv {

__global__ void atomic_probe_kernel(unsigned long long* buf, unsigned long long mask, int ops, int returning,
                                    unsigned long long* sink) {
  const unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  unsigned long long acc = 0;
  for (int i = 0; i < ops; ++i) {
    const unsigned long long h = (t * 0x9E3779B97F4A7C15ull + (unsigned long long)i * 0xD1B54A32D192ED03ull) >> 7;
    const unsigned long long idx = (h * 4ull) & mask;  // one word per 32-byte sector
    const unsigned long long v = (t << 20) ^ (unsigned long long)i;
    if (returning == 2)
      acc += *((volatile const unsigned long long*)(buf + idx));
    else if (returning)
      acc += atomicMin(buf + idx, v);
    else
      atomicMin(buf + idx, v);
  }
  if (returning && acc == 0x123456789ull) *sink = acc;  // keeps the returned values live
}

cudaError_t launch_atomic_probe(unsigned long long* buf, unsigned long long n_words, int ops, int returning,
                                cudaStream_t s) {
  unsigned long long mask = 1;
  while (mask * 2 <= n_words) mask *= 2;
  const int blocks = sm_count() * 8;
  timing_begin("atomic_probe", s);
  atomic_probe_kernel<<<blocks, 256, 0, s>>>(buf, mask - 1, ops, returning, buf);
  timing_end("atomic_probe", s);
  return cudaGetLastError();
}

}  // namespace fhv
