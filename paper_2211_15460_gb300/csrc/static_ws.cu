// static_ws.cu -- fhv_compact_pofa_static: POFA compaction whose scratch
// lives in a fixed device array inside this library, for callers that
// cannot allocate device memory themselves.
//
// The scratch array is a file-scope __device__ array: every GPU that loads
// the library holds it (FHV_STATIC_WS_BYTES) until the process exits. Host
// code cannot use the array's name as a device address, so the first call
// on each device looks the address up with cudaGetSymbolAddress (with that
// device current) and caches it beside the CUDA context it belongs to; a
// call that finds another context current (the device was reset, so the
// module and its array were loaded again) looks the address up again. That
// first call should therefore happen before any stream capture. All calls
// share the one array: the compaction clears the parts that must start at
// zero at the start of every call, and calls whose work overlaps on the GPU
// (other streams, other threads) race on it and must be serialised by the
// caller. The array's first word is the status word of the last call;
// fhv_read_static_status reads it.
#include <cuda.h>

#include <mutex>

#include "kernels.h"

namespace {

__device__ __align__(256) unsigned char g_static_ws[FHV_STATIC_WS_BYTES];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

std::mutex g_mutex;
struct CachedAddress {
  CUcontext ctx;
  void* ptr;
};
CachedAddress g_cache[64] = {};

// The driver's current context, through the runtime's driver entry point
// (no link against libcuda); nullptr if it cannot be asked.
CUcontext current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
    resolved = true;
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device address of g_static_ws on the current device (set up once per
// device and context).
fhv_status static_ws_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return FHV_ERR_CUDA;
  if (dev < 0 || dev >= 64) return FHV_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  CachedAddress& c = g_cache[dev];
  const CUcontext now = current_context();
  if (!c.ptr || !now || now != c.ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || p == nullptr) return FHV_ERR_CUDA;
    c.ptr = p;
    c.ctx = current_context();  // the lookup made the device's context current
  }
  *out = c.ptr;
  return FHV_OK;
}

}  // namespace

extern "C" fhv_status fhv_compact_pofa_static(const fhv_record* d_in, uint64_t n_max, const uint64_t* d_n, int depth,
                                              fhv_record* d_pofa, uint32_t* d_off, uint32_t* d_cnt,
                                              fhv_stream_t stream) {
  if (n_max > FHV_STATIC_MAX_RECORDS) return FHV_ERR_UNSUPPORTED;
  if (depth < 1 || depth > 11) return FHV_ERR_INVALID_ARG;
  if (fhv::compact_ws(depth, n_max).total > FHV_STATIC_WS_BYTES) return FHV_ERR_UNSUPPORTED;
  void* ws = nullptr;
  const fhv_status st = static_ws_address(&ws);
  if (st != FHV_OK) return st;
  return fhv_compact_pofa(d_in, n_max, d_n, depth, d_pofa, d_off, d_cnt, ws, FHV_STATIC_WS_BYTES, stream);
}

extern "C" fhv_status fhv_read_static_status(uint32_t* host_status, fhv_stream_t stream) {
  if (!host_status) return FHV_ERR_INVALID_ARG;
  void* ws = nullptr;
  const fhv_status st = static_ws_address(&ws);
  if (st != FHV_OK) return st;
  return fhv_read_status(ws, host_status, stream);
}
