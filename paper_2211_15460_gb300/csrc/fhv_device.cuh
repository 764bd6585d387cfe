// fhv_device.cuh -- device-side building blocks shared by the FHV kernels:
// record type, Morton coding, the fixed-order float32 helpers of the
// arithmetic contract, warp utilities, acquire/release accesses for the
// decoupled look-back, and the mbarrier / bulk-copy (TMA) primitives of
// sm_100-class GPUs, written as inline PTX.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fhv.h"

namespace fhv {

constexpr int kQBits = 21;
constexpr uint32_t kQMax = (1u << kQBits) - 1u;
constexpr int kIdxBits = 40;
constexpr unsigned long long kIdxMask = (1ull << kIdxBits) - 1ull;
constexpr unsigned long long kVisEmpty = ~0ull;

// Workspace header (first 256 bytes of every call's workspace).
struct WsHeader {
  uint32_t status;      // FHV_DEV_* bits
  uint32_t pad0;
  unsigned long long ticket[4];  // dynamic tile tickets for look-back scans
  unsigned long long total;      // total bbox samples (capture)
  uint32_t huge_count;           // compaction: segments larger than a CTA tile; ray casting: tiles cast per pixel
  uint32_t pad1;
  unsigned long long n_kept;     // direct POFA build: records stored (0 when they exceed the capacity)
  unsigned long long n_huge_buckets;  // sparse compaction: buckets too large for a tile sort
  unsigned long long n_big;      // capture: setups with more than kSmallSamples samples
  unsigned long long big_total;  // capture: their samples
  unsigned long long raster_ticket[3][2];  // capture: per raster pass, batch / item tickets
};
static_assert(sizeof(WsHeader) <= 256, "header");

struct __align__(16) Rec {
  unsigned long long key;
  uint32_t tri;
  uint32_t nrm;
};
static_assert(sizeof(Rec) == sizeof(fhv_record), "record size");

__host__ __device__ inline uint64_t level_offset(int l) {
  return l == 0 ? 0ull : (((1ull << (3 * l)) - 1ull) / 7ull + 3ull);
}

// ------------------------------------------------------------------ Morton

// Spread the low 21 bits of v to every third bit (bit k -> bit 3k).
__device__ __forceinline__ unsigned long long spread3(uint32_t v) {
  unsigned long long x = v & 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// Inverse of spread3.
__device__ __forceinline__ uint32_t compact3(unsigned long long x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

__device__ __forceinline__ unsigned long long morton63(uint32_t x, uint32_t y, uint32_t z) {
  return (spread3(x) << 2) | (spread3(y) << 1) | spread3(z);
}

// ------------------------------------------- float32, one rounding per op

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// ((a.x*b.x) + (a.y*b.y)) + (a.z*b.z)
__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz) {
  return fadd(fadd(fmul(ax, bx), fmul(ay, by)), fmul(az, bz));
}

__device__ __forceinline__ uint32_t quantize1(float p, float cmin, float qscale) {
  float f = floorf(fmul(fsub(p, cmin), qscale));
  if (!(f >= 0.0f)) return 0u;
  if (f >= (float)kQMax) return kQMax;
  return (uint32_t)f;
}

// pixel units -> 1/256 fixed point, guard band +-2^16 px, round half even
__device__ __forceinline__ int32_t snap256(float s) {
  float v = fmul(s, 256.0f);
  v = fminf(fmaxf(v, -16777216.0f), 16777216.0f);
  return __float2int_rn(v);
}

// Octahedral encoding of an (unnormalised) normal to snorm16 x | y << 16.
__device__ __forceinline__ uint32_t oct_encode(float nx, float ny, float nz) {
  float l1 = fadd(fadd(fabsf(nx), fabsf(ny)), fabsf(nz));
  float px = 0.0f, py = 0.0f;
  if (l1 > 0.0f) {
    px = fdiv(nx, l1);
    py = fdiv(ny, l1);
    if (nz < 0.0f) {
      float sx = px >= 0.0f ? 1.0f : -1.0f;
      float sy = py >= 0.0f ? 1.0f : -1.0f;
      float qx = fmul(fsub(1.0f, fabsf(py)), sx);
      float qy = fmul(fsub(1.0f, fabsf(px)), sy);
      px = qx;
      py = qy;
    }
  }
  px = fminf(fmaxf(px, -1.0f), 1.0f);
  py = fminf(fmaxf(py, -1.0f), 1.0f);
  int32_t ex = __float2int_rn(fmul(px, 32767.0f));
  int32_t ey = __float2int_rn(fmul(py, 32767.0f));
  return (uint32_t)(uint16_t)(int16_t)ex | ((uint32_t)(uint16_t)(int16_t)ey << 16);
}

// Normalised normal from the octahedral code (shading only; any rounding).
__device__ __forceinline__ void oct_decode(uint32_t code, float& x, float& y, float& z) {
  x = (float)(int16_t)(uint16_t)(code & 0xffffu) * (1.0f / 32767.0f);
  y = (float)(int16_t)(uint16_t)(code >> 16) * (1.0f / 32767.0f);
  z = 1.0f - fabsf(x) - fabsf(y);
  if (z < 0.0f) {
    float qx = (1.0f - fabsf(y)) * (x >= 0.0f ? 1.0f : -1.0f);
    float qy = (1.0f - fabsf(x)) * (y >= 0.0f ? 1.0f : -1.0f);
    x = qx;
    y = qy;
  }
  float inv = rsqrtf(x * x + y * y + z * z);
  x *= inv;
  y *= inv;
  z *= inv;
}

// ------------------------------------------------------------ warp helpers

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ void set_status(uint32_t* status, uint32_t bits) {
  if (status) atomicOr(status, bits);
}

// ------------------------------------------------- acquire / release words

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// --------------------------------------------------- mbarrier + bulk copies

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// One probe of phase `parity`; true once that phase has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait; returns false if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t max_iter = (1u << 22)) {
  for (uint32_t it = 0; it < max_iter; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

// Bulk global -> shared copy completing on `bar` (bytes multiple of 16,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bulk shared -> global copy (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void* gmem_dst, const void* smem_src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gmem_dst), "r"(smem_u32(smem_src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Make generic-proxy shared-memory writes visible to the async (bulk) proxy.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace fhv
