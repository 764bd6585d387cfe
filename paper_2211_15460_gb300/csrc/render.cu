// render.cu -- image generation for novel viewpoints (Section 3.3) by point
// splatting with an exact visibility pass, then local illumination of the
// visible fragment (Section 5).
//
// GB300 layout of the work:
//  * splat: grid-stride over the 16-byte records (coalesced 512 bytes per
//    warp); each fragment is projected with the float32 contract, its depth
//    quantised to 24 bits, and (qdepth << 40 | index) min-combined into a
//    64-bit visibility word per pixel. A plain load first skips the atomic
//    when the pixel already holds a nearer fragment, so deep pixels cost L2
//    reads rather than L2 atomics.
//  * shade: one thread per pixel decodes the winner, gathers its record and
//    material, and sums the lights kept in shared memory.
#include "kernels.h"
#include "splat.cuh"

namespace fhv {

__device__ __forceinline__ unsigned long long render_n(const RenderArgs& a) {
  unsigned long long n = a.n_max;
  if (a.d_n) {
    unsigned long long c = *a.d_n;
    n = c < n ? c : n;
  }
  return n;
}

// Grid-stride splat of the records. For k = 1 a thread takes kSplatBatch
// records a stride apart per iteration and issues their record loads, then
// their visibility loads, all before the first compare, so several
// dependent memory round trips overlap instead of running one after the
// other.
constexpr int kSplatBatch = 4;

__global__ void __launch_bounds__(256) splat_kernel(RenderArgs a) {
  const unsigned long long n = render_n(a);
  const SplatView sv = make_splat_view(a.cube_min, a.cube_side, a.origin, a.right, a.up, a.fwd, a.pitch, a.width,
                                       a.height, a.z0, a.z1, a.k, a.vis);
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  if (sv.k == 1) {
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n;
         i0 += step * kSplatBatch) {
      uint4 r[kSplatBatch];
#pragma unroll
      for (int b = 0; b < kSplatBatch; ++b) {
        const unsigned long long i = i0 + (unsigned long long)b * step;
        r[b] = i < n ? __ldcs(reinterpret_cast<const uint4*>(a.rec) + i) : make_uint4(0u, 0u, 0u, 0u);
      }
      unsigned long long* ptr[kSplatBatch];
      unsigned long long key[kSplatBatch];
#pragma unroll
      for (int b = 0; b < kSplatBatch; ++b) {
        const unsigned long long i = i0 + (unsigned long long)b * step;
        ptr[b] = nullptr;
        key[b] = kVisEmpty;
        if (i >= n) continue;
        float p[3];
        dequantize((unsigned long long)r[b].x | ((unsigned long long)r[b].y << 32), sv, p);
        const Projected pr = project_point(p, sv);
        if (pr.ax < 0 || pr.ax >= sv.W || pr.ay < 0 || pr.ay >= sv.H) continue;
        ptr[b] = sv.vis + (unsigned long long)pr.ay * sv.W + pr.ax;
        key[b] = ((unsigned long long)pr.qd << kIdxBits) | (a.index_base + i);
      }
      unsigned long long cur[kSplatBatch];
#pragma unroll
      for (int b = 0; b < kSplatBatch; ++b) cur[b] = ptr[b] ? ld_vis(ptr[b]) : 0ull;
#pragma unroll
      for (int b = 0; b < kSplatBatch; ++b)
        if (ptr[b] && cur[b] > key[b]) atomicMin(ptr[b], key[b]);
    }
    return;
  }
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    const uint4 r = __ldcs(reinterpret_cast<const uint4*>(a.rec) + i);
    const unsigned long long key = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
    float p[3];
    dequantize(key, sv, p);
    splat_point(p, a.index_base + i, sv);
  }
}

__global__ void __launch_bounds__(256) shade_kernel(RenderArgs a) {
  __shared__ float s_l[64 * 8];
  for (int i = threadIdx.x; i < a.n_lights * 8; i += blockDim.x) s_l[i] = a.lights[i];
  __syncthreads();
  const unsigned long long np = (unsigned long long)a.width * a.height;
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += step)
    reinterpret_cast<float4*>(a.rgba)[p] =
        shade_pixel(a.vis[p], a.rec, a.tri_material, a.albedo, a.cube_min, a.cube_side, s_l, a.n_lights);
}

// Shading of a slice of the fragments: pixels whose winner is record
// index_base + j (j < n) get that record's colour, all others zero, so that
// the slices' images add up to the whole image.
__global__ void __launch_bounds__(256) shade_owned_kernel(RenderArgs a) {
  __shared__ float s_l[64 * 8];
  for (int i = threadIdx.x; i < a.n_lights * 8; i += blockDim.x) s_l[i] = a.lights[i];
  __syncthreads();
  const unsigned long long n = render_n(a);
  const unsigned long long np = (unsigned long long)a.width * a.height;
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += step) {
    const unsigned long long v = a.vis[p];
    const unsigned long long idx = v & kIdxMask;
    float4 c = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (v != ~0ull && idx >= a.index_base && idx - a.index_base < n)
      c = shade_pixel(v - a.index_base, a.rec, a.tri_material, a.albedo, a.cube_min, a.cube_side, s_l, a.n_lights);
    reinterpret_cast<float4*>(a.rgba)[p] = c;
  }
}

// Splat grid: one batch of kSplatBatch records per thread for up to
// 16 CTAs per SM, grid-stride beyond, so a list of a few million records
// runs in one pass without a tail of half-empty second iterations.
static unsigned splat_grid(unsigned long long n_max) {
  const unsigned long long need = (n_max + 256ull * kSplatBatch - 1) / (256ull * kSplatBatch);
  const unsigned long long most = (unsigned long long)sm_count() * 16ull;
  return (unsigned)(need < most ? (need > 0 ? need : 1ull) : most);
}

cudaError_t launch_splat(const RenderArgs& a, cudaStream_t s) {
  if (a.n_max > 0) {
    timing_begin("splat", s);
    splat_kernel<<<splat_grid(a.n_max), 256, 0, s>>>(a);
    timing_end("splat", s);
  }
  return cudaGetLastError();
}

cudaError_t launch_shade_owned(const RenderArgs& a, cudaStream_t s) {
  const unsigned long long np = (unsigned long long)a.width * a.height;
  unsigned long long blocks = (np + 255) / 256;
  if (blocks > (unsigned long long)sm_count() * 32) blocks = (unsigned long long)sm_count() * 32;
  timing_begin("shade", s);
  shade_owned_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  timing_end("shade", s);
  return cudaGetLastError();
}

cudaError_t launch_render(const RenderArgs& a, cudaStream_t s) {
  const int grid = sm_count() * 8;
  if (a.n_max > 0) {
    timing_begin("splat", s);
    splat_kernel<<<splat_grid(a.n_max), 256, 0, s>>>(a);
    timing_end("splat", s);
  }
  const unsigned long long np = (unsigned long long)a.width * a.height;
  unsigned long long blocks = (np + 255) / 256;
  if (blocks > (unsigned long long)grid * 4) blocks = (unsigned long long)grid * 4;
  timing_begin("shade", s);
  shade_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  timing_end("shade", s);
  return cudaGetLastError();
}

}  // namespace fhv
