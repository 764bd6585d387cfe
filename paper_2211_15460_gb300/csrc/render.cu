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

namespace fhv {

__device__ __forceinline__ unsigned long long render_n(const RenderArgs& a) {
  unsigned long long n = a.n_max;
  if (a.d_n) {
    unsigned long long c = *a.d_n;
    n = c < n ? c : n;
  }
  return n;
}

__global__ void __launch_bounds__(256) splat_kernel(RenderArgs a) {
  const unsigned long long n = render_n(a);
  const float cell = fmul(a.cube_side, 1.0f / 2097152.0f);
  const float inv_pitch = fdiv(1.0f, a.pitch);
  const float hw = fmul(0.5f, (float)a.width), hh = fmul(0.5f, (float)a.height);
  const float qscale = fdiv(16777216.0f, fsub(a.z1, a.z0));
  const float half = fmul(0.5f, (float)(a.k - 1));
  const int W = a.width, H = a.height, k = a.k;
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    const uint4 r = __ldcs(reinterpret_cast<const uint4*>(a.rec) + i);
    const unsigned long long key = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
    const uint32_t q[3] = {compact3(key >> 2), compact3(key >> 1), compact3(key)};
    float p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = fadd(a.cube_min[c], fmul(fadd((float)q[c], 0.5f), cell));
    const float dx = fsub(p[0], a.origin[0]), dy = fsub(p[1], a.origin[1]), dz = fsub(p[2], a.origin[2]);
    const float sx = fadd(fmul(dot3(dx, dy, dz, a.right[0], a.right[1], a.right[2]), inv_pitch), hw);
    const float sy = fadd(fmul(dot3(dx, dy, dz, a.up[0], a.up[1], a.up[2]), inv_pitch), hh);
    const float z = dot3(dx, dy, dz, a.fwd[0], a.fwd[1], a.fwd[2]);
    const float fz = floorf(fmul(fsub(z, a.z0), qscale));
    uint32_t qd;
    if (!(fz >= 0.0f)) qd = 0u;
    else if (fz >= 16777215.0f) qd = (1u << 24) - 1u;
    else qd = (uint32_t)fz;
    const float fx = fminf(fmaxf(floorf(fsub(sx, half)), -1073741824.0f), 1073741824.0f);
    const float fy = fminf(fmaxf(floorf(fsub(sy, half)), -1073741824.0f), 1073741824.0f);
    const int ax = (int)fx, ay = (int)fy;
    const unsigned long long v = ((unsigned long long)qd << kIdxBits) | i;
    for (int b = 0; b < k; ++b) {
      const int y = ay + b;
      if (y < 0 || y >= H) continue;
      for (int c = 0; c < k; ++c) {
        const int x = ax + c;
        if (x < 0 || x >= W) continue;
        unsigned long long* px = a.vis + (unsigned long long)y * W + x;
        if (*((volatile unsigned long long*)px) > v) atomicMin(px, v);
      }
    }
  }
}

__global__ void __launch_bounds__(256) shade_kernel(RenderArgs a) {
  __shared__ float s_l[64 * 8];
  for (int i = threadIdx.x; i < a.n_lights * 8; i += blockDim.x) s_l[i] = a.lights[i];
  __syncthreads();
  const unsigned long long np = (unsigned long long)a.width * a.height;
  const float cell = a.cube_side * (1.0f / 2097152.0f);
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += step) {
    const unsigned long long v = a.vis[p];
    float4 out = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (v != kVisEmpty) {
      const uint4 r = reinterpret_cast<const uint4*>(a.rec)[v & kIdxMask];
      const unsigned long long key = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
      float pos[3];
      pos[0] = a.cube_min[0] + ((float)compact3(key >> 2) + 0.5f) * cell;
      pos[1] = a.cube_min[1] + ((float)compact3(key >> 1) + 0.5f) * cell;
      pos[2] = a.cube_min[2] + ((float)compact3(key) + 0.5f) * cell;
      float nx, ny, nz;
      oct_decode(r.w, nx, ny, nz);
      const uint32_t m = a.tri_material[r.z];
      float acc_r = 0.0f, acc_g = 0.0f, acc_b = 0.0f;
      for (int l = 0; l < a.n_lights; ++l) {
        const float* L = s_l + 8 * l;
        float dx = L[1], dy = L[2], dz = L[3];
        if (L[0] != 0.0f) {
          dx -= pos[0];
          dy -= pos[1];
          dz -= pos[2];
        }
        const float len2 = dx * dx + dy * dy + dz * dz;
        if (!(len2 > 0.0f)) continue;
        const float ndl = fmaxf(0.0f, (nx * dx + ny * dy + nz * dz) * rsqrtf(len2));
        acc_r += L[4] * ndl;
        acc_g += L[5] * ndl;
        acc_b += L[6] * ndl;
      }
      out = make_float4(a.albedo[3 * m] * acc_r, a.albedo[3 * m + 1] * acc_g, a.albedo[3 * m + 2] * acc_b, 1.0f);
    }
    reinterpret_cast<float4*>(a.rgba)[p] = out;
  }
}

cudaError_t launch_render(const RenderArgs& a, cudaStream_t s) {
  const int grid = sm_count() * 8;
  if (a.n_max > 0) {
    timing_begin("splat", s);
    splat_kernel<<<grid, 256, 0, s>>>(a);
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
