// splat.cuh -- per-fragment splatting and per-pixel shading (Section 3.3,
// Section 5), shared by the single-view and the batched renderers so that
// both produce identical bits.
#pragma once

#include "fhv_device.cuh"

namespace fhv {

// Orthographic view as the splat needs it, derived once per kernel/view
// with the float32 contract (every operation rounded on its own). Laid out
// as seven 16-byte groups, the projection's first, so that a copy held in
// shared memory is read back with vector loads (load_view).
struct __align__(16) SplatView {
  float o[3], inv_pitch;
  float r[3], hw;
  float u[3], hh;
  float f[3], z0;
  float qscale, half;
  int W, H;
  unsigned long long* vis;
  int k;
  float cell;
  float cmin[3], pad;
};
static_assert(sizeof(SplatView) == 112, "seven 16-byte groups");

// A SplatView read from (shared) memory in 16-byte loads; groups whose
// fields go unused are not loaded.
__device__ __forceinline__ SplatView load_view(const SplatView* p) {
  const float4* q = reinterpret_cast<const float4*>(p);
  SplatView v;
  const float4 a = q[0], b = q[1], c = q[2], d = q[3], e = q[4], h = q[6];
  const uint4 g = reinterpret_cast<const uint4*>(p)[5];
  v.o[0] = a.x, v.o[1] = a.y, v.o[2] = a.z, v.inv_pitch = a.w;
  v.r[0] = b.x, v.r[1] = b.y, v.r[2] = b.z, v.hw = b.w;
  v.u[0] = c.x, v.u[1] = c.y, v.u[2] = c.z, v.hh = c.w;
  v.f[0] = d.x, v.f[1] = d.y, v.f[2] = d.z, v.z0 = d.w;
  v.qscale = e.x, v.half = e.y, v.W = __float_as_int(e.z), v.H = __float_as_int(e.w);
  v.vis = reinterpret_cast<unsigned long long*>((unsigned long long)g.x | ((unsigned long long)g.y << 32));
  v.k = (int)g.z, v.cell = __uint_as_float(g.w);
  v.cmin[0] = h.x, v.cmin[1] = h.y, v.cmin[2] = h.z, v.pad = h.w;
  return v;
}

__device__ __forceinline__ SplatView make_splat_view(const float* cube_min, float cube_side, const float* origin,
                                                     const float* right, const float* up, const float* fwd,
                                                     float pitch, int W, int H, float z0, float z1, int k,
                                                     unsigned long long* vis) {
  SplatView v;
  for (int c = 0; c < 3; ++c) {
    v.cmin[c] = cube_min[c];
    v.o[c] = origin[c];
    v.r[c] = right[c];
    v.u[c] = up[c];
    v.f[c] = fwd[c];
  }
  v.cell = fmul(cube_side, 1.0f / 2097152.0f);
  v.inv_pitch = fdiv(1.0f, pitch);
  v.hw = fmul(0.5f, (float)W);
  v.hh = fmul(0.5f, (float)H);
  v.z0 = z0;
  v.qscale = fdiv(16777216.0f, fsub(z1, z0));
  v.half = fmul(0.5f, (float)(k - 1));
  v.W = W;
  v.H = H;
  v.k = k;
  v.vis = vis;
  v.pad = 0.0f;
  return v;
}

// Cell centre of a quantised position: cube_min + (q + 1/2) * cell.
__device__ __forceinline__ void dequantize(unsigned long long key, const SplatView& v, float p[3]) {
  const uint32_t q[3] = {compact3(key >> 2), compact3(key >> 1), compact3(key)};
#pragma unroll
  for (int c = 0; c < 3; ++c) p[c] = fadd(v.cmin[c], fmul(fadd((float)q[c], 0.5f), v.cell));
}

// Load of a visibility word for the "already nearer?" test. Keys only ever
// decrease while a view is splatted, so a value older than the current one
// is >= it: the test can only cause a redundant atomicMin, never a wrong
// skip. (Measured: a volatile load beats L1- or L2-cached loads here.)
__device__ __forceinline__ unsigned long long ld_vis(const unsigned long long* p) {
  return *((volatile const unsigned long long*)p);
}

// Projection of one fragment position: footprint anchor (ax, ay) =
// floor(s - (k-1)/2) per screen axis and the 24-bit quantised depth.
struct Projected {
  int ax, ay;
  uint32_t qd;
};

__device__ __forceinline__ Projected project_point(const float p[3], const SplatView& v) {
  const float dx = fsub(p[0], v.o[0]), dy = fsub(p[1], v.o[1]), dz = fsub(p[2], v.o[2]);
  const float sx = fadd(fmul(dot3(dx, dy, dz, v.r[0], v.r[1], v.r[2]), v.inv_pitch), v.hw);
  const float sy = fadd(fmul(dot3(dx, dy, dz, v.u[0], v.u[1], v.u[2]), v.inv_pitch), v.hh);
  const float z = dot3(dx, dy, dz, v.f[0], v.f[1], v.f[2]);
  const float fz = floorf(fmul(fsub(z, v.z0), v.qscale));
  Projected pr;
  if (!(fz >= 0.0f)) pr.qd = 0u;
  else if (fz >= 16777215.0f) pr.qd = (1u << 24) - 1u;
  else pr.qd = (uint32_t)fz;
  const float fx = fminf(fmaxf(floorf(fsub(sx, v.half)), -1073741824.0f), 1073741824.0f);
  const float fy = fminf(fmaxf(floorf(fsub(sy, v.half)), -1073741824.0f), 1073741824.0f);
  pr.ax = (int)fx;
  pr.ay = (int)fy;
  return pr;
}

// project_point for k = 1 (half = 0, so floor(sx - half) = floor(sx)),
// with the on-screen test made on the floored floats before any conversion
// (an integer-valued float in [0, W) converts to the same pixel as the
// clamped integer; NaN and far values fail both tests). False when off the
// screen.
__device__ __forceinline__ bool project_k1(const float p[3], const SplatView& v, uint32_t& ax, uint32_t& ay,
                                           uint32_t& qd) {
  const float dx = fsub(p[0], v.o[0]), dy = fsub(p[1], v.o[1]), dz = fsub(p[2], v.o[2]);
  const float sx = fadd(fmul(dot3(dx, dy, dz, v.r[0], v.r[1], v.r[2]), v.inv_pitch), v.hw);
  const float sy = fadd(fmul(dot3(dx, dy, dz, v.u[0], v.u[1], v.u[2]), v.inv_pitch), v.hh);
  const float fx = floorf(sx), fy = floorf(sy);
  if (!(fx >= 0.0f && fx < (float)v.W && fy >= 0.0f && fy < (float)v.H)) return false;
  const float z = dot3(dx, dy, dz, v.f[0], v.f[1], v.f[2]);
  const float fz = floorf(fmul(fsub(z, v.z0), v.qscale));
  qd = !(fz >= 0.0f) ? 0u : fz >= 16777215.0f ? (1u << 24) - 1u : (uint32_t)fz;
  ax = (uint32_t)fx;
  ay = (uint32_t)fy;
  return true;
}

// Project one fragment position and min-combine (qdepth << 40 | index) into
// its k x k footprint (k = 1: the pixel containing the projection). A load
// first skips the atomic when the pixel already holds a nearer fragment.
__device__ __forceinline__ void splat_point(const float p[3], unsigned long long index, const SplatView& v) {
  const Projected pr = project_point(p, v);
  const int ax = pr.ax, ay = pr.ay;
  const unsigned long long key = ((unsigned long long)pr.qd << kIdxBits) | index;
  if (v.k == 1) {
    if (ax >= 0 && ax < v.W && ay >= 0 && ay < v.H) {
      unsigned long long* px = v.vis + (unsigned long long)ay * v.W + ax;
      if (ld_vis(px) > key) atomicMin(px, key);
    }
    return;
  }
  for (int b = 0; b < v.k; ++b) {
    const int y = ay + b;
    if (y < 0 || y >= v.H) continue;
    for (int c = 0; c < v.k; ++c) {
      const int x = ax + c;
      if (x < 0 || x >= v.W) continue;
      unsigned long long* px = v.vis + (unsigned long long)y * v.W + x;
      if (ld_vis(px) > key) atomicMin(px, key);
    }
  }
}

// Colour of one pixel from its visibility word: albedo of the winner's
// material times the sum over lights of intensity * max(0, n . l); alpha 1;
// (0, 0, 0, 0) when nothing covers the pixel. Lights: 8 floats each
// {type, x, y, z, r, g, b, unused}, type 0 = direction, 1 = position.
__device__ __forceinline__ float4 shade_pixel(unsigned long long v, const Rec* rec, const uint32_t* tri_material,
                                              const float* albedo, const float* cube_min, float cube_side,
                                              const float* lights, int n_lights) {
  if (v == kVisEmpty) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float cell = cube_side * (1.0f / 2097152.0f);
  const uint4 r = reinterpret_cast<const uint4*>(rec)[v & kIdxMask];
  const unsigned long long key = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
  float pos[3];
  pos[0] = cube_min[0] + ((float)compact3(key >> 2) + 0.5f) * cell;
  pos[1] = cube_min[1] + ((float)compact3(key >> 1) + 0.5f) * cell;
  pos[2] = cube_min[2] + ((float)compact3(key) + 0.5f) * cell;
  float nx, ny, nz;
  oct_decode(r.w, nx, ny, nz);
  const uint32_t m = tri_material[r.z];
  float acc_r = 0.0f, acc_g = 0.0f, acc_b = 0.0f;
  for (int l = 0; l < n_lights; ++l) {
    const float* L = lights + 8 * l;
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
  return make_float4(albedo[3 * m] * acc_r, albedo[3 * m + 1] * acc_g, albedo[3 * m + 2] * acc_b, 1.0f);
}

}  // namespace fhv
