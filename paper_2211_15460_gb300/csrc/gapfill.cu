// gapfill.cu -- inputs, loss and optimiser of the learned gap-filler (no
// counterpart in the paper; see conv.cu).
//
//  * features: per pixel of a 1 x 1 splat, 8 BF16 channels: shaded RGB,
//    quantised depth / 2^24, coverage (1 where a fragment won, else 0), the
//    winner's normal projected on the camera's right and up axes, and 0;
//  * loss: squared error of the network's first three output channels, plus
//    the splat's RGB when a base is given (the network predicts a residual),
//    against the target RGB, summed in double, and its gradient
//    grad_scale * (out + base - target) as BF16 (other channels 0);
//  * compose: the final image, RGB = out + base, alpha 1;
//  * Adam on FP32 master parameters (bias-corrected moments), writing the
//    BF16 copy the convolutions read and clearing the gradient.
#include "kernels.h"

namespace fhv {

__global__ void splat_features_kernel(const unsigned long long* vis, const float4* rgba, const Rec* rec, float r0,
                                      float r1, float r2, float u0, float u1, float u2, long long pixels,
                                      __nv_bfloat16* feat) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < pixels;
       p += (long long)gridDim.x * blockDim.x) {
    const unsigned long long v = vis[p];
    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (v != kVisEmpty) {
      const float4 c = rgba[p];
      const uint4 r = reinterpret_cast<const uint4*>(rec)[v & kIdxMask];
      float nx, ny, nz;
      oct_decode(r.w, nx, ny, nz);
      f[0] = c.x;
      f[1] = c.y;
      f[2] = c.z;
      f[3] = (float)(v >> kIdxBits) * (1.0f / 16777216.0f);
      f[4] = 1.0f;
      f[5] = nx * r0 + ny * r1 + nz * r2;
      f[6] = nx * u0 + ny * u1 + nz * u2;
    }
    __nv_bfloat162 o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    reinterpret_cast<uint4*>(feat)[p] = *reinterpret_cast<const uint4*>(o);
  }
}

__device__ __forceinline__ void base_rgb(const __nv_bfloat16* base, long long p, float& b0, float& b1, float& b2) {
  b0 = b1 = b2 = 0.0f;
  if (base) {
    const uint2 v = reinterpret_cast<const uint2*>(base)[2 * p];  // channels 0..3 of 8
    b0 = __uint_as_float(v.x << 16);
    b1 = __uint_as_float(v.x & 0xFFFF0000u);
    b2 = __uint_as_float(v.y << 16);
  }
}

__global__ void gapfill_loss_kernel(const __nv_bfloat16* out, const __nv_bfloat16* base, const float4* target,
                                    long long pixels, float gscale, double* loss_sum, __nv_bfloat16* grad) {
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < pixels;
       p += (long long)gridDim.x * blockDim.x) {
    const uint4 o = reinterpret_cast<const uint4*>(out)[2 * p];  // channels 0..7 of 16
    const float4 t = target[p];
    const float o0 = __uint_as_float(o.x << 16), o1 = __uint_as_float(o.x & 0xFFFF0000u),
                o2 = __uint_as_float(o.y << 16);
    float b0, b1, b2;
    base_rgb(base, p, b0, b1, b2);
    const float d0 = (o0 + b0) - t.x, d1 = (o1 + b1) - t.y, d2 = (o2 + b2) - t.z;
    acc += (double)d0 * d0 + (double)d1 * d1 + (double)d2 * d2;
    if (grad) {
      const __nv_bfloat162 g01 = __floats2bfloat162_rn(gscale * d0, gscale * d1);
      const __nv_bfloat162 g2 = __floats2bfloat162_rn(gscale * d2, 0.0f);
      uint4 w0;
      w0.x = *reinterpret_cast<const uint32_t*>(&g01);
      w0.y = *reinterpret_cast<const uint32_t*>(&g2);
      w0.z = 0u;
      w0.w = 0u;
      reinterpret_cast<uint4*>(grad)[2 * p] = w0;
      reinterpret_cast<uint4*>(grad)[2 * p + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(~0u, acc, o);
  if ((threadIdx.x & 31) == 0 && loss_sum) atomicAdd(loss_sum, acc);
}

__global__ void gapfill_compose_kernel(const __nv_bfloat16* out, const __nv_bfloat16* base, long long pixels,
                                       float4* rgba) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < pixels;
       p += (long long)gridDim.x * blockDim.x) {
    const uint4 o = reinterpret_cast<const uint4*>(out)[2 * p];
    float b0, b1, b2;
    base_rgb(base, p, b0, b1, b2);
    rgba[p] = make_float4(__uint_as_float(o.x << 16) + b0, __uint_as_float(o.x & 0xFFFF0000u) + b1,
                          __uint_as_float(o.y << 16) + b2, 1.0f);
  }
}

__global__ void adam_kernel(float* param, float* grad, float* m, float* v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2, __nv_bfloat16* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float p = param[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    param[i] = p;
    grad[i] = 0.0f;
    if (out) out[i] = __float2bfloat16_rn(p);
  }
}

cudaError_t launch_splat_features(const unsigned long long* vis, const float4* rgba, const Rec* rec,
                                  const float* right, const float* up, long long pixels, __nv_bfloat16* feat,
                                  cudaStream_t s) {
  const long long blocks = std::min<long long>((pixels + 255) / 256, (long long)sm_count() * 16);
  if (blocks > 0)
    splat_features_kernel<<<(unsigned)blocks, 256, 0, s>>>(vis, rgba, rec, right[0], right[1], right[2], up[0], up[1],
                                                          up[2], pixels, feat);
  return cudaGetLastError();
}

cudaError_t launch_gapfill_loss(const __nv_bfloat16* out, const __nv_bfloat16* base, const float4* target,
                                long long pixels, float grad_scale, double* loss_sum, __nv_bfloat16* grad,
                                cudaStream_t s) {
  const long long blocks = std::min<long long>((pixels + 255) / 256, (long long)sm_count() * 16);
  if (blocks > 0) {
    timing_begin("gapfill_loss", s);
    gapfill_loss_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, base, target, pixels, grad_scale, loss_sum, grad);
    timing_end("gapfill_loss", s);
  }
  return cudaGetLastError();
}

cudaError_t launch_gapfill_compose(const __nv_bfloat16* out, const __nv_bfloat16* base, long long pixels,
                                   float4* rgba, cudaStream_t s) {
  const long long blocks = std::min<long long>((pixels + 255) / 256, (long long)sm_count() * 16);
  if (blocks > 0) gapfill_compose_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, base, pixels, rgba);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* param, float* grad, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, int step, __nv_bfloat16* out_bf16, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  const long long blocks = std::min<long long>((n + 255) / 256, (long long)sm_count() * 4);
  if (blocks > 0) adam_kernel<<<(unsigned)blocks, 256, 0, s>>>(param, grad, m, v, n, lr, b1, b2, eps, c1, c2, out_bf16);
  return cudaGetLastError();
}

}  // namespace fhv
