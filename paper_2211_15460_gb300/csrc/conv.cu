// conv.cu -- 3x3 convolutions of the learned gap-filler on the fifth-
// generation tensor cores (tcgen05): BF16 operands in shared memory, FP32
// accumulators in tensor memory. No counterpart in the paper: the network
// stands in for part of the novel-view reconstruction (filling the holes of
// sparse splats, Section 3.3's undersampling remark).
//
// Activations are NHWC BF16 with C in {8, 16, 32}; weights are
// [cout][ky][kx][cin] BF16 (a K-major operand: row = output channel,
// K = (ky * 3 + kx) * cin + c); zero padding outside the image.
//
// Forward (implicit GEMM, D[128 pixels][cout] = A[128][9 cin] * W^T): a tile
// is 128 consecutive pixels of one output row. Input rows are staged as
// [channel chunk of 8][pixel x0-1 .. x0+128][16 bytes]; inside a chunk the
// pixels are 16 bytes apart, so the A operand of tap (ky, kx) is the staged
// row y+ky-1 read from a start shifted by kx pixels: the nine taps cost no
// copies. A persistent CTA walks down a run of rows of one 128-pixel column
// with a ring of six staged rows (each output row stages one new input row)
// and two 128 x cout TMEM accumulators, its warps specialised: a producer
// warp stages rows, one lane issues the 6-9-18 MMAs (K = 16 each) of a row,
// four epilogue warps (one per TMEM lane quarter) apply bias, ReLU and an
// optional mask (x 1[mask > 0], the ReLU derivative of the backward pass) and
// store 32 or 64 bytes per pixel; mbarriers hand rows and accumulators
// between them.
// Weight gradient (D[128 rows of (tap, cin)][cout] = sum over pixels of
// X(pixel + tap)[cin] * dY(pixel)[cout]): both operands are MN-major -- a
// 16-byte core-matrix row holds 8 consecutive channels of one pixel, exactly
// an NHWC chunk -- so each K stage of 64 pixels is gathered by plain 16-byte
// async copies (each thread computes its pixel's coordinates once per stage),
// by producer warps that run ahead of the MMA lane through a ring of three
// stages (mbarrier hand-offs). A CTA reduces a range of pixels in
// TMEM and adds its partial sums to the FP32 gradient with atomics. One
// spare row of the last row tile holds ones, which yields the bias gradient
// sum over pixels of dY in the same MMAs.
#include "kernels.h"
#include "tc.cuh"

namespace fhv {

namespace {

constexpr int kHaloW = 130;  // staged pixels per input row: x0 - 1 .. x0 + 128
// MMAs (K = 16) of one forward tile: 9 taps x cin / 16, or for cin = 8 two
// taps per MMA within one kernel row (3 rows x 2 MMAs, the last of each row
// half zero)
template <int CIN>
constexpr int kFwdMmas = CIN == 8 ? 6 : 9 * CIN / 16;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

}  // namespace

// Forward: the roles are split over warps and handed over through mbarriers
// (no CTA-wide barrier per row):
//   warp 0       producer: stages input rows into a ring with async copies,
//                each slot signalled full when its copies land;
//   warp 1       MMA issuer (one lane): waits for the three rows of an output
//                row and a free accumulator, issues the row's MMAs, commits
//                "accumulator full" and frees the ring slot it no longer needs;
//   warps 2 - 5  epilogue, one per TMEM lane quarter: drain an accumulator,
//                free it, then bias, ReLU, mask and store.
constexpr int kWsWarps = 6;
constexpr int kWsRing = 6;

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWsWarps * 32) conv_fwd_ws_kernel(const __grid_constant__ ConvArgs a) {
  constexpr int CH = CIN / 8;
  constexpr int ROW_BYTES = CH * kHaloW * 16;
  constexpr int RING = kWsRing;
  constexpr int STAGE_PAD = (RING * ROW_BYTES + 1024 + 1023) & ~1023;
  constexpr int NMMA = kFwdMmas<CIN>;
  constexpr int NT = kWsWarps * 32;
  constexpr uint32_t IDESC = tc::idesc_bf16(128, COUT, false, false);
  extern __shared__ __align__(1024) unsigned char conv_smem[];
  unsigned char* sX = conv_smem;
  unsigned char* sW = conv_smem + STAGE_PAD;
  __shared__ __align__(8) uint64_t full[RING], empty[RING], accf[2], acce[2], done;
  __shared__ uint32_t tslot;
  __shared__ float s_bias[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the padded K chunk of cin = 8 reads a little past the ring: keep it finite
  for (int i = RING * ROW_BYTES / 16 + tid; i < STAGE_PAD / 16; i += NT)
    reinterpret_cast<uint4*>(sX)[i] = make_uint4(0u, 0u, 0u, 0u);
  // Weights: K chunk q = 2j + e of MMA j, rows = output channels. For cin >= 16
  // chunk q is (tap q / CH, channels 8 (q % CH) ..); for cin = 8 MMA j covers
  // row ky = j / 2, taps kx = 2 (j % 2) and kx + 1 (zero when kx + 1 = 3), so
  // that no MMA spans two ring slots.
  for (int i = tid; i < 2 * NMMA * COUT; i += NT) {
    const int q = i / COUT, n = i % COUT;
    int tap, c8;
    bool ok = true;
    if (CH == 1) {
      const int j = q >> 1, kx = 2 * (j & 1) + (q & 1);
      ok = kx < 3;
      tap = (j >> 1) * 3 + kx;
      c8 = 0;
    } else {
      tap = q / CH;
      c8 = q % CH;
    }
    const uint32_t dst = tc::smem_addr(sW) + (uint32_t)(q * (COUT / 8) * 128 + (n >> 3) * 128 + (n & 7) * 16);
    tc::cp16(dst, ok ? (const void*)(a.weight + ((size_t)n * 9 + tap) * CIN + c8 * 8) : (const void*)a.weight,
             ok ? 16u : 0u);
  }
  tc::cp_commit();
  if (tid < 32) s_bias[tid] = (a.bias && tid < COUT) ? a.bias[tid] : 0.0f;
  if (warp == 0) tc::tmem_alloc(&tslot, 64);
  if (tid == 0) {
    for (int i = 0; i < RING; ++i) {
      tc::mbar_init(&full[i], 32);  // one arrival per producer lane
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&accf[i], 1);
      tc::mbar_init(&acce[i], 4);  // one arrival per epilogue warp
    }
    tc::mbar_init(&done, 1);
  }
  tc::cp_wait<0>();
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;

  const int segs = (a.w + 127) >> 7;
  const int per_col = (a.h + a.rows_per_item - 1) / a.rows_per_item;
  const long long items = (long long)a.n * segs * per_col;
  auto item_of = [&](long long it, long long& img, int& x0, int& ya, int& yb) {
    const int chunk = (int)(it % per_col);
    const long long col = it / per_col;
    x0 = (int)(col % segs) * 128;
    img = col / segs;
    ya = chunk * a.rows_per_item;
    yb = min(a.h, ya + a.rows_per_item);
  };
  bool ok = true;

  if (warp == 0) {
    // ---- producer: rows ya - 1 .. yb of every item, in order, into the ring
    uint32_t n = 0;  // rows staged so far
    for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
      long long img;
      int x0, ya, yb;
      item_of(it, img, x0, ya, yb);
      for (int r = ya - 1; r <= yb; ++r, ++n) {
        const uint32_t slot = n % RING, use = n / RING;
        if (use > 0 && !tc::mbar_wait(&empty[slot], (use - 1) & 1u)) {
          ok = false;
          break;
        }
        const uint32_t base = tc::smem_addr(sX) + slot * ROW_BYTES;
        const bool row_ok = r >= 0 && r < a.h;
        for (int i = lane; i < CH * kHaloW; i += 32) {
          const int px = i % kHaloW, c8 = i / kHaloW;
          const int xx = x0 + px - 1;
          const bool in = row_ok && xx >= 0 && xx < a.w;
          const __nv_bfloat16* src = in ? a.x + (((size_t)img * a.h + r) * a.w + xx) * CIN + c8 * 8 : a.x;
          tc::cp16(base + (uint32_t)((c8 * kHaloW + px) * 16), src, in ? 16u : 0u);
        }
        tc::cp_arrive_noinc(&full[slot]);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      uint32_t n = 0, acc = 0;  // ring rows consumed, accumulators filled
      for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
        long long img;
        int x0, ya, yb;
        item_of(it, img, x0, ya, yb);
        const uint32_t base = n;  // ring index of row ya - 1
        for (int i = 0; i < yb - ya && ok; ++i) {
          for (uint32_t q = (i == 0 ? base : base + i + 2); q <= base + i + 2; ++q)
            if (!tc::mbar_wait(&full[q % RING], (q / RING) & 1u)) ok = false;
          const uint32_t b = acc & 1u, use = acc >> 1;
          if (ok && use > 0 && !tc::mbar_wait(&acce[b], (use - 1) & 1u)) ok = false;
          if (!ok) break;
          tc::fence_async_smem();  // the rows' async copies, seen through the barrier, to the tensor cores
          tc::fence_after();
          const uint32_t xs = tc::smem_addr(sX), ws = tc::smem_addr(sW);
#pragma unroll
          for (int j = 0; j < NMMA; ++j) {
            uint32_t o0, lbo;
            if (CH == 1) {
              const int ky = j >> 1, kx = 2 * (j & 1);
              o0 = (uint32_t)((((base + i + ky) % RING) * kHaloW + kx) * 16);
              lbo = 16u;
            } else {
              const int qq = 2 * j, t = qq / CH, c = qq % CH, ky = t / 3, kx = t % 3;
              o0 = (uint32_t)(((((base + i + ky) % RING) * CH + c) * kHaloW + kx) * 16);
              lbo = (uint32_t)(kHaloW * 16);
            }
            const uint64_t ad = tc::smem_desc(xs + o0, lbo, 128);
            const uint64_t bd = tc::smem_desc(ws + (uint32_t)(j * 2 * (COUT / 8) * 128), (COUT / 8) * 128, 128);
            tc::mma_bf16(tmem + 32u * b, ad, bd, IDESC, j > 0);
          }
          tc::commit(&accf[b]);
          tc::commit(&empty[(base + i) % RING]);  // row y - 1: this was its last reader
          if (i == yb - ya - 1) {                 // the item's last rows
            tc::commit(&empty[(base + i + 1) % RING]);
            tc::commit(&empty[(base + i + 2) % RING]);
          }
          ++acc;
        }
        n = base + (uint32_t)(yb - ya + 2);
      }
      tc::commit(&done);
      tc::mbar_wait(&done, 0);  // every MMA complete before the teardown
    }
  } else {
    // ---- epilogue: warp quarter q reads TMEM lanes 32 q ..
    const int quarter = warp & 3;
    uint32_t acc = 0;
    for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
      long long img;
      int x0, ya, yb;
      item_of(it, img, x0, ya, yb);
      for (int y = ya; y < yb; ++y, ++acc) {
        const uint32_t b = acc & 1u, use = acc >> 1;
        if (!tc::mbar_wait(&accf[b], use & 1u)) {
          ok = false;
          break;
        }
        tc::fence_after();
        float v[COUT];
        {
          const uint32_t ta = tmem + 32u * b + ((uint32_t)(quarter * 32) << 16);
          if constexpr (COUT == 32) {
            uint32_t r[32];
            tc::tmem_ld32(ta, r);
            tc::tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
          } else {
            uint32_t r[16];
            tc::tmem_ld16(ta, r);
            tc::tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
          }
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acce[b]);
        const int x = x0 + quarter * 32 + lane;
        if (x < a.w) {
          const size_t p = ((size_t)img * a.h + y) * a.w + x;
#pragma unroll
          for (int c = 0; c < COUT; ++c) {
            v[c] += s_bias[c];
            if (a.relu) v[c] = fmaxf(v[c], 0.0f);
          }
          if (a.mask) {
            const uint4* mk = reinterpret_cast<const uint4*>(a.mask + p * COUT);
#pragma unroll
            for (int q = 0; q < COUT / 8; ++q) {
              const uint4 m = __ldg(mk + q);
              const uint32_t mw[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                if (!(bf16_lo(mw[e]) > 0.0f)) v[8 * q + 2 * e] = 0.0f;
                if (!(bf16_hi(mw[e]) > 0.0f)) v[8 * q + 2 * e + 1] = 0.0f;
              }
            }
          }
          uint4* dst = reinterpret_cast<uint4*>(a.y + p * COUT);
#pragma unroll
          for (int q = 0; q < COUT / 8; ++q)
            dst[q] = make_uint4(pack_bf16x2(v[8 * q], v[8 * q + 1]), pack_bf16x2(v[8 * q + 2], v[8 * q + 3]),
                                pack_bf16x2(v[8 * q + 4], v[8 * q + 5]), pack_bf16x2(v[8 * q + 6], v[8 * q + 7]));
        }
      }
    }
  }
  if (!ok && lane == 0) set_status(&a.hdr->status, FHV_DEV_TIMEOUT);
  tc::cp_wait<0>();
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 64);
}

// Weight gradient; see the file comment. Grid: (row tiles, pixel ranges).
// Warps 0 - 3 gather 64-pixel stages into a ring (each thread one pixel, its
// coordinates computed once per stage) and signal a stage full when its
// copies land; warp 4's first lane issues each stage's four MMAs and frees
// the stage when they complete. At the end warps 0 - 3 (one per TMEM lane
// quarter) read the accumulators and add them to the gradients.
constexpr int kWgProducers = 128;  // gathering threads (4 warps)
constexpr int kWgRing = 3;         // stages in flight

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWgProducers + 32) conv_wgrad_kernel(const __grid_constant__ ConvArgs a) {
  constexpr int ROWS = 9 * CIN;                 // (tap, cin) rows; row ROWS is the ones row
  constexpr int KS = 64;                        // pixels per stage
  constexpr int A_BYTES = 16 * (KS / 8) * 128;  // 128 rows x 64 pixels
  constexpr int B_BYTES = (COUT / 8) * (KS / 8) * 128;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr int NST = kWgRing;
  constexpr uint32_t IDESC = tc::idesc_bf16(128, COUT, true, true);
  extern __shared__ __align__(1024) unsigned char conv_smem[];
  __shared__ __align__(8) uint64_t full[NST], empty[NST], done;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row0 = blockIdx.x * 128;  // first (tap, cin) row of this tile
  const long long P = (long long)a.n * a.h * a.w;
  const long long p_beg = (long long)blockIdx.y * a.pixels_per_cta;
  const long long p_end = min(P, p_beg + a.pixels_per_cta);
  const int nst = (int)((p_end - p_beg + KS - 1) / KS);
  // The A tile of one stage: core matrix (row group g, pixel group q) at
  // q * 2048 + g * 128, row = pixel % 8 (16 bytes = 8 channels). The ones
  // row (ROWS, if it falls in this tile) gives the bias gradient.
  const int ones_g = (ROWS - row0) >= 0 && (ROWS - row0) < 128 ? (ROWS - row0) >> 3 : -1;
  // Rows past ROWS are set once per buffer and never gathered: the ones row
  // is 1 for every pixel (pixels past the range have dY = 0), the rest 0.
  for (int st = 0; st < NST; ++st) {
    unsigned char* sa = conv_smem + st * STAGE;
    for (int i = tid; i < 16 * KS; i += blockDim.x) {
      const int k = i % KS, g = i / KS;
      if (row0 + 8 * g < ROWS) continue;
      uint4 z = make_uint4(0u, 0u, 0u, 0u);
      if (g == ones_g) z.x = 0x3F80u;  // bf16 1.0 in element 0 (row ROWS), 0 in rows ROWS + 1 ..
      *reinterpret_cast<uint4*>(sa + (k >> 3) * 2048 + g * 128 + (k & 7) * 16) = z;
    }
  }
  if (warp == 0) tc::tmem_alloc(&tslot, 32);
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      tc::mbar_init(&full[i], kWgProducers);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(&done, 1);
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  bool ok = true;

  if (tid < kWgProducers) {
    // ---- gather: thread t takes pixel k = t % 64 and every other row group
    const int k = tid & (KS - 1), g0 = tid / KS;
    for (int st = 0; st < nst; ++st) {
      const int b = st % NST;
      if (st >= NST && !tc::mbar_wait(&empty[b], ((st / NST) - 1) & 1)) {
        ok = false;
        break;
      }
      unsigned char* sa = conv_smem + b * STAGE;
      unsigned char* sb = sa + A_BYTES;
      const long long p = p_beg + (long long)st * KS + k;
      const bool valid = p < p_end;
      int x = 0, y = 0;
      long long img = 0;
      if (valid) {
        const long long r2 = p / a.w;
        x = (int)(p - r2 * a.w);
        img = r2 / a.h;
        y = (int)(r2 - img * a.h);
      }
      const uint32_t arow = tc::smem_addr(sa) + (uint32_t)((k >> 3) * 2048 + (k & 7) * 16);
#pragma unroll
      for (int g = g0; g < 16; g += kWgProducers / KS) {
        const int row = row0 + 8 * g;
        if (row >= ROWS) continue;
        const int tap = row / CIN, c8 = (row % CIN) >> 3;
        const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
        const bool in = valid && yy >= 0 && yy < a.h && xx >= 0 && xx < a.w;
        const __nv_bfloat16* src = in ? a.x + (((size_t)img * a.h + yy) * a.w + xx) * CIN + c8 * 8 : a.x;
        tc::cp16(arow + (uint32_t)(g * 128), src, in ? 16u : 0u);
      }
      const uint32_t brow = tc::smem_addr(sb) + (uint32_t)((k >> 3) * ((COUT / 8) * 128) + (k & 7) * 16);
#pragma unroll
      for (int g = g0; g < COUT / 8; g += kWgProducers / KS) {
        const __nv_bfloat16* src = valid ? a.dy + (size_t)p * COUT + g * 8 : a.dy;
        tc::cp16(brow + (uint32_t)(g * 128), src, valid ? 16u : 0u);
      }
      tc::cp_arrive_noinc(&full[b]);
    }
  } else if (tid == kWgProducers) {
    // ---- MMA issuer
    for (int st = 0; st < nst; ++st) {
      const int b = st % NST;
      if (!tc::mbar_wait(&full[b], (st / NST) & 1)) {
        ok = false;
        break;
      }
      tc::fence_async_smem();
      tc::fence_after();
      const uint32_t sa = tc::smem_addr(conv_smem + b * STAGE), sb = sa + A_BYTES;
#pragma unroll
      for (int j = 0; j < KS / 16; ++j) {
        const uint64_t ad = tc::smem_desc(sa + j * 2 * 2048, 2048, 128);
        const uint64_t bd = tc::smem_desc(sb + j * 2 * (COUT / 8) * 128, (COUT / 8) * 128, 128);
        tc::mma_bf16(tmem, ad, bd, IDESC, st > 0 || j > 0);
      }
      tc::commit(&empty[b]);
    }
    tc::commit(&done);
  }
  // ---- accumulators to the gradients (warps 0 - 3, one per lane quarter)
  if (tid < kWgProducers) {
    const bool fin = tc::mbar_wait(&done, 0);
    if (ok && fin && nst > 0) {
      tc::fence_after();
      uint32_t r[32];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
      if constexpr (COUT == 32) {
        tc::tmem_ld32(ta, r);
      } else {
        uint32_t r16[16];
        tc::tmem_ld16(ta, r16);
#pragma unroll
        for (int c = 0; c < 16; ++c) r[c] = r16[c];
      }
      tc::tmem_wait_ld();
      const int row = row0 + tid;
      if (row < ROWS) {
        const int tap = row / CIN, ci = row % CIN;
#pragma unroll
        for (int c = 0; c < COUT; ++c)
          atomicAdd(a.dweight + ((size_t)c * 9 + tap) * CIN + ci, __uint_as_float(r[c]));
      } else if (row == ROWS && a.dbias) {
#pragma unroll
        for (int c = 0; c < COUT; ++c) atomicAdd(a.dbias + c, __uint_as_float(r[c]));
      }
    }
    if (!fin) ok = false;
  }
  if (!ok) set_status(&a.hdr->status, FHV_DEV_TIMEOUT);
  tc::cp_wait<0>();
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 32);
}

// Flipped, transposed weights for the backward data pass:
// out[cin][ky][kx][cout] = w[cout][2 - ky][2 - kx][cin].
__global__ void conv_flip_kernel(const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* out) {
  const int n = 9 * cin * cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int co = i % cout, tap = (i / cout) % 9, ci = i / (cout * 9);
    out[i] = w[((size_t)co * 9 + (8 - tap)) * cin + ci];
  }
}

template <int CIN, int COUT>
static cudaError_t launch_fwd_t(ConvArgs a, cudaStream_t s) {
  constexpr int CH = CIN / 8;
  constexpr int STAGE_PAD = (kWsRing * CH * kHaloW * 16 + 1024 + 1023) & ~1023;
  const int smem = STAGE_PAD + 2 * kFwdMmas<CIN> * (COUT / 8) * 128;
  if (cudaFuncSetAttribute(conv_fwd_ws_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return cudaGetLastError();
  // CTAs per SM from the shared-memory budget (static part ~1.3 KB each),
  // at most 8 (8 x 64 TMEM columns); one run of rows per CTA
  int per_sm = (int)((227 * 1024) / (smem + 1408));
  per_sm = std::max(1, std::min(8, per_sm));
  const long long ctas = (long long)sm_count() * per_sm;
  const long long cols = (long long)a.n * ((a.w + 127) / 128);
  const long long per_col = std::max<long long>(1, std::min<long long>(a.h, ctas / std::max<long long>(1, cols)));
  a.rows_per_item = (int)((a.h + per_col - 1) / per_col);
  const long long items = cols * ((a.h + a.rows_per_item - 1) / a.rows_per_item);
  const long long grid = std::min<long long>(items, ctas);
  timing_begin("conv_fwd", s);
  conv_fwd_ws_kernel<CIN, COUT><<<(unsigned)grid, kWsWarps * 32, smem, s>>>(a);
  timing_end("conv_fwd", s);
  return cudaGetLastError();
}

template <int CIN, int COUT>
static cudaError_t launch_wgrad_t(ConvArgs a, cudaStream_t s) {
  constexpr int STAGE = 16 * 8 * 128 + (COUT / 8) * 8 * 128;
  const int smem = kWgRing * STAGE;
  if (cudaFuncSetAttribute(conv_wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return cudaGetLastError();
  const long long P = (long long)a.n * a.h * a.w;
  const int row_tiles = (9 * CIN + 1 + 127) / 128;
  // one wave: as many CTAs as are resident (shared-memory limit), pixel
  // ranges a multiple of 64
  const int per_sm = std::max(1, std::min(8, (227 * 1024) / (smem + 1280)));
  long long ranges = std::max<long long>(1, (long long)sm_count() * per_sm / row_tiles);
  long long per = (P + ranges - 1) / ranges;
  per = std::max<long long>(256, (per + 63) / 64 * 64);
  ranges = (P + per - 1) / per;
  a.pixels_per_cta = per;
  timing_begin("conv_wgrad", s);
  conv_wgrad_kernel<CIN, COUT><<<dim3((unsigned)row_tiles, (unsigned)ranges), kWgProducers + 32, smem, s>>>(a);
  timing_end("conv_wgrad", s);
  return cudaGetLastError();
}

cudaError_t launch_conv_fwd(const ConvArgs& a, cudaStream_t s) {
  if (a.cin == 8 && a.cout == 32) return launch_fwd_t<8, 32>(a, s);
  if (a.cin == 8 && a.cout == 16) return launch_fwd_t<8, 16>(a, s);
  if (a.cin == 16 && a.cout == 32) return launch_fwd_t<16, 32>(a, s);
  if (a.cin == 16 && a.cout == 16) return launch_fwd_t<16, 16>(a, s);
  if (a.cin == 32 && a.cout == 32) return launch_fwd_t<32, 32>(a, s);
  if (a.cin == 32 && a.cout == 16) return launch_fwd_t<32, 16>(a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_conv_wgrad(const ConvArgs& a, cudaStream_t s) {
  if (a.cin == 8 && a.cout == 32) return launch_wgrad_t<8, 32>(a, s);
  if (a.cin == 8 && a.cout == 16) return launch_wgrad_t<8, 16>(a, s);
  if (a.cin == 16 && a.cout == 32) return launch_wgrad_t<16, 32>(a, s);
  if (a.cin == 16 && a.cout == 16) return launch_wgrad_t<16, 16>(a, s);
  if (a.cin == 32 && a.cout == 32) return launch_wgrad_t<32, 32>(a, s);
  if (a.cin == 32 && a.cout == 16) return launch_wgrad_t<32, 16>(a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_conv_flip(const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* out, cudaStream_t s) {
  conv_flip_kernel<<<std::max(1, std::min(1024, (9 * cin * cout + 255) / 256)), 256, 0, s>>>(w, cin, cout, out);
  return cudaGetLastError();
}

}  // namespace fhv
