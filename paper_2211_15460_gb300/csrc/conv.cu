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
// Forward (implicit GEMM): a tile is 128 consecutive pixels of one output
// row, M = 128 pixels. Input rows are staged as [channel chunk of 8][pixel
// x0-1 .. x0+128][16 bytes] by tensor copies; inside a chunk the pixels are
// 16 bytes apart, so tap kx is the staged row read from a start shifted by kx
// pixels. Each staged row is multiplied once by the weights of all three
// kernel rows (N = 3 cout) into the accumulators of the three output rows it
// feeds, which sit in consecutive TMEM slots. A persistent CTA walks down a
// run of rows of one 128-pixel column with a ring of staged rows; a producer
// lane, an MMA lane and four epilogue warps (bias, ReLU, an optional mask
// x 1[mask > 0] -- the ReLU derivative of the backward pass --, 32 or 64
// bytes stored per pixel) hand rows and accumulators over through mbarriers.
// Weight gradient: the pixels of an output row segment are K; the three
// kernel rows share one MMA (M = 3 cout rows of dY against one staged input
// row), and the three kernel columns are shifted descriptor starts on that
// row, so every input and dY row is staged once. The accumulators stay in
// TMEM for the CTA's whole share of rows; a column of ones in the input
// operand gives the bias gradient.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "kernels.h"
#include "tc.cuh"

namespace fhv {

namespace {

constexpr int kHaloW = 130;  // staged pixels per input row: x0 - 1 .. x0 + 128
// pixel slots per staged channel chunk (kHaloW used): 2176 bytes keeps every
// tensor-copy target 128-byte aligned
constexpr int kChunk = 136;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

}  // namespace

// Forward. An input row r feeds three output rows: r + 1 through kernel row
// ky = 0, r through ky = 1 and r - 1 through ky = 2. So one MMA takes A = the
// staged row r at the kx shift (M = 128 pixels, K = 16 channels or, for
// cin = 8, two taps) and B = the weights of all three kernel rows side by
// side (N = 3 cout), and writes three output rows' accumulators at once: the
// accumulators are slots of cout TMEM columns, output row O in slot
// (-O) mod NA, so that rows O + 2, O + 1, O are consecutive slots (at the two
// wrap positions the MMA is split in two). Every staged row is read by one
// batch of MMAs (6 for cin = 32 instead of 18 with M = 128, N = cout).
// The MMAs always accumulate: the epilogue clears a slot (tcgen05.st of
// zeros) after draining it, and every slot is cleared at the start. A run of
// output rows [ya, yb) of one 128-pixel column stages input rows ya - 1 .. yb
// and passes through output rows ya - 2 .. yb + 1; the four outside the run
// collect partial sums that the epilogue drains and drops.
// Roles (mbarrier hand-offs, no CTA-wide barrier per row):
//   warp 0       lane 0 stages input rows into a ring with tensor copies;
//   warp 1       lane 0 issues the MMAs of each staged row, frees its ring
//                slot and signals every output row it completes;
//   warps 2 - 5  epilogue, one per TMEM lane quarter: drain a slot, clear it,
//                free it, then bias, ReLU, mask and store.
constexpr int kFwWarps = 6;
constexpr int kFwRing = 6;     // staged input rows
constexpr int kFwCols = 256;   // TMEM columns: 256 / cout accumulator slots

template <int CIN>
constexpr int kFwRowMmas = CIN == 8 ? 2 : 3 * CIN / 16;  // MMAs (K = 16) per staged row

template <int CIN, int COUT>
__global__ void __launch_bounds__(kFwWarps * 32)
    conv_fwd_kernel(const __grid_constant__ ConvArgs a, const __grid_constant__ CUtensorMap mx) {
  constexpr int CH = CIN / 8;
  constexpr int ROW_BYTES = CH * kChunk * 16;
  constexpr int RING = kFwRing;
  constexpr int STAGE_PAD = (RING * ROW_BYTES + 1024 + 1023) & ~1023;
  constexpr int J = kFwRowMmas<CIN>;
  constexpr int NA = kFwCols / COUT;    // accumulator slots
  constexpr int N3 = 3 * COUT;
  constexpr int WB = 2 * (N3 / 8) * 128;  // one MMA's B tile: 2 K chunks x N3 rows x 16 B
  constexpr int NT = kFwWarps * 32;
  static_assert(NA >= 4, "three slots per MMA and one more to drain");
  extern __shared__ __align__(1024) unsigned char conv_smem[];
  unsigned char* sX = conv_smem;
  unsigned char* sW = conv_smem + STAGE_PAD;
  __shared__ __align__(8) uint64_t full[RING], empty[RING], accf[NA], acce[NA], done;
  __shared__ uint32_t tslot;
  __shared__ float s_bias[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the zero-weight half of cin = 8's second MMA reads one pixel past the
  // halo, into the chunk's padding or past the ring: keep both finite (the
  // tensor copies never write them)
  for (int i = RING * ROW_BYTES / 16 + tid; i < STAGE_PAD / 16; i += NT)
    reinterpret_cast<uint4*>(sX)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < RING * CH * (kChunk - kHaloW); i += NT)
    reinterpret_cast<uint4*>(sX)[(i / (kChunk - kHaloW)) * kChunk + kHaloW + i % (kChunk - kHaloW)] =
        make_uint4(0u, 0u, 0u, 0u);
  // Weights: B tile of MMA j, K chunk q (0, 1), N row n = ky * cout + co. For
  // cin >= 16, MMA j is tap kx = j / (CH / 2) with channel chunks
  // 2 (j % (CH / 2)) + q; for cin = 8 it is taps kx = 2 j + q (zero when 3).
  for (int i = tid; i < J * 2 * N3; i += NT) {
    const int j = i / (2 * N3), q = (i / N3) & 1, n = i % N3;
    const int ky = n / COUT, co = n % COUT;
    int kx, c8;
    bool ok = true;
    if constexpr (CH == 1) {
      kx = 2 * j + q;
      ok = kx < 3;
      c8 = 0;
    } else {
      kx = j / (CH / 2);
      c8 = 2 * (j % (CH / 2)) + q;
    }
    const uint32_t dst = tc::smem_addr(sW) + (uint32_t)(j * WB + q * (N3 / 8) * 128 + (n >> 3) * 128 + (n & 7) * 16);
    tc::cp16(dst, ok ? (const void*)(a.weight + ((size_t)co * 9 + ky * 3 + kx) * CIN + c8 * 8) : (const void*)a.weight,
             ok ? 16u : 0u);
  }
  tc::cp_commit();
  if (tid < 32) s_bias[tid] = (a.bias && tid < COUT) ? a.bias[tid] : 0.0f;
  if (warp == 0) tc::tmem_alloc(&tslot, kFwCols);
  if (tid == 0) {
    for (int i = 0; i < RING; ++i) {
      tc::mbar_init(&full[i], 1);  // the producer's expect-tx arrival
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < NA; ++i) {
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
  if (warp >= 2) {  // every slot starts cleared
    const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll
    for (int c = 0; c < kFwCols; c += 32) tc::tmem_zero32(tmem + lanes + (uint32_t)c);
    tc::tmem_wait_st();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();

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
  auto slot_of = [](uint32_t o) -> uint32_t { return (uint32_t)((NA - (int)(o % NA)) % NA); };
  bool ok = true;

  if (warp == 0) {
    // ---- producer (lane 0): rows ya - 1 .. yb of every item, in order, into
    // the ring, one tensor copy per 8-channel chunk (pixels and rows outside
    // the image come back as zeros)
    uint32_t n = 0;  // rows staged so far
    for (long long it = blockIdx.x; it < items && ok && lane == 0; it += gridDim.x) {
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
        tc::mbar_expect_tx(&full[slot], (uint32_t)(CH * kHaloW * 16));
        for (int c8 = 0; c8 < CH; ++c8)
          tc::tma_load_4d(base + c8 * (kChunk * 16), &mx, c8 * 8, x0 - 1, r, (int)img, &full[slot]);
      }
    }
    // every copy issued has landed before the CTA may leave (n = 0 on lanes 1..31)
    for (uint32_t sl = 0; sl < RING && sl < n; ++sl)
      if (!tc::mbar_wait(&full[sl], ((sl + ((n - 1 - sl) / RING) * RING) / RING) & 1u)) ok = false;
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      uint32_t n = 0, o0 = 0;  // rows consumed; first output row (a phantom) of the current item
      const uint32_t xs0 = tc::smem_addr(sX), ws = tc::smem_addr(sW);
      for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
        long long img;
        int x0, ya, yb;
        item_of(it, img, x0, ya, yb);
        const int len = yb - ya;
        for (int i = 0; i < len + 2 && ok; ++i) {
          const uint32_t q = n + (uint32_t)i;
          if (!tc::mbar_wait(&full[q % RING], (q / RING) & 1u)) {
            ok = false;
            break;
          }
          // this row writes output rows o0 + i + 2 (new), o0 + i + 1, o0 + i;
          // a new row's slot must have been drained and cleared
          for (uint32_t o = (i == 0 ? o0 : o0 + i + 2); o <= o0 + i + 2 && ok; ++o)
            if (o >= NA && !tc::mbar_wait(&acce[slot_of(o)], ((o / NA) - 1) & 1u)) ok = false;
          if (!ok) break;
          tc::fence_after();
          const uint32_t s0 = slot_of(o0 + i + 2), xs = xs0 + (q % RING) * ROW_BYTES;
#pragma unroll
          for (int j = 0; j < J; ++j) {
            uint32_t off, lbo;
            if constexpr (CH == 1) {
              off = (uint32_t)(2 * j * 16);
              lbo = 16u;
            } else {
              const int kx = j / (CH / 2), c = 2 * (j % (CH / 2));
              off = (uint32_t)((c * kChunk + kx) * 16);
              lbo = (uint32_t)(kChunk * 16);
            }
            const uint64_t ad = tc::smem_desc(xs + off, lbo, 128);
            const uint32_t wb = ws + (uint32_t)(j * WB);
            constexpr uint32_t KB = (N3 / 8) * 128;  // B: distance between K chunks
            constexpr uint32_t PART = (COUT / 8) * 128;  // B: one kernel row's N block
            if (s0 + 3 <= NA) {
              tc::mma_bf16(tmem + s0 * COUT, ad, tc::smem_desc(wb, KB, 128), tc::idesc_bf16(128, N3, false, false),
                           true);
            } else if (s0 == NA - 2) {
              tc::mma_bf16(tmem + s0 * COUT, ad, tc::smem_desc(wb, KB, 128),
                           tc::idesc_bf16(128, 2 * COUT, false, false), true);
              tc::mma_bf16(tmem, ad, tc::smem_desc(wb + 2 * PART, KB, 128), tc::idesc_bf16(128, COUT, false, false),
                           true);
            } else {
              tc::mma_bf16(tmem + s0 * COUT, ad, tc::smem_desc(wb, KB, 128), tc::idesc_bf16(128, COUT, false, false),
                           true);
              tc::mma_bf16(tmem, ad, tc::smem_desc(wb + PART, KB, 128), tc::idesc_bf16(128, 2 * COUT, false, false),
                           true);
            }
          }
          tc::commit(&empty[q % RING]);     // the staged row has no other reader
          tc::commit(&accf[slot_of(o0 + i)]);  // output row o0 + i is complete
          if (i == len + 1) {
            tc::commit(&accf[slot_of(o0 + len + 2)]);
            tc::commit(&accf[slot_of(o0 + len + 3)]);
          }
        }
        n += (uint32_t)(len + 2);
        o0 += (uint32_t)(len + 4);
      }
      tc::commit(&done);
      tc::mbar_wait(&done, 0);  // every MMA complete before the teardown
    }
  } else {
    // ---- epilogue: warp quarter q reads TMEM lanes 32 q ..
    const int quarter = warp & 3;
    const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
    uint32_t o = 0;
    for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
      long long img;
      int x0, ya, yb;
      item_of(it, img, x0, ya, yb);
      const int len = yb - ya;
      for (int k = 0; k < len + 4; ++k, ++o) {
        const uint32_t sl = slot_of(o);
        if (!tc::mbar_wait(&accf[sl], (o / NA) & 1u)) {
          ok = false;
          break;
        }
        tc::fence_after();
        float v[COUT];
        {
          const uint32_t ta = tmem + sl * COUT + lanes;
          if constexpr (COUT == 32) {
            uint32_t r[32];
            tc::tmem_ld32(ta, r);
            tc::tmem_wait_ld();
            tc::tmem_zero32(ta);
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
          } else {
            uint32_t r[16];
            tc::tmem_ld16(ta, r);
            tc::tmem_wait_ld();
            tc::tmem_zero16(ta);
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
          }
          tc::tmem_wait_st();
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acce[sl]);
        const int y = ya - 2 + k;
        const int x = x0 + quarter * 32 + lane;
        if (k >= 2 && k < len + 2 && x < a.w) {
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
  if (warp == 0) tc::tmem_free(tmem, kFwCols);
}

// Weight gradient. For a staged input row r and a shift kx, one MMA group
// computes D_kx[(2 - ky) * cout + co][ci] += sum over the 128 pixels p of an
// output row segment of dY[r + 1 - ky][p][co] * X[r][p + kx - 1][ci], for
// the three ky at once: A (M = 128, MN-major) is the window of dY rows r - 1,
// r, r + 1 read straight from a ring whose slots are consecutive in shared
// memory (two mirror slots after the last one keep every window contiguous;
// rows beyond 3 * cout read whatever follows and are never used), B
// (MN-major) is the staged input row read from a start shifted by kx pixels.
// Summed over the input rows, D_kx[(2 - ky) * cout + co][ci] is the weight
// gradient of tap (ky, kx). A run of output rows [ya, yb) of one column
// segment stages the input rows ya - 1 .. yb and the dY rows ya - 2 .. yb + 1
// with the four outside the run set to zero, so every dY row is counted once
// by each tap. A column of ones in the kx = 1 operand gives the bias
// gradient on the ky = 1 rows. The accumulators stay in TMEM for the CTA's
// whole range of rows and are added to the FP32 gradients at the end.
// Roles: one lane of warp 0 loads dY rows and one of warp 2 input rows with
// tensor (TMA) copies (one box of 8 channels x 128 or 130 pixels each; the
// halo, rows outside the image and the zero rows come back zero-filled),
// warp 1 lane 0 issues the MMAs; all four warps read TMEM out at the end and
// add to the gradients with 16-byte vector reductions.
constexpr int kWgX = 3;  // staged input rows
constexpr int kWgD = 5;  // staged dY rows (+ 2 mirror slots)

template <int CIN>
__host__ __device__ constexpr int kWgN(int kx) {  // N of shift kx: channels (+ zero, ones chunks for kx = 1), rounded to 16
  return ((((CIN / 8) + (kx == 1 ? 2 : 0)) * 8 + 15) / 16) * 16;
}
template <int CIN>
__host__ __device__ constexpr int kWgTmem() {  // TMEM columns allocated: a power of two >= 32
  int c = 32;
  while (c < kWgN<CIN>(0) + kWgN<CIN>(1) + kWgN<CIN>(2)) c *= 2;
  return c;
}
template <int CIN, int COUT>
struct WgradSmem {
  static constexpr int XROW = (CIN / 8 + 3) * kChunk * 16;  // one staged input row (+ zero, ones, zero chunks)
  static constexpr int DSLOT = (COUT / 8) * 128 * 16;        // one dY row segment
  static constexpr int DREAD = 16 * 128 * 16;                // what one A operand (M = 128) spans
  static constexpr int D_BYTES =
      (kWgD + 2) * DSLOT > (kWgD - 1) * DSLOT + DREAD ? (kWgD + 2) * DSLOT : (kWgD - 1) * DSLOT + DREAD;
  static constexpr int BYTES = D_BYTES + kWgX * XROW;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
    conv_wgrad_kernel(const __grid_constant__ ConvArgs a, const __grid_constant__ CUtensorMap mx,
                      const __grid_constant__ CUtensorMap mdy) {
  using L = WgradSmem<CIN, COUT>;
  constexpr int CH = CIN / 8;
  constexpr int NCOL = kWgTmem<CIN>();
  static_assert(3 * COUT <= 128, "three dY rows must fit the 128 accumulator rows");
  static_assert(L::XROW % 128 == 0 && L::DSLOT % 128 == 0 && L::D_BYTES % 128 == 0, "tensor-copy targets");
  extern __shared__ __align__(1024) unsigned char conv_smem[];
  unsigned char* sD = conv_smem;
  unsigned char* sX = conv_smem + L::D_BYTES;
  __shared__ __align__(8) uint64_t xfull[kWgX], xempty[kWgX], dfull[kWgD], dempty[kWgD], done;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // constant chunks of every input slot: zeros, ones (1 in channel 0), zeros
  for (int i = tid; i < kWgX * 3 * kHaloW; i += blockDim.x) {
    const int px = i % kHaloW, e = (i / kHaloW) % 3, slot = i / (3 * kHaloW);
    uint4 z = make_uint4(0u, 0u, 0u, 0u);
    if (e == 1) z.x = 0x3F80u;
    *reinterpret_cast<uint4*>(sX + slot * L::XROW + ((CH + e) * kChunk + px) * 16) = z;
  }
  // bytes after the mirror slots that only unused accumulator rows read
  for (int i = (kWgD + 2) * L::DSLOT / 16 + tid; i < L::D_BYTES / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sD)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tc::tmem_alloc(&tslot, NCOL);
  if (tid == 0) {
    for (int i = 0; i < kWgX; ++i) {
      tc::mbar_init(&xfull[i], 1);
      tc::mbar_init(&xempty[i], 1);
    }
    for (int i = 0; i < kWgD; ++i) {
      tc::mbar_init(&dfull[i], 1);
      tc::mbar_init(&dempty[i], 1);
    }
    tc::mbar_init(&done, 1);
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;

  // this CTA's share of the rows, flattened as (image, column segment, row)
  const int segs = (a.w + 127) >> 7;
  const long long total = (long long)a.n * segs * a.h;
  const long long lo = total * blockIdx.x / gridDim.x, hi = total * (blockIdx.x + 1) / gridDim.x;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // ---- dY rows ya - 2 .. yb + 1 of every run; the four outside the run are
    // loaded from row -1, which the tensor copy fills with zeros
    uint32_t nd = 0;
    for (long long r = lo; r < hi && ok;) {
      const long long col = r / a.h;
      const int ya = (int)(r % a.h), len = (int)min((long long)(a.h - ya), hi - r);
      const int img = (int)(col / segs), x0 = (int)(col % segs) * 128;
      r += len;
      for (int e = 0; e < len + 4; ++e) {
        const uint32_t slot = nd % kWgD, use = nd / kWgD;
        if (use > 0 && !tc::mbar_wait(&dempty[slot], (use - 1) & 1u)) {
          ok = false;
          break;
        }
        const int y = (e >= 2 && e < len + 2) ? ya - 2 + e : -1;
        const uint32_t base = tc::smem_addr(sD) + slot * L::DSLOT;
        tc::mbar_expect_tx(&dfull[slot], (uint32_t)L::DSLOT * (slot < 2 ? 2u : 1u));
        for (int g = 0; g < COUT / 8; ++g) {
          tc::tma_load_4d(base + g * 2048, &mdy, g * 8, x0, y, img, &dfull[slot]);
          if (slot < 2) tc::tma_load_4d(base + kWgD * L::DSLOT + g * 2048, &mdy, g * 8, x0, y, img, &dfull[slot]);
        }
        ++nd;
      }
    }
    // every copy issued has landed before the CTA may leave
    for (uint32_t sl = 0; sl < kWgD && sl < nd; ++sl)
      if (!tc::mbar_wait(&dfull[sl], ((sl + ((nd - 1 - sl) / kWgD) * kWgD) / kWgD) & 1u)) ok = false;
  } else if (warp == 2 && lane == 0) {
    // ---- input rows ya - 1 .. yb of every run (rows outside the image and
    // pixels outside it come back as zeros)
    uint32_t nx = 0;
    for (long long r = lo; r < hi && ok;) {
      const long long col = r / a.h;
      const int ya = (int)(r % a.h), len = (int)min((long long)(a.h - ya), hi - r);
      const int img = (int)(col / segs), x0 = (int)(col % segs) * 128;
      r += len;
      for (int i = 0; i < len + 2; ++i) {
        const uint32_t slot = nx % kWgX, use = nx / kWgX;
        if (use > 0 && !tc::mbar_wait(&xempty[slot], (use - 1) & 1u)) {
          ok = false;
          break;
        }
        const uint32_t base = tc::smem_addr(sX) + slot * L::XROW;
        tc::mbar_expect_tx(&xfull[slot], (uint32_t)(CH * kHaloW * 16));
        for (int c8 = 0; c8 < CH; ++c8)
          tc::tma_load_4d(base + c8 * (kChunk * 16), &mx, c8 * 8, x0 - 1, ya - 1 + i, img, &xfull[slot]);
        ++nx;
      }
    }
    for (uint32_t sl = 0; sl < kWgX && sl < nx; ++sl)
      if (!tc::mbar_wait(&xfull[sl], ((sl + ((nx - 1 - sl) / kWgX) * kWgX) / kWgX) & 1u)) ok = false;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    uint32_t nx = 0, nd = 0;
    bool first = true;
    const uint32_t d_base = tc::smem_addr(sD), x_base = tc::smem_addr(sX);
    for (long long r = lo; r < hi && ok;) {
      const int ya = (int)(r % a.h), len = (int)min((long long)(a.h - ya), hi - r);
      r += len;
      const uint32_t d0 = nd;
      for (int i = 0; i < len + 2 && ok; ++i) {
        const uint32_t xs = nx % kWgX;
        ok = tc::mbar_wait(&xfull[xs], (nx / kWgX) & 1u);
        for (uint32_t q = (i == 0 ? d0 : d0 + i + 2); q <= d0 + i + 2 && ok; ++q)
          ok = tc::mbar_wait(&dfull[q % kWgD], (q / kWgD) & 1u);
        if (!ok) break;
        tc::fence_after();
        const uint32_t da = d_base + ((d0 + i) % kWgD) * L::DSLOT, xa = x_base + xs * L::XROW;
#pragma unroll
        for (int j = 0; j < 8; ++j) {  // 16 pixels per MMA
          const uint64_t ad = tc::smem_desc(da + j * 256, 128, 128 * 16);
          uint32_t col = 0;
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            const uint64_t bd = tc::smem_desc(xa + kx * 16 + j * 256, 128, kChunk * 16);
            tc::mma_bf16(tmem + col, ad, bd, tc::idesc_bf16(128, kWgN<CIN>(kx), true, true), !(first && j == 0));
            col += kWgN<CIN>(kx);
          }
        }
        first = false;
        tc::commit(&xempty[xs]);
        tc::commit(&dempty[(d0 + i) % kWgD]);  // dY entry d0 + i: this was its last reader
        ++nx;
      }
      if (!ok) break;
      tc::commit(&dempty[(d0 + len + 2) % kWgD]);
      tc::commit(&dempty[(d0 + len + 3) % kWgD]);
      nd = d0 + len + 4;
    }
    tc::commit(&done);
  }
  // ---- read-out: warp w holds TMEM lanes 32 w .. 32 w + 31 = (2 - ky) * cout + co
  __syncwarp();
  __syncthreads();
  const bool fin = tc::mbar_wait(&done, 0);
  if (!fin) ok = false;
  if (fin && warp * 32 < 3 * COUT) {
    tc::fence_after();
    const int row = warp * 32 + lane;
    const int ky = 2 - row / COUT, co = row % COUT;
    const bool mine = row < 3 * COUT;
    uint32_t col = 0;
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
      for (int c0 = 0; c0 < kWgN<CIN>(kx); c0 += 16) {
        uint32_t v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + col + (uint32_t)c0, v);
        tc::tmem_wait_ld();
        if (mine) {
          float* dst = a.dweight + ((size_t)co * 9 + ky * 3 + kx) * CIN;
#pragma unroll
          for (int c = 0; c < 16; c += 4)
            if (c0 + c < CIN)
              atomicAdd(reinterpret_cast<float4*>(dst + c0 + c),
                        make_float4(__uint_as_float(v[c]), __uint_as_float(v[c + 1]), __uint_as_float(v[c + 2]),
                                    __uint_as_float(v[c + 3])));
          constexpr int kOnes = (CH + 1) * 8;  // column of the ones chunk
          if (kx == 1 && ky == 1 && c0 <= kOnes && kOnes < c0 + 16 && a.dbias)
            atomicAdd(a.dbias + co, __uint_as_float(v[kOnes - c0]));
        }
      }
      col += kWgN<CIN>(kx);
    }
  }
  if (!ok) set_status(&a.hdr->status, FHV_DEV_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, NCOL);
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

// Tensor map of an NHWC BF16 activation [n][h][w][c] read in boxes of 8
// channels x box_px pixels of one row.
static cudaError_t make_act_map(CUtensorMap* m, const void* base, int c, int w, int h, int n, int box_px) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {(cuuint64_t)c, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
  const cuuint64_t strides[3] = {(cuuint64_t)c * 2, (cuuint64_t)w * c * 2, (cuuint64_t)h * w * c * 2};
  const cuuint32_t box[4] = {8, (cuuint32_t)box_px, 1, 1};
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, elem,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CIN, int COUT>
static cudaError_t launch_fwd_t(ConvArgs a, cudaStream_t s) {
  constexpr int CH = CIN / 8;
  constexpr int STAGE_PAD = (kFwRing * CH * kChunk * 16 + 1024 + 1023) & ~1023;
  const int smem = STAGE_PAD + kFwRowMmas<CIN> * 2 * (3 * COUT / 8) * 128;
  CUtensorMap mx;
  const cudaError_t e = make_act_map(&mx, a.x, CIN, a.w, a.h, a.n, kHaloW);
  if (e != cudaSuccess) return e;
  if (cudaFuncSetAttribute(conv_fwd_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return cudaGetLastError();
  // CTAs per SM: as many as TMEM (512 columns) and shared memory allow; one
  // run of rows per CTA
  int per_sm = (int)((227 * 1024) / (smem + 1408));
  per_sm = std::max(1, std::min(512 / kFwCols, per_sm));
  const long long ctas = (long long)sm_count() * per_sm;
  const long long cols = (long long)a.n * ((a.w + 127) / 128);
  const long long per_col = std::max<long long>(1, std::min<long long>(a.h, ctas / std::max<long long>(1, cols)));
  a.rows_per_item = (int)((a.h + per_col - 1) / per_col);
  const long long items = cols * ((a.h + a.rows_per_item - 1) / a.rows_per_item);
  const long long grid = std::min<long long>(items, ctas);
  timing_begin("conv_fwd", s);
  conv_fwd_kernel<CIN, COUT><<<(unsigned)grid, kFwWarps * 32, smem, s>>>(a, mx);
  timing_end("conv_fwd", s);
  return cudaGetLastError();
}

template <int CIN, int COUT>
static cudaError_t launch_wgrad_t(ConvArgs a, cudaStream_t s) {
  constexpr int smem = WgradSmem<CIN, COUT>::BYTES;
  CUtensorMap mx, mdy;
  cudaError_t e = make_act_map(&mx, a.x, CIN, a.w, a.h, a.n, kHaloW);
  if (e == cudaSuccess) e = make_act_map(&mdy, a.dy, COUT, a.w, a.h, a.n, 128);
  if (e != cudaSuccess) return e;
  if (cudaFuncSetAttribute(conv_wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return cudaGetLastError();
  // resident CTAs: shared memory and TMEM (512 columns per SM); each CTA takes
  // an equal share of the rows
  int per_sm = (int)((227 * 1024) / (smem + 1280));
  per_sm = std::max(1, std::min(per_sm, 512 / kWgTmem<CIN>()));
  const long long total = (long long)a.n * ((a.w + 127) / 128) * a.h;
  const long long grid = std::min<long long>(total, (long long)sm_count() * per_sm);
  timing_begin("conv_wgrad", s);
  conv_wgrad_kernel<CIN, COUT><<<(unsigned)grid, 128, smem, s>>>(a, mx, mdy);
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
