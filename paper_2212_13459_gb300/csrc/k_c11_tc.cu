// k_c11_tc.cu -- conv1_1 (3 -> 64 channels) on the tensor cores, forward and input gradient.
//
// conv1_1 is the only convolution whose input is the image itself: 27 taps x channels per output
// pixel, too few for the implicit-GEMM kernels. Both directions become small GEMMs here:
//
//  * forward (Algorithm 1, both steps): the block images are first staged as 16-byte BF16
//    pixels (hi_0..2, lo_0..2, 0, 0) with hi = bf16(x), lo = bf16(x - hi), so each image value
//    enters within 2^-17 |x| of its FP32 value; then D[p][n] = sum_k A[p][k] B[n][k] over a
//    16 x 8 output patch with K = 9 taps x 8, every tap a shifted view of one TMA halo box (see
//    the kernel). The epilogue adds the bias, applies ReLU, zeroes pixels outside the block's
//    valid extent and stores the BF16 row. In the passes that take the Gram statistics it also
//    adds T^T T of every owned output tile T to a per-CTA ReLU1_1 Gram (Eq. 4), on the tensor
//    cores from the tile it stages for the store (see kFwdGramIdesc).
//  * input gradient (last line of Algorithm 1): P[q][j] = sum_co g[q][co] Wt[j][co] with
//    j = 3 tap + ci (27 of N = 32 columns), over an 18 x 14 box of the gated ReLU1_1 gradient
//    loaded by TMA (zero outside the buffer); the epilogue forms
//    dx[ci](y, x) = sum_tap P[(y, x) - offset(tap)][3 tap + ci] for the 16 x 12 owned pixels of
//    the box's centre and writes them at image coordinates. Every owned pixel is written once, by
//    one thread, with a fixed summation order (deterministic).
#include <algorithm>

#include "nst_internal.cuh"
#include "nst_kernels.h"
#include "tc_ptx.cuh"

namespace nst {
namespace {

using namespace nst::tc;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_half, float hi_half) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo_half, hi_half);  // .x = lo_half (low bits)
  return *reinterpret_cast<const uint32_t *>(&h);
}

// byte offset of the 16-byte chunk c of row r in a 128-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t sw128_chunk(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

// ------------------------------------------------------------------------------------------------
// forward
// ------------------------------------------------------------------------------------------------
// Step 1: the block image in the BF16 form, one 16-byte pixel per buffer pixel:
// xs[b][y][x] = (hi_0, hi_1, hi_2, lo_0, lo_1, lo_2, 0, 0) inside the block's valid extent, zero
// elsewhere (the block is a standalone image with zero padding).
__global__ void __launch_bounds__(256) conv11_stage_kernel(const float *__restrict__ img, int H,
                                                           int W, const BlockGeom *__restrict__ geom,
                                                           int B, int Hb, int Wb,
                                                           uint4 *__restrict__ xs) {
  const int npix = B * Hb * Wb;
  const size_t plane = (size_t)H * W;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    const unsigned q = (unsigned)p / (unsigned)Wb;
    const int x = p - (int)q * Wb, y = (int)(q % (unsigned)Hb), b = (int)(q / (unsigned)Hb);
    const BlockGeom g = geom[b];
    uint4 o = make_uint4(0u, 0u, 0u, 0u);
    if (y < g.eh && x < g.ew) {
      const size_t off = (size_t)(g.ey0 + y) * W + g.ex0 + x;
      float hi[3], lo[3];
#pragma unroll
      for (int ci = 0; ci < 3; ci++) {
        const float v = __ldg(img + ci * plane + off);
        hi[ci] = __bfloat162float(__float2bfloat16_rn(v));
        lo[ci] = v - hi[ci];   // exact in FP32; rounded to BF16 by the packing below
      }
      o = make_uint4(pack_bf16x2(hi[0], hi[1]), pack_bf16x2(hi[2], lo[0]),
                     pack_bf16x2(lo[1], lo[2]), 0u);
    }
    xs[p] = o;
  }
}

// Step 2: the convolution, D[p][n] = sum_k A[p][k] B[n][k] with M = a 16 x 8 output patch and
// K = 9 taps x 8 values (hi, lo, 2 zeros) + 8 zero columns = 80. One TMA box of 18 x 10 staged
// pixels (16 bytes each, no swizzle) feeds all taps: in the K-major no-swizzle layout a "core
// matrix" is 8 rows x 16 bytes, so row i of the patch (8 pixels) is one core matrix at
// 160-byte steps (SBO) and the two taps of one K = 16 instruction are two core matrices of the
// same box whose distance is the instruction's LBO. Five instructions per tile: taps (0,1),
// (2,3), (4,5), (6,7), (8, -) with zero weights in the last one's second half.
constexpr int kFwdThreads = 192;   // warp 0 TMA, warp 1 MMA + TMEM, warps 2-5 epilogue
constexpr int kFwdStages = 6;
constexpr int kFwdTH = 16, kFwdTW = 8, kFwdBoxH = kFwdTH + 2, kFwdBoxW = kFwdTW + 2;
constexpr uint32_t kFwdBoxBytes = kFwdBoxH * kFwdBoxW * 16;   // 2,880
constexpr uint32_t kFwdStage = 3072;                         // box + zeroed tail
constexpr uint32_t kFwdB = 16384;                            // 5 x 2 KB used, rest zero
constexpr uint32_t kFwdOut = 128 * 128;                      // one output tile, 128-B swizzle
constexpr int kFwdOutBufs = 4;                               // output tiles in flight per CTA
constexpr uint32_t kFwdZero = 8192;                          // zero rows: the Gram's A channels 64..127
constexpr size_t kFwdSmem =
    1024 + kFwdB + kFwdStages * kFwdStage + kFwdOutBufs * kFwdOut + kFwdZero;
static_assert(2 * (kFwdSmem + 1024) <= 228 * 1024, "two conv1_1 CTAs per SM");
// Gram of the ReLU1_1 output over the owned pixels (Eq. 4), fused: G += T^T T for each owned
// output tile T (128 pixels x 64 channels, the staged BF16 tile the TMA store reads), on the
// tensor cores with both operands MN-major in that tile (M = 128 rows of channels, 64..127 read
// from zero rows, N = 64, K = 16 pixels per instruction, eight instructions a tile), FP32 in
// TMEM columns 128..191; each CTA writes its 64 x 64 partial (rows of 64 floats, 128-row stride).
constexpr uint32_t kFwdGramIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                   ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr int kFwdGramRun = 128 * 64;   // floats per CTA partial

__device__ __forceinline__ uint64_t desc_k_none(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version; layout type 0 = no swizzle
  return d;
}
__host__ __device__ constexpr uint32_t fwd_tap_off(int tap) {   // byte offset of a tap in the box
  return (uint32_t)(((tap / 3) * kFwdBoxW + tap % 3) * 16);
}

// patches: optional list of 16 x 8 output patches {block, y0, x0, 0} (each block's needed
// rectangle); without it every patch of the buffer, tiles_x x tiles_y per block
__global__ void __launch_bounds__(kFwdThreads, 2)
    conv11_fwd_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                         const __grid_constant__ CUtensorMap tmO, const float *__restrict__ w11,
                         const float *__restrict__ bias, const BlockGeom *__restrict__ geom,
                         int B, int Hb, int Wb, int tiles_x, int tiles_y,
                         const int4 *__restrict__ patches, int npatches,
                         float *__restrict__ gram_part, unsigned *err) {
  constexpr uint32_t IDESC = idesc_bf16_m128(64);
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kFwdStages], empty_bar[kFwdStages];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2];
  __shared__ __align__(8) uint64_t gram_bar[kFwdOutBufs], gram_done;   // fused Gram MMAs read
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  __shared__ __align__(16) float bias_sh[64];
  __shared__ int epi_ok, gram_ok, gram_any, gram_fin;   // broadcasts of single-thread waits

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t *smem_gen = smem_raw + (smem_base - smem_u32(smem_raw));
  const uint32_t b_base = smem_base, a_base = smem_base + kFwdB;
  const uint32_t o_off = kFwdB + kFwdStages * kFwdStage;   // output staging tiles
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = patches ? npatches : B * tiles_x * tiles_y;
  auto origin = [&](int t, int &b, int &y0, int &x0) {
    if (patches) {
      const int4 q = __ldg(patches + t);
      b = q.x;
      y0 = q.y;
      x0 = q.z;
    } else {
      b = t / (tiles_x * tiles_y);
      y0 = ((t / tiles_x) % tiles_y) * kFwdTH;
      x0 = (t % tiles_x) * kFwdTW;
    }
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kFwdStages; s++) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(smem_u32(&tfull_bar[i]), 1);
      mbar_init(smem_u32(&tempty_bar[i]), 128);
    }
    for (int i = 0; i < kFwdOutBufs; i++) mbar_init(smem_u32(&gram_bar[i]), 1);
    mbar_init(smem_u32(&gram_done), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B: instruction i's 64 x 16 block at i * 2048: K half h (tap 2i + h) at + h * 1024, output
  // channel n at + n * 16, holding (w[n][0][tap], w[n][1][tap], w[n][2][tap]) twice (for hi and
  // lo) and two zeros; everything else zero. The stage tails past each box are zeroed too, so the
  // K padding of the last instruction multiplies finite values by zero weights.
  for (int i = threadIdx.x; i < (int)(kFwdB / 16); i += kFwdThreads) {
    const int ins = i >> 7, h = (i >> 6) & 1, n = i & 63;
    const int tap = 2 * ins + h;
    float w0 = 0.f, w1 = 0.f, w2 = 0.f;
    if (ins < 5 && tap < 9) {
      w0 = w11[n * 27 + tap];
      w1 = w11[n * 27 + 9 + tap];
      w2 = w11[n * 27 + 18 + tap];
    }
    *reinterpret_cast<uint4 *>(smem_gen + (size_t)i * 16) =
        make_uint4(pack_bf16x2(w0, w1), pack_bf16x2(w2, w0), pack_bf16x2(w1, w2), 0u);
  }
  for (int i = threadIdx.x; i < kFwdStages * (int)((kFwdStage - kFwdBoxBytes) / 16);
       i += kFwdThreads) {
    const int st = i / (int)((kFwdStage - kFwdBoxBytes) / 16);
    const int k = i % (int)((kFwdStage - kFwdBoxBytes) / 16);
    *reinterpret_cast<uint4 *>(smem_gen + kFwdB + (size_t)st * kFwdStage + kFwdBoxBytes + k * 16) =
        make_uint4(0u, 0u, 0u, 0u);
  }
  if (gram_part)   // zero rows after the output tiles: the Gram's A channels 64..127
    for (int i = threadIdx.x; i < (int)(kFwdZero / 16); i += kFwdThreads)
      *reinterpret_cast<uint4 *>(smem_gen + o_off + kFwdOutBufs * kFwdOut + (size_t)i * 16) =
          make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x < 64) bias_sh[threadIdx.x] = bias[threadIdx.x];
  fence_proxy_async_smem();
  const uint32_t tmem_cols = gram_part ? 256u : 128u;   // two accumulators (+ the Gram's)
  if (warp == 1) tmem_alloc(smem_u32(&tmem_base_sh), tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmX)) : "memory");
      int it = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
        const int stage = it % kFwdStages;
        const uint32_t phase = (uint32_t)(it / kFwdStages) & 1u;
        int b, oy, ox;
        origin(t, b, oy, ox);
        if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1u, &abort_flag, err)) break;
        const uint32_t fb = smem_u32(&full_bar[stage]);
        mbar_expect_tx(fb, kFwdBoxBytes);
        tma_load_4d(a_base + stage * kFwdStage, &tmX, fb, 0, ox - 1, oy - 1, b);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
        const int stage = it % kFwdStages;
        const uint32_t phase = (uint32_t)(it / kFwdStages) & 1u;
        const int acc = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (!mbar_wait(smem_u32(&tempty_bar[acc]), (use & 1u) ^ 1u, &abort_flag, err)) break;
        tc_fence_after();
        if (!mbar_wait(smem_u32(&full_bar[stage]), phase, &abort_flag, err)) break;
        tc_fence_after();
        const uint32_t sa = a_base + stage * kFwdStage;
        const uint32_t d = tmem_base + (uint32_t)(acc * 64);
#pragma unroll
        for (int ins = 0; ins < 5; ins++) {
          const uint32_t o0 = fwd_tap_off(2 * ins);
          const uint32_t lbo = ins < 4 ? fwd_tap_off(2 * ins + 1) - o0 : 16u;
          mma_bf16(d, desc_k_none(sa + o0, lbo, kFwdBoxW * 16),
                   desc_k_none(b_base + ins * 2048, 1024, 128), IDESC, ins > 0 ? 1u : 0u);
        }
        mma_commit(smem_u32(&empty_bar[stage]));
        mma_commit(smem_u32(&tfull_bar[acc]));
      }
    }
  } else {
    // ---------------- epilogue: bias, ReLU, valid-extent mask, BF16 tile -> TMA store ----------------
    // Each thread writes its pixel's 128-byte row into a 128-byte-swizzled staging tile (chunk c
    // of row r at c ^ (r & 7): conflict-free), and one thread stores the 16 x 8 x 64 tile with
    // one TMA copy (full-line writes; rows / columns past the buffer are clipped). Four staging
    // tiles rotate (several stores in flight); a tile is rewritten only after its store has
    // finished reading it.
    const int q = warp & 3;
    const int row = q * 32 + lane;   // patch pixel (row / 8, row % 8)
    const int et = threadIdx.x - 64;
    // thread et = 0 issues the stores, et = 32 (the next warp) the fused Gram MMAs; per staging
    // buffer, whether Gram MMAs reading it are in flight (gpend) and the parity of its next
    // completion (gph)
    uint32_t gpend = 0u, gph = 0u;
    bool gfirst = true;   // no Gram MMA issued yet (the first one overwrites the accumulator)
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
      const int acc = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      const int ob = it % kFwdOutBufs;
      // one thread waits (bounded) and broadcasts, so all 128 threads leave the loop together;
      // the same barrier tells everyone that staging tile ob is free again (its store has read
      // it, see below, and so have the Gram MMAs of its last tile)
      if (et == 0) epi_ok = mbar_wait_sleep(smem_u32(&tfull_bar[acc]), use & 1u, &abort_flag, err);
      if (et == 32) {
        gram_ok = 1;
        if ((gpend >> ob) & 1u) {
          gram_ok = mbar_wait_sleep(smem_u32(&gram_bar[ob]), (gph >> ob) & 1u, &abort_flag, err);
          gph ^= 1u << ob;
          gpend &= ~(1u << ob);
        }
      }
      named_bar_sync(1, 128);
      if (!gram_ok) break;
      if (!epi_ok) break;
      tc_fence_after();
      float v[64];
      const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 64);
      tmem_ld32(tb, v);
      tmem_ld32(tb + 32, v + 32);
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty_bar[acc]));
      int b, oy, ox;
      origin(t, b, oy, ox);
      const int y = oy + row / kFwdTW, x = ox + row % kFwdTW;
      const BlockGeom g = geom[b];
      const bool valid = y < g.eh && x < g.ew;
      uint8_t *orow = smem_gen + o_off + (size_t)ob * kFwdOut + (size_t)row * 128;
#pragma unroll
      for (int c = 0; c < 8; c++) {
        const float4 b0 = *reinterpret_cast<const float4 *>(bias_sh + c * 8);
        const float4 b1 = *reinterpret_cast<const float4 *>(bias_sh + c * 8 + 4);
        const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        float r[8];
#pragma unroll
        for (int j = 0; j < 8; j++) r[j] = valid ? fmaxf(v[c * 8 + j] + bb[j], 0.f) : 0.f;
        *reinterpret_cast<uint4 *>(orow + ((c ^ (row & 7)) << 4)) =
            make_uint4(pack_bf16x2(r[0], r[1]), pack_bf16x2(r[2], r[3]),
                       pack_bf16x2(r[4], r[5]), pack_bf16x2(r[6], r[7]));
      }
      fence_proxy_async_smem();
      named_bar_sync(1, 128);
      const uint32_t tile = smem_base + o_off + (uint32_t)ob * kFwdOut;
      if (et == 0) {
        tma_store_4d(&tmO, tile, 0, ox, oy, b);
        bulk_commit();
        bulk_wait_read_3();   // the tile written next (it + 1) was stored at it + 1 - 4
      }
      if (et == 32) {
        // an owned tile (the patch list's fourth field) adds T^T T to the Gram accumulator: its
        // 16-pixel row pairs are the K steps, read in place by the tensor cores
        if (gram_part && patches && __ldg(patches + t).w) {
          tc_fence_after();
          const uint32_t zero = smem_base + o_off + kFwdOutBufs * kFwdOut;
#pragma unroll
          for (int kk = 0; kk < 8; kk++) {
            const uint32_t a0 = tile + (uint32_t)kk * 2048u;
            mma_bf16(tmem_base + 128u, sw128_desc_mn(a0, zero + (uint32_t)(kk & 3) * 2048u - a0),
                     sw128_desc_mn(a0, kFwdZero), kFwdGramIdesc, gfirst && kk == 0 ? 0u : 1u);
          }
          gfirst = false;
          mma_commit(smem_u32(&gram_bar[ob]));
          gpend |= 1u << ob;
        }
      }
    }
    if (et == 0) bulk_wait_all();
    if (gram_part) {
      // this CTA's Gram partial: one commit after the last MMA covers all of them
      if (et == 32) {
        int ok = 1;
        if (!gfirst) {
          mma_commit(smem_u32(&gram_done));
          ok = mbar_wait_sleep(smem_u32(&gram_done), 0u, &abort_flag, err);
        }
        // (own variables: a thread that left the loop on an abort may not have read epi_ok yet)
        gram_fin = ok;
        gram_any = gfirst ? 0 : 1;
      }
      named_bar_sync(1, 128);
      tc_fence_after();
      if (q < 2) {   // rows = channels 0..63 (TMEM lanes 64..127 hold the zero rows' products)
        float v[64];
        if (gram_any && gram_fin) {
          const uint32_t tg = tmem_base + ((uint32_t)(q * 32) << 16) + 128u;
          tmem_ld32(tg, v);
          tmem_ld32(tg + 32, v + 32);
        } else {
#pragma unroll
          for (int j = 0; j < 64; j++) v[j] = 0.f;
        }
        float4 *dst = reinterpret_cast<float4 *>(gram_part + (size_t)blockIdx.x * kFwdGramRun +
                                                 (size_t)row * 64);
#pragma unroll
        for (int j = 0; j < 16; j++)
          dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, tmem_cols);
  }
}

// ------------------------------------------------------------------------------------------------
// input gradient
// ------------------------------------------------------------------------------------------------
constexpr int kDgThreads = 192;   // warp 0 TMA, warp 1 MMA + TMEM allocation, warps 2-5 epilogue
constexpr int kDgStages = 2;
constexpr int kDgOutW = 16, kDgOutH = 12;
constexpr int kDgBoxW = kDgOutW + 2, kDgBoxH = kDgOutH + 2;    // 18 x 14 = 252 pixels
constexpr uint32_t kDgBoxBytes = kDgBoxW * kDgBoxH * 128;      // 32,256
constexpr uint32_t kDgStage = 256 * 128;                       // two M = 128 halves
constexpr uint32_t kDgB = 32 * 128;                            // 32 rows (27 used) x 64 BF16
constexpr int kDgPs = 256;                                     // P row stride (floats)
constexpr size_t kDgSmem = 1024 + kDgB + kDgStages * kDgStage + 27 * kDgPs * 4;

__global__ void __launch_bounds__(kDgThreads, 2)
    conv11_dgrad_tc_kernel(const __grid_constant__ CUtensorMap tmG, const float *__restrict__ w11,
                           const BlockGeom *__restrict__ geom, const OwnRect *__restrict__ inner,
                           int B, int tiles_x, int tiles_y, float *__restrict__ grad, int H, int W,
                           unsigned *err) {
  constexpr uint32_t IDESC = idesc_bf16_m128(32);
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kDgStages], empty_bar[kDgStages];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  __shared__ int epi_ok;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t *smem_gen = smem_raw + (smem_base - smem_u32(smem_raw));
  const uint32_t b_base = smem_base, a_base = smem_base + kDgB;
  float *Ps = reinterpret_cast<float *>(smem_gen + kDgB + kDgStages * kDgStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_block = tiles_x * tiles_y;
  const int ntiles = B * per_block;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kDgStages; s++) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(smem_u32(&tfull_bar[i]), 1);
      mbar_init(smem_u32(&tempty_bar[i]), 128);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B tile: row j = 3 tap + ci (27 rows, then zeros), K = co: W1[co][ci][tap]
  for (int i = threadIdx.x; i < 32 * 8; i += kDgThreads) {
    const int j = i >> 3, c = i & 7;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
      const int co = c * 8 + e;
      v[e] = j < 27 ? w11[co * 27 + (j % 3) * 9 + j / 3] : 0.f;
    }
    *reinterpret_cast<uint4 *>(smem_gen + sw128_chunk(j, c)) =
        make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                   pack_bf16x2(v[6], v[7]));
  }
  fence_proxy_async_smem();
  if (warp == 1) tmem_alloc(smem_u32(&tmem_base_sh), 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  // tile t -> block b, patch origin (y0, x0) in block-local level-0 coordinates; tiles past the
  // block's owned rectangle are skipped identically by every role
  auto tile_at = [&](int t, int &b, int &y0, int &x0, OwnRect &r) -> bool {
    b = t / per_block;
    const int k = t % per_block;
    r = inner[b];
    y0 = r.y0 + (k / tiles_x) * kDgOutH;
    x0 = r.x0 + (k % tiles_x) * kDgOutW;
    return y0 < r.y1 && x0 < r.x1;
  };

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmG)) : "memory");
      int it = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int b, y0, x0;
        OwnRect r;
        if (!tile_at(t, b, y0, x0, r)) continue;
        const int stage = it % kDgStages;
        const uint32_t phase = (uint32_t)(it / kDgStages) & 1u;
        if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1u, &abort_flag, err)) break;
        const uint32_t fb = smem_u32(&full_bar[stage]);
        mbar_expect_tx(fb, kDgBoxBytes);
        tma_load_4d(a_base + stage * kDgStage, &tmG, fb, 0, x0 - 1, y0 - 1, b);
        it++;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int b, y0, x0;
        OwnRect r;
        if (!tile_at(t, b, y0, x0, r)) continue;
        const int stage = it % kDgStages;
        const uint32_t phase = (uint32_t)(it / kDgStages) & 1u;
        const int acc = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (!mbar_wait(smem_u32(&tempty_bar[acc]), (use & 1u) ^ 1u, &abort_flag, err)) break;
        tc_fence_after();
        if (!mbar_wait(smem_u32(&full_bar[stage]), phase, &abort_flag, err)) break;
        tc_fence_after();
        const uint32_t sa = a_base + stage * kDgStage;
        const uint64_t db = sw128_desc(b_base);
#pragma unroll
        for (int h = 0; h < 2; h++) {   // box rows 0..127 and 128..255 (252 loaded)
          const uint64_t da = sw128_desc(sa + h * 128 * 128);
          const uint32_t d = tmem_base + (uint32_t)(acc * 64 + h * 32);
#pragma unroll
          for (int k = 0; k < 4; k++)
            mma_bf16(d, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), IDESC, k > 0 ? 1u : 0u);
        }
        mma_commit(smem_u32(&empty_bar[stage]));
        mma_commit(smem_u32(&tfull_bar[acc]));
        it++;
      }
    }
  } else {
    // ---------------- epilogue: P -> shared memory, 9-tap gather, FP32 stores ----------------
    const int q = warp & 3;
    const int et = threadIdx.x - 64;   // 0..127
    const int row = q * 32 + lane;
    const size_t plane = (size_t)H * W;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      int b, y0, x0;
      OwnRect r;
      if (!tile_at(t, b, y0, x0, r)) continue;
      const int acc = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      // one thread waits (bounded) and broadcasts the outcome, so the 128 threads leave together;
      // the barrier also orders the previous tile's reads of P before this tile's writes
      if (et == 0) epi_ok = mbar_wait_sleep(smem_u32(&tfull_bar[acc]), use & 1u, &abort_flag, err);
      named_bar_sync(1, 128);
      if (!epi_ok) break;
      tc_fence_after();
      float v[32];
      const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 64);
      tmem_ld32(tb, v);
#pragma unroll
      for (int j = 0; j < 27; j++) Ps[j * kDgPs + row] = v[j];
      tmem_ld32(tb + 32, v);
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty_bar[acc]));
      if (128 + row < kDgBoxW * kDgBoxH) {
#pragma unroll
        for (int j = 0; j < 27; j++) Ps[j * kDgPs + 128 + row] = v[j];
      }
      named_bar_sync(1, 128);
      const BlockGeom gm = geom[b];
      for (int o = et; o < kDgOutW * kDgOutH; o += 128) {
        const int oy = o / kDgOutW, ox = o % kDgOutW;
        const int Y = y0 + oy, X = x0 + ox;
        if (Y >= r.y1 || X >= r.x1) continue;
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
        for (int ky = 0; ky < 3; ky++)
#pragma unroll
          for (int kx = 0; kx < 3; kx++) {
            const int src = (oy + 2 - ky) * kDgBoxW + (ox + 2 - kx);
            const int j = (ky * 3 + kx) * 3;
            d0 += Ps[j * kDgPs + src];
            d1 += Ps[(j + 1) * kDgPs + src];
            d2 += Ps[(j + 2) * kDgPs + src];
          }
        const size_t off = (size_t)(gm.ey0 + Y) * W + gm.ex0 + X;
        grad[off] = d0;
        grad[plane + off] = d1;
        grad[2 * plane + off] = d2;
      }
      it++;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 128);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

cudaError_t launch_conv11_fwd_tc(const float *img, int H, int W, const float *w11,
                                 const float *bias, const BlockGeom *geom, int B, int Hb, int Wb,
                                 void *stage_buf, __nv_bfloat16 *out, const int4 *patches,
                                 int npatches, float *gram_part, int *gram_runs, unsigned *err,
                                 cudaStream_t s) {
  if (gram_runs) *gram_runs = 0;
  if (gram_part && (!patches || !gram_runs)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(conv11_fwd_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long npix = (long long)B * Hb * Wb;
  if (npix >= (1LL << 31)) return cudaErrorInvalidValue;
  if (npix <= 0) return cudaSuccess;
  if (reinterpret_cast<uintptr_t>(stage_buf) % 16) return cudaErrorInvalidValue;
  const int sgrid = (int)std::min<long long>((npix + 255) / 256, 32LL * tc_num_sms());
  conv11_stage_kernel<<<sgrid, 256, 0, s>>>(img, H, W, geom, B, Hb, Wb,
                                            reinterpret_cast<uint4 *>(stage_buf));
  EncodeTiledFn enc = reinterpret_cast<EncodeTiledFn>(tc_encode_tiled_fn());
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap m;
  cuuint64_t dims[4] = {8, (cuuint64_t)Wb, (cuuint64_t)Hb, (cuuint64_t)B};
  cuuint64_t strides[3] = {16, (cuuint64_t)Wb * 16, (cuuint64_t)Hb * Wb * 16};
  cuuint32_t box[4] = {8, kFwdBoxW, kFwdBoxH, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, stage_buf, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  CUtensorMap mo;
  cuuint64_t odims[4] = {64, (cuuint64_t)Wb, (cuuint64_t)Hb, (cuuint64_t)B};
  cuuint64_t ostrides[3] = {128, (cuuint64_t)Wb * 128, (cuuint64_t)Hb * Wb * 128};
  cuuint32_t obox[4] = {64, kFwdTW, kFwdTH, 1};
  r = enc(&mo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, out, odims, ostrides, obox, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int tiles_x = (Wb + kFwdTW - 1) / kFwdTW, tiles_y = (Hb + kFwdTH - 1) / kFwdTH;
  const long long ntiles = patches ? npatches : (long long)B * tiles_x * tiles_y;
  if (ntiles <= 0) return cudaSuccess;
  // with the Gram, always two CTAs per SM: CTA c sums the owned patches c, c + grid, ... (the
  // list puts them first), a split that depends on the owned patches alone
  const int grid = gram_part ? 2 * tc_num_sms()
                             : (int)std::min<long long>(ntiles, 2LL * tc_num_sms());
  conv11_fwd_tc_kernel<<<grid, kFwdThreads, kFwdSmem, s>>>(m, mo, w11, bias, geom, B, Hb, Wb,
                                                           tiles_x, tiles_y, patches,
                                                           (int)ntiles, gram_part, err);
  if (gram_runs) *gram_runs = gram_part ? grid : 0;
  return cudaGetLastError();
}

cudaError_t launch_conv11_dgrad_tc(const __nv_bfloat16 *g, const float *w11,
                                   const BlockGeom *geom, const OwnRect *inner, int B, int Hb,
                                   int Wb, int max_inner_h, int max_inner_w, float *grad, int H,
                                   int W, unsigned *err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(conv11_dgrad_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDgSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (B <= 0 || max_inner_h <= 0 || max_inner_w <= 0) return cudaSuccess;
  EncodeTiledFn enc = reinterpret_cast<EncodeTiledFn>(tc_encode_tiled_fn());
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap m;
  cuuint64_t dims[4] = {64, (cuuint64_t)Wb, (cuuint64_t)Hb, (cuuint64_t)B};
  cuuint64_t strides[3] = {64 * 2, (cuuint64_t)Wb * 64 * 2, (cuuint64_t)Hb * Wb * 64 * 2};
  cuuint32_t box[4] = {64, kDgBoxW, kDgBoxH, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(g), dims,
                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int tiles_x = (max_inner_w + kDgOutW - 1) / kDgOutW;
  const int tiles_y = (max_inner_h + kDgOutH - 1) / kDgOutH;
  const long long ntiles = (long long)B * tiles_x * tiles_y;
  const int grid = (int)std::min<long long>(ntiles, 2LL * tc_num_sms());
  conv11_dgrad_tc_kernel<<<grid, kDgThreads, kDgSmem, s>>>(m, w11, geom, inner, B, tiles_x,
                                                           tiles_y, grad, H, W, err);
  return cudaGetLastError();
}

}  // namespace nst
