// k_c11_tc.cu -- conv1_1 (3 -> 64 channels) on the tensor cores, forward and input gradient.
//
// conv1_1 is the only convolution whose input is the image itself: 27 taps x channels per output
// pixel, too few for the implicit-GEMM kernels. Both directions become small GEMMs here:
//
//  * forward (Algorithm 1, both steps): D[p][n] = sum_k A[p][k] B[n][k] over 128 consecutive
//    buffer pixels p, with A the im2col rows of the block (zero outside its valid extent) built
//    by four producer warps straight into the 128-byte-swizzled K-major layout, and B the 64 x 64
//    weight tile. The image stays FP32-accurate: each input value enters as hi + lo, two BF16
//    numbers (hi = bf16(x), lo = bf16(x - hi), within 2^-17 |x| of x), A's row holding
//    [27 hi | 27 lo | 10 zero] against B's [27 w | 27 w | 10 zero]. The epilogue adds the bias,
//    applies ReLU, zeroes pixels outside the block's valid extent and stores the BF16 row.
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
constexpr int kFwdThreads = 288;   // warps 0-3 im2col, 4-7 epilogue, 8 MMA + TMEM allocation
constexpr int kFwdStages = 4;
constexpr uint32_t kFwdTile = 128 * 128;   // 128 rows x 64 BF16
constexpr uint32_t kFwdB = 64 * 128;       // 64 rows x 64 BF16
constexpr size_t kFwdSmem = 1024 + kFwdB + kFwdStages * kFwdTile;

__global__ void __launch_bounds__(kFwdThreads, 2)
    conv11_fwd_tc_kernel(const float *__restrict__ img, int H, int W,
                         const float *__restrict__ w11, const float *__restrict__ bias,
                         const BlockGeom *__restrict__ geom, int B, int Hb, int Wb,
                         __nv_bfloat16 *__restrict__ out, unsigned *err) {
  constexpr uint32_t IDESC = idesc_bf16_m128(64);
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kFwdStages], empty_bar[kFwdStages];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t *smem_gen = smem_raw + (smem_base - smem_u32(smem_raw));
  const uint32_t b_base = smem_base, a_base = smem_base + kFwdB;
  __shared__ __align__(16) float bias_sh[64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int npix = B * Hb * Wb;   // < 2^31 (checked by the launcher)
  const int ntiles = (npix + 127) / 128;
  // pixel p0 + r of the flattened [B][Hb][Wb] buffer -> (b, y, x), from p0's coordinates
  auto locate = [&](int p0, int r, int &b, int &y, int &x) {
    const unsigned q = (unsigned)p0 / (unsigned)Wb;
    x = p0 - (int)q * Wb + r;
    y = (int)(q % (unsigned)Hb);
    b = (int)(q / (unsigned)Hb);
    while (x >= Wb) {
      x -= Wb;
      if (++y == Hb) { y = 0; ++b; }
    }
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kFwdStages; s++) {
      mbar_init(smem_u32(&full_bar[s]), 128);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(smem_u32(&tfull_bar[i]), 1);
      mbar_init(smem_u32(&tempty_bar[i]), 128);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B tile: row n = output channel, K = [w(27) | w(27) | 0(10)], w = W1[n][ci][ky][kx]
  for (int i = threadIdx.x; i < 64 * 8; i += kFwdThreads) {
    const int n = i >> 3, c = i & 7;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int k = c * 8 + j;
      v[j] = k < 27 ? w11[n * 27 + k] : (k < 54 ? w11[n * 27 + k - 27] : 0.f);
    }
    *reinterpret_cast<uint4 *>(smem_gen + sw128_chunk(n, c)) =
        make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                   pack_bf16x2(v[6], v[7]));
  }
  if (threadIdx.x < 64) bias_sh[threadIdx.x] = bias[threadIdx.x];
  fence_proxy_async_smem();
  if (warp == 8) tmem_alloc(smem_u32(&tmem_base_sh), 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  if (warp < 4) {
    // ---------------- im2col producer: one pixel (row) per thread ----------------
    const int row = threadIdx.x;
    const size_t plane = (size_t)H * W;
    auto gather = [&](int t, float *in) {
      bool live = t * 128 + row < npix;
      int x = 0, y = 0, b = 0;
      if (live) locate(t * 128, row, b, y, x);
      const BlockGeom g = geom[live ? b : 0];
      live = live && y < g.eh && x < g.ew;
#pragma unroll
      for (int ky = 0; ky < 3; ky++)
#pragma unroll
        for (int kx = 0; kx < 3; kx++) {
          const int yy = y + ky - 1, xx = x + kx - 1;
          const bool ok = live && yy >= 0 && yy < g.eh && xx >= 0 && xx < g.ew;
          const size_t o = ok ? (size_t)(g.ey0 + yy) * W + g.ex0 + xx : 0;
#pragma unroll
          for (int ci = 0; ci < 3; ci++)
            in[ci * 9 + ky * 3 + kx] = ok ? __ldg(img + ci * plane + o) : 0.f;
        }
    };
    float cur[27], nxt[27];
    int it = 0;
    int t = blockIdx.x;
    if (t < ntiles) gather(t, cur);
    for (; t < ntiles; t += gridDim.x, it++) {
      const int stage = it % kFwdStages;
      const uint32_t phase = (uint32_t)(it / kFwdStages) & 1u;
      const int tn = t + gridDim.x;
      if (tn < ntiles) gather(tn, nxt);   // next tile's loads in flight while this one is stored
      if (!mbar_wait_sleep(smem_u32(&empty_bar[stage]), phase ^ 1u, &abort_flag, err)) break;
      float hi[27], lo[27];
#pragma unroll
      for (int k = 0; k < 27; k++) {
        hi[k] = __bfloat162float(__float2bfloat16_rn(cur[k]));
        lo[k] = cur[k] - hi[k];   // exact in FP32
      }
      uint8_t *arow = smem_gen + kFwdB + (size_t)stage * kFwdTile;
#pragma unroll
      for (int c = 0; c < 8; c++) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const int k = c * 8 + j;
          v[j] = k < 27 ? hi[k] : (k < 54 ? lo[k - 27] : 0.f);
        }
        *reinterpret_cast<uint4 *>(arow + sw128_chunk(row, c)) =
            make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                       pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
      }
      fence_proxy_async_smem();
      mbar_arrive(smem_u32(&full_bar[stage]));
#pragma unroll
      for (int k = 0; k < 27; k++) cur[k] = nxt[k];
    }
  } else if (warp < 8) {
    // ---------------- epilogue: bias, ReLU, valid-extent mask, BF16 row store ----------------
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
      const int acc = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      if (!mbar_wait_sleep(smem_u32(&tfull_bar[acc]), use & 1u, &abort_flag, err)) break;
      tc_fence_after();
      float v[64];
      const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 64);
      tmem_ld32(tb, v);
      tmem_ld32(tb + 32, v + 32);
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty_bar[acc]));
      const int p = t * 128 + row;
      if (p < npix) {
        int b, y, x;
        locate(t * 128, row, b, y, x);
        const BlockGeom g = geom[b];
        const bool valid = y < g.eh && x < g.ew;
        uint4 *o = reinterpret_cast<uint4 *>(out + (size_t)p * 64);
#pragma unroll
        for (int c = 0; c < 8; c++) {
          const float4 b0 = *reinterpret_cast<const float4 *>(bias_sh + c * 8);
          const float4 b1 = *reinterpret_cast<const float4 *>(bias_sh + c * 8 + 4);
          const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
          float r[8];
#pragma unroll
          for (int j = 0; j < 8; j++) r[j] = valid ? fmaxf(v[c * 8 + j] + bb[j], 0.f) : 0.f;
          o[c] = make_uint4(pack_bf16x2(r[0], r[1]), pack_bf16x2(r[2], r[3]),
                            pack_bf16x2(r[4], r[5]), pack_bf16x2(r[6], r[7]));
        }
      }
    }
  } else if (lane == 0) {
    // ---------------- MMA issuer ----------------
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
      const uint64_t da = sw128_desc(a_base + stage * kFwdTile), db = sw128_desc(b_base);
      const uint32_t d = tmem_base + (uint32_t)(acc * 64);
#pragma unroll
      for (int k = 0; k < 4; k++)
        mma_bf16(d, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), IDESC, k > 0 ? 1u : 0u);
      mma_commit(smem_u32(&empty_bar[stage]));
      mma_commit(smem_u32(&tfull_bar[acc]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 128);
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
                                 __nv_bfloat16 *out, unsigned *err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(conv11_fwd_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long npix = (long long)B * Hb * Wb;
  if (npix >= (1LL << 31) - 128) return cudaErrorInvalidValue;
  const long long ntiles = (npix + 127) / 128;
  if (ntiles <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(ntiles, 2LL * tc_num_sms());
  conv11_fwd_tc_kernel<<<grid, kFwdThreads, kFwdSmem, s>>>(img, H, W, w11, bias, geom, B, Hb, Wb,
                                                           out, err);
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
