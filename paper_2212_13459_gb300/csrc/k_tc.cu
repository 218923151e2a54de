// k_tc.cu -- tensor-core implicit-GEMM 3x3 convolution for sm_103a: tcgen05.mma (BF16 inputs,
// FP32 accumulator in tensor memory), operands staged in shared memory by TMA, warp-specialised
// and persistent. It runs every convolution of the VGG-19 trunk except conv1_1 (Cin = 3):
//   forward:  out = relu(W * in + b), zero outside each block's valid region (Section 3.1);
//   backward: out = (W^T * g [+ V R_L] [+ 2 lambda (V - V_u)]) gated by the ReLU mask, i.e. the
//             input gradient of a convolution with the style-loss feature gradient V R_L
//             (Table 1 row 2, R_L = 4 w_L (G - G_ref) / n_p) fused as extra K, and the content
//             gradient (Table 1 row 1) fused in the epilogue (Algorithm 1, Step 2).
//
// GEMM view: M = output pixels of a TH x TW patch (TH * TW = 128), N = output channels (tile BN),
// K = 9 taps x Cin (+ K2). The A tile of one (tap, 64-channel) K-block is one 4-D TMA box of the
// NHWC activation at the tap's offset: out-of-range coordinates read as zero, which is exactly
// the convolution's zero padding. Both operands use the 128-byte swizzled K-major layout.
//
// Roles (320 threads): warp 0 issues TMA, warp 1 owns TMEM and issues tcgen05.mma, warps 2..9
// drain the accumulator (tcgen05.ld), apply the epilogue and store BF16. Two TMEM accumulators
// let the epilogue of one tile overlap the main loop of the next. Every mbarrier wait is bounded:
// on timeout the kernel latches kErrTimeout in the status word and returns.
#include <cuda.h>

#include <mutex>

#include "nst_internal.cuh"
#include "nst_kernels.h"
#include "tc_ptx.cuh"

namespace nst {
namespace {

using namespace nst::tc;

// warp 0: TMA, warp 1: TMEM + MMA, warps 2..9: epilogue (two warps per TMEM lane quarter, each
// draining half of the accumulator's columns)
constexpr int kThreads = 320;
constexpr int kEpiThreads = 256;
constexpr int kBK = 64;                           // channels per K-block (128 bytes of BF16)

struct TcGeom {
  int TH, TW;           // output patch per tile (TH * TW <= the tile's pixel rows; the rows past
                        // TH * TW read stale shared memory and are never stored)
  int tx_bytes;         // bytes one stage's TMA loads deliver
  int tiles_x, tiles_y; // patches per block image
  int n_tiles;          // N tiles (cout / BN)
  int total;            // M tiles * N tiles
  int kb_main;          // taps * cin / 64
  int kb2;              // k2 / 64
  int cin_blocks;       // cin / 64
};

// Origin of output patch (M tile) mt: from the launch's patch list when it has one (each
// block's needed rectangle only), else patch (mt % tiles_x, mt / tiles_x) of block
// mt / (tiles_x tiles_y) on the regular grid over the whole buffer.
__device__ __forceinline__ void patch_origin(const ConvArgs &a, const TcGeom &tg, int mt, int &b,
                                             int &y0, int &x0) {
  if (a.tiles) {
    const int4 t = __ldg(a.tiles + mt);
    b = t.x;
    y0 = t.y;
    x0 = t.z;
  } else {
    const int tx = mt % tg.tiles_x, ty = (mt / tg.tiles_x) % tg.tiles_y;
    b = mt / (tg.tiles_x * tg.tiles_y);
    y0 = ty * tg.TH;
    x0 = tx * tg.TW;
  }
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M = 128, N = n.
__host__ __device__ constexpr uint32_t make_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

// ---- epilogue for 32 consecutive channels of one pixel ------------------------------------------
__device__ __forceinline__ void ld_bf16x8(const __nv_bfloat16 *p, float *v) {
  uint4 t = *reinterpret_cast<const uint4 *>(p);
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&t);
#pragma unroll
  for (int i = 0; i < 4; i++) {
    float2 f = __bfloat1622float2(h[i]);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}
__device__ __forceinline__ void st_bf16x8(__nv_bfloat16 *p, const float *v) {
  uint4 t;
  __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&t);
#pragma unroll
  for (int i = 0; i < 4; i++) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
  *reinterpret_cast<uint4 *>(p) = t;
}

// mrow: when non-null, the ReLU mask of this pixel is read from shared memory instead of a.mask:
// the pixel's 128-byte row (64 channels) of a TMA box with the 128-byte swizzle, whose 16-byte
// chunk j sits at chunk j ^ mswz (mswz = the row's index within its 1024-byte group).
__device__ __forceinline__ void epilogue32(const ConvArgs &a, const BlockGeom &g, int b, int y,
                                           int x, int n, float *v, const uint8_t *mrow = nullptr,
                                           int mswz = 0) {
  const bool valid = y < (g.eh >> a.level) && x < (g.ew >> a.level);
  const size_t o = (((size_t)b * a.Hb + y) * a.Wb + x) * a.cout + n;
  if (a.mode == kEpiForward) {
    const float4 *b4 = reinterpret_cast<const float4 *>(a.bias + n);
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const float4 bb = __ldg(b4 + q);
      v[4 * q] = valid ? fmaxf(v[4 * q] + bb.x, 0.f) : 0.f;
      v[4 * q + 1] = valid ? fmaxf(v[4 * q + 1] + bb.y, 0.f) : 0.f;
      v[4 * q + 2] = valid ? fmaxf(v[4 * q + 2] + bb.z, 0.f) : 0.f;
      v[4 * q + 3] = valid ? fmaxf(v[4 * q + 3] + bb.w, 0.f) : 0.f;
    }
  } else {
    if (!valid) {
#pragma unroll
      for (int j = 0; j < 32; j++) v[j] = 0.f;
    } else {
      if (a.cact) {
        const int gy = (g.ey0 >> a.level) + y, gx = (g.ex0 >> a.level) + x;
        if (gy < a.Hc && gx < a.Wc) {
          const __nv_bfloat16 *ca = reinterpret_cast<const __nv_bfloat16 *>(a.cact) + o;
          const __nv_bfloat16 *ct = reinterpret_cast<const __nv_bfloat16 *>(a.ctgt) +
                                    ((size_t)gy * a.Wc + gx) * a.cout + n;
#pragma unroll
          for (int q = 0; q < 4; q++) {
            float c8[8], t8[8];
            ld_bf16x8(ca + 8 * q, c8);
            ld_bf16x8(ct + 8 * q, t8);
#pragma unroll
            for (int j = 0; j < 8; j++) v[8 * q + j] += a.two_lambda * (c8[j] - t8[j]);
          }
        }
      }
      if (a.addvec) {
#pragma unroll
        for (int j = 0; j < 32; j++) v[j] += __ldg(a.addvec + n + j);
      }
      if (mrow) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint4 raw = *reinterpret_cast<const uint4 *>(
              mrow + ((((n & 63) / 8 + q) ^ mswz) << 4));
          const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&raw);
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const float2 f = __bfloat1622float2(h[i]);
            v[8 * q + 2 * i] = f.x > 0.f ? v[8 * q + 2 * i] : 0.f;
            v[8 * q + 2 * i + 1] = f.y > 0.f ? v[8 * q + 2 * i + 1] : 0.f;
          }
        }
      } else if (a.mask) {
        const __nv_bfloat16 *mk = reinterpret_cast<const __nv_bfloat16 *>(a.mask) + o;
#pragma unroll
        for (int q = 0; q < 4; q++) {
          float m8[8];
          ld_bf16x8(mk + 8 * q, m8);
#pragma unroll
          for (int j = 0; j < 8; j++) v[8 * q + j] = m8[j] > 0.f ? v[8 * q + j] : 0.f;
        }
      }
    }
  }
  if (!a.out) return;   // forward with fused pooling and window positions: nothing else reads it
  __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(a.out) + o;
#pragma unroll
  for (int q = 0; q < 4; q++) st_bf16x8(out + 8 * q, v + 8 * q);
}

// ---- fused 2x2 max pooling in the forward epilogue ---------------------------------------------
// Outside the block's valid pooled region the pooled map is zero. The decision is taken on the
// FP32 activations (accumulator + bias, ReLU), before they are rounded for storage: rounding to
// BF16 merges values that differ by less than half an ulp
// (2^-9 relative), which at a smooth input would turn most windows into exact ties. The pooled
// value is the window max rounded once to BF16; as rounding is monotone, that equals pooling
// the rounded activations.
//
// Window positions for the backward (pool_idx, when a backward pass follows): 4 bits per pooled
// value, bit q set when window pixel q (row-major: 0 = (y, x), 1 = (y, x+1), 2 = (y+1, x),
// 3 = (y+1, x+1)) equals the FP32 window max and that max is positive. The gradient goes to the
// lowest set bit, the first maximum; no bit = the ReLU gate is shut. Layout: one 32-bit word per
// 8 channels c .. c+7 at byte (pooled pixel * C + c) / 2, the nibble of channel c+k at bit
// 8 (k & 3) + 4 (k >> 2).
__device__ __forceinline__ uint32_t pool_nibble_shift(int k) { return 8 * (k & 3) + 4 * (k >> 2); }

// ---- fused 2x2 max pooling of the 64-channel halo kernel, read in the 16x256b layout ------------
// Forward of a 64-channel layer followed by pooling (conv1_2) on 16 x 8 patches: TMEM lane L =
// patch pixel (L / 8, L % 8). One 16x256b read of the 16 lanes 16g .. 16g + 15 of this warp's
// quarter gives thread t the pixels (2r, c) and (2r + 1, c), r = the lanes' pixel-row pair,
// c = t / 4, i.e. the two vertically adjacent pixels of a pooling-window column, for the channel
// pairs 8k + 2(t % 4), +1 (k = 0..3) of the 32 channels at n. The vertical half of each window
// max is in registers, the horizontal half one shuffle away (thread t ^ 4 holds column c ^ 1),
// and the pooled BF16 pairs are formed in place. Bias + ReLU in FP32, zero outside the valid
// region, first maximum decided on the FP32 values, the max rounded once (as in swap_pool8).
//
// Window positions: the 8 threads of a window pair (t / 8 equal) hold disjoint bits of the four
// 32-bit words of its 32 channels (thread t: channels 8k + 2(t % 4), +1 of word k, its column's
// two pixels). A reduce-scatter leaves word j = t % 4 at thread t, OR-ed over the channel pairs
// (exchanges with t ^ 2, then t ^ 1, each passing on the words the partner keeps) and over the
// window's two columns (t ^ 4): 4 shuffles where an OR of all four words at every thread takes 12.
// (Reading both 16-lane halves behind one wait and interleaving them measured 6-7 % slower.)
// pb[k]: the bias of channels n + 8k + 2(t % 4), +1 (loaded once per warp, see the kernel)
__device__ __forceinline__ void halo_pool16(const ConvArgs &a, const BlockGeom &g, int b, int py0,
                                            int px0, int n, uint32_t taddr, const float2 *pb) {
  const int t = threadIdx.x & 31, j = t & 3, c = t >> 2;   // j: channel pair, c: patch column
  float v[16];
  tmem_ld16x256b_x4(taddr, v);
  const int y0 = py0, x = px0 + c;   // top pixel of this thread's column pair (y0 even)
  const int ehl = g.eh >> a.level, ewl = g.ew >> a.level;
  const bool vt = y0 < ehl && x < ewl, vb = y0 + 1 < ehl && x < ewl;
  float m[8];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const float2 bb = pb[k];
#pragma unroll
    for (int e = 0; e < 2; e++) {
      const float bias = e ? bb.y : bb.x;
      float &top = v[4 * k + e], &bot = v[4 * k + 2 + e];
      top = vt ? fmaxf(top + bias, 0.f) : 0.f;
      bot = vb ? fmaxf(bot + bias, 0.f) : 0.f;
      const float mv = fmaxf(top, bot);
      m[2 * k + e] = fmaxf(mv, __shfl_xor_sync(0xffffffffu, mv, 4));
    }
  }
  const bool left = !(c & 1);
  uint32_t idx = 0u;
  if (a.pool_idx) {
    const int qt = left ? 0 : 1;   // window positions of this thread's top / bottom pixel
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      w[k] = 0u;
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const float mm = m[2 * k + e];
        const uint32_t sh = pool_nibble_shift(2 * j + e) + qt;
        w[k] |= (v[4 * k + e] == mm && mm > 0.f) ? 1u << sh : 0u;
        w[k] |= (v[4 * k + 2 + e] == mm && mm > 0.f) ? 1u << (sh + 2) : 0u;
      }
    }
    // keep words {0, 1} (j < 2) or {2, 3}; pass the other two to t ^ 2
    const bool hi = (j & 2) != 0, odd = (j & 1) != 0;
    uint32_t k0 = hi ? w[2] : w[0], k1 = hi ? w[3] : w[1];
    k0 |= __shfl_xor_sync(0xffffffffu, hi ? w[0] : w[2], 2);
    k1 |= __shfl_xor_sync(0xffffffffu, hi ? w[1] : w[3], 2);
    // keep word j; pass the other to t ^ 1
    uint32_t kj = odd ? k1 : k0;
    kj |= __shfl_xor_sync(0xffffffffu, odd ? k0 : k1, 1);
    idx = kj | __shfl_xor_sync(0xffffffffu, kj, 4);   // the window's other column
  }
  if (!left) return;
  const int py = y0 >> 1, px = x >> 1, Hp = a.Hb >> 1, Wp = a.Wb >> 1;
  if (py >= Hp || px >= Wp) return;
  const bool valid = py < (g.eh >> (a.level + 1)) && px < (g.ew >> (a.level + 1));
  const size_t po = (((size_t)b * Hp + py) * Wp + px) * a.cout + n;
  if (a.pool_idx)   // word j: channels n + 8j .. n + 8j + 7
    *reinterpret_cast<uint32_t *>(a.pool_idx + po / 2 + 4 * j) = valid ? idx : 0u;
  __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(a.pool_out) + po + 2 * j;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const __nv_bfloat162 p2 = __floats2bfloat162_rn(valid ? m[2 * k] : 0.f,
                                                   valid ? m[2 * k + 1] : 0.f);
    *reinterpret_cast<__nv_bfloat162 *>(out + 8 * k) = p2;
  }
}

// ---- epilogue through a per-warp transpose tile -----------------------------------------------------
// A warp's 32 x 32 chunk (pixels x channels, FP32) goes to a 4 KB shared-memory tile (row =
// pixel, 16-byte chunks XOR-swizzled by row) and comes back four lanes per pixel, 8 channels
// each: a 16-byte store instruction then covers 8 pixels x 64 contiguous bytes instead of 32
// pixels x 16 bytes at the pixel stride.
constexpr uint32_t kTileT = 32 * 32 * 4;

// 8 consecutive channels (group cg) of chunk pixel j from the warp's transpose tile (row j,
// logical 16-byte chunks 2cg and 2cg + 1, stored at chunk ^ (j % 8))
__device__ __forceinline__ void swap_tile_read8(const uint8_t *tsm, int j, int cg, float *r) {
  const float4 f0 = *reinterpret_cast<const float4 *>(tsm + j * 128 + (((2 * cg) ^ (j & 7)) << 4));
  const float4 f1 =
      *reinterpret_cast<const float4 *>(tsm + j * 128 + (((2 * cg + 1) ^ (j & 7)) << 4));
  r[0] = f0.x; r[1] = f0.y; r[2] = f0.z; r[3] = f0.w;
  r[4] = f1.x; r[5] = f1.y; r[6] = f1.z; r[7] = f1.w;
}

// 8 consecutive FP32 biases (16-byte aligned)
__device__ __forceinline__ void load8_bias(const float *p, float *bb) {
  const float4 b0 = __ldg(reinterpret_cast<const float4 *>(p));
  const float4 b1 = __ldg(reinterpret_cast<const float4 *>(p + 4));
  bb[0] = b0.x; bb[1] = b0.y; bb[2] = b0.z; bb[3] = b0.w;
  bb[4] = b1.x; bb[5] = b1.y; bb[6] = b1.z; bb[7] = b1.w;
}

// epilogue32 for 8 channels n .. n+7 of one pixel; bias8 (forward, optional): their bias,
// already in registers
__device__ __forceinline__ void epilogue8(const ConvArgs &a, const BlockGeom &g, int b, int y,
                                          int x, int n, float *v, const float *bias8 = nullptr) {
  const bool valid = y < (g.eh >> a.level) && x < (g.ew >> a.level);
  const size_t o = (((size_t)b * a.Hb + y) * a.Wb + x) * a.cout + n;
  if (a.mode == kEpiForward) {
    float bb[8];
    if (bias8) {
#pragma unroll
      for (int j = 0; j < 8; j++) bb[j] = bias8[j];
    } else {
      load8_bias(a.bias + n, bb);
    }
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = valid ? fmaxf(v[j] + bb[j], 0.f) : 0.f;
  } else if (!valid) {
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = 0.f;
  } else {
    if (a.cact) {
      const int gy = (g.ey0 >> a.level) + y, gx = (g.ex0 >> a.level) + x;
      if (gy < a.Hc && gx < a.Wc) {
        float c8[8], t8[8];
        ld_bf16x8(reinterpret_cast<const __nv_bfloat16 *>(a.cact) + o, c8);
        ld_bf16x8(reinterpret_cast<const __nv_bfloat16 *>(a.ctgt) +
                      ((size_t)gy * a.Wc + gx) * a.cout + n, t8);
#pragma unroll
        for (int j = 0; j < 8; j++) v[j] += a.two_lambda * (c8[j] - t8[j]);
      }
    }
    if (a.addvec) {
#pragma unroll
      for (int j = 0; j < 8; j++) v[j] += __ldg(a.addvec + n + j);
    }
    if (a.mask) {
      float m8[8];
      ld_bf16x8(reinterpret_cast<const __nv_bfloat16 *>(a.mask) + o, m8);
#pragma unroll
      for (int j = 0; j < 8; j++) v[j] = m8[j] > 0.f ? v[j] : 0.f;
    }
  }
  if (a.out) st_bf16x8(reinterpret_cast<__nv_bfloat16 *>(a.out) + o, v);
}

// fused 2 x 2 max pool of a 32-pixel chunk (whole rows of a patch 8 or 16 wide) from the warp's
// transpose tile: lane = (window, 8-channel group); the window's four values are recomputed in
// FP32 as the forward epilogue forms them (bias, ReLU, valid region), the first maximum is
// decided on those FP32 values, and the max is rounded once to BF16 for the pooled map
__device__ __forceinline__ void swap_pool8(const ConvArgs &a, const BlockGeom &g, int b,
                                           int oy, int ox, const TcGeom &tg, int c, int n,
                                           const uint8_t *tsm, const float *bias8 = nullptr) {
  const int lane = threadIdx.x & 31;
  const int w = lane >> 2, cg = lane & 3;
  const int wpr = tg.TW >> 1;   // windows per row pair
  const int j0 = 2 * (w / wpr) * tg.TW + 2 * (w % wpr);
  const int pp0 = c + j0;
  const int y = oy + pp0 / tg.TW, x = ox + pp0 % tg.TW;
  if (pp0 >= tg.TH * tg.TW || y >= a.Hb || x >= a.Wb) return;
  float bb[8];
  if (bias8) {
#pragma unroll
    for (int j = 0; j < 8; j++) bb[j] = bias8[j];
  } else {
    load8_bias(a.bias + n + cg * 8, bb);
  }
  const int ehl = g.eh >> a.level, ewl = g.ew >> a.level;
  float m[8];
  int k8[8];   // window position (row-major) of the first maximum
#pragma unroll
  for (int qq = 0; qq < 4; qq++) {
    // odd windows visit their pixels in the order 1, 0, 3, 2: the two windows of a quarter-warp
    // then read rows of opposite parity, whose swizzled chunks fall on different banks
    const int q = qq ^ (w & 1);
    const int j = j0 + (q >> 1) * tg.TW + (q & 1);
    const bool valid = y + (q >> 1) < ehl && x + (q & 1) < ewl;
    float r[8];
    swap_tile_read8(tsm, j, cg, r);
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const float s = valid ? fmaxf(r[i] + bb[i], 0.f) : 0.f;
      if (qq == 0 || s > m[i] || (s == m[i] && q < k8[i])) {
        m[i] = s;
        k8[i] = q;
      }
    }
  }
  const int py = y >> 1, px = x >> 1, Hp = a.Hb >> 1, Wp = a.Wb >> 1;
  const bool pv = py < (g.eh >> (a.level + 1)) && px < (g.ew >> (a.level + 1));
  if (!pv) {
#pragma unroll
    for (int i = 0; i < 8; i++) m[i] = 0.f;
  }
  const size_t po = (((size_t)b * Hp + py) * Wp + px) * a.cout + n + cg * 8;
  st_bf16x8(reinterpret_cast<__nv_bfloat16 *>(a.pool_out) + po, m);
  if (a.pool_idx) {   // window positions, in the nibble format above (first max only)
    uint32_t w = 0u;
#pragma unroll
    for (int i = 0; i < 8; i++)
      if (m[i] > 0.f) w |= (1u << k8[i]) << pool_nibble_shift(i);
    *reinterpret_cast<uint32_t *>(a.pool_idx + po / 2) = w;
  }
}

// ---- the kernel -------------------------------------------------------------------------------------
template <int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmA2,
                   const __grid_constant__ CUtensorMap tmB2, const ConvArgs a, const TcGeom tg) {
  constexpr uint32_t A_BYTES = 128 * kBK * 2;
  constexpr uint32_t B_BYTES = BN * kBK * 2;
  constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr uint32_t TMEM_COLS = 2 * BN;
  constexpr uint32_t IDESC = make_idesc(BN);

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(smem_u32(&tfull_bar[i]), 1);
      mbar_init(smem_u32(&tempty_bar[i]), kEpiThreads / 32);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_base_sh), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;
  const int kb_total = tg.kb_main + tg.kb2;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tg.total && ok; t += gridDim.x) {
        const int nt = t % tg.n_tiles, mt = t / tg.n_tiles;
        int b, y0, x0;
        patch_origin(a, tg, mt, b, y0, x0);
        const int n0 = nt * BN;
        for (int kb = 0; kb < kb_total; kb++) {
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          const uint32_t sa = smem_base + stage * STAGE_BYTES, sb = sa + A_BYTES;
          mbar_expect_tx(fb, (uint32_t)tg.tx_bytes);
          if (kb < tg.kb_main) {
            const int tap = kb / tg.cin_blocks, cb = kb % tg.cin_blocks;
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            tma_load_4d(sa, &tmA, fb, cb * kBK, x0 + dx, y0 + dy, b);
            tma_load_2d(sb, &tmB, fb, tap * a.cin + cb * kBK, n0);
          } else {
            const int cb = kb - tg.kb_main;
            tma_load_4d(sa, &tmA2, fb, cb * kBK, x0, y0, b);
            tma_load_2d(sb, &tmB2, fb, cb * kBK, n0);
          }
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tg.total && ok; t += gridDim.x, it++) {
        const int acc = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (!mbar_wait(smem_u32(&tempty_bar[acc]), (use & 1) ^ 1, &abort_flag, a.err)) break;
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * BN);
        for (int kb = 0; kb < kb_total; kb++) {
          if (!mbar_wait(smem_u32(&full_bar[stage]), phase, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_base + stage * STAGE_BYTES, sb = sa + A_BYTES;
          const uint64_t da = sw128_desc(sa), db = sw128_desc(sb);
#pragma unroll
          for (int k = 0; k < kBK / 16; k++)
            mma_bf16(d, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), IDESC,
                     (kb > 0 || k > 0) ? 1u : 0u);
          mma_commit(smem_u32(&empty_bar[stage]));
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
        if (ok) mma_commit(smem_u32(&tfull_bar[acc]));
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int q = warp & 3;           // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2; // which half of the accumulator columns it drains
    uint8_t *tsm = smem_raw + ((smem_base - smem_u32(smem_raw)) + STAGES * STAGE_BYTES +
                               (size_t)(warp - 2) * kTileT);
    int it = 0;
    for (int t = blockIdx.x; t < tg.total; t += gridDim.x, it++) {
      const int acc = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      // lane 0 waits (bounded) and the warp leaves together: the epilogue's warp-wide
      // shuffles and __syncwarp need every lane
      int ready = 0;
      if (lane == 0) ready = mbar_wait_sleep(smem_u32(&tfull_bar[acc]), use & 1, &abort_flag, a.err);
      if (!__shfl_sync(0xffffffffu, ready, 0)) break;
      tc_fence_after();
      const int nt = t % tg.n_tiles, mt = t / tg.n_tiles;
      int b, oy, ox;
      patch_origin(a, tg, mt, b, oy, ox);
      const BlockGeom g = a.geom[b];
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
      const int cg = lane & 3;
#pragma unroll 1
      for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 32) {
        float v[32];
        tmem_ld32(tbase + (uint32_t)c, v);   // row = this lane's pixel, 32 channels
#pragma unroll
        for (int k = 0; k < 8; k++)
          *reinterpret_cast<float4 *>(tsm + lane * 128 + ((k ^ (lane & 7)) << 4)) =
              make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
        __syncwarp();
        float cbias[8];   // (forward) the bias of this thread's 8 channels of the chunk
        if (a.mode == kEpiForward) load8_bias(a.bias + nt * BN + c + cg * 8, cbias);
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int j = k * 8 + (lane >> 2);
          const int pp = q * 32 + j;
          const int y = oy + pp / tg.TW, x = ox + pp % tg.TW;
          if (pp < tg.TH * tg.TW && y < a.Hb && x < a.Wb) {
            float r[8];
            swap_tile_read8(tsm, j, cg, r);
            epilogue8(a, g, b, y, x, nt * BN + c + cg * 8, r,
                      a.mode == kEpiForward ? cbias : nullptr);
          }
        }
        if (a.pool_out) swap_pool8(a, g, b, oy, ox, tg, q * 32, nt * BN + c, tsm);
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();   // every lane of the warp has finished its TMEM reads
      if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[acc]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}


// ---- halo-reuse variant for the narrow layers ----------------------------------------------------
// For the 64/128-channel layers the weights of one N slice (<= 160 KB) stay in shared memory for
// the life of the CTA, and each 64-channel K-block loads ONE activation box of 18 rows x 10
// pixels around a 16 x 8 output patch. The nine taps are nine descriptors into that box,
// shifted by whole 128-byte pixel rows (the patch's 8-pixel rows are 1,280 bytes apart); the
// hardware applies the 128-byte swizzle to absolute shared-memory address bits, so the shifted
// starts read exactly what the TMA wrote. Every input pixel crosses L2 -> shared memory once
// per K-block instead of nine times. Phase-2 K-blocks (the fused V R term) use the centre tap.
constexpr int kHaloTH = 16, kHaloTW = 8, kHaloBoxW = kHaloTW + 2, kHaloBoxH = kHaloTH + 2;
constexpr uint32_t kHaloBoxBytes = kHaloBoxW * kHaloBoxH * 128;        // 23,040
constexpr uint32_t kHaloStage = (kHaloBoxBytes + 1023u) & ~1023u;      // 23,552
constexpr uint32_t kHaloSmemMax = 227 * 1024;
// the fused input-gradient form (MASK_SMEM): main-phase boxes in kMaskAStages stages, the tile's
// own 16 x 8 phase-2 box (16 KB) in a ring of kMaskVStages
constexpr int kMaskAStages = 3, kMaskVStages = 4;
constexpr uint32_t kMaskVStage = 128 * 128;

template <int BN, int KB, int P2KB, int NT>
struct HaloCfg {
  static constexpr uint32_t TILE_B = BN * 128;                  // one (tap, K-block) weight tile
  static constexpr uint32_t W_BYTES = (9 * KB + P2KB) * TILE_B;
  static constexpr int STAGES_RAW = (int)((kHaloSmemMax - 1024 - W_BYTES) / kHaloStage);
  // two boxes per tile (the fused V R phase) get three tiles in flight; one box per tile keeps
  // four stages (six measured slower on conv1_2's forward, faster on its input gradient)
  static constexpr int CAP = P2KB ? 6 : 4;
  static constexpr int STAGES = STAGES_RAW > CAP ? CAP : STAGES_RAW;
  static constexpr size_t SMEM = 1024 + W_BYTES + (size_t)STAGES * kHaloStage;
};

template <int BN, int KB, int P2KB, int NT, bool MASK_SMEM>
__global__ void __launch_bounds__(kThreads, 1)
    conv_tc_halo_kernel(const __grid_constant__ CUtensorMap tmA,
                        const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmA2,
                        const __grid_constant__ CUtensorMap tmB2, const ConvArgs a,
                        const TcGeom tg) {
  using Cfg = HaloCfg<BN, KB, P2KB, NT>;
  constexpr int STAGES = Cfg::STAGES;
  // four accumulators in TMEM (512 columns at N = 128): the tiles are short, and more tiles in
  // flight keep the tensor pipe fed while the epilogue drains
  constexpr int NACC = 4;
  constexpr uint32_t TMEM_COLS = NACC * BN;
  constexpr uint32_t IDESC = make_idesc(BN);
  constexpr int KBT = KB + P2KB;   // K-blocks per tile
  // MASK_SMEM: the phase-2 K-block is the fused V R term of an input gradient whose ReLU mask
  // is that same activation V. Its box is the tile's own 16 x 8 pixels (the V R term reads the
  // centre tap only, the mask the pixel itself): 16 KB in a ring of its own (SV stages), read by
  // the MMAs and then by the epilogue, whose warps release it; the main-phase boxes keep SA
  // stages, released by the MMA.
  static_assert(!MASK_SMEM || (KB == 1 && P2KB == 1 && NT == 1 && BN == 64),
                "mask from the phase-2 box");
  constexpr int SA = MASK_SMEM ? kMaskAStages : STAGES;
  constexpr int SV = MASK_SMEM ? kMaskVStages : 1;

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], w_bar;
  __shared__ __align__(8) uint64_t vfull_bar[SV], vempty_bar[SV];
  __shared__ __align__(8) uint64_t tfull_bar[NACC], tempty_bar[NACC];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t w_base = smem_base, a_base = smem_base + Cfg::W_BYTES;
  const uint32_t v_base = a_base + SA * kHaloStage;   // (MASK_SMEM) the phase-2 ring
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this CTA's N slice, and its share of the M tiles
  const int nt = blockIdx.x % NT, m_first = blockIdx.x / NT, m_step = gridDim.x / NT;
  const int m_total = tg.total;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; s++) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int s = 0; s < SV; s++) {
      mbar_init(smem_u32(&vfull_bar[s]), 1);
      mbar_init(smem_u32(&vempty_bar[s]), kEpiThreads / 32);
    }
    mbar_init(smem_u32(&w_bar), 1);
    for (int i = 0; i < NACC; i++) {
      mbar_init(smem_u32(&tfull_bar[i]), 1);
      mbar_init(smem_u32(&tempty_bar[i]), kEpiThreads);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_base_sh), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      // resident weights of slice nt: tile (tap, cb) at w_base + (tap * KB + cb) * TILE_B, then
      // the phase-2 tiles (R rows of the slice)
      const uint32_t wb = smem_u32(&w_bar);
      mbar_expect_tx(wb, Cfg::W_BYTES);
      for (int tap = 0; tap < 9; tap++)
        for (int cb = 0; cb < KB; cb++)
          tma_load_2d(w_base + (tap * KB + cb) * Cfg::TILE_B, &tmB, wb, tap * a.cin + cb * kBK,
                      nt * BN);
      for (int cb = 0; cb < P2KB; cb++)
        tma_load_2d(w_base + (9 * KB + cb) * Cfg::TILE_B, &tmB2, wb, cb * kBK, nt * BN);
      int stage = 0, vst = 0;
      uint32_t phase = 0, vph = 0;
      bool ok = true;
      for (int t = m_first; t < m_total && ok; t += m_step) {
        int b, oy, ox;
        patch_origin(a, tg, t, b, oy, ox);
        for (int kb = 0; kb < KBT; kb++) {
          if (MASK_SMEM && kb == KB) {   // the tile's own pixels of V (no halo)
            if (!mbar_wait(smem_u32(&vempty_bar[vst]), vph ^ 1, &abort_flag, a.err)) {
              ok = false;
              break;
            }
            const uint32_t fb = smem_u32(&vfull_bar[vst]);
            mbar_expect_tx(fb, kMaskVStage);
            tma_load_4d(v_base + vst * kMaskVStage, &tmA2, fb, 0, ox, oy, b);
            if (++vst == SV) { vst = 0; vph ^= 1; }
            continue;
          }
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          mbar_expect_tx(fb, kHaloBoxBytes);
          const uint32_t sa = a_base + stage * kHaloStage;
          if (kb < KB)
            tma_load_4d(sa, &tmA, fb, kb * kBK, ox - 1, oy - 1, b);
          else
            tma_load_4d(sa, &tmA2, fb, (kb - KB) * kBK, ox - 1, oy - 1, b);
          if (++stage == SA) { stage = 0; phase ^= 1; }
        }
      }
    }
  } else if (warp == 1) {
    // The whole warp runs the issue loop (its waits and loop control are warp-uniform), and one
    // elected lane issues each K-block's MMAs and commit: a loop run by a single lane issues
    // several times slower once epilogue warps keep this warp's scheduler busy, and a 64-wide
    // MMA takes only 48 cycles. (The 256-wide MMAs of the other kernels take 128 cycles; there
    // the single-lane loop keeps up and measured slightly faster.)
    bool ok = mbar_wait_warp(smem_u32(&w_bar), 0, &abort_flag, a.err);
    int stage = 0, vst = 0;
    uint32_t phase = 0, vph = 0;
    int it = 0;
    for (int t = m_first; t < m_total && ok; t += m_step, it++) {
      const int acc = it % NACC;
      const uint32_t use = (uint32_t)(it / NACC);
      if (!mbar_wait_warp(smem_u32(&tempty_bar[acc]), (use & 1) ^ 1, &abort_flag, a.err)) break;
      tc_fence_after();
      const uint32_t d = tmem_base + (uint32_t)(acc * BN);
      for (int kb = 0; kb < KBT; kb++) {
        if (MASK_SMEM && kb == KB) {   // V R from the tile's own 16 x 8 box (no commit: the
          // epilogue reads the mask from it and releases the stage)
          if (!mbar_wait_warp(smem_u32(&vfull_bar[vst]), vph, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (elect_one()) {
            const uint64_t da = sw128_desc(v_base + vst * kMaskVStage);
            const uint64_t db = sw128_desc(w_base + 9 * KB * Cfg::TILE_B);
#pragma unroll
            for (int k = 0; k < kBK / 16; k++)
              mma_bf16(d, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), IDESC, 1u);
          }
          __syncwarp();
          if (++vst == SV) { vst = 0; vph ^= 1; }
          continue;
        }
        if (!mbar_wait_warp(smem_u32(&full_bar[stage]), phase, &abort_flag, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = a_base + stage * kHaloStage;
        // shifted by whole 128-byte rows; the swizzle follows absolute address bits, so the
        // phase field stays 0 (the box itself starts 1024-aligned). Descriptors are the stage's
        // base descriptors plus compile-time offsets (address field in 16-byte units).
        // One lane (the same one each time) is elected per K-block and issues its unrolled run
        // of MMAs and the commit: one branch per K-block instead of one per MMA.
        if (elect_one()) {
          const uint64_t da0 = sw128_desc_k(sa, kHaloBoxW * 128, 0);
          if (kb < KB) {
            const uint64_t db0 = sw128_desc(w_base + kb * Cfg::TILE_B);
#pragma unroll
            for (int tap = 0; tap < 9; tap++) {
              const uint64_t da = da0 + (uint64_t)(((tap / 3) * kHaloBoxW + tap % 3) * 8);
              const uint64_t db = db0 + (uint64_t)(tap * KB * (Cfg::TILE_B >> 4));
#pragma unroll
              for (int k = 0; k < kBK / 16; k++)
                mma_bf16(d, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), IDESC,
                         kb == 0 && tap == 0 && k == 0 ? 0u : 1u);
            }
          } else {   // phase 2: the V R term, centre tap only (after phase 1: accumulate)
            const uint64_t da = da0 + (uint64_t)((kHaloBoxW + 1) * 8);
            const uint64_t db = sw128_desc(w_base + (9 * KB + kb - KB) * Cfg::TILE_B);
#pragma unroll
            for (int k = 0; k < kBK / 16; k++)
              mma_bf16(d, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), IDESC, 1u);
          }
          mma_commit(smem_u32(&empty_bar[stage]));
        }
        __syncwarp();
        if (++stage == SA) { stage = 0; phase ^= 1; }
      }
      if (!ok) break;
      if (elect_one()) mma_commit(smem_u32(&tfull_bar[acc]));
    }
  } else {
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    // pooled forward (BN = 64: one 32-channel chunk per warp): the bias pairs this thread
    // applies on every tile, loaded once
    float2 pbias[4] = {};
    if (a.pool_out && BN == 64)
#pragma unroll
      for (int k = 0; k < 4; k++)
        pbias[k] = __ldg(reinterpret_cast<const float2 *>(a.bias + nt * BN + half * (BN / 2) +
                                                          8 * k + 2 * (lane & 3)));
    int it = 0;
    for (int t = m_first; t < m_total; t += m_step, it++) {
      const int acc = it % NACC;
      const uint32_t use = (uint32_t)(it / NACC);
      // lane 0 waits (bounded) and the warp leaves together: the epilogue's warp-wide
      // shuffles and __syncwarp need every lane
      int ready = 0;
      if (lane == 0) ready = mbar_wait_sleep(smem_u32(&tfull_bar[acc]), use & 1, &abort_flag, a.err);
      if (!__shfl_sync(0xffffffffu, ready, 0)) break;
      tc_fence_after();
      int b, oy, ox;
      patch_origin(a, tg, t, b, oy, ox);
      const int y = oy + row / kHaloTW, x = ox + row % kHaloTW;
      const bool inb = y < a.Hb && x < a.Wb;
      const BlockGeom g = a.geom[b];
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
      // the ReLU mask from the tile's phase-2 box (this pixel's row: box pixel = patch pixel);
      // its full barrier completed before the MMAs that the accumulator waited for, and waiting
      // on it here acquires the TMA's writes
      const uint8_t *mrow = nullptr;
      int mswz = 0, ms = 0;
      if constexpr (MASK_SMEM) {
        ms = it % SV;
        int mok = 0;
        if (lane == 0)
          mok = mbar_wait_sleep(smem_u32(&vfull_bar[ms]), (uint32_t)(it / SV) & 1u, &abort_flag,
                                a.err);
        if (!__shfl_sync(0xffffffffu, mok, 0)) break;
        mrow = smem_raw + (v_base - smem_u32(smem_raw)) + (size_t)ms * kMaskVStage +
               (size_t)row * 128;
        mswz = row & 7;
      }
      if (a.pool_out) {
        // pooled forward: two 16-lane reads of the 16x256b layout (pixel-row pairs 4q, 4q + 2)
#pragma unroll 1
        for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 32) {
          float2 pb[4];   // (other widths: this chunk's bias pairs)
          const float2 *bp = pbias;
          if constexpr (BN != 64) {
#pragma unroll
            for (int k = 0; k < 4; k++)
              pb[k] = __ldg(reinterpret_cast<const float2 *>(a.bias + nt * BN + c + 8 * k +
                                                             2 * (lane & 3)));
            bp = pb;
          }
#pragma unroll
          for (int grp = 0; grp < 2; grp++)
            halo_pool16(a, g, b, oy + 4 * q + 2 * grp, ox, nt * BN + c,
                        tbase + ((uint32_t)(16 * grp) << 16) + (uint32_t)c, bp);
        }
      } else {
#pragma unroll 1
        for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 32) {
          float v[32];
          tmem_ld32(tbase + (uint32_t)c, v);
          if (inb) epilogue32(a, g, b, y, x, nt * BN + c, v, mrow, mswz);
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty_bar[acc]));
      if constexpr (MASK_SMEM) {   // every lane has read its mask row: release the box's stage
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&vempty_bar[ms]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// ---- pixels-as-N variant for 128-channel outputs ---------------------------------------------------
// With Cout = 128 the natural tile (M = 128 pixels, N = 128 channels) issues MMAs half as wide as
// the 256-channel layers, and a narrow MMA costs nearly as much issue time as a wide one. Here the
// roles swap: M = the 128 output channels (A = a 128 x 64 weight box), N = 256 output pixels of a
// TH x TW patch (B = the activation box), so every tcgen05.mma is 128 x 256 x 16 like the widest
// layers. The accumulator holds D[channel][pixel]; each epilogue warp reads 32 channels x 32
// pixels, transposes them through a private 4 KB shared-memory tile (16-byte chunks XOR-swizzled
// by row, conflict-free both ways) and then runs the same per-pixel epilogue as the other kernels
// (one pixel per lane, 32 consecutive channels).
constexpr int kSwapBN = 128;                    // output channels per tile (M)
constexpr int kSwapBP = 256;                    // output pixels per tile (N)
constexpr uint32_t kSwapA = kSwapBN * kBK * 2;  // 16 KB weight box
constexpr uint32_t kSwapB = kSwapBP * kBK * 2;  // 32 KB activation box

template <int STAGES>
__global__ void __launch_bounds__(kThreads, 1)
    conv_tc_swap_kernel(const __grid_constant__ CUtensorMap tmA,
                        const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmA2,
                        const __grid_constant__ CUtensorMap tmB2, const ConvArgs a,
                        const TcGeom tg) {
  constexpr uint32_t STAGE_BYTES = kSwapA + kSwapB;
  constexpr uint32_t TMEM_COLS = 2 * kSwapBP;
  constexpr uint32_t IDESC = make_idesc(kSwapBP);

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t *smem_gen = smem_raw + (smem_base - smem_u32(smem_raw));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(smem_u32(&tfull_bar[i]), 1);
      mbar_init(smem_u32(&tempty_bar[i]), kEpiThreads / 32);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_base_sh), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;
  const int kb_total = tg.kb_main + tg.kb2;

  if (warp == 0) {
    // ---------------- TMA producer: weight box (A) + activation box (B) per K-block ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tg.total && ok; t += gridDim.x) {
        const int nt = t % tg.n_tiles, mt = t / tg.n_tiles;
        int b, y0, x0;
        patch_origin(a, tg, mt, b, y0, x0);
        const int n0 = nt * kSwapBN;
        for (int kb = 0; kb < kb_total; kb++) {
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          const uint32_t sw = smem_base + stage * STAGE_BYTES, sx = sw + kSwapA;
          mbar_expect_tx(fb, (uint32_t)tg.tx_bytes);
          if (kb < tg.kb_main) {
            const int tap = kb / tg.cin_blocks, cb = kb % tg.cin_blocks;
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            tma_load_2d(sw, &tmB, fb, tap * a.cin + cb * kBK, n0);
            tma_load_4d(sx, &tmA, fb, cb * kBK, x0 + dx, y0 + dy, b);
          } else {
            const int cb = kb - tg.kb_main;
            tma_load_2d(sw, &tmB2, fb, cb * kBK, n0);
            tma_load_4d(sx, &tmA2, fb, cb * kBK, x0, y0, b);
          }
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: D[128 ch][256 px] += W[128 x 64] X[256 x 64]^T ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tg.total && ok; t += gridDim.x, it++) {
        const int acc = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (!mbar_wait(smem_u32(&tempty_bar[acc]), (use & 1) ^ 1, &abort_flag, a.err)) break;
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * kSwapBP);
        for (int kb = 0; kb < kb_total; kb++) {
          if (!mbar_wait(smem_u32(&full_bar[stage]), phase, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sw = smem_base + stage * STAGE_BYTES, sx = sw + kSwapA;
          const uint64_t dw = sw128_desc(sw), dx = sw128_desc(sx);
#pragma unroll
          for (int k = 0; k < kBK / 16; k++)
            mma_bf16(d, dw + (uint64_t)(k * 2), dx + (uint64_t)(k * 2), IDESC,
                     (kb > 0 || k > 0) ? 1u : 0u);
          mma_commit(smem_u32(&empty_bar[stage]));
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
        if (ok) mma_commit(smem_u32(&tfull_bar[acc]));
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int q = warp & 3;            // TMEM lane quarter = channels q*32 .. q*32+31 of the tile
    const int half = (warp - 2) >> 2;  // pixels half*128 .. half*128+127 of the patch
    uint8_t *tsm = smem_gen + STAGES * STAGE_BYTES + (size_t)(warp - 2) * kTileT;
    // forward with one channel tile: this thread's 8 channels (q * 32 + 8 (lane % 4)) are the
    // same on every tile, so their bias is loaded once
    float sbias[8];
    const bool hoist = a.mode == kEpiForward && tg.n_tiles == 1;
    if (hoist) load8_bias(a.bias + q * 32 + (lane & 3) * 8, sbias);
    int it = 0;
    for (int t = blockIdx.x; t < tg.total; t += gridDim.x, it++) {
      const int acc = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      // lane 0 waits (bounded) and the warp leaves together: the epilogue's warp-wide
      // shuffles and __syncwarp need every lane
      int ready = 0;
      if (lane == 0) ready = mbar_wait_sleep(smem_u32(&tfull_bar[acc]), use & 1, &abort_flag, a.err);
      if (!__shfl_sync(0xffffffffu, ready, 0)) break;
      tc_fence_after();
      const int nt = t % tg.n_tiles, mt = t / tg.n_tiles;
      int b, oy, ox;
      patch_origin(a, tg, mt, b, oy, ox);
      const BlockGeom g = a.geom[b];
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kSwapBP);
      const int n = nt * kSwapBN + q * 32;
#pragma unroll 1
      for (int c = half * (kSwapBP / 2); c < (half + 1) * (kSwapBP / 2); c += 32) {
        float v[32];
        tmem_ld32(tbase + (uint32_t)c, v);   // v[j] = D[channel n + lane][pixel c + j]
        // transpose: row j of the tile = pixel c + j, 16-byte chunk (lane / 4) ^ (j % 8)
#pragma unroll
        for (int j = 0; j < 32; j++)
          *reinterpret_cast<float *>(tsm + j * 128 + ((((lane >> 2) ^ (j & 7)) << 4) |
                                                      ((lane & 3) << 2))) = v[j];
        __syncwarp();
        // read back four lanes per pixel (8 channels each): every 16-byte store of the warp then
        // covers 8 pixels x 64 contiguous bytes
        const int cg = lane & 3;
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int j = k * 8 + (lane >> 2);   // pixel of the chunk
          float r[8];
          swap_tile_read8(tsm, j, cg, r);
          const int pp = c + j;
          const int y = oy + pp / tg.TW, x = ox + pp % tg.TW;
          if (pp < tg.TH * tg.TW && y < a.Hb && x < a.Wb)
            epilogue8(a, g, b, y, x, n + cg * 8, r, hoist ? sbias : nullptr);
        }
        if (a.pool_out) swap_pool8(a, g, b, oy, ox, tg, c, n, tsm, hoist ? sbias : nullptr);
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();   // every lane of the warp has finished its TMEM reads
      if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[acc]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// ---- pixels-as-N halo variant for 64 -> 128 channels ------------------------------------------------
// conv2_1's forward: M = the 128 output channels (A = one tap's 128 x 64 weight tile, streamed
// from L2 tap by tap), N = the 256 pixels of a 32 x 8 output patch (B = ONE 34 x 10 activation
// box per tile; the nine taps are nine descriptors into it, shifted by whole 128-byte pixel rows,
// with 8-row groups one box row = 1,280 bytes apart). Every tcgen05.mma is 128 x 256 x 16, the
// full-rate shape (a 64-channel input gives the M = pixels form 128-wide MMAs that read both
// operands at the shared-memory bandwidth), and each activation pixel crosses L2 -> shared memory
// once per tile instead of once per tap. Epilogue as in the pixels-as-N kernel.
constexpr int kSHTH = 32, kSHTW = 8, kSHBoxW = kSHTW + 2, kSHBoxH = kSHTH + 2;
constexpr uint32_t kSHBoxBytes = kSHBoxW * kSHBoxH * 128;          // 43,520
constexpr uint32_t kSHBoxStage = (kSHBoxBytes + 1023u) & ~1023u;   // 44,032
constexpr int kSHBoxStages = 2;
constexpr uint32_t kSHWTile = kSwapBN * kBK * 2;                   // 16 KB
constexpr int kSHWStages = 4;
constexpr size_t kSHSmem =
    1024 + kSHBoxStages * kSHBoxStage + kSHWStages * kSHWTile + 8 * kTileT;

__global__ void __launch_bounds__(kThreads, 1)
    conv_tc_swap_halo_kernel(const __grid_constant__ CUtensorMap tmA,
                             const __grid_constant__ CUtensorMap tmW, const ConvArgs a,
                             const TcGeom tg) {
  constexpr uint32_t TMEM_COLS = 2 * kSwapBP;
  constexpr uint32_t IDESC = make_idesc(kSwapBP);

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bfull[kSHBoxStages], bempty[kSHBoxStages];
  __shared__ __align__(8) uint64_t wfull[kSHWStages], wempty[kSHWStages];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t *smem_gen = smem_raw + (smem_base - smem_u32(smem_raw));
  const uint32_t box_base = smem_base, w_base = smem_base + kSHBoxStages * kSHBoxStage;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kSHBoxStages; s++) {
      mbar_init(smem_u32(&bfull[s]), 1);
      mbar_init(smem_u32(&bempty[s]), 1);
    }
    for (int s = 0; s < kSHWStages; s++) {
      mbar_init(smem_u32(&wfull[s]), 1);
      mbar_init(smem_u32(&wempty[s]), 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(smem_u32(&tfull_bar[i]), 1);
      mbar_init(smem_u32(&tempty_bar[i]), kEpiThreads / 32);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_base_sh), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  if (warp == 0) {
    // ---------------- TMA producer: one box per tile, one weight tile per tap ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmW)) : "memory");
      int bs = 0, ws = 0;
      uint32_t bph = 0, wph = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tg.total && ok; t += gridDim.x) {
        int b, oy, ox;
        patch_origin(a, tg, t, b, oy, ox);
        if (!mbar_wait(smem_u32(&bempty[bs]), bph ^ 1, &abort_flag, a.err)) break;
        mbar_expect_tx(smem_u32(&bfull[bs]), kSHBoxBytes);
        tma_load_4d(box_base + bs * kSHBoxStage, &tmA, smem_u32(&bfull[bs]), 0, ox - 1, oy - 1, b);
        if (++bs == kSHBoxStages) { bs = 0; bph ^= 1; }
        for (int tap = 0; tap < 9; tap++) {
          if (!mbar_wait(smem_u32(&wempty[ws]), wph ^ 1, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          mbar_expect_tx(smem_u32(&wfull[ws]), kSHWTile);
          tma_load_2d(w_base + ws * kSHWTile, &tmW, smem_u32(&wfull[ws]), tap * kBK, 0);
          if (++ws == kSHWStages) { ws = 0; wph ^= 1; }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: D[128 ch][256 px] += W_tap[128 x 64] X_tap[256 x 64]^T ----------
    if (lane == 0) {
      int bs = 0, ws = 0, it = 0;
      uint32_t bph = 0, wph = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tg.total && ok; t += gridDim.x, it++) {
        const int acc = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (!mbar_wait(smem_u32(&tempty_bar[acc]), (use & 1) ^ 1, &abort_flag, a.err)) break;
        tc_fence_after();
        if (!mbar_wait(smem_u32(&bfull[bs]), bph, &abort_flag, a.err)) break;
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * kSwapBP);
        // the box's 8-row groups (patch rows) are one box row apart; the swizzle follows
        // absolute address bits, so shifted starts keep the phase field at 0
        const uint64_t db0 = sw128_desc_k(box_base + bs * kSHBoxStage, kSHBoxW * 128, 0);
        for (int tap = 0; tap < 9; tap++) {
          if (!mbar_wait(smem_u32(&wfull[ws]), wph, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t da = sw128_desc(w_base + ws * kSHWTile);
          const uint64_t db = db0 + (uint64_t)(((tap / 3) * kSHBoxW + tap % 3) * 8);
#pragma unroll
          for (int k = 0; k < kBK / 16; k++)
            mma_bf16(d, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), IDESC,
                     (tap > 0 || k > 0) ? 1u : 0u);
          mma_commit(smem_u32(&wempty[ws]));
          if (++ws == kSHWStages) { ws = 0; wph ^= 1; }
        }
        if (!ok) break;
        mma_commit(smem_u32(&bempty[bs]));
        if (++bs == kSHBoxStages) { bs = 0; bph ^= 1; }
        mma_commit(smem_u32(&tfull_bar[acc]));
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9), as in the pixels-as-N kernel ----------------
    const int q = warp & 3;            // TMEM lane quarter = channels q*32 .. q*32+31
    const int half = (warp - 2) >> 2;  // pixels half*128 .. half*128+127 of the patch
    uint8_t *tsm = smem_gen + kSHBoxStages * kSHBoxStage + kSHWStages * kSHWTile +
                   (size_t)(warp - 2) * kTileT;
    float sbias[8];   // (forward) this thread's 8 channels' bias, the same on every tile
    const bool hoist = a.mode == kEpiForward;
    if (hoist) load8_bias(a.bias + q * 32 + (lane & 3) * 8, sbias);
    int it = 0;
    for (int t = blockIdx.x; t < tg.total; t += gridDim.x, it++) {
      const int acc = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      int ready = 0;
      if (lane == 0) ready = mbar_wait_sleep(smem_u32(&tfull_bar[acc]), use & 1, &abort_flag, a.err);
      if (!__shfl_sync(0xffffffffu, ready, 0)) break;
      tc_fence_after();
      int b, oy, ox;
      patch_origin(a, tg, t, b, oy, ox);
      const BlockGeom g = a.geom[b];
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kSwapBP);
      const int n = q * 32;
#pragma unroll 1
      for (int c = half * (kSwapBP / 2); c < (half + 1) * (kSwapBP / 2); c += 32) {
        float v[32];
        tmem_ld32(tbase + (uint32_t)c, v);   // v[j] = D[channel n + lane][pixel c + j]
#pragma unroll
        for (int j = 0; j < 32; j++)
          *reinterpret_cast<float *>(tsm + j * 128 + ((((lane >> 2) ^ (j & 7)) << 4) |
                                                      ((lane & 3) << 2))) = v[j];
        __syncwarp();
        const int cg = lane & 3;
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int j = k * 8 + (lane >> 2);
          float r[8];
          swap_tile_read8(tsm, j, cg, r);
          const int pp = c + j;
          const int y = oy + pp / kSHTW, x = ox + pp % kSHTW;
          if (y < a.Hb && x < a.Wb)
            epilogue8(a, g, b, y, x, n + cg * 8, r, hoist ? sbias : nullptr);
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();   // every lane of the warp has finished its TMEM reads
      if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[acc]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// ---- failure path check ----------------------------------------------------------------------------
// One CTA waits on an mbarrier that nothing will complete, with the same bounded wait the
// convolution kernels use but a short limit: the wait runs out, kErrTimeout is latched in the
// status word and the kernel returns. No fault, no hang; the context stays usable.
__global__ void timeout_check_kernel(long long limit, unsigned *err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_limit(smem_u32(&bar), 0, &abort_flag, err, limit);
}

// ---- host side -------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn g_encode = nullptr;
int g_num_sms = 0;
bool g_tc_ok = false;
std::once_flag g_once;

void init_once() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return;
  g_num_sms = prop.multiProcessorCount;
  if (prop.major != 10) return;  // tcgen05 needs a Blackwell data-center part
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return;
  g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  g_tc_ok = true;
}

// NHWC BF16 activation [B][H][W][C] as a 4-D tensor map with a (64, TW, TH, 1) box
cudaError_t encode_act(CUtensorMap *m, const void *ptr, int B, int H, int W, int C, int TH,
                       int TW) {
  cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  cuuint32_t box[4] = {(cuuint32_t)kBK, (cuuint32_t)TW, (cuuint32_t)TH, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(ptr), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// weights [N][K] (K contiguous) as a 2-D tensor map with a (64, BN) box
cudaError_t encode_wt(CUtensorMap *m, const void *ptr, int N, int K, int BN) {
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)N};
  cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)BN};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int STAGES>
cudaError_t launch_bn(const CUtensorMap &A, const CUtensorMap &B, const CUtensorMap &A2,
                      const CUtensorMap &B2, const ConvArgs &a, const TcGeom &tg,
                      cudaStream_t s) {
  constexpr size_t smem = (size_t)STAGES * (128 * kBK * 2 + BN * kBK * 2) + 8 * kTileT + 1024;
  static_assert(smem <= 227 * 1024, "tcgen05 convolution shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<BN, STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int grid = std::min(tg.total, g_num_sms);
  conv_tc_kernel<BN, STAGES><<<grid, kThreads, smem, s>>>(A, B, A2, B2, a, tg);
  return cudaGetLastError();
}

template <int STAGES>
cudaError_t launch_swap(const CUtensorMap &A, const CUtensorMap &B, const CUtensorMap &A2,
                        const CUtensorMap &B2, const ConvArgs &a, const TcGeom &tg,
                        cudaStream_t s) {
  constexpr size_t smem = (size_t)STAGES * (kSwapA + kSwapB) + 8 * kTileT + 1024;
  static_assert(smem <= 227 * 1024, "pixels-as-N kernel shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv_tc_swap_kernel<STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int grid = std::min(tg.total, g_num_sms);
  conv_tc_swap_kernel<STAGES><<<grid, kThreads, smem, s>>>(A, B, A2, B2, a, tg);
  return cudaGetLastError();
}

// Output patch of at most `rows` pixels (the tile's M or N) covering n rectangles h[i] x w[i]
// with the fewest tiles. Without fused pooling any TH x TW <= rows works (a 9 x 14 patch tiles
// an 84 x 98 map with 97 % of the MMA rows in use where 8 x 16 reaches 83 %); with fused pooling
// the 2 x 2 windows must pair up inside a 32-pixel epilogue chunk, so TW is 8 or 16 and
// TH * TW = rows.
void pick_patch_multi(const int *h, const int *w, int n, int rows, bool pool, int &TH, int &TW) {
  long long best_tiles = -1;
  int best_area = 0;
  TH = 1;
  TW = rows;
  for (int th = 1; th <= rows && th <= 256; th++) {
    const int tw = rows / th;
    if (tw < 1 || tw > 256) continue;
    if (pool && !((tw == 8 || tw == 16) && th * tw == rows)) continue;
    long long tiles = 0;
    for (int i = 0; i < n; i++) tiles += (long long)((h[i] + th - 1) / th) * ((w[i] + tw - 1) / tw);
    if (best_tiles < 0 || tiles < best_tiles || (tiles == best_tiles && th * tw > best_area)) {
      best_tiles = tiles;
      best_area = th * tw;
      TH = th;
      TW = tw;
    }
  }
}

void pick_patch_rows(int H, int W, int rows, int &TH, int &TW, bool pool) {
  pick_patch_multi(&H, &W, 1, rows, pool, TH, TW);
}

template <int BN, int KB, int P2KB, int NT, bool MASK_SMEM = false>
cudaError_t launch_halo(const CUtensorMap &A, const CUtensorMap &B, const CUtensorMap &A2,
                        const CUtensorMap &B2, const ConvArgs &a, cudaStream_t s) {
  using Cfg = HaloCfg<BN, KB, P2KB, NT>;
  // (MASK_SMEM: the main-phase ring and the 16 x 8 phase-2 ring)
  constexpr size_t smem = MASK_SMEM ? 1024 + Cfg::W_BYTES + (size_t)kMaskAStages * kHaloStage +
                                          (size_t)kMaskVStages * kMaskVStage
                                    : Cfg::SMEM;
  static_assert(Cfg::STAGES >= 2, "halo kernel needs two activation stages");
  static_assert(smem <= kHaloSmemMax, "halo kernel shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv_tc_halo_kernel<BN, KB, P2KB, NT, MASK_SMEM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TcGeom tg{};
  tg.TH = kHaloTH;
  tg.TW = kHaloTW;
  tg.tiles_x = (a.Wb + kHaloTW - 1) / kHaloTW;
  tg.tiles_y = (a.Hb + kHaloTH - 1) / kHaloTH;
  tg.n_tiles = NT;
  // M tiles; every slice covers all of them
  tg.total = a.tiles ? a.n_mtiles : a.B * tg.tiles_x * tg.tiles_y;
  if (tg.total <= 0) return cudaSuccess;
  int grid = std::min(tg.total * NT, g_num_sms);
  grid = std::max(NT, grid / NT * NT);
  conv_tc_halo_kernel<BN, KB, P2KB, NT, MASK_SMEM><<<grid, kThreads, smem, s>>>(A, B, A2, B2, a,
                                                                             tg);
  return cudaGetLastError();
}

// 4-D map of an activation with the halo box (64 ch, 10 px, 18 rows, 1)
cudaError_t encode_act_halo(CUtensorMap *m, const void *ptr, int B, int H, int W, int C) {
  cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  cuuint32_t box[4] = {(cuuint32_t)kBK, (cuuint32_t)kHaloBoxW, (cuuint32_t)kHaloBoxH, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(ptr), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// conv2_1's forward shape (64 -> 128 channels, no fused term): the pixels-as-N halo kernel
bool swap_halo_shape(const ConvArgs &a) {
  return a.taps == 9 && a.cin == 64 && a.cout == kSwapBN && a.k2 == 0 && !a.pool_out;
}

cudaError_t launch_swap_halo(const ConvArgs &a, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv_tc_swap_halo_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSHSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (a.tiles && (a.TH != kSHTH || a.TW != kSHTW)) return cudaErrorInvalidValue;
  CUtensorMap mA, mW;
  cudaError_t e;
  {
    cuuint64_t dims[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.Wb, (cuuint64_t)a.Hb, (cuuint64_t)a.B};
    cuuint64_t strides[3] = {(cuuint64_t)a.cin * 2, (cuuint64_t)a.Wb * a.cin * 2,
                             (cuuint64_t)a.Hb * a.Wb * a.cin * 2};
    cuuint32_t box[4] = {(cuuint32_t)kBK, (cuuint32_t)kSHBoxW, (cuuint32_t)kSHBoxH, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = g_encode(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(a.A), dims,
                          strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  if ((e = encode_wt(&mW, a.Wt, a.cout, 9 * a.cin, kSwapBN)) != cudaSuccess) return e;
  TcGeom tg{};
  tg.TH = kSHTH;
  tg.TW = kSHTW;
  tg.tiles_x = (a.Wb + kSHTW - 1) / kSHTW;
  tg.tiles_y = (a.Hb + kSHTH - 1) / kSHTH;
  tg.n_tiles = 1;
  tg.total = a.tiles ? a.n_mtiles : a.B * tg.tiles_x * tg.tiles_y;
  if (tg.total <= 0) return cudaSuccess;
  const int grid = std::min(tg.total, g_num_sms);
  conv_tc_swap_halo_kernel<<<grid, kThreads, kSHSmem, s>>>(mA, mW, a, tg);
  return cudaGetLastError();
}

// (cin, cout, k2) of the narrow layers -> N slice width and counts; false if not a halo layer
bool halo_shape(const ConvArgs &a, int *BN, int *KB, int *P2KB, int *NT) {
  if (a.taps != 9 || a.cin % kBK || a.k2 % kBK) return false;
  *KB = a.cin / kBK;
  *P2KB = a.k2 / kBK;
  if (a.cin == 64 && a.cout == 64 && a.k2 <= 64) { *BN = 64; *NT = 1; return true; }
  // (conv2_1's forward, 64 -> 128 without a fused term, runs on the pixels-as-N halo kernel)
  // (conv2_1's input gradient, 128 -> 64: 0.47 ms here against 1.12 ms on the main kernel with
  // N = 64, at 3024 x 4032, although the 144 KB of resident weights leave three stages)
  if (a.cin == 128 && a.cout == 64 && a.k2 == 0) { *BN = 64; *NT = 1; return true; }
  // (conv2_2, 128 -> 128, runs faster on the pixels-as-N kernel with 256-wide MMAs than here
  // with two 64-wide N slices; conv2_1, 64 -> 128, is faster here: 0.76 against 0.83 ms at
  // 3024 x 4032, where the pixels-as-N kernel streams a 16 KB weight box with every K-block)
  return false;
}

cudaError_t launch_conv_tc_halo(const ConvArgs &a, int BN, int KB, int P2KB, int NT,
                                cudaStream_t s) {
  CUtensorMap mA, mB, mA2, mB2;
  cudaError_t e;
  if ((e = encode_act_halo(&mA, a.A, a.B, a.Hb, a.Wb, a.cin)) != cudaSuccess) return e;
  if ((e = encode_wt(&mB, a.Wt, a.cout, 9 * a.cin, BN)) != cudaSuccess) return e;
  // the ReLU mask of an input gradient is usually the V of its fused V R term: the kernel then
  // loads that phase as the tile's own 16 x 8 box and reads the mask from it
  const bool mask_smem =
      BN == 64 && KB == 1 && P2KB == 1 && NT == 1 && a.mask == a.A2 && a.k2 == a.cout;
  if (a.k2) {
    e = mask_smem ? encode_act(&mA2, a.A2, a.B, a.Hb, a.Wb, a.k2, kHaloTH, kHaloTW)
                  : encode_act_halo(&mA2, a.A2, a.B, a.Hb, a.Wb, a.k2);
    if (e != cudaSuccess) return e;
    if ((e = encode_wt(&mB2, a.W2, a.cout, a.k2, BN)) != cudaSuccess) return e;
  } else {
    mA2 = mA;
    mB2 = mB;
  }
  if (BN == 64 && KB == 1 && P2KB == 0 && NT == 1) return launch_halo<64, 1, 0, 1>(mA, mB, mA2, mB2, a, s);
  if (BN == 64 && KB == 1 && P2KB == 1 && NT == 1) {
    if (mask_smem) return launch_halo<64, 1, 1, 1, true>(mA, mB, mA2, mB2, a, s);
    return launch_halo<64, 1, 1, 1>(mA, mB, mA2, mB2, a, s);
  }
  if (BN == 128 && KB == 1 && P2KB == 0 && NT == 1) return launch_halo<128, 1, 0, 1>(mA, mB, mA2, mB2, a, s);
  if (BN == 64 && KB == 2 && P2KB == 0 && NT == 1) return launch_halo<64, 2, 0, 1>(mA, mB, mA2, mB2, a, s);
  return cudaErrorInvalidValue;
}

}  // namespace

bool tc_available() {
  std::call_once(g_once, init_once);
  return g_tc_ok;
}

void *tc_encode_tiled_fn() { return tc_available() ? reinterpret_cast<void *>(g_encode) : nullptr; }
int tc_num_sms() {
  tc_available();
  return g_num_sms;
}

cudaError_t launch_timeout_check(long long limit_cycles, unsigned *err, cudaStream_t s) {
  timeout_check_kernel<<<1, 32, 0, s>>>(limit_cycles, err);
  return cudaGetLastError();
}

void conv_tc_patch_rule(int cin, int cout, int taps, int k2, bool pool, int *rows, int *fixed_th,
                        int *fixed_tw) {
  ConvArgs a{};
  a.cin = taps ? cin : 0;
  a.cout = cout;
  a.taps = taps;
  a.k2 = k2;
  a.pool_out = pool ? reinterpret_cast<void *>(1) : nullptr;   // only tested against null
  int bn, kb, p2, nt;
  *fixed_th = *fixed_tw = 0;
  if (swap_halo_shape(a)) {
    *rows = kSwapBP;
    *fixed_th = kSHTH;
    *fixed_tw = kSHTW;
  } else if (halo_shape(a, &bn, &kb, &p2, &nt)) {
    *rows = kHaloTH * kHaloTW;
    *fixed_th = kHaloTH;
    *fixed_tw = kHaloTW;
  } else {
    *rows = cout == kSwapBN ? kSwapBP : 128;
  }
}

void conv_tc_pick_patch(const int *h, const int *w, int n, int rows, int fixed_th, int fixed_tw,
                        bool pool, int *TH, int *TW) {
  if (fixed_th) {
    *TH = fixed_th;
    *TW = fixed_tw;
    return;
  }
  pick_patch_multi(h, w, n, rows, pool, *TH, *TW);
}

cudaError_t launch_conv_tc(const ConvArgs &a, cudaStream_t s) {
  if (!tc_available()) return cudaErrorNotSupported;
  if ((a.taps != 0 && a.taps != 9) || a.cout % 64 || (a.taps && a.cin % 64) || a.k2 % 64 ||
      (a.taps == 0 && a.k2 == 0))
    return cudaErrorInvalidValue;
  if (swap_halo_shape(a)) return launch_swap_halo(a, s);
  int hBN, hKB, hP2, hNT;
  if (halo_shape(a, &hBN, &hKB, &hP2, &hNT)) {
    if (a.tiles && (a.TH != kHaloTH || a.TW != kHaloTW)) return cudaErrorInvalidValue;
    return launch_conv_tc_halo(a, hBN, hKB, hP2, hNT, s);
  }
  // 128 output channels: pixels as the MMA's N (256 wide) instead of channels (128 wide)
  const bool swap = a.cout == kSwapBN;
  const int BN = swap ? kSwapBN : (a.cout >= 256 ? 256 : a.cout);
  const int rows = swap ? kSwapBP : 128;
  TcGeom tg;
  if (a.tiles) {
    // a patch list from the caller: its patch shape must follow this kernel's rule
    if (a.TH < 1 || a.TW < 1 || a.TH * a.TW > rows ||
        (a.pool_out && !((a.TW == 8 || a.TW == 16) && a.TH * a.TW == rows)))
      return cudaErrorInvalidValue;
    tg.TH = a.TH;
    tg.TW = a.TW;
  } else {
    pick_patch_rows(a.Hb, a.Wb, rows, tg.TH, tg.TW, a.pool_out != nullptr);
  }
  tg.tx_bytes = tg.TH * tg.TW * kBK * 2 + BN * kBK * 2;
  tg.tiles_x = (a.Wb + tg.TW - 1) / tg.TW;
  tg.tiles_y = (a.Hb + tg.TH - 1) / tg.TH;
  tg.n_tiles = a.cout / BN;
  tg.total = (a.tiles ? a.n_mtiles : a.B * tg.tiles_x * tg.tiles_y) * tg.n_tiles;
  if (tg.total <= 0) return cudaSuccess;
  tg.cin_blocks = a.taps ? a.cin / kBK : 0;
  tg.kb_main = a.taps * tg.cin_blocks;
  tg.kb2 = a.k2 / kBK;
  CUtensorMap mA, mB, mA2, mB2;
  cudaError_t e;
  if (a.taps) {
    if ((e = encode_act(&mA, a.A, a.B, a.Hb, a.Wb, a.cin, tg.TH, tg.TW)) != cudaSuccess) return e;
    if ((e = encode_wt(&mB, a.Wt, a.cout, a.taps * a.cin, BN)) != cudaSuccess) return e;
  }
  if (a.k2) {
    if ((e = encode_act(&mA2, a.A2, a.B, a.Hb, a.Wb, a.k2, tg.TH, tg.TW)) != cudaSuccess) return e;
    if ((e = encode_wt(&mB2, a.W2, a.cout, a.k2, BN)) != cudaSuccess) return e;
  }
  if (!a.taps) { mA = mA2; mB = mB2; }
  if (!a.k2) { mA2 = mA; mB2 = mB; }
  if (swap) return launch_swap<4>(mA, mB, mA2, mB2, a, tg, s);
  switch (BN) {
    case 64: return launch_bn<64, 8>(mA, mB, mA2, mB2, a, tg, s);
    case 128: return launch_bn<128, 6>(mA, mB, mA2, mB2, a, tg, s);
    case 256: return launch_bn<256, 4>(mA, mB, mA2, mB2, a, tg, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nst
