// nst_internal.cuh -- types shared by the library's translation units (host scheduler and kernels).
//
// Data layout in HBM (one batch of B blocks, Section 4.1 "blocks with margin"):
//   every activation of the VGG-19 trunk is NHWC [B][Hb_l][Wb_l][C] with Hb_l = Hb >> l at pooling
//   level l (Hb, Wb multiples of 16). Block t holds a valid region of (eh_t >> l) x (ew_t >> l)
//   pixels; everything outside it is kept at exactly zero so that each block behaves as a
//   standalone image with zero padding.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nst {

constexpr int kNConv = 13;
constexpr int kNStyle = 5;
constexpr int kCin[kNConv] = {3, 64, 64, 128, 128, 256, 256, 256, 256, 512, 512, 512, 512};
constexpr int kCout[kNConv] = {64, 64, 128, 128, 256, 256, 256, 256, 512, 512, 512, 512, 512};
constexpr int kLevel[kNConv] = {0, 0, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 4};
constexpr bool kPoolAfter[kNConv] = {false, true, false, true, false, false, false, true,
                                     false, false, false, true, false};
constexpr int kStyleConv[kNStyle] = {0, 2, 4, 8, 12};   // ReLU1_1 ReLU2_1 ReLU3_1 ReLU4_1 ReLU5_1
constexpr int kContentConv = 9;                          // ReLU4_2
constexpr int kContentLevel = 3;

// device status word bits
enum : unsigned { kErrTimeout = 1u, kErrNonfinite = 2u };

// per-block geometry, image coordinates at level 0: extended origin and valid extent
struct BlockGeom {
  int ey0, ex0, eh, ew;
};

// owned (inner) feature rectangle of a block at one level, block-local coordinates
struct OwnRect {
  int y0, y1, x0, x1;
};

// ---- element conversions ---------------------------------------------------------------------
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// ---- convolution launch description (shared by the SIMT and tcgen05 engines) ------------------
//
// out[b][y][x][n] = epilogue( sum_{tap,c} A[b][y+dy][x+dx][c] * Wt[n][tap][c]
//                            + sum_c A2[b][y][x][c] * W2[n][c] )
// with zero fill outside [0,Hb) x [0,Wb). taps = 9 gives a 3x3 convolution (dy,dx in -1..1),
// taps = 0 drops the first sum. The second sum (K2 > 0) is the style-gradient term V R of
// Table 1 (row 2), fused into the same accumulator.
enum EpiMode : int {
  kEpiForward = 0,   // relu(acc + bias), zero outside the block's valid region
  kEpiBackward = 1,  // (acc [+ 2 lambda (cact - ctgt)]) * (mask > 0)
};

struct ConvArgs {
  int B, Hb, Wb;        // batch and buffer dims at this layer's level
  int cin, cout, taps;  // main phase
  int k2;               // phase-2 depth (0 = none)
  const void *A, *Wt;   // main phase input [B][Hb][Wb][cin], weights [cout][taps][cin]
  const void *A2, *W2;  // phase 2 input [B][Hb][Wb][k2], weights [cout][k2]
  void *out;            // [B][Hb][Wb][cout]
  int mode;
  const float *bias;    // forward
  const void *mask;     // backward: gate (post-ReLU activation, [B][Hb][Wb][cout]) or null
  const void *cact;     // backward: content feature V^Lc(x) of the block, or null
  const void *ctgt;     // backward: global content target [Hc][Wc][cout]
  int Hc, Wc;
  float two_lambda;
  const BlockGeom *geom;  // [B]
  int level;
  unsigned *err;
  void *pool_out;         // forward, tensor-core engine: also write the 2x2 max pool
                          // [B][Hb/2][Wb/2][cout] (null = no fused pooling)
  const float *addvec;    // backward: per-channel term added at valid pixels before the gate
                          // (alpha of the mean / std loss, Table 1 rows 3-4), or null
  unsigned char *pool_idx;  // forward with pool_out: also the window positions of the maximum,
                            // 4 bits per pooled value ([B][Hb/2][Wb/2][cout] / 2 bytes), or null
  // tensor-core engine: the output patches to compute, one {block, y0, x0, 0} per patch (its
  // origin in the block's [Hb][Wb] buffer), each TH x TW; null = every patch of the buffer
  const int4 *tiles;
  int n_mtiles, TH, TW;
};

}  // namespace nst
