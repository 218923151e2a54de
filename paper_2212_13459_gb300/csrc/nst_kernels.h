// nst_kernels.h -- host-side declarations of the library's kernel launchers.
#pragma once
#include <cuda.h>

#include "nst_internal.cuh"

namespace nst {

// a run of owned pixels [p0, p1) of block b (row-major inside its owned rectangle)
struct GramChunk {
  int b, p0, p1, pad;
};

struct StyleLayerArgs {
  const double *Gacc;  // sum over owned pixels of V V^T (FP64)
  const double *Ghat;  // G^L(v)
  double *Gout;        // G^L(x) = Gacc / np
  void *R;             // (4 w / np)(G - Ghat) + diag(beta), FP32 or BF16
  int C;
  double np;
  double w;
  // mean / std terms (Eq. 5), all optional: channel sums S, targets mu / sigma with weights
  // wm / ws; alpha receives the per-channel gradient offset; mean_out / std_out the moments
  const double *S;
  const double *mu, *sigma;
  double wm, ws;
  float *alpha;
  double *mean_out, *std_out;
};
constexpr int kFinalizeChunks = 65;   // per layer: moment term + 64 residual chunks
struct StyleFinalizeArgs {
  StyleLayerArgs L[kNStyle];
  double *Eparts;   // [5]
  int r_is_bf16;
  double *beta;     // scratch [5][512]
  double *partial;  // scratch [5][kFinalizeChunks]
};

// conv1_1 weights and biases as one kernel parameter (7,168 bytes): w[k][c] = W1[c][k] with
// k = ci * 9 + ky * 3 + kx
struct Conv11W {
  float w[27][64];
  float b[64];
};

// k_simt.cu
template <typename T> void launch_conv_simt(const ConvArgs &a, cudaStream_t s);
template <typename T>
void launch_conv11_fwd(const float *img, int H, int W, const Conv11W &cw, const BlockGeom *geom,
                       int B, int Hb, int Wb, T *out, cudaStream_t s);
template <typename T>
void launch_conv11_dgrad_scatter(const T *g, const float *w11, const BlockGeom *geom,
                                 const OwnRect *inner, int B, int Hb, int Wb, float *grad, int H,
                                 int W, int max_inner_px, cudaStream_t s);
template <typename T>
void launch_pool(const T *in, T *out, int B, int Hp, int Wp, int C, const BlockGeom *geom,
                 int level_out, cudaStream_t s);
template <typename T>
void launch_unpool(const T *gp, const T *act, T *g, int B, int Hp, int Wp, int C,
                   const BlockGeom *geom, int level_out, cudaStream_t s);
// tensor-core form: routing by the window positions the fused forward pooling stored; rects
// (optional, device, one {y0, y1, x0, x1} of pooled positions per block, at most max_rect_px
// positions each) restricts it to those positions
void launch_unpool_idx(const __nv_bfloat16 *gp, const unsigned char *idx, __nv_bfloat16 *g,
                       int B, int Hp, int Wp, int C, const BlockGeom *geom, int level_out,
                       const int4 *rects, int max_rect_px, cudaStream_t s);
template <typename T>
void launch_gram_partial(const T *V, int Hb, int Wb, int C, const OwnRect *own,
                         const GramChunk *chunks, int nchunks, float *part, cudaStream_t s);
template <typename T>
void launch_gram_partial_flat(const T *V, long long npix, int C, long long chunk_len, int nchunks,
                              float *part, cudaStream_t s);
void launch_gram_reduce(const float *part, int nchunks, int C, double *Gacc, cudaStream_t s);
void launch_style_finalize(const StyleFinalizeArgs &a, cudaStream_t s);
template <typename T>
void launch_chansum(const T *V, int Hb, int Wb, int C, const OwnRect *own,
                    const GramChunk *chunks, int nchunks, double *partial, double *S,
                    cudaStream_t s);
template <typename T>
void launch_content_loss(const T *V, int Hb, int Wb, const T *Vu, int Hc, int Wc,
                         const BlockGeom *geom, const OwnRect *own, const GramChunk *chunks,
                         int nchunks, double *partial, double lambda, double *acc, cudaStream_t s);
template <typename T>
void launch_crop_content(const T *V, int B, int Hb, int Wb, const BlockGeom *geom,
                         const OwnRect *own, T *Vu, int Hc, int Wc, int max_own_px,
                         cudaStream_t s);
void launch_check_finite(const float *x, long long n, unsigned *err, cudaStream_t s);
void launch_finish_loss(const double *parts, double *loss, cudaStream_t s);

// k_tc.cu: tcgen05 / TMEM / TMA implicit-GEMM convolution (BF16 in, FP32 accumulate)
// Returns cudaSuccess or the error of tensor-map encoding / launch.
cudaError_t launch_conv_tc(const ConvArgs &a, cudaStream_t s);
// Patch rule of the tensor-core convolution that a launch of this shape runs: a fixed
// *fixed_th x *fixed_tw patch (16 x 8 for the 64-channel halo kernel, 32 x 8 for the
// pixels-as-N halo kernel of conv2_1's forward; 0 = free) or any TH x TW with TH * TW <= *rows
// pixels (128; 256 for the pixels-as-N kernel of 128-channel outputs). pool: fused pooling.
void conv_tc_patch_rule(int cin, int cout, int taps, int k2, bool pool, int *rows, int *fixed_th,
                        int *fixed_tw);
// The patch shape within that rule that covers n rectangles h[i] x w[i] with the fewest
// patches (with fused pooling TW is 8 or 16 and TH * TW = rows).
void conv_tc_pick_patch(const int *h, const int *w, int n, int rows, int fixed_th, int fixed_tw,
                        bool pool, int *TH, int *TW);
bool tc_available();
void *tc_encode_tiled_fn();   // cuTensorMapEncodeTiled (driver entry point), null if unavailable
int tc_num_sms();
// one bounded mbarrier wait that cannot complete: latches kErrTimeout after limit_cycles
cudaError_t launch_timeout_check(long long limit_cycles, unsigned *err, cudaStream_t s);

// k_c11_tc.cu: conv1_1 on the tensor cores (BF16 storage). Forward: out[b][y][x][64] =
// relu(bias + conv1_1(block image)) inside each block's valid extent, zero elsewhere; w11 is
// [64][3][3][3] FP32 holding BF16 values; stage_buf (16 bytes per buffer pixel, 16-byte aligned)
// receives the staged block images; patches (optional, npatches 16 x 8 output patches
// {block, y0, x0, owned}) restricts the convolution to them. gram_part (optional, needs patches):
// the Gram sum_p V_p V_p^T over the patches with owned != 0 (each wholly inside its block's owned
// rectangle, or past the valid extent, where V = 0) is accumulated per CTA on the tensor cores
// and written as *gram_runs partials of 128 x 64 floats (rows 0..63 used), the layout
// launch_gram_tc_reduce reads (C = N = 64, one tile). Input gradient:
// grad[ci][ey0 + y][ex0 + x] for the owned (inner) pixels of every block, from the gated
// ReLU1_1 gradient g [B][Hb][Wb][64].
cudaError_t launch_conv11_fwd_tc(const float *img, int H, int W, const float *w11,
                                 const float *bias, const BlockGeom *geom, int B, int Hb, int Wb,
                                 void *stage_buf, __nv_bfloat16 *out, const int4 *patches,
                                 int npatches, float *gram_part, int *gram_runs, unsigned *err,
                                 cudaStream_t s);
cudaError_t launch_conv11_dgrad_tc(const __nv_bfloat16 *g, const float *w11,
                                   const BlockGeom *geom, const OwnRect *inner, int B, int Hb,
                                   int Wb, int max_inner_h, int max_inner_w, float *grad, int H,
                                   int W, unsigned *err, cudaStream_t s);

// k_gram_tc.cu: Gram statistics on the tensor cores
struct GramTcChunk {
  int b, box0, box1, nbx;  // boxes [box0, box1) of block b's owned rectangle, nbx boxes per row
};
struct GramTcArgs {
  const CUtensorMap *maps;    // per block of the batch: owned rectangle as a 4-D BF16 map
  const GramTcChunk *chunks;  // one run per CTA column
  int C, N, nI, nJ, TH, TW;   // channels, J-tile width, tile counts, box shape (TH * TW = 64)
  float *part;                // [runs][nI * nJ][128][N] FP32 partial tiles
  unsigned *err;
};
void gram_tc_shape(int C, int *N, int *nI, int *nJ);
void gram_tc_patch(int own_h, int own_w, int *TH, int *TW);
cudaError_t encode_gram_map(CUtensorMap *m, const void *base, int C, int own_w, int own_h,
                            long long row_stride_px, int TH, int TW);
cudaError_t launch_gram_tc(const GramTcArgs &a, int nruns, double *Gacc, cudaStream_t s);
// Gacc[i][j] += the sum over nruns FP32 partial tiles (run r at part + r * nI * nJ * 128 * N,
// tile (I, J) of 128 x N floats), fixed order; the reduction launch_gram_tc ends with.
cudaError_t launch_gram_tc_reduce(const float *part, int nruns, int C, int N, int nI, int nJ,
                                  double *Gacc, cudaStream_t s);

// Chunking of a flat [npix][C] feature matrix for the CUDA-core Gram kernels: about 1,216 CTAs
// over the 64 x 64 block pairs (npairs = nb (nb + 1) / 2, nb = C / 64), chunks of a multiple of
// 32 pixels, at least 256. nchunks * npairs <= 1,216 whenever npix > 256 * 1216 / npairs.
inline void gram_flat_plan(long long npix, int C, long long *chunk_len, int *nchunks) {
  const int nb = C / 64, npairs = nb * (nb + 1) / 2;
  const long long target = 1216 / npairs > 1 ? 1216 / npairs : 1;
  long long ch = (npix + target - 1) / target;
  if (ch < 256) ch = 256;
  ch = (ch + 31) / 32 * 32;
  *chunk_len = ch;
  *nchunks = (int)((npix + ch - 1) / ch);
}

// context-free error message (returned by nst_last_error(NULL)); defined in nst_api.cu
void set_last_error_msg(const char *msg);

// k_lbfgs.cu (L-BFGS launchers are declared in nst_lbfgs_dev.h)
void launch_bicubic(const float *x, int C, int h, int w, float *out, int H, int W,
                    cudaStream_t s);
void launch_area(const float *x, int C, int h, int w, float *out, int H, int W, cudaStream_t s);

}  // namespace nst
