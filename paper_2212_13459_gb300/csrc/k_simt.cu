// k_simt.cu -- CUDA-core kernels of the localized loss/gradient path:
//   * the plain FP32 convolution engine (implicit GEMM on CUDA cores, no TF32), used by the FP32
//     form of the path and as a cross-check of the tensor-core engine;
//   * conv1_1 forward straight from the caller's planar image (block gather fused) and conv1_1
//     input-gradient with the inner-part scatter into dE/dx fused (Algorithm 1, last step);
//   * 2x2 max pooling and its adjoint (argmax routing + ReLU gate);
//   * split Gram partial sums over owned pixels and their FP64 reduction (Eq. 4, Algorithm 1
//     Step 1), the style finalisation (Eq. 3 and Table 1 row 2), the content loss over owned
//     pixels (Algorithm 1 Step 2), the content-target crop, and a finiteness check.
#include "nst_internal.cuh"
#include "nst_kernels.h"

namespace nst {

// ---- vector helpers ----------------------------------------------------------------------------
__device__ __forceinline__ void load4(const float *p, float v[4]) {
  float4 t = *reinterpret_cast<const float4 *>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const __nv_bfloat16 *p, float v[4]) {
  uint2 t = *reinterpret_cast<const uint2 *>(p);
  __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&t.x);
  __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&t.y);
  float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}
__device__ __forceinline__ void store4(float *p, const float v[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(__nv_bfloat16 *p, const float v[4]) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
  uint2 t;
  t.x = *reinterpret_cast<unsigned *>(&a);
  t.y = *reinterpret_cast<unsigned *>(&b);
  *reinterpret_cast<uint2 *>(p) = t;
}
__device__ __forceinline__ void load8(const float *p, float v[8]) { load4(p, v); load4(p + 4, v + 4); }
__device__ __forceinline__ void load8(const __nv_bfloat16 *p, float v[8]) {
  uint4 t = *reinterpret_cast<const uint4 *>(p);
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&t);
#pragma unroll
  for (int i = 0; i < 4; i++) {
    float2 f = __bfloat1622float2(h[i]);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}
__device__ __forceinline__ void store8(float *p, const float v[8]) { store4(p, v); store4(p + 4, v + 4); }
__device__ __forceinline__ void store8(__nv_bfloat16 *p, const float v[8]) {
  uint4 t;
  __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&t);
#pragma unroll
  for (int i = 0; i < 4; i++) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
  *reinterpret_cast<uint4 *>(p) = t;
}

// ---- shared epilogue (4 consecutive output channels of one pixel) ------------------------------
template <typename T>
__device__ __forceinline__ void conv_epilogue4(const ConvArgs &a, int b, int y, int x, int n,
                                               float v[4]) {
  const BlockGeom g = a.geom[b];
  const bool valid = y < (g.eh >> a.level) && x < (g.ew >> a.level);
  const size_t o = (((size_t)b * a.Hb + y) * a.Wb + x) * a.cout + n;
  if (a.mode == kEpiForward) {
#pragma unroll
    for (int j = 0; j < 4; j++) v[j] = valid ? fmaxf(v[j] + a.bias[n + j], 0.f) : 0.f;
  } else {
    if (a.cact && valid) {
      const int gy = (g.ey0 >> a.level) + y, gx = (g.ex0 >> a.level) + x;
      if (gy < a.Hc && gx < a.Wc) {
        float ca[4], ct[4];
        load4(reinterpret_cast<const T *>(a.cact) + o, ca);
        load4(reinterpret_cast<const T *>(a.ctgt) + ((size_t)gy * a.Wc + gx) * a.cout + n, ct);
#pragma unroll
        for (int j = 0; j < 4; j++) v[j] += a.two_lambda * (ca[j] - ct[j]);
      }
    }
    if (a.addvec && valid) {
#pragma unroll
      for (int j = 0; j < 4; j++) v[j] += a.addvec[n + j];
    }
    if (a.mask) {
      float m[4];
      load4(reinterpret_cast<const T *>(a.mask) + o, m);
#pragma unroll
      for (int j = 0; j < 4; j++) v[j] = m[j] > 0.f ? v[j] : 0.f;
    }
    if (!valid) v[0] = v[1] = v[2] = v[3] = 0.f;
  }
  store4(reinterpret_cast<T *>(a.out) + o, v);
}

// ---- CUDA-core implicit-GEMM convolution ---------------------------------------------------------
// CTA tile: 8x8 output pixels x 64 output channels; K slices of 16 channels of one tap.
// 256 threads, each 4 pixels x 4 channels, FP32 accumulation.
template <typename T>
__global__ void __launch_bounds__(256) conv_simt_kernel(ConvArgs a) {
  __shared__ __align__(16) float As[16][68];
  __shared__ __align__(16) float Bs[16][68];
  const int tilesX = (a.Wb + 7) >> 3, tilesY = (a.Hb + 7) >> 3;
  int t = blockIdx.x;
  const int tx = t % tilesX;
  t /= tilesX;
  const int ty = t % tilesY;
  const int b = t / tilesY;
  const int n0 = blockIdx.y * 64;
  const int tid = threadIdx.x;
  const int tp = tid & 15, tc = tid >> 4;
  const int lp = tid >> 2, lc = (tid & 3) * 4;
  const int py = ty * 8 + (lp >> 3), px = tx * 8 + (lp & 7);
  const int bn = tid >> 2, bk = (tid & 3) * 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.f;

  auto mac = [&]() {
#pragma unroll
    for (int k = 0; k < 16; k++) {
      float4 av = *reinterpret_cast<const float4 *>(&As[k][tp * 4]);
      float4 bv = *reinterpret_cast<const float4 *>(&Bs[k][tc * 4]);
      float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
    }
  };

  const T *A = reinterpret_cast<const T *>(a.A);
  const T *Wt = reinterpret_cast<const T *>(a.Wt);
  for (int tap = 0; tap < a.taps; tap++) {
    const int y = py + tap / 3 - 1, x = px + tap % 3 - 1;
    const bool in = y >= 0 && y < a.Hb && x >= 0 && x < a.Wb;
    const T *arow = A + (((size_t)b * a.Hb + y) * a.Wb + x) * a.cin;
    const T *brow = Wt + ((size_t)(n0 + bn) * a.taps + tap) * a.cin;
    for (int c0 = 0; c0 < a.cin; c0 += 16) {
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (in) load4(arow + c0 + lc, v);
#pragma unroll
      for (int j = 0; j < 4; j++) As[lc + j][lp] = v[j];
      float w[4];
      load4(brow + c0 + bk, w);
#pragma unroll
      for (int j = 0; j < 4; j++) Bs[bk + j][bn] = w[j];
      __syncthreads();
      mac();
      __syncthreads();
    }
  }
  if (a.k2 > 0) {
    const T *A2 = reinterpret_cast<const T *>(a.A2);
    const T *W2 = reinterpret_cast<const T *>(a.W2);
    const bool in = py < a.Hb && px < a.Wb;
    const T *arow = A2 + (((size_t)b * a.Hb + py) * a.Wb + px) * a.k2;
    const T *brow = W2 + (size_t)(n0 + bn) * a.k2;
    for (int c0 = 0; c0 < a.k2; c0 += 16) {
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (in) load4(arow + c0 + lc, v);
#pragma unroll
      for (int j = 0; j < 4; j++) As[lc + j][lp] = v[j];
      float w[4];
      load4(brow + c0 + bk, w);
#pragma unroll
      for (int j = 0; j < 4; j++) Bs[bk + j][bn] = w[j];
      __syncthreads();
      mac();
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int p = tp * 4 + i;
    const int y = ty * 8 + (p >> 3), x = tx * 8 + (p & 7);
    if (y < a.Hb && x < a.Wb) conv_epilogue4<T>(a, b, y, x, n0 + tc * 4, acc[i]);
  }
}

template <typename T>
void launch_conv_simt(const ConvArgs &a, cudaStream_t s) {
  dim3 grid(((a.Wb + 7) / 8) * ((a.Hb + 7) / 8) * a.B, a.cout / 64);
  conv_simt_kernel<T><<<grid, 256, 0, s>>>(a);
}
template void launch_conv_simt<float>(const ConvArgs &, cudaStream_t);
template void launch_conv_simt<__nv_bfloat16>(const ConvArgs &, cudaStream_t);

// ---- conv1_1 forward from the planar image (block extraction fused) ----------------------------
// out[b][y][x][c] = relu(b1[c] + sum W1[c][ci][ky][kx] * blk(ci, y+ky-1, x+kx-1)), where blk is the
// block's extended rectangle of x and reads zero outside it (the block is a standalone image).
// One thread computes all 64 channels of one pixel. The 27 x 64 weights travel as a
// __grid_constant__ kernel parameter: with the loops unrolled, every FMA takes its weight
// straight from the constant bank, so no load instruction competes with the FMAs. In the BF16 form
// each image value enters as hi + lo (hi = bf16(x), lo = bf16(x - hi)), the representation the
// tensor-core conv1_1 multiplies, so both engines see the same input.
template <typename T>
__global__ void __launch_bounds__(128) conv11_fwd_kernel(const float *__restrict__ img, int H,
                                                         int W, const __grid_constant__ Conv11W cw,
                                                         const BlockGeom *__restrict__ geom,
                                                         int B, int Hb, int Wb, T *__restrict__ out) {
  const long long npix = (long long)B * Hb * Wb;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(p % Wb);
    const int y = (int)((p / Wb) % Hb);
    const int b = (int)(p / ((long long)Wb * Hb));
    const BlockGeom g = geom[b];
    float acc[64];
    if (y < g.eh && x < g.ew) {
      float in[27];
#pragma unroll
      for (int ci = 0; ci < 3; ci++)
#pragma unroll
        for (int ky = 0; ky < 3; ky++)
#pragma unroll
          for (int kx = 0; kx < 3; kx++) {
            const int yy = y + ky - 1, xx = x + kx - 1;
            const bool ok = yy >= 0 && yy < g.eh && xx >= 0 && xx < g.ew;
            float v = ok ? __ldg(img + ((size_t)ci * H + g.ey0 + yy) * W + g.ex0 + xx) : 0.f;
            if (sizeof(T) == 2) {   // the BF16 form reads the image as a BF16 pair hi + lo
              const float hi = __bfloat162float(__float2bfloat16_rn(v));
              v = hi + __bfloat162float(__float2bfloat16_rn(v - hi));
            }
            in[ci * 9 + ky * 3 + kx] = v;
          }
#pragma unroll
      for (int c = 0; c < 64; c++) acc[c] = cw.b[c];
#pragma unroll
      for (int k = 0; k < 27; k++) {
        const float v = in[k];
#pragma unroll
        for (int c = 0; c < 64; c++) acc[c] = fmaf(cw.w[k][c], v, acc[c]);
      }
#pragma unroll
      for (int c = 0; c < 64; c++) acc[c] = fmaxf(acc[c], 0.f);
    } else {
#pragma unroll
      for (int c = 0; c < 64; c++) acc[c] = 0.f;
    }
    T *o = out + (size_t)p * 64;
#pragma unroll
    for (int c8 = 0; c8 < 8; c8++) store8(o + c8 * 8, acc + c8 * 8);
  }
}

template <typename T>
void launch_conv11_fwd(const float *img, int H, int W, const Conv11W &cw, const BlockGeom *geom,
                       int B, int Hb, int Wb, T *out, cudaStream_t s) {
  long long npix = (long long)B * Hb * Wb;
  long long blocks = (npix + 127) / 128;
  int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
  conv11_fwd_kernel<T><<<grid, 128, 0, s>>>(img, H, W, cw, geom, B, Hb, Wb, out);
}
template void launch_conv11_fwd<float>(const float *, int, int, const Conv11W &,
                                       const BlockGeom *, int, int, int, float *, cudaStream_t);
template void launch_conv11_fwd<__nv_bfloat16>(const float *, int, int, const Conv11W &,
                                               const BlockGeom *, int, int, int,
                                               __nv_bfloat16 *, cudaStream_t);

// ---- conv1_1 input gradient + scatter of the inner part into dE/dx --------------------------------
// dx[ci](y,x) = sum_{co,ky,kx} W1[co][ci][ky][kx] * g[y-ky+1][x-kx+1][co] for the owned (inner)
// pixels of each block, written to grad at image coordinates (Algorithm 1, last line).
template <typename T>
__global__ void __launch_bounds__(256) conv11_dgrad_scatter_kernel(
    const T *__restrict__ g, const float *__restrict__ w11, const BlockGeom *__restrict__ geom,
    const OwnRect *__restrict__ inner, int B, int Hb, int Wb, float *__restrict__ grad, int H,
    int W) {
  // Eight lanes per pixel, lane group cg holding channels 8cg..8cg+7: a warp reads four pixels'
  // 128-byte channel vectors as 512 contiguous bytes. ws[k][cg][j] = {W1[co][0][k], W1[co][1][k],
  // W1[co][2][k], 0} with co = 8cg + j, rows padded to 9 float4 so the 8 groups hit distinct banks.
  __shared__ __align__(16) float4 ws[9][8][9];
  for (int i = threadIdx.x; i < 9 * 64; i += blockDim.x) {
    const int k = i / 64, co = i % 64;
    ws[k][co / 8][co % 8] =
        make_float4(w11[co * 27 + k], w11[co * 27 + 9 + k], w11[co * 27 + 18 + k], 0.f);
  }
  __syncthreads();
  const int b = blockIdx.y;
  if (b >= B) return;
  const OwnRect r = inner[b];
  const BlockGeom gm = geom[b];
  const int rw = r.x1 - r.x0, rh = r.y1 - r.y0;
  const long long n = (long long)rw * rh;
  const int cg = threadIdx.x & 7;
  const long long stride = (long long)gridDim.x * (blockDim.x >> 3);
  // every lane of a warp runs the same number of iterations (the bound is per 4-pixel group)
  for (long long q0 = (long long)blockIdx.x * (blockDim.x >> 3) + (threadIdx.x >> 5) * 4;
       q0 < n; q0 += stride) {
    const long long q = q0 + ((threadIdx.x & 31) >> 3);
    const bool live = q < n;
    const int y = live ? r.y0 + (int)(q / rw) : r.y0, x = live ? r.x0 + (int)(q % rw) : r.x0;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll 3
    for (int k = 0; k < 9; k++) {
      const int yy = y - k / 3 + 1, xx = x - k % 3 + 1;
      if (live && yy >= 0 && yy < Hb && xx >= 0 && xx < Wb) {
        float gv[8];
        load8(g + (((size_t)b * Hb + yy) * Wb + xx) * 64 + cg * 8, gv);
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const float4 w = ws[k][cg][j];
          d0 = fmaf(w.x, gv[j], d0);
          d1 = fmaf(w.y, gv[j], d1);
          d2 = fmaf(w.z, gv[j], d2);
        }
      }
    }
#pragma unroll
    for (int m = 1; m < 8; m <<= 1) {
      d0 += __shfl_xor_sync(0xffffffffu, d0, m);
      d1 += __shfl_xor_sync(0xffffffffu, d1, m);
      d2 += __shfl_xor_sync(0xffffffffu, d2, m);
    }
    if (live && cg == 0) {
      const size_t o = (size_t)(gm.ey0 + y) * W + gm.ex0 + x;
      grad[o] = d0;
      grad[(size_t)H * W + o] = d1;
      grad[2 * (size_t)H * W + o] = d2;
    }
  }
}

template <typename T>
void launch_conv11_dgrad_scatter(const T *g, const float *w11, const BlockGeom *geom,
                                 const OwnRect *inner, int B, int Hb, int Wb, float *grad, int H,
                                 int W, int max_inner_px, cudaStream_t s) {
  int gx = (max_inner_px + 31) / 32;   // 32 pixels per 256-thread CTA pass
  if (gx > 2048) gx = 2048;
  if (gx < 1) gx = 1;
  dim3 grid(gx, B);
  conv11_dgrad_scatter_kernel<T><<<grid, 256, 0, s>>>(g, w11, geom, inner, B, Hb, Wb, grad, H, W);
}
template void launch_conv11_dgrad_scatter<float>(const float *, const float *, const BlockGeom *,
                                                 const OwnRect *, int, int, int, float *, int, int,
                                                 int, cudaStream_t);
template void launch_conv11_dgrad_scatter<__nv_bfloat16>(const __nv_bfloat16 *, const float *,
                                                         const BlockGeom *, const OwnRect *, int,
                                                         int, int, float *, int, int, int,
                                                         cudaStream_t);

// ---- 2x2 max pool (floor) and its adjoint ----------------------------------------------------------
// The window's first maximum in row-major order (strict '>') is the argmax, as in the oracle.
__device__ __forceinline__ int argmax4(float v0, float v1, float v2, float v3) {
  int k = 0;
  float m = v0;
  if (v1 > m) { m = v1; k = 1; }
  if (v2 > m) { m = v2; k = 2; }
  if (v3 > m) { k = 3; }
  return k;
}

// in: [B][2Hp][2Wp][C] at level l; out: [B][Hp][Wp][C] at level l+1; zero outside valid region
template <typename T>
__global__ void pool_kernel(const T *__restrict__ in, T *__restrict__ out, int B, int Hp, int Wp,
                            int C, const BlockGeom *__restrict__ geom, int level_out) {
  const int C8 = C / 8;
  const long long n = (long long)B * Hp * Wp * C8;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C8) * 8;
    long long p = i / C8;
    const int x = (int)(p % Wp);
    const int y = (int)((p / Wp) % Hp);
    const int b = (int)(p / ((long long)Wp * Hp));
    const BlockGeom g = geom[b];
    float o[8];
    if (y < (g.eh >> level_out) && x < (g.ew >> level_out)) {
      const int Wi = 2 * Wp;
      const T *base = in + (((size_t)b * 2 * Hp + 2 * y) * Wi + 2 * x) * C + c;
      float v0[8], v1[8], v2[8], v3[8];
      load8(base, v0);
      load8(base + C, v1);
      load8(base + (size_t)Wi * C, v2);
      load8(base + (size_t)Wi * C + C, v3);
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int k = argmax4(v0[j], v1[j], v2[j], v3[j]);
        o[j] = k == 0 ? v0[j] : k == 1 ? v1[j] : k == 2 ? v2[j] : v3[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; j++) o[j] = 0.f;
    }
    store8(out + (size_t)p * C + c, o);
  }
}

// gp: [B][Hp][Wp][C] gradient w.r.t. the pooled map; act: [B][2Hp][2Wp][C] post-ReLU activation;
// g:  [B][2Hp][2Wp][C] gradient w.r.t. the pre-activation = routed gp gated by act > 0
template <typename T>
__global__ void unpool_kernel(const T *__restrict__ gp, const T *__restrict__ act,
                              T *__restrict__ g, int B, int Hp, int Wp, int C,
                              const BlockGeom *__restrict__ geom, int level_out) {
  const int C8 = C / 8;
  const long long n = (long long)B * Hp * Wp * C8;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C8) * 8;
    long long p = i / C8;
    const int x = (int)(p % Wp);
    const int y = (int)((p / Wp) % Hp);
    const int b = (int)(p / ((long long)Wp * Hp));
    const BlockGeom gm = geom[b];
    const int Wi = 2 * Wp;
    const size_t o0 = (((size_t)b * 2 * Hp + 2 * y) * Wi + 2 * x) * C + c;
    const size_t offs[4] = {o0, o0 + C, o0 + (size_t)Wi * C, o0 + (size_t)Wi * C + C};
    float r[4][8];
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
      for (int j = 0; j < 8; j++) r[k][j] = 0.f;
    if (y < (gm.eh >> level_out) && x < (gm.ew >> level_out)) {
      float gv[8], v[4][8];
      load8(gp + (size_t)p * C + c, gv);
#pragma unroll
      for (int k = 0; k < 4; k++) load8(act + offs[k], v[k]);
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int k = argmax4(v[0][j], v[1][j], v[2][j], v[3][j]);
        const float av = k == 0 ? v[0][j] : k == 1 ? v[1][j] : k == 2 ? v[2][j] : v[3][j];
        const float val = av > 0.f ? gv[j] : 0.f;
        r[0][j] = k == 0 ? val : 0.f;
        r[1][j] = k == 1 ? val : 0.f;
        r[2][j] = k == 2 ? val : 0.f;
        r[3][j] = k == 3 ? val : 0.f;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) store8(g + offs[k], r[k]);
  }
}

// Tensor-core form of the same routing: the forward's fused pooling stored 4 bits per pooled
// value, bit q set where window pixel q (row-major) equals the window max and that max is
// positive; the gradient goes to the lowest set bit (the first maximum), none where no bit is
// set (the ReLU gate is shut). One 32-bit word per 8 channels c .. c+7 at byte (p C + c) / 2,
// channel c+k in the nibble at bit 8 (k & 3) + 4 (k >> 2). The backward reads half a byte per
// value instead of the four activations.
// rects (optional): per block, the pooled rectangle {y0, y1, x0, x1} to route (the rest of the
// block's full-resolution gradient is left as it is); grid (n, B), row b = block b. Without
// rects: every pooled position of the buffer, grid-stride over all blocks.
__global__ void unpool_idx_kernel(const __nv_bfloat16 *__restrict__ gp,
                                  const unsigned char *__restrict__ idx,
                                  __nv_bfloat16 *__restrict__ g, int B, int Hp, int Wp, int C,
                                  const BlockGeom *__restrict__ geom, int level_out,
                                  const int4 *__restrict__ rects) {
  const int C8 = C / 8;
  int4 r = make_int4(0, Hp, 0, Wp);
  long long n = (long long)B * Hp * Wp * C8;
  long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (rects) {
    r = rects[blockIdx.y];
    n = (long long)max(0, r.y - r.x) * max(0, r.w - r.z) * C8;
  }
  const int rw = r.w - r.z;
  for (long long i = i0; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C8) * 8;
    const long long q = i / C8;
    int x, y, b;
    if (rects) {
      x = r.z + (int)(q % rw);
      y = r.x + (int)(q / rw);
      b = blockIdx.y;
    } else {
      x = (int)(q % Wp);
      y = (int)((q / Wp) % Hp);
      b = (int)(q / ((long long)Wp * Hp));
    }
    const long long p = ((long long)b * Hp + y) * Wp + x;
    const BlockGeom gm = geom[b];
    const int Wi = 2 * Wp;
    const size_t o0 = (((size_t)b * 2 * Hp + 2 * y) * Wi + 2 * x) * C + c;
    const size_t offs[4] = {o0, o0 + C, o0 + (size_t)Wi * C, o0 + (size_t)Wi * C + C};
    float rv[4][8];
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
      for (int j = 0; j < 8; j++) rv[k][j] = 0.f;
    if (y < (gm.eh >> level_out) && x < (gm.ew >> level_out)) {
      float gv[8];
      load8(gp + (size_t)p * C + c, gv);
      const uint32_t w = *reinterpret_cast<const uint32_t *>(idx + ((size_t)p * C + c) / 2);
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const uint32_t nib = (w >> (8 * (j & 3) + 4 * (j >> 2))) & 0xfu;
        const uint32_t first = nib & (0u - nib);   // lowest set bit, 0 if none
#pragma unroll
        for (int qq = 0; qq < 4; qq++) rv[qq][j] = first == (1u << qq) ? gv[j] : 0.f;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) store8(g + offs[k], rv[k]);
  }
}

static int ew_grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

template <typename T>
void launch_pool(const T *in, T *out, int B, int Hp, int Wp, int C, const BlockGeom *geom,
                 int level_out, cudaStream_t s) {
  pool_kernel<T><<<ew_grid((long long)B * Hp * Wp * C / 8), 256, 0, s>>>(in, out, B, Hp, Wp, C,
                                                                          geom, level_out);
}
template <typename T>
void launch_unpool(const T *gp, const T *act, T *g, int B, int Hp, int Wp, int C,
                   const BlockGeom *geom, int level_out, cudaStream_t s) {
  unpool_kernel<T><<<ew_grid((long long)B * Hp * Wp * C / 8), 256, 0, s>>>(gp, act, g, B, Hp, Wp,
                                                                            C, geom, level_out);
}
void launch_unpool_idx(const __nv_bfloat16 *gp, const unsigned char *idx, __nv_bfloat16 *g,
                       int B, int Hp, int Wp, int C, const BlockGeom *geom, int level_out,
                       const int4 *rects, int max_rect_px, cudaStream_t s) {
  if (rects) {
    if (max_rect_px <= 0) return;
    const long long per = (long long)max_rect_px * C / 8;
    int nx = (int)std::min<long long>((per + 255) / 256, std::max(1, 152 * 32 / B));
    dim3 grid(nx, B);
    unpool_idx_kernel<<<grid, 256, 0, s>>>(gp, idx, g, B, Hp, Wp, C, geom, level_out, rects);
    return;
  }
  unpool_idx_kernel<<<ew_grid((long long)B * Hp * Wp * C / 8), 256, 0, s>>>(gp, idx, g, B, Hp, Wp,
                                                                            C, geom, level_out,
                                                                            nullptr);
}
template void launch_pool<float>(const float *, float *, int, int, int, int, const BlockGeom *,
                                 int, cudaStream_t);
template void launch_pool<__nv_bfloat16>(const __nv_bfloat16 *, __nv_bfloat16 *, int, int, int,
                                         int, const BlockGeom *, int, cudaStream_t);
template void launch_unpool<float>(const float *, const float *, float *, int, int, int, int,
                                   const BlockGeom *, int, cudaStream_t);
template void launch_unpool<__nv_bfloat16>(const __nv_bfloat16 *, const __nv_bfloat16 *,
                                           __nv_bfloat16 *, int, int, int, int, const BlockGeom *,
                                           int, cudaStream_t);

// ---- Gram partial sums over owned pixels (CUDA cores) --------------------------------------------
// chunk c covers pixels [p0, p1) of block b's owned rectangle (row-major inside the rectangle);
// CTA (c, pair) accumulates the 64x64 block (I, J), I <= J, of sum_p V_p V_p^T in FP32 and writes
// it to part[(c * npairs + pair) * 4096 + i * 64 + j].
// With chunks == null, V is one flat [n_flat][C] matrix and CTA c takes pixels
// [c * chunk_len, min((c + 1) * chunk_len, n_flat)).
template <typename T>
__global__ void __launch_bounds__(256) gram_partial_kernel(const T *__restrict__ V, int Hb, int Wb,
                                                           int C, const OwnRect *__restrict__ own,
                                                           const GramChunk *__restrict__ chunks,
                                                           float *__restrict__ part,
                                                           long long chunk_len, long long n_flat) {
  __shared__ __align__(16) float Ai[32][68];
  __shared__ __align__(16) float Aj[32][68];
  const int nb = C / 64;
  const int npairs = nb * (nb + 1) / 2;
  int pair = blockIdx.y, I = 0;
  while (pair >= nb - I) { pair -= nb - I; I++; }
  const int J = I + pair;
  GramChunk ch;
  OwnRect r;
  if (chunks) {
    ch = chunks[blockIdx.x];
    r = own[ch.b];
  } else {
    const long long p0 = (long long)blockIdx.x * chunk_len;
    const long long p1 = p0 + chunk_len < n_flat ? p0 + chunk_len : n_flat;
    ch = {0, (int)p0, (int)p1, 0};
    r = {0, 1, 0, (int)n_flat};
  }
  const int rw = r.x1 - r.x0;
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  const int lp = tid >> 3, lc = (tid & 7) * 8;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.f;
  for (int q0 = ch.p0; q0 < ch.p1; q0 += 32) {
    const int q = q0 + lp;
    float vi[8], vj[8];
    if (q < ch.p1) {
      const int y = r.y0 + q / rw, x = r.x0 + q % rw;
      const T *row = V + (((size_t)ch.b * Hb + y) * Wb + x) * C;
      load8(row + I * 64 + lc, vi);
      load8(row + J * 64 + lc, vj);
    } else {
#pragma unroll
      for (int k = 0; k < 8; k++) vi[k] = vj[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      Ai[lp][lc + k] = vi[k];
      Aj[lp][lc + k] = vj[k];
    }
    __syncthreads();
#pragma unroll 8
    for (int p = 0; p < 32; p++) {
      float4 a4 = *reinterpret_cast<const float4 *>(&Ai[p][ti * 4]);
      float4 b4 = *reinterpret_cast<const float4 *>(&Aj[p][tj * 4]);
      float ar[4] = {a4.x, a4.y, a4.z, a4.w}, br[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *o = part + ((size_t)blockIdx.x * npairs + blockIdx.y) * 4096;
#pragma unroll
  for (int i = 0; i < 4; i++)
    *reinterpret_cast<float4 *>(o + (ti * 4 + i) * 64 + tj * 4) =
        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
}

// Gacc[C][C] += sum over chunks (fixed order, FP64) of the partial blocks; mirrored for I != J
__global__ void gram_reduce_kernel(const float *__restrict__ part, int nchunks, int C,
                                   double *__restrict__ Gacc) {
  const int nb = C / 64;
  const int npairs = nb * (nb + 1) / 2;
  const long long n = (long long)npairs * 4096;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int pair = (int)(e / 4096), I = 0;
    const int k = (int)(e % 4096);
    while (pair >= nb - I) { pair -= nb - I; I++; }
    const int J = I + pair;
    double s = 0.0;
    for (int c = 0; c < nchunks; c++) s += (double)part[((size_t)c * npairs) * 4096 + e];
    const int i = I * 64 + k / 64, j = J * 64 + k % 64;
    Gacc[(size_t)i * C + j] += s;
    if (I != J) Gacc[(size_t)j * C + i] += s;
  }
}

template <typename T>
void launch_gram_partial(const T *V, int Hb, int Wb, int C, const OwnRect *own,
                         const GramChunk *chunks, int nchunks, float *part, cudaStream_t s) {
  const int nb = C / 64;
  dim3 grid(nchunks, nb * (nb + 1) / 2);
  gram_partial_kernel<T><<<grid, 256, 0, s>>>(V, Hb, Wb, C, own, chunks, part, 0, 0);
}

template <typename T>
void launch_gram_partial_flat(const T *V, long long npix, int C, long long chunk_len, int nchunks,
                              float *part, cudaStream_t s) {
  const int nb = C / 64;
  dim3 grid(nchunks, nb * (nb + 1) / 2);
  gram_partial_kernel<T><<<grid, 256, 0, s>>>(V, 1, (int)npix, C, nullptr, nullptr, part,
                                              chunk_len, npix);
}
template void launch_gram_partial_flat<float>(const float *, long long, int, long long, int,
                                              float *, cudaStream_t);
template void launch_gram_partial_flat<__nv_bfloat16>(const __nv_bfloat16 *, long long, int,
                                                      long long, int, float *, cudaStream_t);
template void launch_gram_partial<float>(const float *, int, int, int, const OwnRect *,
                                         const GramChunk *, int, float *, cudaStream_t);
template void launch_gram_partial<__nv_bfloat16>(const __nv_bfloat16 *, int, int, int,
                                                 const OwnRect *, const GramChunk *, int, float *,
                                                 cudaStream_t);
void launch_gram_reduce(const float *part, int nchunks, int C, double *Gacc, cudaStream_t s) {
  const int nb = C / 64;
  long long n = (long long)nb * (nb + 1) / 2 * 4096;
  gram_reduce_kernel<<<ew_grid(n), 256, 0, s>>>(part, nchunks, C, Gacc);
}

// ---- style finalisation: G = Gacc / np, E_L = w ||G - Ghat||^2, R = (4 w / np)(G - Ghat) -------------
// One CTA of 1024 threads per style layer; deterministic reduction.
// Stage 1 (one CTA per layer): mean / std terms of Eq. 5 per channel, from the channel sums and
// diag(G): beta_j (added to R's diagonal), alpha_j (epilogue offset), the moment loss, and the
// moments themselves when requested.
__global__ void __launch_bounds__(512) style_moments_kernel(StyleFinalizeArgs a) {
  __shared__ double red[512];
  const StyleLayerArgs L = a.L[blockIdx.x];
  const double inv = 1.0 / L.np;
  double s = 0.0;
  for (int j = threadIdx.x; j < L.C; j += blockDim.x) {
    double b = 0.0;
    if (L.S) {
      // rounded products (no contraction into an FMA), so the loss pass reproduces the target
      // pass's mean bit for bit when x = v
      const double m = __dmul_rn(L.S[j], inv);
      const double var = __dmul_rn(L.Gacc[(long long)j * L.C + j], inv) - __dmul_rn(m, m);
      const double sd = var > 0.0 ? sqrt(var) : 0.0;
      if (L.mean_out) L.mean_out[j] = m;
      if (L.std_out) L.std_out[j] = sd;
      if (L.mu) {
        s += L.wm * (m - L.mu[j]) * (m - L.mu[j]) + L.ws * (sd - L.sigma[j]) * (sd - L.sigma[j]);
        b = sd > 0.0 ? L.ws * 2.0 * inv * (sd - L.sigma[j]) / sd : 0.0;
        if (L.alpha) L.alpha[j] = (float)(L.wm * 2.0 * inv * (m - L.mu[j]) - b * m);
      }
    }
    a.beta[blockIdx.x * 512 + j] = b;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 256; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.partial[blockIdx.x * kFinalizeChunks] = red[0];
}

// Stage 2 (grid: layer x chunk): G = Gacc / np, R = (4 w / np)(G - Ghat) + diag(beta), and the
// chunk's share of w ||G - Ghat||^2 into partial[layer][1 + chunk]
__global__ void __launch_bounds__(256) style_residual_kernel(StyleFinalizeArgs a) {
  __shared__ double red[256];
  const StyleLayerArgs L = a.L[blockIdx.x];
  const long long n = (long long)L.C * L.C;
  const long long per = (n + gridDim.y - 1) / gridDim.y;
  const long long e0 = blockIdx.y * per, e1 = e0 + per < n ? e0 + per : n;
  const double inv = 1.0 / L.np, rs = 4.0 * L.w / L.np;
  double s = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double G = L.Gacc[e] * inv;
    const double d = G - L.Ghat[e];
    L.Gout[e] = G;
    s += L.w * d * d;
    const int i = (int)(e / L.C), j = (int)(e % L.C);
    const double r = rs * d + (i == j ? a.beta[blockIdx.x * 512 + j] : 0.0);
    if (a.r_is_bf16)
      reinterpret_cast<__nv_bfloat16 *>(L.R)[e] = __float2bfloat16_rn((float)r);
    else
      reinterpret_cast<float *>(L.R)[e] = (float)r;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.partial[blockIdx.x * kFinalizeChunks + 1 + blockIdx.y] = red[0];
}

// Stage 3: E_L = sum of the layer's partials in a fixed order
__global__ void style_sum_kernel(StyleFinalizeArgs a, int chunks) {
  const int l = threadIdx.x;
  if (l < kNStyle) {
    double s = 0.0;
    for (int c = 0; c <= chunks; c++) s += a.partial[l * kFinalizeChunks + c];
    a.Eparts[l] = s;
  }
}

void launch_style_finalize(const StyleFinalizeArgs &a, cudaStream_t s) {
  style_moments_kernel<<<kNStyle, 512, 0, s>>>(a);
  style_residual_kernel<<<dim3(kNStyle, kFinalizeChunks - 1), 256, 0, s>>>(a);
  style_sum_kernel<<<1, 32, 0, s>>>(a, kFinalizeChunks - 1);
}

// channel sums over owned pixels: partial[c][j] = sum over chunk c of V[p][j] (FP32 runs of 64
// pixels added in FP64)
template <typename T>
__global__ void __launch_bounds__(256) chansum_partial_kernel(
    const T *__restrict__ V, int Hb, int Wb, int C, const OwnRect *__restrict__ own,
    const GramChunk *__restrict__ chunks, double *__restrict__ partial) {
  const GramChunk ch = chunks[blockIdx.x];
  const OwnRect r = own[ch.b];
  const int rw = r.x1 - r.x0;
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    double acc = 0.0;
    for (int q0 = ch.p0; q0 < ch.p1; q0 += 64) {
      float f = 0.f;
      const int q1 = q0 + 64 < ch.p1 ? q0 + 64 : ch.p1;
      for (int q = q0; q < q1; q++) {
        const int y = r.y0 + q / rw, x = r.x0 + q % rw;
        f += to_f(V[(((size_t)ch.b * Hb + y) * Wb + x) * C + j]);
      }
      acc += (double)f;
    }
    partial[(size_t)blockIdx.x * C + j] = acc;
  }
}

// S[j] += sum over chunks of partial[c][j]: a CTA takes 32 channels (lane = channel), its 8 warps
// split the chunks (warp w: chunks w, w + 8, ... in order), then the warps are added in order
__global__ void __launch_bounds__(256) chansum_reduce_kernel(const double *__restrict__ partial,
                                                             int nchunks, int C,
                                                             double *__restrict__ S) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (j < C)
    for (int c = warp; c < nchunks; c += 8) s += partial[(size_t)c * C + j];
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && j < C) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; w++) t += red[w][lane];
    S[j] += t;
  }
}

template <typename T>
void launch_chansum(const T *V, int Hb, int Wb, int C, const OwnRect *own,
                    const GramChunk *chunks, int nchunks, double *partial, double *S,
                    cudaStream_t s) {
  if (nchunks <= 0) return;
  chansum_partial_kernel<T><<<nchunks, 256, 0, s>>>(V, Hb, Wb, C, own, chunks, partial);
  chansum_reduce_kernel<<<(C + 31) / 32, 256, 0, s>>>(partial, nchunks, C, S);
}
template void launch_chansum<float>(const float *, int, int, int, const OwnRect *,
                                    const GramChunk *, int, double *, double *, cudaStream_t);
template void launch_chansum<__nv_bfloat16>(const __nv_bfloat16 *, int, int, int,
                                            const OwnRect *, const GramChunk *, int, double *,
                                            double *, cudaStream_t);


// ---- content loss over owned pixels: partial[c] = sum (V - Vu)^2 (FP64) ----------------------------
template <typename T>
__global__ void __launch_bounds__(256) content_partial_kernel(
    const T *__restrict__ V, int Hb, int Wb, const T *__restrict__ Vu, int Hc, int Wc,
    const BlockGeom *__restrict__ geom, const OwnRect *__restrict__ own,
    const GramChunk *__restrict__ chunks, double *__restrict__ partial) {
  __shared__ double red[256];
  const GramChunk ch = chunks[blockIdx.x];
  const OwnRect r = own[ch.b];
  const BlockGeom g = geom[ch.b];
  const int rw = r.x1 - r.x0;
  const int oy = g.ey0 >> kContentLevel, ox = g.ex0 >> kContentLevel;
  double s = 0.0;
  // 64 threads per pixel row of 512 channels (8 each)
  for (int q = ch.p0 + (threadIdx.x >> 6); q < ch.p1; q += 4) {
    const int y = r.y0 + q / rw, x = r.x0 + q % rw;
    const int c = (threadIdx.x & 63) * 8;
    float a[8], t[8];
    load8(V + (((size_t)ch.b * Hb + y) * Wb + x) * 512 + c, a);
    load8(Vu + ((size_t)(oy + y) * Wc + ox + x) * 512 + c, t);
    // differences of two stored values are exact in FP32 (BF16 inputs) or nearly so (FP32
    // inputs); 8 squares summed in FP32, then accumulated in FP64
    float f = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const float d = a[j] - t[j];
      f = fmaf(d, d, f);
    }
    s += (double)f;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// acc += lambda * sum_c partial[c] in a fixed order
// (256 threads: thread t adds partials t, t + 256, ... in order, then a fixed tree; the same
// order every time, several times faster than one thread adding a thousand partials in turn)
__global__ void __launch_bounds__(256) content_reduce_kernel(const double *__restrict__ partial,
                                                             int n, double lambda,
                                                             double *__restrict__ acc) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *acc += lambda * red[0];
}

template <typename T>
void launch_content_loss(const T *V, int Hb, int Wb, const T *Vu, int Hc, int Wc,
                         const BlockGeom *geom, const OwnRect *own, const GramChunk *chunks,
                         int nchunks, double *partial, double lambda, double *acc,
                         cudaStream_t s) {
  if (nchunks > 0) {
    content_partial_kernel<T><<<nchunks, 256, 0, s>>>(V, Hb, Wb, Vu, Hc, Wc, geom, own, chunks,
                                                      partial);
    content_reduce_kernel<<<1, 256, 0, s>>>(partial, nchunks, lambda, acc);
  }
}
template void launch_content_loss<float>(const float *, int, int, const float *, int, int,
                                         const BlockGeom *, const OwnRect *, const GramChunk *,
                                         int, double *, double, double *, cudaStream_t);
template void launch_content_loss<__nv_bfloat16>(const __nv_bfloat16 *, int, int,
                                                 const __nv_bfloat16 *, int, int,
                                                 const BlockGeom *, const OwnRect *,
                                                 const GramChunk *, int, double *, double,
                                                 double *, cudaStream_t);

// ---- content target crop: owned ReLU4_2 features of each block into the global map ------------------
template <typename T>
__global__ void crop_content_kernel(const T *__restrict__ V, int B, int Hb, int Wb,
                                    const BlockGeom *__restrict__ geom,
                                    const OwnRect *__restrict__ own, T *__restrict__ Vu, int Hc,
                                    int Wc) {
  const int b = blockIdx.y;
  const OwnRect r = own[b];
  const BlockGeom g = geom[b];
  const int rw = r.x1 - r.x0;
  const long long n = (long long)(r.y1 - r.y0) * rw * 64;
  const int oy = g.ey0 >> kContentLevel, ox = g.ex0 >> kContentLevel;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % 64) * 8;
    const long long q = i / 64;
    const int y = r.y0 + (int)(q / rw), x = r.x0 + (int)(q % rw);
    float v[8];
    load8(V + (((size_t)b * Hb + y) * Wb + x) * 512 + c, v);
    store8(Vu + ((size_t)(oy + y) * Wc + ox + x) * 512 + c, v);
  }
  (void)B;
  (void)Hc;
}

template <typename T>
void launch_crop_content(const T *V, int B, int Hb, int Wb, const BlockGeom *geom,
                         const OwnRect *own, T *Vu, int Hc, int Wc, int max_own_px,
                         cudaStream_t s) {
  int gx = (int)(((long long)max_own_px * 64 + 255) / 256);
  if (gx > 2048) gx = 2048;
  if (gx < 1) gx = 1;
  crop_content_kernel<T><<<dim3(gx, B), 256, 0, s>>>(V, B, Hb, Wb, geom, own, Vu, Hc, Wc);
}
template void launch_crop_content<float>(const float *, int, int, int, const BlockGeom *,
                                         const OwnRect *, float *, int, int, int, cudaStream_t);
template void launch_crop_content<__nv_bfloat16>(const __nv_bfloat16 *, int, int, int,
                                                 const BlockGeom *, const OwnRect *,
                                                 __nv_bfloat16 *, int, int, int, cudaStream_t);

// ---- misc ---------------------------------------------------------------------------------------
__global__ void check_finite_kernel(const float *__restrict__ x, long long n,
                                    unsigned *__restrict__ err) {
  bool bad = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrNonfinite);
}
void launch_check_finite(const float *x, long long n, unsigned *err, cudaStream_t s) {
  check_finite_kernel<<<ew_grid(n), 256, 0, s>>>(x, n, err);
}

// loss = sum of the five style parts + content part, in fixed order
__global__ void finish_loss_kernel(const double *__restrict__ parts, double *__restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kNStyle + 1; i++) s += parts[i];
    if (loss) *loss = s;
  }
}
void launch_finish_loss(const double *parts, double *loss, cudaStream_t s) {
  finish_loss_kernel<<<1, 32, 0, s>>>(parts, loss);
}

}  // namespace nst
