// k_lbfgs.cu -- HBM-bound vector kernels of the optimiser and of the multiscale initialisation:
//   * the L-BFGS step (Section 3.1, after Nocedal 1980) in the compact representation of the
//     inverse-BFGS matrix (Byrd, Nocedal and Schnabel 1994): with S, Y the stored pairs (oldest
//     first), R the upper triangle of S^T Y, D its diagonal and H0 = gamma I,
//         H g = gamma g + S p - gamma Y u,  u = R^-1 (S^T g),
//                                           p = R^-T ((D + gamma Y^T Y) u - gamma Y^T g),
//     the same matrix the two-loop recursion applies. A step reads every stored vector twice
//     (one fused pass for all dot products, one pass forming the step) instead of four times;
//     S^T Y and Y^T Y are kept up to date from the new pair's dot products. Dots are FP32 chunks
//     summed in FP64 with fixed-order reductions; the small solve runs in FP64 on one thread.
//     History slots are resolved on the device, so a step needs no host round trip.
//   * bicubic x2 upscaling used to initialise each scale after the first (Algorithm 2).
#include "nst_internal.cuh"
#include "nst_kernels.h"
#include "nst_lbfgs_dev.h"

namespace nst {

constexpr int kDotThreads = 256;
constexpr int kDotBlocksTotal = 1216;   // 8 CTAs per SM on 152 SMs, shared among the groups

static int dot_groups(int m) { return (m + 1 + kLbGroup - 1) / kLbGroup; }
static int dot_blocks(int m) {   // CTAs per group; fixed for a given m (reproducible reductions)
  const int b = kDotBlocksTotal / dot_groups(m);
  return b < 152 ? 152 : b;
}
int lbfgs_partials_count(int m) { return 4 * (m + 1) * dot_blocks(m); }

// Position p of the fused pass: p = 0 is the candidate pair (spare slot: last step s and the new
// y), p = 1 .. count the stored pairs order[p - 1]. partials[(4 p + q) * nb + cta] for the dots
// q = 0: s.g, 1: y.g, 2: s.y_new, 3: y.y_new. Elements go four at a time (float4) when every
// vector is 16-byte aligned, with all of an element group's loads issued before its FMAs.
template <int G>
struct DotAcc {
  double acc[G][4];
  float part[G][4];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int j = 0; j < G; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[j][q] = 0.0, part[j][q] = 0.f;
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int j = 0; j < G; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[j][q] += (double)part[j][q], part[j][q] = 0.f;
  }
  __device__ __forceinline__ void add(int j, float sv, float wv, float gv, float yv) {
    part[j][0] = fmaf(sv, gv, part[j][0]);
    part[j][1] = fmaf(wv, gv, part[j][1]);
    part[j][2] = fmaf(sv, yv, part[j][2]);
    part[j][3] = fmaf(wv, yv, part[j][3]);
  }
};

__global__ void __launch_bounds__(kDotThreads) lbfgs_dots_kernel(
    const float *__restrict__ g, const float *__restrict__ g_prev, const float *__restrict__ S,
    float *__restrict__ Y, long long stride, long long n, const LbfgsCtl *__restrict__ c,
    int first, int vec, double *__restrict__ partials) {
  constexpr int G = kLbGroup;
  __shared__ long long off[G];
  __shared__ int nj_sh;
  __shared__ long long sp_off;
  __shared__ double red[kDotThreads / 32][4 * G];
  const int grp = blockIdx.y, nb = gridDim.x;
  if (threadIdx.x == 0) {
    const int count = c->count;
    int nj = 0;
    for (int j = 0; j < G; j++) {
      const int p = grp * G + j;
      off[j] = 0;
      if (p <= count) {
        off[j] = (long long)(p == 0 ? c->spare : c->order[p - 1]) * stride;
        nj = j + 1;
      }
    }
    nj_sh = first ? (grp == 0 ? 1 : 0) : nj;
    sp_off = (long long)c->spare * stride;
  }
  __syncthreads();
  const int nj = nj_sh;
  if (nj == 0) return;
  float *ynew = Y + sp_off;
  const bool own_y = grp == 0;   // group 0 holds the candidate (position 0) and writes its y
  const long long tstride = (long long)nb * kDotThreads;
  const long long t0 = (long long)blockIdx.x * kDotThreads + threadIdx.x;
  DotAcc<G> A;
  A.clear();
  int chunk = 0;
  const long long n4 = vec ? n / 4 : 0;
  for (long long v = t0; v < n4; v += tstride) {
    const float4 gv = reinterpret_cast<const float4 *>(g)[v];
    if (first) {
      A.part[0][0] += fabsf(gv.x) + fabsf(gv.y) + fabsf(gv.z) + fabsf(gv.w);
    } else {
      const float4 gp = reinterpret_cast<const float4 *>(g_prev)[v];
      const float4 yv = make_float4(gv.x - gp.x, gv.y - gp.y, gv.z - gp.z, gv.w - gp.w);
      if (own_y) reinterpret_cast<float4 *>(ynew)[v] = yv;
      float4 sv[G], wv[G];
#pragma unroll
      for (int j = 0; j < G; j++) {
        if (j < nj) {
          sv[j] = reinterpret_cast<const float4 *>(S + off[j])[v];
          wv[j] = (own_y && j == 0) ? yv : reinterpret_cast<const float4 *>(Y + off[j])[v];
        }
      }
#pragma unroll
      for (int j = 0; j < G; j++) {
        if (j < nj) {
          A.add(j, sv[j].x, wv[j].x, gv.x, yv.x);
          A.add(j, sv[j].y, wv[j].y, gv.y, yv.y);
          A.add(j, sv[j].z, wv[j].z, gv.z, yv.z);
          A.add(j, sv[j].w, wv[j].w, gv.w, yv.w);
        }
      }
    }
    if (++chunk == 4) { chunk = 0; A.flush(); }   // FP32 over 16 elements, FP64 across chunks
  }
  for (long long i = n4 * 4 + t0; i < n; i += tstride) {   // scalar path / tail
    const float gv = g[i];
    if (first) {
      A.part[0][0] += fabsf(gv);
    } else {
      const float yv = gv - g_prev[i];
      if (own_y) ynew[i] = yv;
#pragma unroll
      for (int j = 0; j < G; j++)
        if (j < nj) A.add(j, S[off[j] + i], (own_y && j == 0) ? yv : Y[off[j] + i], gv, yv);
    }
    if (++chunk == 16) { chunk = 0; A.flush(); }
  }
  A.flush();
  // fixed-order block reduction: warp shuffles, then the warps in index order
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < G; j++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      double v = A.acc[j][q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][j * 4 + q] = v;
    }
  __syncthreads();
  if (threadIdx.x < 4 * nj) {
    double v = 0.0;
    for (int w = 0; w < kDotThreads / 32; w++) v += red[w][threadIdx.x];
    const int d = grp * G * 4 + threadIdx.x;   // = 4 p + q
    partials[(size_t)d * nb + blockIdx.x] = v;
  }
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

void launch_lbfgs_dots(const float *g, const float *g_prev, const float *S, float *Y,
                       long long stride, long long n, const LbfgsCtl *c, int m, int first,
                       double *partials, cudaStream_t s) {
  dim3 grid(dot_blocks(m), first ? 1 : dot_groups(m));
  const int vec = aligned16(g) && aligned16(g_prev) && aligned16(S) && aligned16(Y) &&
                  stride % 4 == 0;
  lbfgs_dots_kernel<<<grid, kDotThreads, 0, s>>>(g, g_prev, S, Y, stride, n, c, first, vec,
                                                 partials);
}

__global__ void __launch_bounds__(256) lbfgs_solve_kernel(LbfgsCtl *__restrict__ c,
                                                          const double *__restrict__ partials,
                                                          int nb, int m, int first, double eps,
                                                          double *__restrict__ SY,
                                                          double *__restrict__ YY) {
  __shared__ double dots[4 * (kMaxHistory + 1)];
  __shared__ double sg[kMaxHistory + 1], yg[kMaxHistory + 1];   // by slot
  __shared__ double u[kMaxHistory], w[kMaxHistory], pv[kMaxHistory];
  __shared__ int sl[kMaxHistory];
  const int count0 = c->count;
  const int nd = first ? 1 : 4 * (count0 + 1);
  for (int d = threadIdx.x; d < nd; d += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < nb; b++) v += partials[(size_t)d * nb + b];   // fixed order
    dots[d] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (first) {
    const double l1 = dots[0];
    c->k = 0;
    c->cg = (float)-(l1 > 1.0 ? 1.0 / l1 : 1.0);   // t = min(1, 1 / ||g||_1), d = -g
    return;
  }
  const int ld = m + 1;
  const int sp = c->spare;
  sg[sp] = dots[0];
  yg[sp] = dots[1];
  for (int p = 1; p <= count0; p++) {
    sg[c->order[p - 1]] = dots[4 * p];
    yg[c->order[p - 1]] = dots[4 * p + 1];
  }
  const double ys = dots[2], yy = dots[3];
  if (ys > eps) {
    // the candidate becomes the newest pair: its column of S^T Y and row / column of Y^T Y
    for (int p = 1; p <= count0; p++) {
      const int a = c->order[p - 1];
      SY[(size_t)a * ld + sp] = dots[4 * p + 2];
      YY[(size_t)a * ld + sp] = dots[4 * p + 3];
      YY[(size_t)sp * ld + a] = dots[4 * p + 3];
    }
    SY[(size_t)sp * ld + sp] = ys;
    YY[(size_t)sp * ld + sp] = yy;
    c->gamma = ys / yy;
    const int keep = count0 < m ? count0 : m - 1;
    for (int i = keep; i >= 1; i--) c->order[i] = c->order[i - 1];
    c->order[0] = sp;
    c->count = keep + 1;
    for (int i = c->count; i < m; i++) c->order[i] = -1;
    for (int s = 0; s <= m; s++) {   // first slot not in use receives the next step
      bool used = false;
      for (int i = 0; i < c->count; i++) used |= c->order[i] == s;
      if (!used) { c->spare = s; break; }
    }
  }
  const int k = c->count;
  const double gamma = k > 0 ? c->gamma : 1.0;
  for (int i = 0; i < k; i++) sl[i] = c->order[k - 1 - i];   // oldest first
  // u = R^-1 (S^T g), R_ij = s_i . y_j (i <= j)
  for (int i = k - 1; i >= 0; i--) {
    double v = sg[sl[i]];
    for (int j = i + 1; j < k; j++) v -= SY[(size_t)sl[i] * ld + sl[j]] * u[j];
    u[i] = v / SY[(size_t)sl[i] * ld + sl[i]];
  }
  // w = (D + gamma Y^T Y) u - gamma Y^T g
  for (int i = 0; i < k; i++) {
    double v = 0.0;
    for (int j = 0; j < k; j++) v += YY[(size_t)sl[i] * ld + sl[j]] * u[j];
    w[i] = SY[(size_t)sl[i] * ld + sl[i]] * u[i] + gamma * (v - yg[sl[i]]);
  }
  // p = R^-T w
  for (int i = 0; i < k; i++) {
    double v = w[i];
    for (int j = 0; j < i; j++) v -= SY[(size_t)sl[j] * ld + sl[i]] * pv[j];
    pv[i] = v / SY[(size_t)sl[i] * ld + sl[i]];
  }
  // d = -H g = -gamma g - S p + gamma Y u; step length 1
  c->k = k;
  for (int i = 0; i < k; i++) {
    c->slot[i] = sl[i];
    c->cS[i] = (float)(-pv[i]);
    c->cY[i] = (float)(gamma * u[i]);
  }
  c->cg = (float)(-gamma);
}

void launch_lbfgs_solve(LbfgsCtl *c, const double *partials, int m, int first, double eps,
                        double *SY, double *YY, cudaStream_t s) {
  lbfgs_solve_kernel<<<1, 256, 0, s>>>(c, partials, dot_blocks(m), m, first, eps, SY, YY);
}

__global__ void __launch_bounds__(256) lbfgs_combine_kernel(
    float *__restrict__ x, float *__restrict__ S, const float *__restrict__ Y, long long stride,
    float *__restrict__ g_prev, const float *__restrict__ g, long long n,
    const LbfgsCtl *__restrict__ c, int vec) {
  constexpr int U = 8;   // stored pairs whose loads are issued together
  __shared__ float cS[kMaxHistory], cY[kMaxHistory];
  __shared__ long long off[kMaxHistory];
  __shared__ float cg_sh;
  __shared__ int k_sh;
  __shared__ long long sp_off;
  if (threadIdx.x == 0) {
    k_sh = c->k;
    cg_sh = c->cg;
    sp_off = (long long)c->spare * stride;
  }
  for (int i = threadIdx.x; i < kMaxHistory; i += blockDim.x) {
    cS[i] = c->cS[i];
    cY[i] = c->cY[i];
    off[i] = (long long)c->slot[i] * stride;
  }
  __syncthreads();
  const int k = k_sh;
  const float cg = cg_sh;
  float *snew = S + sp_off;
  const long long tstride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n4 = vec ? n / 4 : 0;
  for (long long v = t0; v < n4; v += tstride) {
    const float4 gv = reinterpret_cast<const float4 *>(g)[v];
    float4 d = make_float4(cg * gv.x, cg * gv.y, cg * gv.z, cg * gv.w);
    for (int j0 = 0; j0 < k; j0 += U) {
      float4 sv[U], yv[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (j0 + u < k) {
          sv[u] = reinterpret_cast<const float4 *>(S + off[j0 + u])[v];
          yv[u] = reinterpret_cast<const float4 *>(Y + off[j0 + u])[v];
        }
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (j0 + u < k) {
          const float a = cS[j0 + u], b = cY[j0 + u];
          d.x = fmaf(b, yv[u].x, fmaf(a, sv[u].x, d.x));
          d.y = fmaf(b, yv[u].y, fmaf(a, sv[u].y, d.y));
          d.z = fmaf(b, yv[u].z, fmaf(a, sv[u].z, d.z));
          d.w = fmaf(b, yv[u].w, fmaf(a, sv[u].w, d.w));
        }
      }
    }
    reinterpret_cast<float4 *>(snew)[v] = d;
    float4 xv = reinterpret_cast<float4 *>(x)[v];
    xv.x += d.x; xv.y += d.y; xv.z += d.z; xv.w += d.w;
    reinterpret_cast<float4 *>(x)[v] = xv;
    reinterpret_cast<float4 *>(g_prev)[v] = gv;
  }
  for (long long i = n4 * 4 + t0; i < n; i += tstride) {   // scalar path / tail
    const float gv = g[i];
    float d = cg * gv;
    for (int j = 0; j < k; j++) d = fmaf(cY[j], Y[off[j] + i], fmaf(cS[j], S[off[j] + i], d));
    snew[i] = d;
    x[i] += d;
    g_prev[i] = gv;
  }
}

void launch_lbfgs_combine(float *x, float *S, const float *Y, long long stride, float *g_prev,
                          const float *g, long long n, const LbfgsCtl *c, cudaStream_t s) {
  const int vec = aligned16(x) && aligned16(S) && aligned16(Y) && aligned16(g_prev) &&
                  aligned16(g) && stride % 4 == 0;
  long long b = (n / 4 + 255) / 256;
  const int grid = (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
  lbfgs_combine_kernel<<<grid, 256, 0, s>>>(x, S, Y, stride, g_prev, g, n, c, vec);
}

// ---- bicubic resampling ---------------------------------------------------------------------------
// Keys cubic convolution, a = -0.75, source coordinate (i + 0.5) * h / H - 0.5, clamped indices;
// rows are combined first, then columns.
__device__ __forceinline__ float keys_w(float t) {
  const float A = -0.75f;
  t = fabsf(t);
  if (t <= 1.f) return ((A + 2.f) * t - (A + 3.f)) * t * t + 1.f;
  if (t < 2.f) return ((A * t - 5.f * A) * t + 8.f * A) * t - 4.f * A;
  return 0.f;
}

__global__ void bicubic_kernel(const float *__restrict__ x, int C, int h, int w,
                               float *__restrict__ out, int H, int W) {
  const long long n = (long long)C * H * W;
  const float sy = (float)h / (float)H, sx = (float)w / (float)W;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(i % W);
    const int Y = (int)((i / W) % H);
    const int c = (int)(i / ((long long)W * H));
    const float fy = (Y + 0.5f) * sy - 0.5f, fx = (X + 0.5f) * sx - 0.5f;
    const int iy = (int)floorf(fy), ix = (int)floorf(fx);
    const float ty = fy - iy, tx = fx - ix;
    const float wy[4] = {keys_w(1.f + ty), keys_w(ty), keys_w(1.f - ty), keys_w(2.f - ty)};
    const float wx[4] = {keys_w(1.f + tx), keys_w(tx), keys_w(1.f - tx), keys_w(2.f - tx)};
    const float *src = x + (size_t)c * h * w;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int xx = min(max(ix - 1 + j, 0), w - 1);
      float col = 0.f;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int yy = min(max(iy - 1 + k, 0), h - 1);
        col = fmaf(wy[k], src[(size_t)yy * w + xx], col);
      }
      acc = fmaf(wx[j], col, acc);
    }
    out[i] = acc;
  }
}

void launch_bicubic(const float *x, int C, int h, int w, float *out, int H, int W,
                    cudaStream_t s) {
  long long n = (long long)C * H * W;
  long long b = (n + 255) / 256;
  int grid = (int)(b < 152 * 32 ? b : 152 * 32);
  bicubic_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(x, C, h, w, out, H, W);
}

// ---- area-average downscaling (adaptive average pooling) ---------------------------------------
// out[c][Y][X] = mean of x[c][y][x] over y in [floor(Y h / H), ceil((Y+1) h / H)) and
// x in [floor(X w / W), ceil((X+1) w / W)): the downscaling of (u, v) in Algorithm 2.
__global__ void area_kernel(const float *__restrict__ x, int C, int h, int w,
                            float *__restrict__ out, int H, int W) {
  const long long n = (long long)C * H * W;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(i % W);
    const int Y = (int)((i / W) % H);
    const int c = (int)(i / ((long long)W * H));
    const int y0 = (int)(((long long)Y * h) / H), y1 = (int)(((long long)(Y + 1) * h + H - 1) / H);
    const int x0 = (int)(((long long)X * w) / W), x1 = (int)(((long long)(X + 1) * w + W - 1) / W);
    const float *src = x + (size_t)c * h * w;
    double acc = 0.0;
    for (int y = y0; y < y1; y++) {
      float row = 0.f;
      for (int xx = x0; xx < x1; xx++) row += src[(size_t)y * w + xx];
      acc += (double)row;
    }
    out[i] = (float)(acc / ((double)(y1 - y0) * (double)(x1 - x0)));
  }
}

void launch_area(const float *x, int C, int h, int w, float *out, int H, int W, cudaStream_t s) {
  long long n = (long long)C * H * W;
  long long b = (n + 255) / 256;
  int grid = (int)(b < 152 * 32 ? b : 152 * 32);
  area_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(x, C, h, w, out, H, W);
}

}  // namespace nst
