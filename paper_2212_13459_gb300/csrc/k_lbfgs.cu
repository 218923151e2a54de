// k_lbfgs.cu -- HBM-bound vector kernels of the optimiser and of the multiscale initialisation:
//   * L-BFGS two-loop recursion (Section 3.1, after Nocedal 1980): FP64 dot products with a
//     deterministic two-stage reduction, axpy updates whose coefficients stay in device memory,
//     and the step/update kernel. History slots are resolved on the device, so a step needs no
//     host round trip.
//   * bicubic x2 upscaling used to initialise each scale after the first (Algorithm 2).
#include "nst_internal.cuh"
#include "nst_kernels.h"
#include "nst_lbfgs_dev.h"

namespace nst {

constexpr int kDotBlocks = 1216;   // 8 CTAs per SM on 152 SMs; fixed so reductions are reproducible
constexpr int kDotThreads = 256;
int dot_partials_count() { return kDotBlocks; }

__device__ __forceinline__ const float *resolve(const VecRef &r) {
  if (!r.slot) return r.base;
  const int s = *r.slot;
  return s < 0 ? nullptr : r.base + (size_t)s * r.stride;
}

// partial[blockIdx] = sum over the CTA's grid-stride share of a[i]*b[i] (or |a[i]|), in FP64
__global__ void __launch_bounds__(kDotThreads) dot_partial_kernel(VecRef ra, VecRef rb,
                                                                  long long n, int abs_mode,
                                                                  double *__restrict__ partial) {
  __shared__ double red[kDotThreads];
  const float *a = resolve(ra);
  const float *b = abs_mode ? nullptr : resolve(rb);
  double s = 0.0;
  if (a && (abs_mode || b)) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      if (abs_mode)
        s += fabs((double)a[i]);
      else
        s = fma((double)a[i], (double)b[i], s);
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = kDotThreads / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// *out = mul * sum(partial) in fixed order; mul = rho[*slot] (0 if the slot is empty) or 1.
// In abs mode the result is the first step length min(1, 1 / sum).
__global__ void __launch_bounds__(1024) dot_final_kernel(const double *__restrict__ partial, int np,
                                                         const double *__restrict__ mul_base,
                                                         const int *__restrict__ mul_slot,
                                                         int abs_mode, double *__restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 512; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double r = red[0];
    if (abs_mode) {
      r = r > 1.0 ? 1.0 / r : 1.0;
    } else if (mul_base) {
      const int sl = mul_slot ? *mul_slot : 0;
      r = sl < 0 ? 0.0 : mul_base[sl] * r;
    }
    *out = r;
  }
}

void launch_dot_ref(const VecRef &a, const VecRef &b, long long n, double *partials, double *out,
                    const double *mul_base, const int *mul_slot, int abs_mode, cudaStream_t s) {
  dot_partial_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, n, abs_mode, partials);
  dot_final_kernel<<<1, 1024, 0, s>>>(partials, kDotBlocks, mul_base, mul_slot, abs_mode, out);
}

// y += (c1 - c2) * x, with c1, c2 device scalars (c2 may be null) and x resolved on the device;
// no-op when x's slot is empty
__global__ void axpy_kernel(float *__restrict__ y, VecRef rx, long long n,
                            const double *__restrict__ c1, const double *__restrict__ c2,
                            float sign) {
  const float *x = resolve(rx);
  if (!x) return;
  const float c = sign * (float)(*c1 - (c2 ? *c2 : 0.0));
  // the float4 path needs both vectors 16-byte aligned; otherwise everything goes scalar
  const bool vec = (((uintptr_t)y | (uintptr_t)x) & 15) == 0;
  const long long n4 = vec ? n / 4 : 0;
  float4 *y4 = reinterpret_cast<float4 *>(y);
  const float4 *x4 = reinterpret_cast<const float4 *>(x);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    float4 a = y4[i], b = x4[i];
    a.x = fmaf(c, b.x, a.x);
    a.y = fmaf(c, b.y, a.y);
    a.z = fmaf(c, b.z, a.z);
    a.w = fmaf(c, b.w, a.w);
    y4[i] = a;
  }
  for (long long i = n4 * 4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fmaf(c, x[i], y[i]);
}

static int vec_grid(long long n) {
  long long b = (n / 4 + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

void launch_axpy_ref(float *y, const VecRef &x, long long n, const double *c1, const double *c2,
                     float sign, cudaStream_t s) {
  axpy_kernel<<<vec_grid(n), 256, 0, s>>>(y, x, n, c1, c2, sign);
}

// out = a - b, out resolved on the device (the spare history slot)
__global__ void sub_kernel(VecRef rout, const float *__restrict__ a, const float *__restrict__ b,
                           long long n) {
  float *out = const_cast<float *>(resolve(rout));
  if (!out) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}
void launch_sub_ref(const VecRef &out, const float *a, const float *b, long long n,
                    cudaStream_t s) {
  sub_kernel<<<vec_grid(n * 4), 256, 0, s>>>(out, a, b, n);
}

// y = gamma * x (gamma device scalar)
__global__ void scale_kernel(float *__restrict__ y, const float *__restrict__ x, long long n,
                             const double *__restrict__ gamma) {
  const float g = (float)*gamma;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = g * x[i];
}
void launch_scale_dev(float *y, const float *x, long long n, const double *gamma,
                      cudaStream_t s) {
  scale_kernel<<<vec_grid(n * 4), 256, 0, s>>>(y, x, n, gamma);
}

// s = -t r stored in the spare slot; x += s; g_prev = g
__global__ void lbfgs_finish_kernel(float *__restrict__ x, VecRef rs, float *__restrict__ g_prev,
                                    const float *__restrict__ r, const float *__restrict__ g,
                                    long long n, const double *__restrict__ t) {
  float *sv = const_cast<float *>(resolve(rs));
  const float tt = (float)*t;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float st = -tt * r[i];
    if (sv) sv[i] = st;
    x[i] += st;
    g_prev[i] = g[i];
  }
}
void launch_lbfgs_finish_ref(float *x, const VecRef &s_next, float *g_prev, const float *r,
                             const float *g, long long n, const double *t, cudaStream_t s) {
  lbfgs_finish_kernel<<<vec_grid(n * 4), 256, 0, s>>>(x, s_next, g_prev, r, g, n, t);
}

// Curvature test and history bookkeeping, one thread. ys = y^T s, yy = y^T y of the pair held in
// the spare slot. Accepted pairs go to the front of `order` (newest first); the slot dropped
// from the back (if the history is full) or any slot not in `order` becomes the next spare.
__global__ void lbfgs_accept_kernel(LbfgsCtl *__restrict__ c, double *__restrict__ rho, int m,
                                    double eps) {
  if (threadIdx.x || blockIdx.x) return;
  const double ys = c->ys, yy = c->yy;
  const int sp = c->spare;
  if (ys > eps) {
    rho[sp] = 1.0 / ys;
    c->gamma = ys / yy;
    const int keep = c->count < m ? c->count : m - 1;
    for (int i = keep; i >= 1; i--) c->order[i] = c->order[i - 1];
    c->order[0] = sp;
    c->count = keep + 1;
    for (int i = c->count; i < m; i++) c->order[i] = -1;
    for (int s = 0; s <= m; s++) {
      bool used = false;
      for (int i = 0; i < c->count; i++) used |= c->order[i] == s;
      if (!used) { c->spare = s; break; }
    }
  }
}
void launch_lbfgs_accept(LbfgsCtl *c, double *rho, int m, double eps, cudaStream_t s) {
  lbfgs_accept_kernel<<<1, 32, 0, s>>>(c, rho, m, eps);
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
