// nst_api_opt.cu -- C ABI of the optimiser step (L-BFGS, Section 3.1 / Section 5.1) and of the
// multiscale initialisation (Algorithm 2).
#include <cstring>
#include <string>

#include "../../include/nst.h"
#include "nst_kernels.h"
#include "nst_lbfgs_dev.h"

using namespace nst;

struct nst_lbfgs {
  long long n = 0;
  long long stride = 0;              // slot stride: n rounded up to 64 floats (256-byte slots)
  int m = 0;
  long long iters = 0;
  float *S = nullptr, *Y = nullptr;  // [m+1][n] history slots (device pointers)
  float *S_host = nullptr, *Y_host = nullptr;  // host allocations when the history lives there
  float *g_prev = nullptr;
  double *SY = nullptr, *YY = nullptr;   // [m+1][m+1] s_a . y_b and y_a . y_b by slot
  double *partials = nullptr;
  LbfgsCtl *ctl = nullptr;
};

namespace {
constexpr double kCurvEps = 1e-10;
}

extern "C" {

nst_status nst_lbfgs_create(nst_lbfgs **out, long long n, int m) {
  return nst_lbfgs_create_ex(out, n, m, 0);
}

nst_status nst_lbfgs_create_ex(nst_lbfgs **out, long long n, int m, int flags) {
  if (!out || n <= 0 || m < 1 || m > kMaxHistory || (flags & ~NST_LBFGS_HOST_HISTORY))
    return NST_ERR_INVALID_ARG;
  *out = nullptr;
  nst_lbfgs *st = new nst_lbfgs();
  st->n = n;
  st->m = m;
  st->stride = (n + 63) / 64 * 64;
  const size_t slots = (size_t)(m + 1);
  const size_t hist = slots * st->stride * sizeof(float);
  bool ok = true;
  if (flags & NST_LBFGS_HOST_HISTORY) {
    ok = cudaHostAlloc(&st->S_host, hist, cudaHostAllocMapped | cudaHostAllocPortable) ==
             cudaSuccess &&
         cudaHostAlloc(&st->Y_host, hist, cudaHostAllocMapped | cudaHostAllocPortable) ==
             cudaSuccess &&
         cudaHostGetDevicePointer(&st->S, st->S_host, 0) == cudaSuccess &&
         cudaHostGetDevicePointer(&st->Y, st->Y_host, 0) == cudaSuccess;
    if (ok) {
      std::memset(st->S_host, 0, hist);
      std::memset(st->Y_host, 0, hist);
    }
  } else {
    ok = cudaMalloc(&st->S, hist) == cudaSuccess && cudaMalloc(&st->Y, hist) == cudaSuccess;
    if (ok) ok = cudaMemset(st->S, 0, hist) == cudaSuccess && cudaMemset(st->Y, 0, hist) == cudaSuccess;
  }
  ok = ok &&
            cudaMalloc(&st->g_prev, n * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&st->SY, slots * slots * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&st->YY, slots * slots * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&st->partials, lbfgs_partials_count(m) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&st->ctl, sizeof(LbfgsCtl)) == cudaSuccess;
  if (!ok) {
    nst_lbfgs_destroy(st);
    return NST_ERR_OOM;
  }
  cudaMemset(st->SY, 0, slots * slots * sizeof(double));
  cudaMemset(st->YY, 0, slots * slots * sizeof(double));
  LbfgsCtl c;
  std::memset(&c, 0, sizeof(c));
  c.gamma = 1.0;
  c.count = 0;
  c.spare = 0;
  for (int i = 0; i < kMaxHistory; i++) c.order[i] = -1;
  cudaMemcpy(st->ctl, &c, sizeof(c), cudaMemcpyHostToDevice);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    nst_lbfgs_destroy(st);
    return NST_ERR_CUDA;
  }
  *out = st;
  return NST_OK;
}

nst_status nst_lbfgs_destroy(nst_lbfgs *st) {
  if (!st) return NST_OK;
  cudaDeviceSynchronize();
  if (st->S_host) {
    cudaFreeHost(st->S_host);
    cudaFreeHost(st->Y_host);
  } else {
    cudaFree(st->S);
    cudaFree(st->Y);
  }
  cudaFree(st->g_prev);
  cudaFree(st->SY); cudaFree(st->YY); cudaFree(st->partials); cudaFree(st->ctl);
  delete st;
  return NST_OK;
}

nst_status nst_lbfgs_step(nst_lbfgs *st, float *x, const float *g, void *stream) {
  if (!st || !x || !g) return NST_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int first = st->iters == 0 ? 1 : 0;
  // 1. one pass over g, g_prev and every stored vector: y = g - g_prev into the spare slot and
  //    all dot products of the compact representation (first call: ||g||_1)
  launch_lbfgs_dots(g, st->g_prev, st->S, st->Y, st->stride, st->n, st->ctl, st->m, first,
                    st->partials, s);
  // 2. curvature test, history update, S^T Y / Y^T Y update, small solve (one CTA)
  launch_lbfgs_solve(st->ctl, st->partials, st->m, first, kCurvEps, st->SY, st->YY, s);
  // 3. one pass forming s = t d (into the spare slot), x += s, g_prev = g
  launch_lbfgs_combine(x, st->S, st->Y, st->stride, st->g_prev, g, st->n, st->ctl, s);
  if (cudaGetLastError() != cudaSuccess) return NST_ERR_CUDA;
  st->iters++;
  return NST_OK;
}

nst_status nst_lbfgs_info(nst_lbfgs *st, int *pairs, long long *iters, void *stream) {
  if (!st) return NST_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return NST_ERR_CUDA;
  LbfgsCtl c;
  if (cudaMemcpy(&c, st->ctl, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
    return NST_ERR_CUDA;
  if (pairs) *pairs = c.count;
  if (iters) *iters = st->iters;
  return NST_OK;
}

nst_status nst_upsample_init(const float *xs, int h, int w, float *x, int H, int W,
                             void *stream) {
  if (!xs || !x || h < 1 || w < 1 || H < 1 || W < 1) return NST_ERR_INVALID_ARG;
  launch_bicubic(xs, 3, h, w, x, H, W, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? NST_OK : NST_ERR_CUDA;
}

nst_status nst_downscale(const float *x, int h, int w, float *out, int H, int W, void *stream) {
  if (!x || !out || h < 1 || w < 1 || H < 1 || W < 1 || H > h || W > w) return NST_ERR_INVALID_ARG;
  launch_area(x, 3, h, w, out, H, W, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? NST_OK : NST_ERR_CUDA;
}

}  // extern "C"
