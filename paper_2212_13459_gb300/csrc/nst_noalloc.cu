// nst_noalloc.cu -- nst_gram_noalloc: the Gram statistics of one feature matrix (same kernels
// and result as nst_gram) without any device allocation.
//
// Who needs this: code that runs inside a host application which owns all device memory
// through its own pool (a framework's caching allocator, a real-time renderer's fixed memory
// plan) and does not allow libraries to call cudaMalloc/cudaFree, because those calls
// synchronize the device and fragment or bypass the pool. Such callers can still pass their own
// input and output buffers; the temporary per-chunk partial sums then live in a fixed array
// that this file reserves in the library's device image.
//
// The scratch array below is part of the loaded module: every GPU that loads libnst holds its
// 16 MiB until the process exits, and every call shares it.
#include <algorithm>
#include <mutex>

#include "../../include/nst.h"
#include "nst_kernels.h"

namespace {

// 1,024 blocks of 64 x 64 FP32 partial sums (16 MiB)
constexpr int kScratchBlocks = 1024;
constexpr size_t kScratchFloats = (size_t)kScratchBlocks * 4096;
static __device__ __align__(256) float g_gram_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
// (In host code `g_gram_scratch` is only a host-side shadow; its device address must come from
// the runtime.)
cudaError_t scratch_for_current_device(float **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<float *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" nst_status nst_gram_noalloc(int dtype, const void *V, long long npix, int C,
                                       double *G, void *stream) {
  if ((dtype != NST_PREC_FP32 && dtype != NST_PREC_BF16) || !V || !G || npix < 1 ||
      npix >= (1LL << 31))
    return NST_ERR_INVALID_ARG;
  // the 64 x 64 block pairs of one chunk must fit the scratch: C <= 512 gives at most 36
  if (C < 64 || C > 512 || C % 64) return NST_ERR_SHAPE;
  const int nb = C / 64, npairs = nb * (nb + 1) / 2;
  // as many pixel chunks as the scratch holds (and about as many CTAs as nst_gram uses)
  const long long max_chunks = std::min<long long>(kScratchBlocks / npairs,
                                                   std::max(1, 1216 / npairs));
  long long chunk = std::max(256LL, (npix + max_chunks - 1) / max_chunks);
  chunk = (chunk + 31) / 32 * 32;
  const int nchunks = (int)((npix + chunk - 1) / chunk);
  if ((size_t)nchunks * npairs * 4096 > kScratchFloats) return NST_ERR_SHAPE;
  float *part = nullptr;
  if (scratch_for_current_device(&part) != cudaSuccess) return NST_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the partial kernel overwrites every block it uses; only the output accumulates
  if (cudaMemsetAsync(G, 0, sizeof(double) * C * C, s) != cudaSuccess) return NST_ERR_CUDA;
  if (dtype == NST_PREC_BF16)
    nst::launch_gram_partial_flat<__nv_bfloat16>((const __nv_bfloat16 *)V, npix, C, chunk,
                                                 nchunks, part, s);
  else
    nst::launch_gram_partial_flat<float>((const float *)V, npix, C, chunk, nchunks, part, s);
  nst::launch_gram_reduce(part, nchunks, C, G, s);
  return cudaGetLastError() == cudaSuccess ? NST_OK : NST_ERR_CUDA;
}
