// nst_noalloc.cu -- nst_gram_noalloc: the Gram statistics of one feature matrix (same kernels,
// same chunking and so the same bits as nst_gram) without any device allocation.
//
// Who needs this: code that runs inside a host application which owns all device memory
// through its own pool (a framework's caching allocator, a real-time renderer's fixed memory
// plan) and does not allow libraries to call cudaMalloc/cudaFree, because those calls
// synchronize the device and fragment or bypass the pool. Such callers can still pass their own
// input and output buffers; the temporary per-chunk partial sums then live in a fixed array
// that this file reserves in the library's device image.
//
// The scratch array below is part of the loaded module: every GPU that loads libnst holds its
// 19 MiB until the process exits, and every call shares it.
#include <cuda.h>

#include <mutex>
#include <string>

#include "../../include/nst.h"
#include "nst_kernels.h"

namespace {

// 1,216 blocks of 64 x 64 FP32 partial sums (19 MiB): the most blocks nst_gram's chunk plan
// uses for any C <= 512 (nchunks * npairs <= 1,216), so both entries chunk identically
constexpr int kScratchBlocks = 1216;
constexpr size_t kScratchFloats = (size_t)kScratchBlocks * 4096;
static __device__ __align__(256) float g_gram_scratch[kScratchFloats];

// Device address of the scratch array, looked up with cudaGetSymbolAddress once per device and
// CUDA context, with that device current. (In host code `g_gram_scratch` names a host-side
// shadow, not device memory.) The context is part of the key because the module, and with it
// the array, is loaded again at another address when a device's context is destroyed and
// recreated (cudaDeviceReset) or another context is made current.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchSlot {
  CUcontext ctx = nullptr;
  float *ptr = nullptr;
};
ScratchSlot g_slot[kMaxDevices];
CtxGetCurrentFn g_ctx_get = nullptr;
bool g_ctx_get_tried = false;

cudaError_t scratch_for_current_device(float **out, std::string &why) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { why = "cudaGetDevice"; return e; }
  if (dev < 0 || dev >= kMaxDevices) { why = "device ordinal out of range"; return cudaErrorInvalidDevice; }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ctx_get_tried) {
    g_ctx_get_tried = true;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get = reinterpret_cast<CtxGetCurrentFn>(fn);
  }
  if (!g_ctx_get) {
    why = "cuCtxGetCurrent unavailable";
    return cudaErrorNotSupported;
  }
  // null until the runtime has set up this thread's context; the lookup below does that
  CUcontext ctx = nullptr;
  if (g_ctx_get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  ScratchSlot &s = g_slot[dev];
  if (!ctx || !s.ptr || s.ctx != ctx) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) { why = "cudaGetSymbolAddress"; return e; }
    if (g_ctx_get(&ctx) != CUDA_SUCCESS || !ctx) {
      why = "no current CUDA context";
      return cudaErrorDeviceUninitialized;
    }
    s.ptr = static_cast<float *>(p);
    s.ctx = ctx;
  }
  *out = s.ptr;
  return cudaSuccess;
}

nst_status fail(nst_status st, const std::string &m) {
  nst::set_last_error_msg(m.c_str());
  return st;
}

nst_status cuda_fail(cudaError_t e, const std::string &what) {
  return fail(NST_ERR_CUDA, "nst_gram_noalloc: " + what + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" nst_status nst_gram_noalloc(int dtype, const void *V, long long npix, int C,
                                       double *G, void *stream) {
  if ((dtype != NST_PREC_FP32 && dtype != NST_PREC_BF16) || !V || !G || npix < 1 ||
      npix >= (1LL << 31) || C < 64 || C % 64)
    return fail(NST_ERR_INVALID_ARG, "nst_gram_noalloc: bad arguments");
  // beyond the scratch array: the 64 x 64 block pairs of the chunk plan would not fit it
  if (C > 512)
    return fail(NST_ERR_SHAPE, "nst_gram_noalloc: C > 512 exceeds the fixed scratch array");
  long long chunk;
  int nchunks;
  nst::gram_flat_plan(npix, C, &chunk, &nchunks);
  const int nb = C / 64, npairs = nb * (nb + 1) / 2;
  if ((size_t)nchunks * npairs * 4096 > kScratchFloats)
    return fail(NST_ERR_SHAPE, "nst_gram_noalloc: chunk plan exceeds the fixed scratch array");
  // an error left pending by earlier work is reported as such, before anything is launched
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "CUDA error pending before the call");
  float *part = nullptr;
  std::string why;
  e = scratch_for_current_device(&part, why);
  if (e != cudaSuccess) return cuda_fail(e, why);
  cudaStream_t s = (cudaStream_t)stream;
  // the partial kernel overwrites every block it uses; only the output accumulates
  e = cudaMemsetAsync(G, 0, sizeof(double) * C * C, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (dtype == NST_PREC_BF16)
    nst::launch_gram_partial_flat<__nv_bfloat16>((const __nv_bfloat16 *)V, npix, C, chunk,
                                                 nchunks, part, s);
  else
    nst::launch_gram_partial_flat<float>((const float *)V, npix, C, chunk, nchunks, part, s);
  nst::launch_gram_reduce(part, nchunks, C, G, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return NST_OK;
}
