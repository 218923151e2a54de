// k_gram_tc.cu -- Gram statistics on the tensor cores: sum over owned pixels p of V_p V_p^T
// (Eq. 4, accumulated block by block as in Algorithm 1, Step 1).
//
// GEMM view: D[M x N] = A[M x K] B[K x N] with M = 128 channels of the I tile, N = channels of
// the J tile (64 / 128 / 256), K = pixels. Both operands are the same NHWC activation, so both
// are MN-major in shared memory (64 channels = 128 bytes contiguous per pixel row, 128-byte
// swizzle). One TMA box of 64 pixels feeds every operand slab of a K step. Each block gets its
// own tensor map whose bounds are its owned rectangle, so pixels outside it read as zero and
// never enter the sum. Every CTA accumulates one (I, J) tile over one run of boxes in TMEM
// (FP32) and writes it out; a fixed-order compensated reduction adds the runs (deterministic).
// When the I tile's channels are among the J tile's (C <= 128, and the diagonal tiles of
// larger C), the A operand is read from the B slabs already in shared memory instead of being
// loaded again; A channels past C (C = 64) read a slab of zeros written once per CTA.
#include <algorithm>

#include "nst_internal.cuh"
#include "nst_kernels.h"
#include "tc_ptx.cuh"

namespace nst {
namespace {

using namespace nst::tc;

constexpr int kThreads = 192;
constexpr uint32_t kSlab = 64 * 128;  // one 64-pixel x 64-channel BF16 slab
constexpr uint32_t kSmemMax = 227 * 1024;

// Stages of the box ring: ALOAD (some I tile's channels lie outside the J tile, C = 512) keeps
// room for two A slabs per stage, 4 stages; otherwise A is always read from the B slabs (or the
// zero slab) and a stage is the B slabs alone, so more boxes are in flight (8 at N = 64, 128;
// 6 at N = 256).
template <int N, bool ALOAD>
struct GramCfg {
  static constexpr uint32_t A_BYTES = ALOAD ? 2 * kSlab : 0u;
  static constexpr uint32_t B_BYTES = (N / 64) * kSlab;
  static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int FIT = (int)((kSmemMax - kSlab - 1024) / STAGE_BYTES);
  static constexpr int STAGES = ALOAD ? 4 : (FIT > 8 ? 8 : FIT);
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + kSlab + 1024;
};

template <int N, bool ALOAD>
__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(GramTcArgs a) {
  using Cfg = GramCfg<N, ALOAD>;
  constexpr int kStages = Cfg::STAGES;
  constexpr uint32_t A_BYTES = Cfg::A_BYTES;
  constexpr uint32_t B_BYTES = Cfg::B_BYTES;
  constexpr uint32_t STAGE_BYTES = Cfg::STAGE_BYTES;
  constexpr uint32_t ZERO_OFF = kStages * STAGE_BYTES;   // one slab of zeros after the stages
  constexpr uint32_t TMEM_COLS = N;
  // kind::f16, FP32 D, BF16 A/B, both MN-major, M = 128, N
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                             ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const GramTcChunk ch = a.chunks[blockIdx.x];
  const int tile = blockIdx.y, I = tile / a.nJ, J = tile % a.nJ;
  const CUtensorMap *map = a.maps + ch.b;
  // A slab s (channels I*128 + 64 s ..) is B slab (I*128 + 64 s - J*N) / 64 when it lies inside
  // the J tile, zeros when it lies past C, else loaded
  int a_src[2];
  bool a_load = false;
#pragma unroll
  for (int sl = 0; sl < 2; sl++) {
    const int c0 = I * 128 + 64 * sl;
    if (c0 >= a.C) a_src[sl] = -2;                                   // zeros
    else if (c0 >= J * N && c0 + 64 <= J * N + N) a_src[sl] = (c0 - J * N) / 64;   // B slab
    else { a_src[sl] = -1; a_load = true; }                          // own A slab
  }
  // (without room for A slabs (ALOAD false) the host has checked that no tile needs them)
  const uint32_t tx_bytes = B_BYTES + (ALOAD && a_load ? A_BYTES : 0u);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (a_src[0] == -2 || a_src[1] == -2) {   // the zero slab (read by the MMAs only)
    uint8_t *z = smem_raw + (smem_base - smem_u32(smem_raw)) + ZERO_OFF;
    for (int i = threadIdx.x; i < (int)(kSlab / 16); i += kThreads)
      *reinterpret_cast<uint4 *>(z + (size_t)i * 16) = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
  }
  if (warp == 1) tmem_alloc(smem_u32(&tmem_base_sh), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int k = ch.box0; k < ch.box1; k++) {
        if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, &abort_flag, a.err)) break;
        const uint32_t fb = smem_u32(&full_bar[stage]);
        const uint32_t sa = smem_base + stage * STAGE_BYTES, sb = sa + A_BYTES;
        const int x = (k % ch.nbx) * a.TW, y = (k / ch.nbx) * a.TH;
        mbar_expect_tx(fb, tx_bytes);
        if (ALOAD && a_load) {
          tma_load_4d(sa, map, fb, I * 128, x, y, 0);
          tma_load_4d(sa + kSlab, map, fb, I * 128 + 64, x, y, 0);
        }
#pragma unroll
        for (int j = 0; j < N / 64; j++) tma_load_4d(sb + j * kSlab, map, fb, J * N + j * 64, x, y, 0);
        if (++stage == kStages) { stage = 0; phase ^= 1; }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int k = ch.box0; k < ch.box1; k++) {
        if (!mbar_wait(smem_u32(&full_bar[stage]), phase, &abort_flag, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_base + stage * STAGE_BYTES, sb = sa + A_BYTES;
        // A's two 64-channel atoms: its own slabs, B slabs, or the zero slab (after every stage,
        // so the atom distance, the descriptor's leading byte offset, stays positive)
        uint32_t a0 = sa, lbo = kSlab;
        if (!a_load) {
          a0 = a_src[0] >= 0 ? sb + (uint32_t)a_src[0] * kSlab : smem_base + ZERO_OFF;
          const uint32_t a1 =
              a_src[1] >= 0 ? sb + (uint32_t)a_src[1] * kSlab : smem_base + ZERO_OFF;
          lbo = a1 - a0;
        }
#pragma unroll
        for (int kk = 0; kk < 4; kk++)   // 16 pixels (two 8-row groups) per MMA
          mma_bf16(tmem_base, sw128_desc_mn(a0 + kk * 2048, lbo),
                   sw128_desc_mn(sb + kk * 2048, kSlab), IDESC,
                   (k > ch.box0 || kk > 0) ? 1u : 0u);
        mma_commit(smem_u32(&empty_bar[stage]));
        if (++stage == kStages) { stage = 0; phase ^= 1; }
      }
      if (ok) mma_commit(smem_u32(&done_bar));
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;   // channel I * 128 + row
    // lane 0 waits (bounded); the warp then proceeds or leaves as one (tcgen05.ld is warp-wide)
    int ready = 0;
    if (lane == 0) ready = mbar_wait(smem_u32(&done_bar), 0, &abort_flag, a.err);
    if (__shfl_sync(0xffffffffu, ready, 0)) {
      tc_fence_after();
      float *out = a.part + (((size_t)blockIdx.x * a.nI * a.nJ + tile) * 128 + row) * N;
      const bool live = I * 128 + row < a.C;
#pragma unroll 1
      for (int c = 0; c < N; c += 32) {
        float v[32];
        tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
        if (live) {
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4 *>(out + c + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
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

// Compensated FP32 addition (Knuth's TwoSum): s + c carries the sum of every added value with
// the rounding error of each addition kept in c, so the pair is as exact as an FP64 sum of the
// FP32 inputs up to O(n u^2) (u = 2^-24) and costs seven FP32 operations, where the FP64 unit of
// this GPU retires a few operations per SM and clock.
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x) {
  const float t = s + x;
  const float z = t - s;
  c += (s - (t - z)) + (x - z);
  s = t;
}

// Gacc[i][j] += sum over runs (fixed order, compensated FP32, then FP64) of the FP32 tile
// partials. A CTA takes 32 V consecutive elements (V per lane: one float4 load per run when
// V = 4, coalesced); its NW warps split the runs (warp w sums runs w, w + NW, ... in order) and
// the NW partial pairs are added in warp order (deterministic); each element's pair is converted
// to FP64 once and added to Gacc. A warp issues the loads of up to 8 of its runs before adding
// them (in run order), so the loads are in flight together instead of one after another.
// C^2 is a multiple of 4096 and V consecutive elements stay inside one N-wide tile row, so the
// V elements of a lane are contiguous in every run's partial.
template <int V, int NW>
__global__ void __launch_bounds__(NW * 32) gram_tc_reduce_kernel(const float *__restrict__ part,
                                                                 int nruns, int C, int N, int nI,
                                                                 int nJ,
                                                                 double *__restrict__ Gacc) {
  __shared__ float2 red[NW][32 * V];
  const long long n = (long long)C * C;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t stride = (size_t)nI * nJ * 128 * N;
  for (long long e0 = (long long)blockIdx.x * 32 * V; e0 < n;
       e0 += (long long)gridDim.x * 32 * V) {
    const long long e = e0 + (long long)lane * V;
    float s[V], c[V];
#pragma unroll
    for (int k = 0; k < V; k++) s[k] = c[k] = 0.f;
    if (e < n) {
      const int i = (int)(e / C), j = (int)(e % C);
      const int tile = (i / 128) * nJ + j / N;
      const size_t off = ((size_t)tile * 128 + (i % 128)) * N + (j % N);
      for (int r0 = warp; r0 < nruns; r0 += 8 * NW) {
        float v[8][V];
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const int r = r0 + NW * u;
          if constexpr (V == 4) {
            const float4 q = r < nruns
                                 ? __ldg(reinterpret_cast<const float4 *>(part + (size_t)r * stride + off))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            v[u][0] = q.x; v[u][1] = q.y; v[u][2] = q.z; v[u][3] = q.w;
          } else {
            v[u][0] = r < nruns ? __ldg(part + (size_t)r * stride + off) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 8; u++)
          if (r0 + NW * u < nruns)
#pragma unroll
            for (int k = 0; k < V; k++) two_sum_add(s[k], c[k], v[u][k]);
      }
    }
#pragma unroll
    for (int k = 0; k < V; k++) red[warp][lane * V + k] = make_float2(s[k], c[k]);
    __syncthreads();
    for (int q = threadIdx.x; q < 32 * V; q += NW * 32) {
      if (e0 + q < n) {
        float ts = 0.f, tc = 0.f;
#pragma unroll
        for (int w = 0; w < NW; w++) {
          const float2 p = red[w][q];
          two_sum_add(ts, tc, p.x);
          tc += p.y;
        }
        Gacc[e0 + q] += (double)ts + (double)tc;
      }
    }
    __syncthreads();
  }
}

template <int N, bool ALOAD>
cudaError_t launch_n(const GramTcArgs &a, int nruns, cudaStream_t s) {
  constexpr size_t smem = GramCfg<N, ALOAD>::SMEM;
  static_assert(smem <= kSmemMax, "Gram kernel shared memory");
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<N, ALOAD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  gram_tc_kernel<N, ALOAD><<<dim3(nruns, a.nI * a.nJ), kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// whether some (I, J) tile reads A slabs of its own: an I-tile slab below C that lies outside
// the J tile (the same test the kernel makes per tile)
bool gram_needs_aload(const GramTcArgs &a) {
  for (int I = 0; I < a.nI; I++)
    for (int J = 0; J < a.nJ; J++)
      for (int sl = 0; sl < 2; sl++) {
        const int c0 = I * 128 + 64 * sl;
        if (c0 < a.C && !(c0 >= J * a.N && c0 + 64 <= J * a.N + a.N)) return true;
      }
  return false;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

void gram_tc_shape(int C, int *N, int *nI, int *nJ) {
  *N = C >= 256 ? 256 : C;
  *nI = C <= 128 ? 1 : C / 128;
  *nJ = C / *N;
}

void gram_tc_patch(int own_h, int own_w, int *TH, int *TW) {
  static const int cand[5][2] = {{1, 64}, {2, 32}, {4, 16}, {8, 8}, {16, 4}};
  long long best = -1;
  for (auto &c : cand) {
    const long long area = (long long)((own_h + c[0] - 1) / c[0]) * c[0] *
                           ((own_w + c[1] - 1) / c[1]) * c[1];
    if (best < 0 || area < best) { best = area; *TH = c[0]; *TW = c[1]; }
  }
}

cudaError_t encode_gram_map(CUtensorMap *m, const void *base, int C, int own_w, int own_h,
                            long long row_stride_px, int TH, int TW) {
  EncodeTiledFn enc = reinterpret_cast<EncodeTiledFn>(tc_encode_tiled_fn());
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)std::max(own_w, 1),
                        (cuuint64_t)std::max(own_h, 1), 1};
  cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)row_stride_px * C * 2,
                           (cuuint64_t)row_stride_px * C * 2 * std::max(own_h, 1)};
  cuuint32_t box[4] = {64, (cuuint32_t)TW, (cuuint32_t)TH, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims,
                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_gram_tc(const GramTcArgs &a, int nruns, double *Gacc, cudaStream_t s) {
  if (nruns <= 0) return cudaSuccess;
  cudaError_t e;
  const bool aload = gram_needs_aload(a);
  switch (a.N) {
    case 64: e = aload ? launch_n<64, true>(a, nruns, s) : launch_n<64, false>(a, nruns, s); break;
    case 128: e = aload ? launch_n<128, true>(a, nruns, s) : launch_n<128, false>(a, nruns, s); break;
    case 256: e = aload ? launch_n<256, true>(a, nruns, s) : launch_n<256, false>(a, nruns, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return launch_gram_tc_reduce(a.part, nruns, a.C, a.N, a.nI, a.nJ, Gacc, s);
}

cudaError_t launch_gram_tc_reduce(const float *part, int nruns, int C, int N, int nI, int nJ,
                                  double *Gacc, cudaStream_t s) {
  if (nruns <= 0) return cudaSuccess;
  // float4 lanes where that still gives two CTAs per SM; otherwise one element per lane and 16
  // warps per CTA splitting the runs (C = 64, 128: few elements, several hundred runs)
  const long long n = (long long)C * C;
  const int sms = tc_num_sms();
  if (n / 128 >= 2LL * sms) {
    const int grid = (int)std::min<long long>(n / 128, 8LL * sms);
    gram_tc_reduce_kernel<4, 8><<<grid, 256, 0, s>>>(part, nruns, C, N, nI, nJ, Gacc);
  } else {
    const int grid = (int)std::min<long long>(n / 32, 4LL * sms);
    gram_tc_reduce_kernel<1, 16><<<grid, 512, 0, s>>>(part, nruns, C, N, nI, nJ, Gacc);
  }
  return cudaGetLastError();
}

}  // namespace nst
