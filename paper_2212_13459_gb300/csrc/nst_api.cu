// nst_api.cu -- the C ABI of libnst and its host-side scheduler.
//
// One evaluation of Algorithm 1 (Section 4.2) is
//   Step 1: for every batch of blocks (extended by margin1): VGG-19 forward to ReLU5_1, Gram partial
//           sums of the owned pixels at the five style layers, reduced into G^L(x) (FP64);
//           then E_style and the style residuals R_L = (4 w_L / n_p)(G^L(x) - G^L(v)) (Eq. 3,
//           Table 1 row 2);
//   Step 2: for every batch of blocks (extended by margin2): forward again keeping activations,
//           feature gradients (style residual fused into the input-gradient convolution that
//           produces dE/dReLU_k_1, content residual 2 lambda (V - V_u) fused at ReLU4_2, Table 1
//           rows 1-2), input-gradient chain back to the pixels, inner part scattered into dE/dx,
//           and the content loss of the owned pixels.
// Blocks of a batch are processed together in every launch (one NHWC buffer per layer).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/nst.h"
#include "nst_internal.cuh"
#include "nst_kernels.h"
#include "nst_lbfgs_dev.h"

using namespace nst;

namespace {

constexpr int kGramTotal = 64 * 64 + 128 * 128 + 256 * 256 + 512 * 512 + 512 * 512;  // 610304
constexpr int kMomentTotal = 64 + 128 + 256 + 512 + 512;                               // 1472
constexpr int kStyleC[kNStyle] = {64, 128, 256, 512, 512};
constexpr long long kDefaultWorkspace = 48LL << 30;

std::mutex g_err_mu;
std::string g_err;

void set_global_err(const std::string &m) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = m;
}

long long gram_offset(int s) {
  long long o = 0;
  for (int i = 0; i < s; i++) o += (long long)kStyleC[i] * kStyleC[i];
  return o;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int moment_offset(int s) {
  int o = 0;
  for (int i = 0; i < s; i++) o += kStyleC[i];
  return o;
}

// ---- block partition ---------------------------------------------------------------------------
// Interior boundaries on multiples of 16. Border blocks have no margin on their image side, so
// they get `margin` more inner pixels than interior blocks whenever the image is large enough:
// all extended blocks then have about the same size (less padding when they share one buffer).
int round16(double t) { return 16 * (int)std::floor(t / 16.0 + 0.5); }

bool plan_1d(int L, int k, int margin, std::vector<int> &b) {
  b.assign(k + 1, 0);
  b[k] = L;
  if (k < 1) return false;
  const double a = (double)(L - 2 * margin) / k;
  const bool balanced = k >= 2 && a >= 16.0;
  for (int i = 1; i < k; i++)
    b[i] = balanced ? round16(a + margin + (i - 1) * a) : round16((double)i * L / k);
  for (int i = 0; i < k; i++)
    if (b[i + 1] <= b[i]) return false;
  return true;
}

struct Tile {
  int iy0, iy1, ix0, ix1, ey0, ey1, ex0, ex1;
};

bool make_tiles(int H, int W, int kh, int kw, int margin, std::vector<Tile> &t) {
  std::vector<int> by, bx;
  if (!plan_1d(H, kh, margin, by) || !plan_1d(W, kw, margin, bx)) return false;
  t.clear();
  for (int i = 0; i < kh; i++)
    for (int j = 0; j < kw; j++) {
      Tile r;
      r.iy0 = by[i]; r.iy1 = by[i + 1]; r.ix0 = bx[j]; r.ix1 = bx[j + 1];
      r.ey0 = std::max(0, r.iy0 - margin); r.ey1 = std::min(H, r.iy1 + margin);
      r.ex0 = std::max(0, r.ix0 - margin); r.ex1 = std::min(W, r.ix1 + margin);
      if (r.ey1 - r.ey0 < 16 || r.ex1 - r.ex0 < 16) return false;
      t.push_back(r);
    }
  return true;
}

// feature rows j (stride s) owned by inner [i0, i1): s*j in [i0, i1) and j < n_glob
void owned(int i0, int i1, int s, int n_glob, int &j0, int &j1) {
  j0 = (i0 + s - 1) / s;
  j1 = std::min((i1 + s - 1) / s, n_glob);
  if (j1 < j0) j1 = j0;
}

// own-rect slots per block: 0..4 style levels, 5 content (level 3), 6 inner pixels (level 0)
constexpr int kOwnSlots = 7;
constexpr int kOwnContent = 5, kOwnInner = 6;

// One tensor-core convolution launch's patch list: entries [off, off + n) of the plan's patch
// table, TH x TW patches.
struct PatchList {
  int off, n, TH, TW;
};
// The passes whose convolutions are restricted to what the owned pixels need (see needed_axis):
// Step-1 statistics (also the style targets), the content target, the Step-2 forward.
enum FwdKind { kFwdStats = 0, kFwdContent = 1, kFwdStep2 = 2, kFwdKinds = 3 };

struct Batch {
  int t0, B;                                  // first block index, block count
  PatchList fwd[kFwdKinds][kNConv];           // forward conv l (l >= 1) per pass kind
  PatchList bwd[kNConv];                      // input-gradient conv l (l >= 1)
  PatchList vr;                               // the V R seed of conv5_1's gradient
  PatchList unpool[kNConv];                   // pooled layer l: one pooled rectangle per block
                                              // ({y0, y1, x0, x1}; TH = largest area)
  int chunk_off[kNStyle + 1], nchunks[kNStyle + 1];  // Gram chunks per style layer; [5] content
  int tc_off[kNStyle], tc_runs[kNStyle];      // tensor-core Gram runs per style layer
  int max_inner_px, max_content_px;
  int max_inner_h, max_inner_w;
};

struct PassPlan {
  int H, W, kh, kw, margin;
  int Hb, Wb, Bmax;
  std::vector<Tile> tiles;
  std::vector<Batch> batches;
  BlockGeom *d_geom = nullptr;    // [ntiles]
  OwnRect *d_own = nullptr;       // [kOwnSlots][ntiles]
  GramChunk *d_chunks = nullptr;  // all chunks
  size_t gram_part_floats = 0;    // largest nchunks * npairs * 4096 (or tensor-core tiles)
  int max_content_chunks = 0;
  size_t chansum_doubles = 0;     // largest nchunks * C (channel-sum partials)
  // tensor-core Gram: box shape per style layer, runs, and per-block owned-rectangle maps
  int tc_TH[kNStyle], tc_TW[kNStyle];
  GramTcChunk *d_tcchunks = nullptr;
  CUtensorMap *d_maps = nullptr;   // [kNStyle][ntiles]
  const void *maps_ws = nullptr;   // workspace the maps were encoded for
  std::vector<OwnRect> own_host;   // [kOwnSlots][ntiles]
  int4 *d_patches = nullptr;       // patch table of every launch of every batch
};

struct Workspace {
  void *act[kNConv] = {};
  void *pool[kNConv] = {};
  void *g[2] = {};
};

}  // namespace

void nst::set_last_error_msg(const char *msg) { set_global_err(msg ? msg : ""); }

struct nst_ctx {
  int device = 0;
  nst_config cfg{};
  bool bf16 = true;
  bool use_tc = false;
  size_t esz = 2;
  std::string err;
  // weights
  float *d_w11 = nullptr;       // conv1_1 [64][3][3][3]
  Conv11W h_c11{};              // conv1_1 weights / bias as a kernel parameter
  float *d_bias[kNConv] = {};
  void *d_wf[kNConv] = {};      // [cout][9][cin]
  void *d_wd[kNConv] = {};      // [cin][9][cout], taps flipped
  // targets
  double *d_ghat = nullptr;
  bool have_style = false;
  void *d_ctgt = nullptr;
  size_t ctgt_cap = 0;
  int H = 0, W = 0, Hc = 0, Wc = 0;
  bool have_content = false;
  bool resident = false;   // the last evaluation kept every block's activations (one forward)
  int pass_batches = 0;    // Step-2 batches of the last evaluation
  // evaluation state
  double *d_gacc = nullptr, *d_gx = nullptr, *d_parts = nullptr, *d_loss = nullptr;
  void *d_R = nullptr;
  double *d_cpart = nullptr;
  size_t cpart_cap = 0;
  float *d_gpart = nullptr;
  // the ReLU1_1 Gram partials the conv1_1 forward writes (one 128 x 64 tile per CTA) and their
  // count for the batch's Gram reduction (0: that forward took no Gram)
  float *d_g11part = nullptr;
  int g11_runs = 0;
  size_t gpart_cap = 0;
  unsigned *d_err = nullptr;
  // mean / std terms (Eq. 5)
  bool aug = false;
  double *d_sacc = nullptr, *d_mu = nullptr, *d_sigma = nullptr, *d_cspart = nullptr;
  float *d_alpha = nullptr;
  size_t cspart_cap = 0;
  double *d_fin = nullptr;   // style finaliser scratch: beta [5][512] then partials
  // workspace (grow-only)
  void *d_ws = nullptr;
  size_t ws_cap = 0;
  // host-buffer path
  float *d_xh = nullptr, *d_gh = nullptr;
  size_t xh_cap = 0;
  // cached pass plans
  std::map<std::tuple<int, int, int, int, int>, PassPlan> plans;
  // timing
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_marks;  // (class, event index)
  double conv_flops = 0;
  long long conv_launches = 0, launches = 0;
};

namespace {

nst_status fail(nst_ctx *c, nst_status st, const std::string &m) {
  if (c) c->err = m; else set_global_err(m);
  return st;
}

nst_status cuda_fail(nst_ctx *c, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, NST_ERR_OOM, m);
  return fail(c, NST_ERR_CUDA, m);
}

#define CK(call)                                                  \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);      \
  } while (0)

// ---- timing helpers -------------------------------------------------------------------------------
enum TimeClass { kTConv = 0, kTGram = 1, kTOther = 2 };

struct Timer {
  nst_ctx *c;
  int cls;
  size_t idx;
  cudaStream_t s;
  Timer(nst_ctx *ctx, int k, cudaStream_t st) : c(ctx), cls(k), idx(0), s(st) {
    if (!c->timing) return;
    if (c->ev_used == c->ev_pool.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      c->ev_pool.push_back({a, b});
    }
    idx = c->ev_used++;
    cudaEventRecord(c->ev_pool[idx].first, s);
  }
  ~Timer() {
    if (!c->timing) return;
    cudaEventRecord(c->ev_pool[idx].second, s);
    c->ev_marks.push_back({cls, idx});
  }
};

uint16_t f2bf(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);  // inf / nan
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

float bf2f(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// ---- pass plan --------------------------------------------------------------------------------------
// Bytes of the per-layer buffer of conv l: its activation, or, for a layer followed by pooling in
// the tensor-core form, the window positions of the fused pooling (4 bits per pooled value; the
// full-resolution activation is then never stored).
size_t layer_bytes(int l, size_t px, size_t esz, bool pool_positions) {
  if (pool_positions && kPoolAfter[l]) return (px >> (2 * (kLevel[l] + 1))) * kCout[l] / 2;
  return (px >> (2 * kLevel[l])) * kCout[l] * esz;
}

size_t tile_bytes(int Hb, int Wb, size_t esz, bool pool_positions) {
  size_t px = (size_t)Hb * Wb, tot = 0;
  for (int l = 0; l < kNConv; l++) {
    tot += layer_bytes(l, px, esz, pool_positions);
    if (kPoolAfter[l]) tot += (px >> (2 * (kLevel[l] + 1))) * kCout[l] * esz;
  }
  tot += 2 * px * 64 * esz;  // two gradient buffers
  return tot;
}

// ---- needed rectangles ----------------------------------------------------------------------------
// The owned (inner) pixels of a block depend, at each layer, only on a rectangle of that layer's
// map that grows with the receptive field: Step 1 needs ReLU5_1 on the owned pixels only, and
// each earlier layer one pixel more per 3x3 convolution (twice that across a pooling); Step 2's
// backward needs dE/dReLU1_1 on the inner pixels +- 1 and one pixel more per convolution going
// deeper; its forward needs the activations where the backward reads them (ReLU masks, V of
// V R, the pooling windows, the content feature) plus the forward reach of the deeper layers.
// Each convolution therefore computes only those rectangles of each block, not the whole
// extended block: the values there are the same sums of the same inputs in the same order, so
// E and dE/dx are unchanged, bit for bit. Intervals are per axis (every step is separable),
// half-open, in global feature coordinates of their level.
struct Iv {
  int a, b;
  bool empty() const { return b <= a; }
};
Iv iv_inter(Iv p, Iv q) { return {std::max(p.a, q.a), std::min(p.b, q.b)}; }
Iv iv_union(Iv p, Iv q) {
  if (p.empty()) return q;
  if (q.empty()) return p;
  return {std::min(p.a, q.a), std::max(p.b, q.b)};
}
Iv iv_grow(Iv p, int d) { return p.empty() ? p : Iv{p.a - d, p.b + d}; }
Iv iv_pooldown(Iv p) { return p.empty() ? p : Iv{p.a >> 1, ((p.b - 1) >> 1) + 1}; }   // windows
Iv iv_poolup(Iv p) { return p.empty() ? p : Iv{2 * p.a, 2 * p.b}; }                    // pixels

struct AxisNeed {
  Iv F[kFwdKinds][kNConv];   // forward: outputs of conv l needed, per pass kind
  Iv D[kNConv];              // backward: input gradient of conv l (level of conv l)
  Iv G12;                    // backward seed: gradient of conv5_1's output
};

void needed_axis(int L, int i0, int i1, int e0, int e1, AxisNeed &n) {
  Iv val[5], own[5];
  for (int lv = 0; lv < 5; lv++) {
    val[lv] = {e0 >> lv, e1 >> lv};
    int j0, j1;
    owned(i0, i1, 1 << lv, L >> lv, j0, j1);
    own[lv] = {j0, j1};
  }
  // backward: G[l] = gradient of conv l's output, D[l] = conv l's input gradient
  Iv G[kNConv];
  G[0] = iv_inter(iv_grow(Iv{i0, i1}, 1), val[0]);
  n.D[0] = Iv{0, 0};
  for (int l = 1; l < kNConv; l++) {
    const int lv = kLevel[l];
    n.D[l] = kPoolAfter[l - 1] ? iv_inter(iv_pooldown(G[l - 1]), val[lv]) : G[l - 1];
    G[l] = iv_inter(iv_grow(n.D[l], 1), val[lv]);
  }
  n.G12 = G[kNConv - 1];
  for (int k = 0; k < kFwdKinds; k++) {
    const int last = k == kFwdContent ? kContentConv : kNConv - 1;
    for (int l = 0; l < kNConv; l++) n.F[k][l] = Iv{0, 0};
    for (int l = last; l >= 0; l--) {
      const int lv = kLevel[l];
      Iv need{0, 0};
      bool style = false;
      for (int si = 0; si < kNStyle; si++) style |= kStyleConv[si] == l;
      if (k != kFwdContent && style) need = own[lv];                  // Gram of the owned pixels
      if (k == kFwdContent && l == kContentConv) need = own[lv];      // the content target
      if (k == kFwdStep2) {
        need = iv_union(need, G[l]);                                  // masks, V R, content
        if (l == kContentConv) need = iv_union(need, own[lv]);        // content loss
        if (kPoolAfter[l] && l < last) need = iv_union(need, iv_poolup(n.D[l + 1]));  // routing
      }
      if (l < last) {   // the next convolution's input, one pixel around what it computes
        if (kPoolAfter[l])
          need = iv_union(need, iv_poolup(iv_inter(iv_grow(n.F[k][l + 1], 1), val[lv + 1])));
        else
          need = iv_union(need, iv_inter(iv_grow(n.F[k][l + 1], 1), val[lv]));
      }
      n.F[k][l] = iv_inter(need, val[lv]);
    }
  }
}

// One block's rectangle of a launch in its buffer ([0, buf) at the launch's level; the valid
// extent is [0, ext)): global interval -> block-local, and a rectangle that reaches the valid
// extent runs on to the buffer's end, so the launch also writes the zeros past the block's edge
// that the next layer reads as padding. With fused pooling (pool) the ends are even (whole
// windows) and the edge is that of the pooled map: the last whole window ends at ext & ~1 (floor
// pooling drops an odd last pixel), and the windows after it give the pooled map's zeros.
Iv local_rect(Iv g, int e0_level, int ext, int buf, bool pool) {
  if (g.empty()) return Iv{0, 0};
  Iv r{g.a - e0_level, g.b - e0_level};
  if (pool) {
    r.a &= ~1;
    r.b = (r.b + 1) & ~1;
    ext &= ~1;
  }
  if (r.b >= ext) r.b = buf;
  return iv_inter(r, Iv{0, buf});
}

nst_status build_plan(nst_ctx *ctx, int H, int W, int margin, PassPlan **out) {
  auto key = std::make_tuple(H, W, ctx->cfg.tiles_h, ctx->cfg.tiles_w, margin);
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) { *out = &it->second; return NST_OK; }
  PassPlan p;
  p.H = H; p.W = W; p.kh = ctx->cfg.tiles_h; p.kw = ctx->cfg.tiles_w; p.margin = margin;
  if (!make_tiles(H, W, p.kh, p.kw, margin, p.tiles))
    return fail(ctx, NST_ERR_SHAPE, "tile grid does not fit the image (blocks < 16 px)");
  const int nt = (int)p.tiles.size();
  int mh = 0, mw = 0;
  for (auto &t : p.tiles) { mh = std::max(mh, t.ey1 - t.ey0); mw = std::max(mw, t.ex1 - t.ex0); }
  p.Hb = (mh + 15) / 16 * 16;
  p.Wb = (mw + 15) / 16 * 16;
  long long limit = ctx->cfg.workspace_limit_bytes > 0 ? ctx->cfg.workspace_limit_bytes
                                                       : kDefaultWorkspace;
  long long per = (long long)tile_bytes(p.Hb, p.Wb, ctx->esz, ctx->use_tc);
  int B = (int)std::max(1LL, limit / std::max(per, 1LL));
  if (ctx->cfg.max_batch_tiles > 0) B = std::min(B, ctx->cfg.max_batch_tiles);
  B = std::min(B, nt);
  p.Bmax = B;
  // host metadata
  std::vector<BlockGeom> geom(nt);
  std::vector<OwnRect> own((size_t)kOwnSlots * nt);
  for (int i = 0; i < nt; i++) {
    const Tile &t = p.tiles[i];
    geom[i] = {t.ey0, t.ex0, t.ey1 - t.ey0, t.ex1 - t.ex0};
    for (int s = 0; s < kOwnSlots; s++) {
      const int lv = s < kNStyle ? s : (s == kOwnContent ? kContentLevel : 0);
      const int st = 1 << lv;
      int y0, y1, x0, x1;
      owned(t.iy0, t.iy1, st, H / st, y0, y1);
      owned(t.ix0, t.ix1, st, W / st, x0, x1);
      own[(size_t)s * nt + i] = {y0 - t.ey0 / st, y1 - t.ey0 / st, x0 - t.ex0 / st,
                                 x1 - t.ex0 / st};
    }
  }
  std::vector<GramChunk> chunks;
  std::vector<GramTcChunk> tcchunks;
  for (int t0 = 0; t0 < nt; t0 += B) {
    Batch bt{};
    bt.t0 = t0;
    bt.B = std::min(B, nt - t0);
    for (int s = 0; s <= kNStyle; s++) {
      const int slot = s < kNStyle ? s : kOwnContent;
      const int C = s < kNStyle ? kStyleC[s] : 512;
      const int nb = C / 64, npairs = nb * (nb + 1) / 2;
      long long tot = 0;
      for (int i = t0; i < t0 + bt.B; i++) {
        const OwnRect &r = own[(size_t)slot * nt + i];
        tot += (long long)(r.y1 - r.y0) * (r.x1 - r.x0);
      }
      const long long target = s < kNStyle ? std::max(1, 1216 / npairs) : 608;
      long long ch = std::max(256LL, (tot + target - 1) / target);
      ch = (ch + 31) / 32 * 32;
      bt.chunk_off[s] = (int)chunks.size();
      for (int i = t0; i < t0 + bt.B; i++) {
        const OwnRect &r = own[(size_t)slot * nt + i];
        const long long n = (long long)(r.y1 - r.y0) * (r.x1 - r.x0);
        for (long long q = 0; q < n; q += ch)
          chunks.push_back({i - t0, (int)q, (int)std::min(n, q + ch), 0});
      }
      bt.nchunks[s] = (int)chunks.size() - bt.chunk_off[s];
      if (s < kNStyle) {
        p.gram_part_floats = std::max(p.gram_part_floats, (size_t)bt.nchunks[s] * npairs * 4096);
        p.chansum_doubles = std::max(p.chansum_doubles, (size_t)bt.nchunks[s] * C);
      }
      else
        p.max_content_chunks = std::max(p.max_content_chunks, bt.nchunks[s]);
    }
    for (int si = 0; si < kNStyle; si++) {
      int N, nI, nJ;
      gram_tc_shape(kStyleC[si], &N, &nI, &nJ);
      if (t0 == 0) {
        long long h = 0, w = 0;
        for (int i = 0; i < nt; i++) {
          const OwnRect &r = own[(size_t)si * nt + i];
          h = std::max<long long>(h, r.y1 - r.y0);
          w = std::max<long long>(w, r.x1 - r.x0);
        }
        gram_tc_patch((int)h, (int)w, &p.tc_TH[si], &p.tc_TW[si]);
      }
      const int TH = p.tc_TH[si], TW = p.tc_TW[si];
      long long boxes = 0;
      for (int i = t0; i < t0 + bt.B; i++) {
        const OwnRect &r = own[(size_t)si * nt + i];
        boxes += (long long)((r.y1 - r.y0 + TH - 1) / TH) * ((r.x1 - r.x0 + TW - 1) / TW);
      }
      const long long per = std::max(2LL, (boxes * nI * nJ + 303) / 304);
      bt.tc_off[si] = (int)tcchunks.size();
      for (int i = t0; i < t0 + bt.B; i++) {
        const OwnRect &r = own[(size_t)si * nt + i];
        const int nbx = (r.x1 - r.x0 + TW - 1) / TW, nby = (r.y1 - r.y0 + TH - 1) / TH;
        const long long nb = (long long)nbx * nby;
        for (long long k = 0; k < nb; k += per)
          tcchunks.push_back({i - t0, (int)k, (int)std::min(nb, k + per), nbx});
      }
      bt.tc_runs[si] = (int)tcchunks.size() - bt.tc_off[si];
      p.gram_part_floats = std::max(p.gram_part_floats,
                                    (size_t)bt.tc_runs[si] * nI * nJ * 128 * N);
    }
    bt.max_inner_px = 0;
    bt.max_content_px = 0;
    bt.max_inner_h = bt.max_inner_w = 0;
    for (int i = t0; i < t0 + bt.B; i++) {
      const OwnRect &r = own[(size_t)kOwnInner * nt + i];
      bt.max_inner_px = std::max(bt.max_inner_px, (r.y1 - r.y0) * (r.x1 - r.x0));
      bt.max_inner_h = std::max(bt.max_inner_h, r.y1 - r.y0);
      bt.max_inner_w = std::max(bt.max_inner_w, r.x1 - r.x0);
      const OwnRect &c = own[(size_t)kOwnContent * nt + i];
      bt.max_content_px = std::max(bt.max_content_px, (c.y1 - c.y0) * (c.x1 - c.x0));
    }
    p.batches.push_back(bt);
  }
  // patch tables of the tensor-core convolutions: per batch, per launch, each block's needed
  // rectangle covered by patches of the launch's shape
  std::vector<AxisNeed> ny(nt), nx(nt);
  for (int i = 0; i < nt; i++) {
    const Tile &t = p.tiles[i];
    needed_axis(H, t.iy0, t.iy1, t.ey0, t.ey1, ny[i]);
    needed_axis(W, t.ix0, t.ix1, t.ex0, t.ex1, nx[i]);
  }
  std::vector<int4> patches;
  auto add_list = [&](const Batch &bt, int level, int cin, int cout, int taps, int k2, bool pool,
                      auto pick) -> PatchList {
    PatchList pl{(int)patches.size(), 0, 0, 0};
    int rows, fth, ftw;
    conv_tc_patch_rule(cin, cout, taps, k2, pool, &rows, &fth, &ftw);
    std::vector<Iv> ry(bt.B), rx(bt.B);
    std::vector<int> hs(bt.B), wsz(bt.B);
    for (int j = 0; j < bt.B; j++) {
      const Tile &t = p.tiles[bt.t0 + j];
      Iv gy, gx;
      pick(bt.t0 + j, gy, gx);
      ry[j] = local_rect(gy, t.ey0 >> level, (t.ey1 - t.ey0) >> level, p.Hb >> level, pool);
      rx[j] = local_rect(gx, t.ex0 >> level, (t.ex1 - t.ex0) >> level, p.Wb >> level, pool);
      hs[j] = std::max(0, ry[j].b - ry[j].a);
      wsz[j] = std::max(0, rx[j].b - rx[j].a);
    }
    conv_tc_pick_patch(hs.data(), wsz.data(), bt.B, rows, fth, ftw, pool, &pl.TH, &pl.TW);
    for (int j = 0; j < bt.B; j++)
      for (int y = ry[j].a; y < ry[j].b; y += pl.TH)
        for (int x = rx[j].a; x < rx[j].b; x += pl.TW) patches.push_back(make_int4(j, y, x, 0));
    pl.n = (int)patches.size() - pl.off;
    return pl;
  };
  for (Batch &bt : p.batches) {
    for (int k = 0; k < kFwdKinds; k++) {
      // conv1_1 (its own kernel, 16 x 8 patches)
      PatchList &c11 = bt.fwd[k][0];
      c11 = PatchList{(int)patches.size(), 0, 16, 8};
      // Passes that take the Grams (Step 1, the style targets, the resident pass): the patch
      // grid sits on multiples of 16 x 8 px of the block buffer, as do the owned rectangle's
      // edges (block bounds and margins are multiples of 16 px; at the image edge the owned
      // rectangle ends with the valid extent, past which the activation is zero), so every
      // patch is wholly owned or wholly not, and the fused ReLU1_1 Gram takes whole patches:
      // the fourth field flags the patches that meet the owned rectangle. The owned patches
      // come first, block by block in row order: the same image positions in the same order
      // under either margin, so the kernel's fixed split of them over its CTAs (and the FP32
      // order of each CTA's sum) does not depend on the pass.
      const bool gram = k != kFwdContent;
      std::vector<int4> rest;
      for (int j = 0; j < bt.B; j++) {
        const Tile &t = p.tiles[bt.t0 + j];
        const Iv ry = local_rect(ny[bt.t0 + j].F[k][0], t.ey0, t.ey1 - t.ey0, p.Hb, false);
        const Iv rx = local_rect(nx[bt.t0 + j].F[k][0], t.ex0, t.ex1 - t.ex0, p.Wb, false);
        const OwnRect &o = own[bt.t0 + j];   // style layer 0 (ReLU1_1), level 0
        const int ya = gram ? ry.a / 16 * 16 : ry.a, xa = gram ? rx.a / 8 * 8 : rx.a;
        for (int y = ya; y < ry.b; y += 16)
          for (int x = xa; x < rx.b; x += 8) {
            const bool op = gram && y < o.y1 && y + 16 > o.y0 && x < o.x1 && x + 8 > o.x0;
            (op ? patches : rest).push_back(make_int4(j, y, x, op ? 1 : 0));
          }
      }
      patches.insert(patches.end(), rest.begin(), rest.end());
      c11.n = (int)patches.size() - c11.off;
    }
    for (int k = 0; k < kFwdKinds; k++)
      for (int l = 1; l < kNConv; l++)
        bt.fwd[k][l] = add_list(bt, kLevel[l], kCin[l], kCout[l], 9, 0, kPoolAfter[l],
                                [&](int i, Iv &gy, Iv &gx) {
                                  gy = ny[i].F[k][l];
                                  gx = nx[i].F[k][l];
                                });
    for (int l = 1; l < kNConv; l++) {
      const int lp = l - 1;
      int k2 = 0;
      for (int si = 0; si < kNStyle; si++)
        if (kStyleConv[si] == lp && !kPoolAfter[lp]) k2 = kCout[lp];
      bt.bwd[l] = add_list(bt, kLevel[l], kCout[l], kCin[l], 9, k2, false,
                           [&](int i, Iv &gy, Iv &gx) {
                             gy = ny[i].D[l];
                             gx = nx[i].D[l];
                           });
    }
    bt.vr = add_list(bt, kLevel[kNConv - 1], 0, kCout[kNConv - 1], 0, kCout[kNConv - 1], false,
                     [&](int i, Iv &gy, Iv &gx) {
                       gy = ny[i].G12;
                       gx = nx[i].G12;
                     });
    // the unpool after pooled layer l routes the pooled gradient of the pooled positions that
    // the next input-gradient convolution computed (D[l + 1]), with the same edge rule
    for (int l = 0; l + 1 < kNConv; l++) {
      if (!kPoolAfter[l]) continue;
      const int lv = kLevel[l] + 1;
      PatchList &pl = bt.unpool[l];
      pl = PatchList{(int)patches.size(), bt.B, 0, 0};
      for (int j = 0; j < bt.B; j++) {
        const Tile &t = p.tiles[bt.t0 + j];
        const Iv ry = local_rect(ny[bt.t0 + j].D[l + 1], t.ey0 >> lv, (t.ey1 - t.ey0) >> lv,
                                 p.Hb >> lv, false);
        const Iv rx = local_rect(nx[bt.t0 + j].D[l + 1], t.ex0 >> lv, (t.ex1 - t.ex0) >> lv,
                                 p.Wb >> lv, false);
        patches.push_back(make_int4(ry.a, std::max(ry.a, ry.b), rx.a, std::max(rx.a, rx.b)));
        pl.TH = std::max(pl.TH, std::max(0, ry.b - ry.a) * std::max(0, rx.b - rx.a));
      }
    }
  }
  // device copies (one-time per geometry; synchronous so host arrays may be dropped)
  CK(cudaMalloc(&p.d_patches, sizeof(int4) * std::max<size_t>(1, patches.size())));
  if (!patches.empty())
    CK(cudaMemcpy(p.d_patches, patches.data(), sizeof(int4) * patches.size(),
                  cudaMemcpyHostToDevice));
  CK(cudaMalloc(&p.d_geom, sizeof(BlockGeom) * nt));
  CK(cudaMalloc(&p.d_own, sizeof(OwnRect) * own.size()));
  CK(cudaMalloc(&p.d_chunks, sizeof(GramChunk) * std::max<size_t>(1, chunks.size())));
  CK(cudaMemcpy(p.d_geom, geom.data(), sizeof(BlockGeom) * nt, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p.d_own, own.data(), sizeof(OwnRect) * own.size(), cudaMemcpyHostToDevice));
  if (!chunks.empty())
    CK(cudaMemcpy(p.d_chunks, chunks.data(), sizeof(GramChunk) * chunks.size(),
                  cudaMemcpyHostToDevice));
  CK(cudaMalloc(&p.d_tcchunks, sizeof(GramTcChunk) * std::max<size_t>(1, tcchunks.size())));
  if (!tcchunks.empty())
    CK(cudaMemcpy(p.d_tcchunks, tcchunks.data(), sizeof(GramTcChunk) * tcchunks.size(),
                  cudaMemcpyHostToDevice));
  CK(cudaMalloc(&p.d_maps, sizeof(CUtensorMap) * kNStyle * nt));
  p.own_host = own;
  auto res = ctx->plans.emplace(key, std::move(p));
  *out = &res.first->second;
  return NST_OK;
}

nst_status ensure_buffers(nst_ctx *ctx, const PassPlan &p, Workspace &ws) {
  const size_t per = tile_bytes(p.Hb, p.Wb, ctx->esz, ctx->use_tc);
  const size_t need = per * p.Bmax + 64 * 256;
  if (need > ctx->ws_cap) {
    if (ctx->d_ws) CK(cudaFree(ctx->d_ws));
    ctx->d_ws = nullptr;
    ctx->ws_cap = 0;
    CK(cudaMalloc(&ctx->d_ws, need));
    ctx->ws_cap = need;
  }
  char *q = (char *)ctx->d_ws;
  const size_t px = (size_t)p.Bmax * p.Hb * p.Wb;
  for (int l = 0; l < kNConv; l++) {
    ws.act[l] = q;
    q += align256(layer_bytes(l, px, ctx->esz, ctx->use_tc));
    ws.pool[l] = nullptr;
    if (kPoolAfter[l]) {
      ws.pool[l] = q;
      q += align256((px >> (2 * (kLevel[l] + 1))) * kCout[l] * ctx->esz);
    }
  }
  for (int i = 0; i < 2; i++) {
    ws.g[i] = q;
    q += align256(px * 64 * ctx->esz);
  }
  if (p.gram_part_floats > ctx->gpart_cap) {
    if (ctx->d_gpart) CK(cudaFree(ctx->d_gpart));
    ctx->d_gpart = nullptr;
    CK(cudaMalloc(&ctx->d_gpart, p.gram_part_floats * sizeof(float)));
    ctx->gpart_cap = p.gram_part_floats;
  }
  if (p.chansum_doubles > ctx->cspart_cap) {
    if (ctx->d_cspart) CK(cudaFree(ctx->d_cspart));
    ctx->d_cspart = nullptr;
    CK(cudaMalloc(&ctx->d_cspart, sizeof(double) * p.chansum_doubles));
    ctx->cspart_cap = p.chansum_doubles;
  }
  if ((size_t)p.max_content_chunks > ctx->cpart_cap) {
    if (ctx->d_cpart) CK(cudaFree(ctx->d_cpart));
    ctx->d_cpart = nullptr;
    CK(cudaMalloc(&ctx->d_cpart, sizeof(double) * p.max_content_chunks));
    ctx->cpart_cap = p.max_content_chunks;
  }
  return NST_OK;
}

// ---- convolution dispatch -----------------------------------------------------------------------
// the tensor-core engine computes only the launch's patch list (the CUDA-core engine ignores it
// and computes whole blocks, with the same values where the list's patches lie)
void use_patches(ConvArgs &a, const PassPlan &p, const PatchList &pl) {
  a.tiles = p.d_patches + pl.off;
  a.n_mtiles = pl.n;
  a.TH = pl.TH;
  a.TW = pl.TW;
}

nst_status run_conv(nst_ctx *ctx, ConvArgs a, cudaStream_t s) {
  a.err = ctx->d_err;
  ctx->launches++;
  ctx->conv_launches++;
  const double px = ctx->use_tc && a.tiles ? (double)a.n_mtiles * a.TH * a.TW
                                           : (double)a.B * a.Hb * a.Wb;
  ctx->conv_flops += 2.0 * px * a.cout * ((double)a.taps * a.cin + a.k2);
  Timer tm(ctx, kTConv, s);
  if (ctx->use_tc) {
    cudaError_t e = launch_conv_tc(a, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tcgen05 convolution launch");
  } else if (ctx->bf16) {
    launch_conv_simt<__nv_bfloat16>(a, s);
  } else {
    launch_conv_simt<float>(a, s);
  }
  return NST_OK;
}

template <typename T>
nst_status forward_batch(nst_ctx *ctx, const PassPlan &p, const Batch &bt, const Workspace &ws,
                         const float *img, int last_conv, bool for_backward, cudaStream_t s,
                         bool grams = false) {
  const BlockGeom *geom = p.d_geom + bt.t0;
  ctx->g11_runs = 0;
  // grams: gram_batch follows; on the tensor cores the conv1_1 forward also takes the ReLU1_1
  // Gram of its owned patches (partials reduced there)
  const bool fuse_g11 = grams && ctx->use_tc;
  if (fuse_g11 && !ctx->d_g11part)
    CK(cudaMalloc(&ctx->d_g11part, (size_t)2 * tc_num_sms() * 128 * 64 * sizeof(float)));
  {
    Timer tm(ctx, kTOther, s);
    ctx->launches += ctx->use_tc ? 2 : 1;   // tensor-core form: staging + convolution
    if (ctx->use_tc) {
      // the staged BF16-pair image goes to the (not yet used) second gradient buffer
      const PatchList &pl = bt.fwd[last_conv == kContentConv ? kFwdContent
                                  : (for_backward ? kFwdStep2 : kFwdStats)][0];
      cudaError_t e = launch_conv11_fwd_tc(img, p.H, p.W, ctx->d_w11, ctx->d_bias[0], geom, bt.B,
                                           p.Hb, p.Wb, ws.g[1], (__nv_bfloat16 *)ws.act[0],
                                           p.d_patches + pl.off, pl.n,
                                           fuse_g11 ? ctx->d_g11part : nullptr, &ctx->g11_runs,
                                           ctx->d_err, s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "conv1_1 tensor-core forward launch");
    } else {
      launch_conv11_fwd<T>(img, p.H, p.W, ctx->h_c11, geom, bt.B, p.Hb, p.Wb, (T *)ws.act[0], s);
    }
  }
  const int kind = last_conv == kContentConv ? kFwdContent
                                             : (for_backward ? kFwdStep2 : kFwdStats);
  for (int l = 1; l <= last_conv; l++) {
    const int lv = kLevel[l];
    ConvArgs a{};
    a.B = bt.B; a.Hb = p.Hb >> lv; a.Wb = p.Wb >> lv;
    a.cin = kCin[l]; a.cout = kCout[l]; a.taps = 9; a.k2 = 0;
    use_patches(a, p, bt.fwd[kind][l]);
    a.A = kPoolAfter[l - 1] ? ws.pool[l - 1] : ws.act[l - 1];
    a.Wt = ctx->d_wf[l];
    a.out = ws.act[l];
    a.mode = kEpiForward;
    a.bias = ctx->d_bias[l];
    a.geom = geom;
    a.level = lv;
    // the tensor-core epilogue writes the pooled map and, when a backward pass follows, the
    // window position of each pooled value (the backward's routing) in place of the activation
    const bool fuse_pool = ctx->use_tc && kPoolAfter[l];
    if (fuse_pool) {
      if (l >= last_conv) return fail(ctx, NST_ERR_STATE, "pass ends at a pooled layer");
      a.pool_out = ws.pool[l];
      a.out = nullptr;
      a.pool_idx = for_backward ? (unsigned char *)ws.act[l] : nullptr;
    }
    nst_status st = run_conv(ctx, a, s);
    if (st) return st;
    if (kPoolAfter[l] && l < last_conv && !fuse_pool) {
      Timer tm(ctx, kTOther, s);
      ctx->launches++;
      launch_pool<T>((const T *)ws.act[l], (T *)ws.pool[l], bt.B, p.Hb >> (lv + 1),
                     p.Wb >> (lv + 1), kCout[l], geom, lv + 1, s);
    }
  }
  return NST_OK;
}

// per-block owned-rectangle tensor maps of the style layers, for the current workspace
nst_status ensure_gram_maps(nst_ctx *ctx, PassPlan &p, const Workspace &ws) {
  if (p.maps_ws == ctx->d_ws) return NST_OK;
  const int nt = (int)p.tiles.size();
  std::vector<CUtensorMap> maps((size_t)kNStyle * nt);
  for (const Batch &bt : p.batches)
    for (int si = 0; si < kNStyle; si++) {
      const int l = kStyleConv[si], lv = kLevel[l], C = kCout[l];
      const long long Hl = p.Hb >> lv, Wl = p.Wb >> lv;
      for (int i = bt.t0; i < bt.t0 + bt.B; i++) {
        const OwnRect &r = p.own_host[(size_t)si * nt + i];
        const char *base = (const char *)ws.act[l] +
                           ((((long long)(i - bt.t0) * Hl + r.y0) * Wl + r.x0) * C) * 2;
        cudaError_t e = encode_gram_map(&maps[(size_t)si * nt + i], base, C, r.x1 - r.x0,
                                        r.y1 - r.y0, Wl, p.tc_TH[si], p.tc_TW[si]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "Gram tensor map");
      }
    }
  CK(cudaMemcpy(p.d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                cudaMemcpyHostToDevice));
  p.maps_ws = ctx->d_ws;
  return NST_OK;
}

template <typename T>
nst_status gram_batch(nst_ctx *ctx, PassPlan &p, const Batch &bt, const Workspace &ws,
                      cudaStream_t s, bool moments) {
  const int nt = (int)p.tiles.size();
  if (moments)
    for (int si = 0; si < kNStyle; si++) {
      const int l = kStyleConv[si], lv = kLevel[l];
      Timer tm(ctx, kTGram, s);
      ctx->launches += 2;
      launch_chansum<T>((const T *)ws.act[l], p.Hb >> lv, p.Wb >> lv, kCout[l],
                        p.d_own + (size_t)si * nt + bt.t0, p.d_chunks + bt.chunk_off[si],
                        bt.nchunks[si], ctx->d_cspart, ctx->d_sacc + moment_offset(si), s);
    }
  if (ctx->use_tc) {
    nst_status st = ensure_gram_maps(ctx, p, ws);
    if (st) return st;
  }
  for (int si = 0; si < kNStyle; si++) {
    const int l = kStyleConv[si], lv = kLevel[l];
    Timer tm(ctx, kTGram, s);
    ctx->launches += 2;
    if (ctx->use_tc && si == 0 && ctx->g11_runs > 0) {
      // ReLU1_1: the conv1_1 forward took the Gram of its owned patches; reduce its partials
      cudaError_t e = launch_gram_tc_reduce(ctx->d_g11part, ctx->g11_runs, 64, 64, 1, 1,
                                            ctx->d_gacc + gram_offset(0), s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "ReLU1_1 Gram reduction launch");
      continue;
    }
    if (ctx->use_tc) {
      GramTcArgs a{};
      a.maps = p.d_maps + (size_t)si * nt + bt.t0;
      a.chunks = p.d_tcchunks + bt.tc_off[si];
      a.C = kCout[l];
      gram_tc_shape(a.C, &a.N, &a.nI, &a.nJ);
      a.TH = p.tc_TH[si];
      a.TW = p.tc_TW[si];
      a.part = ctx->d_gpart;
      a.err = ctx->d_err;
      cudaError_t e = launch_gram_tc(a, bt.tc_runs[si], ctx->d_gacc + gram_offset(si), s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core Gram launch");
      continue;
    }
    if (bt.nchunks[si] == 0) continue;
    launch_gram_partial<T>((const T *)ws.act[l], p.Hb >> lv, p.Wb >> lv, kCout[l],
                           p.d_own + (size_t)si * nt + bt.t0, p.d_chunks + bt.chunk_off[si],
                           bt.nchunks[si], ctx->d_gpart, s);
    launch_gram_reduce(ctx->d_gpart, bt.nchunks[si], kCout[l], ctx->d_gacc + gram_offset(si), s);
  }
  return NST_OK;
}

template <typename T>
nst_status backward_batch(nst_ctx *ctx, const PassPlan &p, const Batch &bt, const Workspace &ws,
                          float *grad, cudaStream_t s) {
  const int nt = (int)p.tiles.size();
  const BlockGeom *geom = p.d_geom + bt.t0;
  const size_t Rbase[kNStyle] = {(size_t)gram_offset(0), (size_t)gram_offset(1),
                                 (size_t)gram_offset(2), (size_t)gram_offset(3),
                                 (size_t)gram_offset(4)};
  auto Rptr = [&](int si) { return (const char *)ctx->d_R + Rbase[si] * ctx->esz; };
  int cur = 0;
  // dE/d pre-activation of conv5_1 = [ReLU5_1 > 0] * (V R_5)   (Table 1 row 2 at ReLU5_1)
  {
    const int l = 12, lv = kLevel[l];
    ConvArgs a{};
    a.B = bt.B; a.Hb = p.Hb >> lv; a.Wb = p.Wb >> lv;
    a.cin = 0; a.cout = kCout[l]; a.taps = 0;
    a.k2 = kCout[l]; a.A2 = ws.act[l]; a.W2 = Rptr(4);
    if (ctx->aug) a.addvec = ctx->d_alpha + moment_offset(4);
    a.out = ws.g[cur];
    a.mode = kEpiBackward;
    a.mask = ws.act[l];
    a.geom = geom;
    a.level = lv;
    use_patches(a, p, bt.vr);
    nst_status st = run_conv(ctx, a, s);
    if (st) return st;
  }
  for (int l = 12; l >= 1; l--) {
    const int lv = kLevel[l];
    const int lp = l - 1;
    ConvArgs a{};
    a.B = bt.B; a.Hb = p.Hb >> lv; a.Wb = p.Wb >> lv;
    a.cin = kCout[l]; a.cout = kCin[l]; a.taps = 9;
    a.A = ws.g[cur]; a.Wt = ctx->d_wd[l];
    a.out = ws.g[1 - cur];
    a.mode = kEpiBackward;
    a.geom = geom;
    a.level = lv;
    use_patches(a, p, bt.bwd[l]);
    if (!kPoolAfter[lp]) {
      a.mask = ws.act[lp];
      for (int si = 0; si < kNStyle; si++)
        if (kStyleConv[si] == lp) {
          a.k2 = kCout[lp];
          a.A2 = ws.act[lp];
          a.W2 = Rptr(si);
          if (ctx->aug) a.addvec = ctx->d_alpha + moment_offset(si);
        }
      if (lp == kContentConv) {
        a.cact = ws.act[lp];
        a.ctgt = ctx->d_ctgt;
        a.Hc = ctx->Hc;
        a.Wc = ctx->Wc;
        a.two_lambda = 2.f * ctx->cfg.lambda_c;
      }
    }
    nst_status st = run_conv(ctx, a, s);
    if (st) return st;
    if (kPoolAfter[lp]) {
      Timer tm(ctx, kTOther, s);
      ctx->launches++;
      if (ctx->use_tc)
        launch_unpool_idx((const __nv_bfloat16 *)ws.g[1 - cur], (const unsigned char *)ws.act[lp],
                          (__nv_bfloat16 *)ws.g[cur], bt.B, p.Hb >> lv, p.Wb >> lv, kCout[lp],
                          geom, lv, p.d_patches + bt.unpool[lp].off, bt.unpool[lp].TH, s);
      else
        launch_unpool<T>((const T *)ws.g[1 - cur], (const T *)ws.act[lp], (T *)ws.g[cur], bt.B,
                         p.Hb >> lv, p.Wb >> lv, kCout[lp], geom, lv, s);
    } else {
      cur = 1 - cur;
    }
  }
  {
    Timer tm(ctx, kTOther, s);
    ctx->launches++;
    const OwnRect *inner = p.d_own + (size_t)kOwnInner * nt + bt.t0;
    if (ctx->use_tc) {
      cudaError_t e = launch_conv11_dgrad_tc((const __nv_bfloat16 *)ws.g[cur], ctx->d_w11, geom,
                                             inner, bt.B, p.Hb, p.Wb, bt.max_inner_h,
                                             bt.max_inner_w, grad, p.H, p.W, ctx->d_err, s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "conv1_1 tensor-core input-gradient launch");
    } else {
      launch_conv11_dgrad_scatter<T>((const T *)ws.g[cur], ctx->d_w11, geom, inner, bt.B, p.Hb,
                                     p.Wb, grad, p.H, p.W, bt.max_inner_px, s);
    }
  }
  return NST_OK;
}

enum PassKind { kPassStyleStats, kPassContentTarget };

template <typename T>
nst_status stats_pass(nst_ctx *ctx, const float *img, int H, int W, PassKind kind,
                      cudaStream_t s, bool moments = false) {
  PassPlan *p = nullptr;
  nst_status st = build_plan(ctx, H, W, ctx->cfg.margin1, &p);
  if (st) return st;
  Workspace ws;
  st = ensure_buffers(ctx, *p, ws);
  if (st) return st;
  const int nt = (int)p->tiles.size();
  for (const Batch &bt : p->batches) {
    const int last = kind == kPassContentTarget ? kContentConv : kNConv - 1;
    st = forward_batch<T>(ctx, *p, bt, ws, img, last, false, s, kind == kPassStyleStats);
    if (st) return st;
    if (kind == kPassStyleStats) {
      st = gram_batch<T>(ctx, *p, bt, ws, s, moments);
      if (st) return st;
    } else {
      ctx->launches++;
      launch_crop_content<T>((const T *)ws.act[kContentConv], bt.B, p->Hb >> kContentLevel,
                             p->Wb >> kContentLevel, p->d_geom + bt.t0,
                             p->d_own + (size_t)kOwnContent * nt + bt.t0, (T *)ctx->d_ctgt,
                             ctx->Hc, ctx->Wc, bt.max_content_px, s);
    }
  }
  return NST_OK;
}

template <typename T>
nst_status loss_grad_impl(nst_ctx *ctx, const float *x, float *grad, double *loss,
                          cudaStream_t s) {
  const int H = ctx->H, W = ctx->W;
  ctx->launches++;
  launch_check_finite(x, 3LL * H * W, ctx->d_err, s);
  // Step 1: global statistics of x
  CK(cudaMemsetAsync(ctx->d_gacc, 0, sizeof(double) * kGramTotal, s));
  if (ctx->aug) CK(cudaMemsetAsync(ctx->d_sacc, 0, sizeof(double) * kMomentTotal, s));
  PassPlan *p = nullptr;
  nst_status st = build_plan(ctx, H, W, ctx->cfg.margin2, &p);
  if (st) return st;
  Workspace ws;
  st = ensure_buffers(ctx, *p, ws);
  if (st) return st;
  // Resident mode: when every block with the Step-2 margin fits in the workspace at once, one
  // forward pass of all blocks serves both steps. The statistics come from the owned pixels of
  // those blocks (exact, as the Step-2 margin exceeds Step 1's), and Step 2 back-propagates
  // through the activations already in HBM instead of recomputing them.
  const bool resident = p->batches.size() == 1 && ctx->cfg.schedule != NST_SCHED_TWO_PASS;
  ctx->resident = resident;
  ctx->pass_batches = (int)p->batches.size();
  if (resident) {
    const Batch &bt = p->batches[0];
    st = forward_batch<T>(ctx, *p, bt, ws, x, kNConv - 1, true, s, true);
    if (st) return st;
    st = gram_batch<T>(ctx, *p, bt, ws, s, ctx->aug);
    if (st) return st;
  } else {
    st = stats_pass<T>(ctx, x, H, W, kPassStyleStats, s, ctx->aug);
    if (st) return st;
    st = ensure_buffers(ctx, *p, ws);   // the Step-1 plan may have moved the workspace
    if (st) return st;
  }
  StyleFinalizeArgs fa{};
  for (int si = 0; si < kNStyle; si++) {
    const int stv = 1 << si;
    fa.L[si].Gacc = ctx->d_gacc + gram_offset(si);
    fa.L[si].Ghat = ctx->d_ghat + gram_offset(si);
    fa.L[si].Gout = ctx->d_gx + gram_offset(si);
    fa.L[si].R = (char *)ctx->d_R + gram_offset(si) * ctx->esz;
    fa.L[si].C = kStyleC[si];
    fa.L[si].np = (double)(H / stv) * (double)(W / stv);
    fa.L[si].w = ctx->cfg.w_style[si];
    if (ctx->aug) {
      const int mo = moment_offset(si);
      fa.L[si].S = ctx->d_sacc + mo;
      fa.L[si].mu = ctx->d_mu + mo;
      fa.L[si].sigma = ctx->d_sigma + mo;
      fa.L[si].wm = ctx->cfg.w_mean[si];
      fa.L[si].ws = ctx->cfg.w_std[si];
      fa.L[si].alpha = ctx->d_alpha + mo;
    }
  }
  fa.Eparts = ctx->d_parts;
  fa.r_is_bf16 = ctx->bf16 ? 1 : 0;
  fa.beta = ctx->d_fin;
  fa.partial = ctx->d_fin + kNStyle * 512;
  ctx->launches += 3;   // moments, residuals, sums
  launch_style_finalize(fa, s);
  // Step 2: loss and gradient block by block
  CK(cudaMemsetAsync(ctx->d_parts + kNStyle, 0, sizeof(double), s));
  const int nt = (int)p->tiles.size();
  for (const Batch &bt : p->batches) {
    if (!resident) {
      st = forward_batch<T>(ctx, *p, bt, ws, x, kNConv - 1, true, s);
      if (st) return st;
    }
    {
      Timer tm(ctx, kTOther, s);
      ctx->launches += 2;
      launch_content_loss<T>((const T *)ws.act[kContentConv], p->Hb >> kContentLevel,
                             p->Wb >> kContentLevel, (const T *)ctx->d_ctgt, ctx->Hc, ctx->Wc,
                             p->d_geom + bt.t0, p->d_own + (size_t)kOwnContent * nt + bt.t0,
                             p->d_chunks + bt.chunk_off[kNStyle], bt.nchunks[kNStyle],
                             ctx->d_cpart, (double)ctx->cfg.lambda_c, ctx->d_parts + kNStyle, s);
    }
    st = backward_batch<T>(ctx, *p, bt, ws, grad, s);
    if (st) return st;
  }
  ctx->launches++;
  launch_finish_loss(ctx->d_parts, loss ? loss : ctx->d_loss, s);
  CK(cudaGetLastError());
  return NST_OK;
}

nst_status check_img(nst_ctx *ctx, const void *p, int H, int W) {
  if (!ctx) return fail(nullptr, NST_ERR_INVALID_ARG, "null context");
  if (!p) return fail(ctx, NST_ERR_INVALID_ARG, "null image pointer");
  if (H < 16 || W < 16) return fail(ctx, NST_ERR_SHAPE, "image smaller than 16 x 16");
  return NST_OK;
}

void reset_counters(nst_ctx *ctx) {
  ctx->ev_used = 0;
  ctx->ev_marks.clear();
  ctx->conv_flops = 0;
  ctx->conv_launches = 0;
  ctx->launches = 0;
}

}  // namespace

// =================================================================================================
// C ABI
// =================================================================================================
extern "C" {

const char *nst_version(void) { return "libnst 0.1 (sm_103a)"; }

const char *nst_last_error(nst_ctx *ctx) {
  if (ctx) return ctx->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  static thread_local std::string copy;
  copy = g_err;
  return copy.c_str();
}

nst_status nst_config_default(nst_config *cfg) {
  if (!cfg) return fail(nullptr, NST_ERR_INVALID_ARG, "null config");
  std::memset(cfg, 0, sizeof(*cfg));
  for (int i = 0; i < 5; i++) cfg->w_style[i] = 0.2f;
  cfg->lambda_c = 1e-3f;
  cfg->tiles_h = cfg->tiles_w = 1;
  cfg->margin1 = 80;
  cfg->margin2 = 160;
  cfg->precision = NST_PREC_BF16;
  cfg->conv_engine = NST_CONV_AUTO;
  cfg->max_batch_tiles = 0;
  cfg->workspace_limit_bytes = 0;
  return NST_OK;
}

nst_status nst_tile_plan(int H, int W, int tiles_h, int tiles_w, int margin, int *rects_out) {
  if (!rects_out || tiles_h < 1 || tiles_w < 1 || margin < 0 || margin % 16)
    return fail(nullptr, NST_ERR_INVALID_ARG, "bad tile-plan arguments");
  std::vector<Tile> t;
  if (!make_tiles(H, W, tiles_h, tiles_w, margin, t))
    return fail(nullptr, NST_ERR_SHAPE, "tile grid does not fit the image");
  for (size_t i = 0; i < t.size(); i++) {
    int *r = rects_out + 8 * i;
    r[0] = t[i].iy0; r[1] = t[i].iy1; r[2] = t[i].ix0; r[3] = t[i].ix1;
    r[4] = t[i].ey0; r[5] = t[i].ey1; r[6] = t[i].ex0; r[7] = t[i].ex1;
  }
  return NST_OK;
}

nst_status nst_create(nst_ctx **out, const float *params, long long n_params,
                      const nst_config *cfg) {
  if (!out || !params || !cfg) return fail(nullptr, NST_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  long long expect = 0;
  for (int l = 0; l < kNConv; l++) expect += (long long)kCout[l] * kCin[l] * 9 + kCout[l];
  if (n_params != expect) return fail(nullptr, NST_ERR_INVALID_ARG, "n_params mismatch");
  if (cfg->tiles_h < 1 || cfg->tiles_w < 1 || cfg->margin1 < 0 || cfg->margin2 < 0 ||
      cfg->margin1 % 16 || cfg->margin2 % 16 ||
      (cfg->precision != NST_PREC_FP32 && cfg->precision != NST_PREC_BF16) ||
      cfg->conv_engine < 0 || cfg->conv_engine > 2 || cfg->max_batch_tiles < 0 ||
      cfg->schedule < 0 || cfg->schedule > 1)
    return fail(nullptr, NST_ERR_INVALID_ARG, "invalid configuration");
  if (cfg->conv_engine == NST_CONV_TC && cfg->precision != NST_PREC_BF16)
    return fail(nullptr, NST_ERR_INVALID_ARG, "the tensor-core engine needs BF16 precision");
  nst_ctx *ctx = new nst_ctx();
  ctx->cfg = *cfg;
  ctx->bf16 = cfg->precision == NST_PREC_BF16;
  ctx->esz = ctx->bf16 ? 2 : 4;
  ctx->use_tc = ctx->bf16 && cfg->conv_engine != NST_CONV_SIMT;
  auto bad = [&](nst_status st) { nst_destroy(ctx); return st; };
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) { cuda_fail(nullptr, e, "cudaGetDevice"); return bad(NST_ERR_CUDA); }
  if (ctx->use_tc && !tc_available()) {
    fail(nullptr, NST_ERR_CUDA, "tcgen05 engine unavailable on this device");
    return bad(NST_ERR_CUDA);
  }
  // weights
  std::vector<uint16_t> hb;
  std::vector<float> hf;
  const float *p = params;
  for (int l = 0; l < kNConv; l++) {
    const int ci = kCin[l], co = kCout[l];
    const float *Wl = p;
    const float *bl = p + (size_t)co * ci * 9;
    p = bl + co;
    if (cudaMalloc(&ctx->d_bias[l], sizeof(float) * co) != cudaSuccess) return bad(NST_ERR_OOM);
    cudaMemcpy(ctx->d_bias[l], bl, sizeof(float) * co, cudaMemcpyHostToDevice);
    if (l == 0) {
      // the BF16 form holds every weight, conv1_1's included, as a BF16 value (kept here as the
      // float it converts to exactly); the FP32 form keeps them as given
      std::vector<float> w1(Wl, Wl + (size_t)co * ci * 9);
      if (ctx->bf16)
        for (float &w : w1) w = bf2f(f2bf(w));
      for (int o = 0; o < co; o++) {
        for (int k = 0; k < 27; k++) ctx->h_c11.w[k][o] = w1[(size_t)o * 27 + k];
        ctx->h_c11.b[o] = bl[o];
      }
      if (cudaMalloc(&ctx->d_w11, sizeof(float) * co * ci * 9) != cudaSuccess)
        return bad(NST_ERR_OOM);
      cudaMemcpy(ctx->d_w11, w1.data(), sizeof(float) * co * ci * 9, cudaMemcpyHostToDevice);
      continue;
    }
    const size_t n = (size_t)co * ci * 9;
    for (int dir = 0; dir < 2; dir++) {
      hf.assign(n, 0.f);
      for (int o = 0; o < co; o++)
        for (int i = 0; i < ci; i++)
          for (int t = 0; t < 9; t++) {
            const float w = Wl[((size_t)o * ci + i) * 9 + t];
            if (dir == 0)
              hf[((size_t)o * 9 + t) * ci + i] = w;  // [cout][tap][cin]
            else
              hf[((size_t)i * 9 + (8 - t)) * co + o] = w;  // [cin][flipped tap][cout]
          }
      void **dst = dir == 0 ? &ctx->d_wf[l] : &ctx->d_wd[l];
      if (cudaMalloc(dst, n * ctx->esz) != cudaSuccess) return bad(NST_ERR_OOM);
      if (ctx->bf16) {
        hb.resize(n);
        for (size_t k = 0; k < n; k++) hb[k] = f2bf(hf[k]);
        cudaMemcpy(*dst, hb.data(), n * 2, cudaMemcpyHostToDevice);
      } else {
        cudaMemcpy(*dst, hf.data(), n * 4, cudaMemcpyHostToDevice);
      }
    }
  }
  if (cudaMalloc(&ctx->d_ghat, sizeof(double) * kGramTotal) != cudaSuccess ||
      cudaMalloc(&ctx->d_gacc, sizeof(double) * kGramTotal) != cudaSuccess ||
      cudaMalloc(&ctx->d_gx, sizeof(double) * kGramTotal) != cudaSuccess ||
      cudaMalloc(&ctx->d_R, ctx->esz * kGramTotal) != cudaSuccess ||
      cudaMalloc(&ctx->d_parts, sizeof(double) * 8) != cudaSuccess ||
      cudaMalloc(&ctx->d_loss, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_err, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&ctx->d_sacc, sizeof(double) * kMomentTotal) != cudaSuccess ||
      cudaMalloc(&ctx->d_mu, sizeof(double) * kMomentTotal) != cudaSuccess ||
      cudaMalloc(&ctx->d_sigma, sizeof(double) * kMomentTotal) != cudaSuccess ||
      cudaMalloc(&ctx->d_alpha, sizeof(float) * kMomentTotal) != cudaSuccess ||
      cudaMalloc(&ctx->d_fin, sizeof(double) * (kNStyle * 512 + kNStyle * kFinalizeChunks)) !=
          cudaSuccess)
    return bad(NST_ERR_OOM);
  for (int i = 0; i < 5; i++) ctx->aug |= cfg->w_mean[i] != 0.f || cfg->w_std[i] != 0.f;
  cudaMemset(ctx->d_err, 0, sizeof(unsigned));
  cudaMemset(ctx->d_parts, 0, sizeof(double) * 8);
  cudaMemset(ctx->d_gx, 0, sizeof(double) * kGramTotal);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { cuda_fail(nullptr, e, "nst_create"); return bad(NST_ERR_CUDA); }
  *out = ctx;
  return NST_OK;
}

nst_status nst_destroy(nst_ctx *ctx) {
  if (!ctx) return NST_OK;
  cudaDeviceSynchronize();
  cudaFree(ctx->d_w11);
  for (int l = 0; l < kNConv; l++) {
    cudaFree(ctx->d_bias[l]);
    cudaFree(ctx->d_wf[l]);
    cudaFree(ctx->d_wd[l]);
  }
  cudaFree(ctx->d_ghat); cudaFree(ctx->d_ctgt); cudaFree(ctx->d_gacc); cudaFree(ctx->d_gx);
  cudaFree(ctx->d_R); cudaFree(ctx->d_parts); cudaFree(ctx->d_loss); cudaFree(ctx->d_cpart);
  cudaFree(ctx->d_gpart); cudaFree(ctx->d_g11part); cudaFree(ctx->d_err); cudaFree(ctx->d_ws);
  cudaFree(ctx->d_xh); cudaFree(ctx->d_gh);
  cudaFree(ctx->d_sacc); cudaFree(ctx->d_mu); cudaFree(ctx->d_sigma); cudaFree(ctx->d_alpha);
  cudaFree(ctx->d_cspart);
  cudaFree(ctx->d_fin);
  for (auto &kv : ctx->plans) {
    cudaFree(kv.second.d_geom);
    cudaFree(kv.second.d_own);
    cudaFree(kv.second.d_chunks);
    cudaFree(kv.second.d_tcchunks);
    cudaFree(kv.second.d_maps);
    cudaFree(kv.second.d_patches);
  }
  for (auto &ev : ctx->ev_pool) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
  delete ctx;
  return NST_OK;
}

nst_status nst_style_targets(nst_ctx *ctx, const float *v, int Hv, int Wv, void *stream) {
  nst_status st = check_img(ctx, v, Hv, Wv);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(ctx->d_gacc, 0, sizeof(double) * kGramTotal, s));
  CK(cudaMemsetAsync(ctx->d_sacc, 0, sizeof(double) * kMomentTotal, s));
  st = ctx->bf16 ? stats_pass<__nv_bfloat16>(ctx, v, Hv, Wv, kPassStyleStats, s, true)
                 : stats_pass<float>(ctx, v, Hv, Wv, kPassStyleStats, s, true);
  if (st) return st;
  // G^L(v) = sum / n_p: the finaliser with w = 0 against a zero reference
  StyleFinalizeArgs fa{};
  CK(cudaMemsetAsync(ctx->d_gx, 0, sizeof(double) * kGramTotal, s));
  for (int si = 0; si < kNStyle; si++) {
    const int stv = 1 << si;
    fa.L[si].Gacc = ctx->d_gacc + gram_offset(si);
    fa.L[si].Ghat = ctx->d_gx + gram_offset(si);  // zero reference
    fa.L[si].Gout = ctx->d_ghat + gram_offset(si);
    fa.L[si].R = (char *)ctx->d_R + gram_offset(si) * ctx->esz;
    fa.L[si].C = kStyleC[si];
    fa.L[si].np = (double)(Hv / stv) * (double)(Wv / stv);
    fa.L[si].w = 0.0;
    const int mo = moment_offset(si);
    fa.L[si].S = ctx->d_sacc + mo;
    fa.L[si].mean_out = ctx->d_mu + mo;
    fa.L[si].std_out = ctx->d_sigma + mo;
  }
  fa.Eparts = ctx->d_parts;
  fa.r_is_bf16 = ctx->bf16 ? 1 : 0;
  fa.beta = ctx->d_fin;
  fa.partial = ctx->d_fin + kNStyle * 512;
  launch_style_finalize(fa, s);
  CK(cudaGetLastError());
  ctx->have_style = true;
  return NST_OK;
}

nst_status nst_content_targets(nst_ctx *ctx, const float *u, int H, int W, void *stream) {
  nst_status st = check_img(ctx, u, H, W);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int Hc = H / 8, Wc = W / 8;
  const size_t need = (size_t)Hc * Wc * 512 * ctx->esz;
  if (need > ctx->ctgt_cap) {
    if (ctx->d_ctgt) CK(cudaFree(ctx->d_ctgt));
    ctx->d_ctgt = nullptr;
    ctx->ctgt_cap = 0;
    CK(cudaMalloc(&ctx->d_ctgt, need));
    ctx->ctgt_cap = need;
  }
  ctx->H = H; ctx->W = W; ctx->Hc = Hc; ctx->Wc = Wc;
  CK(cudaMemsetAsync(ctx->d_ctgt, 0, need, s));
  st = ctx->bf16 ? stats_pass<__nv_bfloat16>(ctx, u, H, W, kPassContentTarget, s)
                 : stats_pass<float>(ctx, u, H, W, kPassContentTarget, s);
  if (st) return st;
  CK(cudaGetLastError());
  ctx->have_content = true;
  return NST_OK;
}

nst_status nst_loss_grad(nst_ctx *ctx, const float *x, int H, int W, float *grad, double *loss,
                         void *stream) {
  nst_status st = check_img(ctx, x, H, W);
  if (st) return st;
  if (!grad) return fail(ctx, NST_ERR_INVALID_ARG, "null gradient pointer");
  if (!ctx->have_style || !ctx->have_content)
    return fail(ctx, NST_ERR_STATE, "style and content targets must be set first");
  if (H != ctx->H || W != ctx->W)
    return fail(ctx, NST_ERR_SHAPE, "image size differs from the content target's");
  cudaStream_t s = (cudaStream_t)stream;
  return ctx->bf16 ? loss_grad_impl<__nv_bfloat16>(ctx, x, grad, loss, s)
                   : loss_grad_impl<float>(ctx, x, grad, loss, s);
}

nst_status nst_loss_grad_host(nst_ctx *ctx, const float *xh, int H, int W, float *gh,
                              double *lossh, void *stream) {
  nst_status st = check_img(ctx, xh, H, W);
  if (st) return st;
  if (!gh) return fail(ctx, NST_ERR_INVALID_ARG, "null gradient pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = 3ULL * H * W;
  if (n > ctx->xh_cap) {
    cudaFree(ctx->d_xh);
    cudaFree(ctx->d_gh);
    ctx->d_xh = ctx->d_gh = nullptr;
    ctx->xh_cap = 0;
    CK(cudaMalloc(&ctx->d_xh, n * sizeof(float)));
    CK(cudaMalloc(&ctx->d_gh, n * sizeof(float)));
    ctx->xh_cap = n;
  }
  // A page-locked gradient buffer is device-accessible: the last kernel of the evaluation (the
  // conv1_1 input gradient, one store per owned pixel) writes it over the host link itself, in
  // place of a separate device-to-host copy after it. (Copy engine and kernel stores move the
  // same bytes per second over this link; the kernel's own work then hides under its writes.)
  // Other buffers go through the device copy.
  float *gdst = ctx->d_gh;
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, gh) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeHost && pa.devicePointer) gdst = (float *)pa.devicePointer;
  } else {
    cudaGetLastError();   // the query's own error (an unknown pointer), not a pending one
  }
  CK(cudaMemcpyAsync(ctx->d_xh, xh, n * sizeof(float), cudaMemcpyHostToDevice, s));
  st = nst_loss_grad(ctx, ctx->d_xh, H, W, gdst, ctx->d_loss, stream);
  if (st) return st;
  if (gdst == ctx->d_gh)
    CK(cudaMemcpyAsync(gh, ctx->d_gh, n * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (lossh) CK(cudaMemcpyAsync(lossh, ctx->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return NST_OK;
}

nst_status nst_set_schedule(nst_ctx *ctx, int schedule) {
  if (!ctx) return fail(nullptr, NST_ERR_INVALID_ARG, "null context");
  if (schedule < 0 || schedule > 1) return fail(ctx, NST_ERR_INVALID_ARG, "unknown schedule");
  ctx->cfg.schedule = schedule;
  return NST_OK;
}

nst_status nst_pass_info(nst_ctx *ctx, int *batches, int *resident) {
  if (!ctx) return fail(nullptr, NST_ERR_INVALID_ARG, "null context");
  if (batches) *batches = ctx->pass_batches;
  if (resident) *resident = ctx->resident ? 1 : 0;
  return NST_OK;
}

nst_status nst_get_stats(nst_ctx *ctx, double *parts, double *grams, void *stream) {
  if (!ctx || !parts) return fail(ctx, NST_ERR_INVALID_ARG, "null argument");
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CK(cudaMemcpy(parts, ctx->d_parts, sizeof(double) * 6, cudaMemcpyDeviceToHost));
  if (grams) CK(cudaMemcpy(grams, ctx->d_gx, sizeof(double) * kGramTotal, cudaMemcpyDeviceToHost));
  return NST_OK;
}

nst_status nst_get_style_grams(nst_ctx *ctx, double *grams, void *stream) {
  if (!ctx || !grams) return fail(ctx, NST_ERR_INVALID_ARG, "null argument");
  if (!ctx->have_style) return fail(ctx, NST_ERR_STATE, "no style targets");
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CK(cudaMemcpy(grams, ctx->d_ghat, sizeof(double) * kGramTotal, cudaMemcpyDeviceToHost));
  return NST_OK;
}

nst_status nst_get_style_moments(nst_ctx *ctx, double *mean, double *sd, void *stream) {
  if (!ctx || !mean || !sd) return fail(ctx, NST_ERR_INVALID_ARG, "null argument");
  if (!ctx->have_style) return fail(ctx, NST_ERR_STATE, "no style targets");
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CK(cudaMemcpy(mean, ctx->d_mu, sizeof(double) * kMomentTotal, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(sd, ctx->d_sigma, sizeof(double) * kMomentTotal, cudaMemcpyDeviceToHost));
  return NST_OK;
}

nst_status nst_set_timing(nst_ctx *ctx, int enable) {
  if (!ctx) return fail(nullptr, NST_ERR_INVALID_ARG, "null context");
  if (ctx->timing) {
    cudaError_t e = cudaDeviceSynchronize();  // pending events must complete before reuse
    if (e != cudaSuccess) return cuda_fail(ctx, e, "nst_set_timing");
  }
  ctx->timing = enable != 0;
  reset_counters(ctx);
  return NST_OK;
}

nst_status nst_get_timing(nst_ctx *ctx, double *out, void *stream) {
  if (!ctx || !out) return fail(ctx, NST_ERR_INVALID_ARG, "null argument");
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  double ms[3] = {0, 0, 0};
  for (auto &m : ctx->ev_marks) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ctx->ev_pool[m.second].first, ctx->ev_pool[m.second].second) ==
        cudaSuccess)
      ms[m.first] += t;
  }
  out[0] = ms[kTConv];
  out[1] = ctx->conv_flops;
  out[2] = ms[kTGram];
  out[3] = ms[kTOther];
  out[4] = (double)ctx->conv_launches;
  out[5] = (double)ctx->launches;
  return NST_OK;
}

nst_status nst_sync_status(nst_ctx *ctx, void *stream) {
  if (!ctx) return fail(nullptr, NST_ERR_INVALID_ARG, "null context");
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned e = 0;
  CK(cudaMemcpy(&e, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  CK(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
  if (e & kErrTimeout) return fail(ctx, NST_ERR_TIMEOUT, "a device-side wait ran out");
  if (e & kErrNonfinite) return fail(ctx, NST_ERR_NONFINITE, "non-finite value in x");
  return NST_OK;
}

nst_status nst_check_timeout_path(nst_ctx *ctx, long long limit_cycles, void *stream) {
  if (!ctx) return fail(nullptr, NST_ERR_INVALID_ARG, "null context");
  if (limit_cycles < 1 || limit_cycles > 4000000000LL)
    return fail(ctx, NST_ERR_INVALID_ARG, "limit out of range");
  cudaError_t e = launch_timeout_check(limit_cycles, ctx->d_err, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "timeout check launch");
  return NST_OK;
}

nst_status nst_conv3x3(int dtype, int engine, int B, int H, int W, int cin, int cout, int taps,
                       const void *in, const void *w, int k2, const void *in2, const void *w2,
                       const float *bias, int mode, const void *mask, const int *geom, void *out,
                       void *stream) {
  nst_ctx *ctx = nullptr;
  if ((dtype != NST_PREC_FP32 && dtype != NST_PREC_BF16) ||
      (engine != NST_CONV_SIMT && engine != NST_CONV_TC) || (taps != 0 && taps != 9) || B < 1 ||
      H < 1 || W < 1 || cout < 1 || cout % 64 || k2 < 0 || (taps && (!in || !w || cin < 16)) ||
      (k2 && (!in2 || !w2)) || (!taps && !k2) || !geom || !out || (mode != 0 && mode != 1) ||
      (mode == 0 && !bias))
    return fail(nullptr, NST_ERR_INVALID_ARG, "bad convolution arguments");
  if (engine == NST_CONV_TC && (dtype != NST_PREC_BF16 || (taps && cin % 64) || k2 % 64))
    return fail(nullptr, NST_ERR_INVALID_ARG, "tensor-core engine: BF16, channels % 64");
  if (engine == NST_CONV_SIMT && ((taps && cin % 16) || k2 % 16))
    return fail(nullptr, NST_ERR_INVALID_ARG, "CUDA-core engine: channels % 16");
  ConvArgs a{};
  a.B = B; a.Hb = H; a.Wb = W;
  a.cin = taps ? cin : 0; a.cout = cout; a.taps = taps;
  a.k2 = k2; a.A = in; a.Wt = w; a.A2 = in2; a.W2 = w2;
  a.out = out;
  a.mode = mode;
  a.bias = bias;
  a.mask = mask;
  a.geom = reinterpret_cast<const BlockGeom *>(geom);
  a.level = 0;
  a.err = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (engine == NST_CONV_TC)
    e = launch_conv_tc(a, s);
  else if (dtype == NST_PREC_BF16)
    launch_conv_simt<__nv_bfloat16>(a, s);
  else
    launch_conv_simt<float>(a, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "nst_conv3x3");
  return NST_OK;
}

nst_status nst_gram(int dtype, const void *V, long long npix, int C, double *G, void *stream) {
  nst_ctx *ctx = nullptr;
  if ((dtype != NST_PREC_FP32 && dtype != NST_PREC_BF16) || !V || !G || C < 64 || C > 512 ||
      C % 64 || npix < 1 || npix >= (1LL << 31))
    return fail(nullptr, NST_ERR_INVALID_ARG, "bad Gram arguments");
  cudaStream_t s = (cudaStream_t)stream;
  long long chunk_len;
  int nchunks;
  gram_flat_plan(npix, C, &chunk_len, &nchunks);
  const int nb = C / 64, npairs = nb * (nb + 1) / 2;
  float *part = nullptr;
  CK(cudaMallocAsync((void **)&part, (size_t)nchunks * npairs * 4096 * sizeof(float), s));
  CK(cudaMemsetAsync(G, 0, sizeof(double) * C * C, s));
  if (dtype == NST_PREC_BF16)
    launch_gram_partial_flat<__nv_bfloat16>((const __nv_bfloat16 *)V, npix, C, chunk_len, nchunks,
                                            part, s);
  else
    launch_gram_partial_flat<float>((const float *)V, npix, C, chunk_len, nchunks, part, s);
  launch_gram_reduce(part, nchunks, C, G, s);
  CK(cudaFreeAsync(part, s));
  CK(cudaGetLastError());
  return NST_OK;
}

}  // extern "C"


