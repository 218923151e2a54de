/*
 * nst_oracle.c -- FP64 CPU oracle for the localized style-transfer loss and its image gradient
 * (Galerne et al., "Scaling Painting Style Transfer", Sections 3-4, Table 1, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
 * load this file. The library under test never calls it and shares no code with it.
 *
 * Everything is the plain definition, written out in double precision, with no blocking, fusion
 * or reordering beyond what the definition states:
 *   - VGG-19 features up to ReLU5_1 (Section 3.1): 13 convolutions 3x3 (zero padding 1, stride 1)
 *     each followed by a ReLU, and a 2x2 stride-2 max pool after conv1_2, conv2_2, conv3_4 and
 *     conv4_4.
 *   - Gram matrices G^L = V^T V / n_p (Section 3.1, Eq. 4), Gram style loss (Eq. 3), content loss
 *     and transfer loss (Eq. 1-2).
 *   - Feature gradients of Table 1 (rows 1-4) and a hand-written reverse pass (ReLU mask, max-pool
 *     routing, transposed 3x3 convolution) back to the image.
 *   - The augmented style loss of Eq. 5 (Section 3.2): Gram term plus w'_L ||mean - mu||^2 and
 *     w''_L ||std - sigma||^2, with std = (diag(G) - mean^2)^(1/2) (Algorithm 1, Step 1),
 *     population statistics over the n_p feature pixels; a channel with std = 0 is constant, so
 *     its std-term gradient (V - mean) * (...) / std is 0 (taken as 0, not 0/0).
 *   - Algorithm 1 (two passes over blocks extracted with a margin), literally, for the exactness
 *     and margin tests.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - style/content features are the post-ReLU outputs ReLU_k_1 and ReLU_4_2;
 *   - pooling is max pooling, 2x2 stride 2, floor mode (a trailing odd row/column is dropped);
 *   - ties in a pooling window go to the first maximum in row-major window order (strict '>');
 *   - the ReLU derivative at 0 is 0 (mask = pre-activation > 0, i.e. post-activation > 0);
 *   - the image enters the network as is (RGB in [0,1], no mean subtraction);
 *   - n_p^L is the feature-pixel count of the whole image, floor(H/s) * floor(W/s), s = 2^pools;
 *   - a feature pixel j of stride s belongs to the block whose inner rectangle holds image pixel
 *     (s*j_y, s*j_x); the content loss of Step 2 sums over those owned pixels only.
 *
 * Storage precision (orc_set_storage): the network's gradient is discontinuous where a ReLU input
 * or a pooling window's top two values meet, so a ReLU mask or pooling argmax decided in one
 * precision cannot be compared with one decided in another. In mode 1 (float32) or 2 (bfloat16)
 * the oracle rounds, round-to-nearest-even, every value the evaluated form stores: the image as
 * it enters conv1_1 (bfloat16 mode only: a hi + lo pair of bfloat16 numbers), the weights of
 * all thirteen convolutions (bfloat16 mode only), every post-ReLU activation, the style residuals
 * R_L = 4 w_L (G - G_ref) / n_p, and every masked feature gradient before it enters the next
 * transposed convolution; the reverse pass stays the exact adjoint of the rounded forward values.
 * Mode 0 (the default) is the plain FP64 definition.
 *
 * Layout: images and activations are planar C x H x W (channel-major) doubles. Parameters are one
 * flat array: for conv l = 0..12, W_l[Cout][Cin][3][3] followed by b_l[Cout].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NCONV 13
#define NSTYLE 5

static const int kCin[NCONV] = {3, 64, 64, 128, 128, 256, 256, 256, 256, 512, 512, 512, 512};
static const int kCout[NCONV] = {64, 64, 128, 128, 256, 256, 256, 256, 512, 512, 512, 512, 512};
/* a max pool follows conv1_2, conv2_2, conv3_4 and conv4_4 */
static const int kPoolAfter[NCONV] = {0, 1, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0};
/* style layers ReLU1_1, ReLU2_1, ReLU3_1, ReLU4_1, ReLU5_1 (Section 3.1) as conv indices */
static const int kStyleConv[NSTYLE] = {0, 2, 4, 8, 12};
static const int kStyleStride[NSTYLE] = {1, 2, 4, 8, 16};
/* content layer ReLU4_2 */
#define CONTENT_CONV 9
#define CONTENT_STRIDE 8

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_SHAPE = 2, ORC_ERR_OOM = 3 };

static int g_storage = 0; /* 0: float64 (exact), 1: float32, 2: bfloat16 */

void orc_set_storage(int mode) { g_storage = (mode >= 0 && mode <= 2) ? mode : 0; }

/* round to the storage type (via float32, as a float32 value is what gets narrowed) */
static double q(double v) {
  if (g_storage == 0) return v;
  float f = (float)v;
  if (g_storage == 1) return (double)f;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}
static void q_array(double *a, long n) {
  if (g_storage)
    for (long i = 0; i < n; i++) a[i] = q(a[i]);
}
/* the bfloat16 form stores the weights of every convolution in bfloat16 */
static double qw(double w, int layer) {
  (void)layer;
  return g_storage == 2 ? q(w) : w;
}

/* the bfloat16 form reads the image as a pair of bfloat16 numbers: hi = bf16(v), lo = bf16(v - hi);
 * the pair carries v to within 2^-17 |v| */
static double q_pair(double v) {
  const double hi = q(v);
  return hi + q(v - hi);
}

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }

/* ------------------------------------------------------------------------------------------- */
/* parameters                                                                                   */

long orc_param_count(void) {
  long n = 0;
  for (int l = 0; l < NCONV; l++) n += (long)kCout[l] * kCin[l] * 9 + kCout[l];
  return n;
}

static void param_ptrs(const double *params, const double **W, const double **b) {
  const double *p = params;
  for (int l = 0; l < NCONV; l++) {
    W[l] = p;
    p += (long)kCout[l] * kCin[l] * 9;
    b[l] = p;
    p += kCout[l];
  }
}

/* ------------------------------------------------------------------------------------------- */
/* layers                                                                                       */

/* out[co][y][x] = b[co] + sum_{ci,ky,kx} W[co][ci][ky][kx] * in[ci][y+ky-1][x+kx-1],
 * with in = 0 outside [0,h) x [0,w) (zero padding 1, stride 1). */
static void conv3x3_forward(const double *in, int cin, int h, int w, const double *W,
                            const double *b, int cout, double *out, int layer) {
  long hw = (long)h * w;
  double *in_pair = NULL;
  if (layer == 0 && g_storage == 2) {
    in_pair = (double *)malloc(sizeof(double) * (size_t)cin * hw + 8);
    if (in_pair) {
      for (long i = 0; i < cin * hw; i++) in_pair[i] = q_pair(in[i]);
      in = in_pair;
    }
  }
#pragma omp parallel for schedule(static)
  for (int co = 0; co < cout; co++) {
    double *o = out + co * hw;
    for (long i = 0; i < hw; i++) o[i] = b[co];
    for (int ci = 0; ci < cin; ci++) {
      const double *src = in + ci * hw;
      for (int ky = 0; ky < 3; ky++)
        for (int kx = 0; kx < 3; kx++) {
          double wt = qw(W[((long)co * cin + ci) * 9 + ky * 3 + kx], layer);
          int dy = ky - 1, dx = kx - 1;
          int y0 = imax(0, -dy), y1 = imin(h, h - dy);
          int x0 = imax(0, -dx), x1 = imin(w, w - dx);
          for (int y = y0; y < y1; y++) {
            const double *srow = src + (long)(y + dy) * w + dx;
            double *orow = o + (long)y * w;
            for (int x = x0; x < x1; x++) orow[x] += wt * srow[x];
          }
        }
    }
  }
  free(in_pair);
}

/* Adjoint of conv3x3_forward with respect to its input:
 * din[ci][y][x] = sum_{co,ky,kx} W[co][ci][ky][kx] * dout[co][y-ky+1][x-kx+1] (valid terms). */
static void conv3x3_backward_data(const double *dout, int cout, int h, int w, const double *W,
                                  int cin, double *din, int layer) {
  long hw = (long)h * w;
#pragma omp parallel for schedule(static)
  for (int ci = 0; ci < cin; ci++) {
    double *d = din + ci * hw;
    for (long i = 0; i < hw; i++) d[i] = 0.0;
    for (int co = 0; co < cout; co++) {
      const double *g = dout + co * hw;
      for (int ky = 0; ky < 3; ky++)
        for (int kx = 0; kx < 3; kx++) {
          double wt = qw(W[((long)co * cin + ci) * 9 + ky * 3 + kx], layer);
          int dy = 1 - ky, dx = 1 - kx; /* y' = y + dy */
          int y0 = imax(0, -dy), y1 = imin(h, h - dy);
          int x0 = imax(0, -dx), x1 = imin(w, w - dx);
          for (int y = y0; y < y1; y++) {
            const double *grow = g + (long)(y + dy) * w + dx;
            double *drow = d + (long)y * w;
            for (int x = x0; x < x1; x++) drow[x] += wt * grow[x];
          }
        }
    }
  }
}

static void relu_inplace(double *a, long n) {
  for (long i = 0; i < n; i++)
    if (!(a[i] > 0.0)) a[i] = 0.0;
}

/* index (0..3) of the first maximum of a 2x2 window in row-major order, strict '>' */
static int window_argmax(const double *a, int w, int y, int x) {
  const double v0 = a[(long)(2 * y) * w + 2 * x], v1 = a[(long)(2 * y) * w + 2 * x + 1];
  const double v2 = a[(long)(2 * y + 1) * w + 2 * x], v3 = a[(long)(2 * y + 1) * w + 2 * x + 1];
  int k = 0;
  double m = v0;
  if (v1 > m) { m = v1; k = 1; }
  if (v2 > m) { m = v2; k = 2; }
  if (v3 > m) { m = v3; k = 3; }
  return k;
}

/* 2x2 stride-2 max pool, floor mode: out is c x (h/2) x (w/2) */
static void maxpool_forward(const double *in, int c, int h, int w, double *out) {
  int ph = h / 2, pw = w / 2;
  for (int ch = 0; ch < c; ch++) {
    const double *a = in + (long)ch * h * w;
    double *o = out + (long)ch * ph * pw;
    for (int y = 0; y < ph; y++)
      for (int x = 0; x < pw; x++) {
        int k = window_argmax(a, w, y, x);
        o[(long)y * pw + x] = a[(long)(2 * y + k / 2) * w + 2 * x + k % 2];
      }
  }
}

/* adjoint of maxpool_forward: the pooled gradient goes to the window's argmax */
static void maxpool_backward(const double *gout, const double *in, int c, int h, int w,
                             double *gin) {
  int ph = h / 2, pw = w / 2;
  memset(gin, 0, sizeof(double) * (size_t)c * h * w);
  for (int ch = 0; ch < c; ch++) {
    const double *a = in + (long)ch * h * w;
    const double *g = gout + (long)ch * ph * pw;
    double *d = gin + (long)ch * h * w;
    for (int y = 0; y < ph; y++)
      for (int x = 0; x < pw; x++) {
        int k = window_argmax(a, w, y, x);
        d[(long)(2 * y + k / 2) * w + 2 * x + k % 2] += g[(long)y * pw + x];
      }
  }
}

/* ------------------------------------------------------------------------------------------- */
/* the network                                                                                  */

typedef struct {
  int h[NCONV], w[NCONV];   /* spatial size of conv l (input = output size) */
  double *a[NCONV];         /* post-ReLU output of conv l */
  double *p[NCONV];         /* pooled output after conv l (kPoolAfter[l]) */
} acts_t;

static void acts_free(acts_t *A) {
  for (int l = 0; l < NCONV; l++) {
    free(A->a[l]);
    free(A->p[l]);
    A->a[l] = A->p[l] = NULL;
  }
}

static int acts_alloc(acts_t *A, int H, int W) {
  memset(A, 0, sizeof(*A));
  int h = H, w = W;
  for (int l = 0; l < NCONV; l++) {
    A->h[l] = h;
    A->w[l] = w;
    A->a[l] = (double *)malloc(sizeof(double) * (size_t)kCout[l] * h * w + 8);
    if (!A->a[l]) { acts_free(A); return ORC_ERR_OOM; }
    if (kPoolAfter[l]) {
      h /= 2;
      w /= 2;
      A->p[l] = (double *)malloc(sizeof(double) * (size_t)kCout[l] * h * w + 8);
      if (!A->p[l]) { acts_free(A); return ORC_ERR_OOM; }
    }
  }
  return ORC_OK;
}

/* VGG-19 forward to ReLU5_1 on an image of 3 x H x W; keeps every activation */
static void vgg_forward(const double *params, const double *img, acts_t *A) {
  const double *W[NCONV], *b[NCONV];
  param_ptrs(params, W, b);
  const double *in = img;
  for (int l = 0; l < NCONV; l++) {
    int h = A->h[l], w = A->w[l];
    conv3x3_forward(in, kCin[l], h, w, W[l], b[l], kCout[l], A->a[l], l);
    relu_inplace(A->a[l], (long)kCout[l] * h * w);
    q_array(A->a[l], (long)kCout[l] * h * w);
    in = A->a[l];
    if (kPoolAfter[l]) {
      maxpool_forward(A->a[l], kCout[l], h, w, A->p[l]);
      in = A->p[l];
    }
  }
}

/* Reverse pass: feat_grad[l] (may be NULL) is dE/d(post-ReLU output of conv l); returns dE/dimg.
 * Each step is the adjoint of one forward step, taken in reverse order. */
static int vgg_backward(const double *params, const acts_t *A, double *const *feat_grad,
                        double *dimg) {
  const double *W[NCONV], *b[NCONV];
  param_ptrs(params, W, b);
  long maxn = 0;
  for (int l = 0; l < NCONV; l++) {
    long n = (long)kCout[l] * A->h[l] * A->w[l];
    if (n > maxn) maxn = n;
  }
  double *g = (double *)calloc((size_t)maxn + 8, sizeof(double));   /* dE/d a[l] */
  double *t = (double *)calloc((size_t)maxn + 8, sizeof(double));   /* scratch */
  if (!g || !t) { free(g); free(t); return ORC_ERR_OOM; }
  /* start at conv5_1: nothing consumes its output except the style loss */
  int l = NCONV - 1;
  long n = (long)kCout[l] * A->h[l] * A->w[l];
  for (long i = 0; i < n; i++) g[i] = feat_grad[l] ? feat_grad[l][i] : 0.0;
  for (;;) {
    int h = A->h[l], w = A->w[l];
    n = (long)kCout[l] * h * w;
    /* ReLU: gradient passes where the output is positive */
    for (long i = 0; i < n; i++)
      if (!(A->a[l][i] > 0.0)) g[i] = 0.0;
    q_array(g, n);
    /* conv l: gradient with respect to its input */
    double *din = (l == 0) ? dimg : t;
    conv3x3_backward_data(g, kCout[l], h, w, W[l], kCin[l], din, l);
    if (l == 0) break;
    int lp = l - 1;   /* producer of conv l's input */
    long np = (long)kCout[lp] * A->h[lp] * A->w[lp];
    if (kPoolAfter[lp]) {
      q_array(t, (long)kCout[lp] * A->h[l] * A->w[l]);
      maxpool_backward(t, A->a[lp], kCout[lp], A->h[lp], A->w[lp], g);
    } else {
      memcpy(g, t, sizeof(double) * (size_t)np);
    }
    if (feat_grad[lp])
      for (long i = 0; i < np; i++) g[i] += feat_grad[lp][i];
    l = lp;
  }
  free(g);
  free(t);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------- */
/* statistics and feature losses (Section 3.1, Table 1)                                         */

/* S[i][j] = sum over the listed pixels of V[i][p] V[j][p]; V is c x (h*w), pixels restricted
 * to rows [y0,y1) and columns [x0,x1) of the h x w map */
static void gram_sum_rect(const double *V, int c, int h, int w, int y0, int y1, int x0, int x1,
                          double *S) {
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < c; i++)
    for (int j = i; j < c; j++) {
      double s = 0.0;
      for (int y = y0; y < y1; y++)
        for (int x = x0; x < x1; x++) {
          long p = (long)y * w + x;
          s += V[(long)i * h * w + p] * V[(long)j * h * w + p];
        }
      S[(long)i * c + j] = s;
      S[(long)j * c + i] = s;
    }
}

/* Table 1, row 2: E = w ||G - Gref||_F^2 and dE/dV = w (4/np) V (G - Gref) (V is np x nc there;
 * here V is nc x npix and the gradient is written in the same layout). */
static double gram_loss_grad_ab(const double *V, int c, long npix, double np, const double *G,
                                const double *Gref, double w, const double *beta,
                                const double *alpha, double *gV) {
  double E = 0.0;
  for (long k = 0; k < (long)c * c; k++) {
    double d = G[k] - Gref[k];
    E += d * d;
  }
  E *= w;
  if (gV) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < c; j++) {
      double *gj = gV + (long)j * npix;
      const double aj = alpha ? (g_storage ? (double)(float)alpha[j] : alpha[j]) : 0.0;
      for (long p = 0; p < npix; p++) gj[p] = aj;
      for (int i = 0; i < c; i++) {
        double rij = (G[(long)i * c + j] - Gref[(long)i * c + j]) * (4.0 * w / np);
        if (beta && i == j) rij += beta[j];
        const double dij = q(rij);
        const double *vi = V + (long)i * npix;
        for (long p = 0; p < npix; p++) gj[p] += vi[p] * dij;
      }
    }
  }
  return E;
}

static double gram_loss_grad(const double *V, int c, long npix, double np, const double *G,
                             const double *Gref, double w, double *gV) {
  return gram_loss_grad_ab(V, c, npix, np, G, Gref, w, NULL, NULL, gV);
}

/* Mean and std terms of Eq. 5 from the layer statistics: mean_j = S_j / n_p (S = channel sums),
 * std_j = (G_jj - mean_j^2)^(1/2) (Algorithm 1, Step 1). Returns w' |mean - mu|^2 +
 * w'' |std - sigma|^2 and the per-channel affine feature gradient of Table 1 rows 3-4:
 * dE/dV_kj = alpha_j + beta_j V_kj with beta_j = w'' (2/n_p)(std_j - sigma_j)/std_j and
 * alpha_j = w' (2/n_p)(mean_j - mu_j) - beta_j mean_j (beta_j = 0 when std_j = 0). */
static double moment_terms(int c, double np, const double *G, const double *mean,
                           const double *mu, const double *sigma, double wm, double ws,
                           double *std_out, double *alpha, double *beta) {
  double E = 0.0;
  for (int j = 0; j < c; j++) {
    const double m = mean[j];
    const double var = G[(long)j * c + j] - m * m;
    const double sd = var > 0.0 ? sqrt(var) : 0.0;
    if (std_out) std_out[j] = sd;
    E += wm * (m - mu[j]) * (m - mu[j]) + ws * (sd - sigma[j]) * (sd - sigma[j]);
    const double b = sd > 0.0 ? ws * 2.0 / np * (sd - sigma[j]) / sd : 0.0;
    if (beta) beta[j] = b;
    if (alpha) alpha[j] = wm * 2.0 / np * (m - mu[j]) - b * m;
  }
  return E;
}

/* Standalone Table 1 rows for the feature-level tests. V is np x nc, row-major (the paper's
 * layout). Gram: G = V^T V / np. */
void orc_table1_gram(const double *V, int np, int nc, const double *Gref, double w, double *E,
                     double *gV) {
  double *G = (double *)calloc((size_t)nc * nc, sizeof(double));
  for (int i = 0; i < nc; i++)
    for (int j = 0; j < nc; j++) {
      double s = 0.0;
      for (int k = 0; k < np; k++) s += V[(long)k * nc + i] * V[(long)k * nc + j];
      G[(long)i * nc + j] = s / np;
    }
  double e = 0.0;
  for (long k = 0; k < (long)nc * nc; k++) e += (G[k] - Gref[k]) * (G[k] - Gref[k]);
  *E = w * e;
  for (int k = 0; k < np; k++)
    for (int j = 0; j < nc; j++) {
      double s = 0.0;
      for (int i = 0; i < nc; i++) s += V[(long)k * nc + i] * (G[(long)i * nc + j] - Gref[(long)i * nc + j]);
      gV[(long)k * nc + j] = w * 4.0 / np * s;
    }
  free(G);
}

/* Table 1, row 1: E = lambda ||V - Vref||^2, dE/dV = 2 lambda (V - Vref) */
void orc_table1_mse(const double *V, const double *Vref, long n, double lambda, double *E,
                    double *gV) {
  double e = 0.0;
  for (long i = 0; i < n; i++) {
    double d = V[i] - Vref[i];
    e += d * d;
    gV[i] = 2.0 * lambda * d;
  }
  *E = lambda * e;
}

/* Table 1, row 3: E = w ||mean(V) - mu||^2, (dE/dV)_k = w (2/np) (mean(V) - mu) for every row k.
 * V is np x nc row-major. */
void orc_table1_mean(const double *V, int np, int nc, const double *mu, double w, double *E,
                     double *gV) {
  double e = 0.0;
  for (int j = 0; j < nc; j++) {
    double m = 0.0;
    for (int k = 0; k < np; k++) m += V[(long)k * nc + j];
    m /= np;
    e += (m - mu[j]) * (m - mu[j]);
    for (int k = 0; k < np; k++) gV[(long)k * nc + j] = w * 2.0 / np * (m - mu[j]);
  }
  *E = w * e;
}

/* Table 1, row 4: E = w ||std(V) - sigma||^2 (population std),
 * (dE/dV)_kj = w (2/np) (V_kj - mean_j) (std_j - sigma_j) / std_j. */
void orc_table1_std(const double *V, int np, int nc, const double *sigma, double w, double *E,
                    double *gV) {
  double e = 0.0;
  for (int j = 0; j < nc; j++) {
    double m = 0.0, m2 = 0.0;
    for (int k = 0; k < np; k++) {
      m += V[(long)k * nc + j];
      m2 += V[(long)k * nc + j] * V[(long)k * nc + j];
    }
    m /= np;
    m2 /= np;
    double var = m2 - m * m;
    double sd = var > 0.0 ? sqrt(var) : 0.0;
    e += (sd - sigma[j]) * (sd - sigma[j]);
    for (int k = 0; k < np; k++)
      gV[(long)k * nc + j] =
          sd > 0.0 ? w * 2.0 / np * (V[(long)k * nc + j] - m) * (sd - sigma[j]) / sd : 0.0;
  }
  *E = w * e;
}

/* ------------------------------------------------------------------------------------------- */
/* untiled evaluation (the plain definition)                                                    */

static int check_size(int H, int W) { return (H >= 16 && W >= 16) ? ORC_OK : ORC_ERR_SHAPE; }

/* post-ReLU features of conv index `conv` (0..12) of image x (3 x H x W) */
int orc_features(const double *params, const double *x, int H, int W, int conv, double *out) {
  if (conv < 0 || conv >= NCONV) return ORC_ERR_ARG;
  if (check_size(H, W)) return ORC_ERR_SHAPE;
  acts_t A;
  if (acts_alloc(&A, H, W)) return ORC_ERR_OOM;
  vgg_forward(params, x, &A);
  memcpy(out, A.a[conv], sizeof(double) * (size_t)kCout[conv] * A.h[conv] * A.w[conv]);
  acts_free(&A);
  return ORC_OK;
}

/* style statistics G^L(v), L in L_s, concatenated (64^2 + 128^2 + 256^2 + 512^2 + 512^2) */
int orc_style_grams(const double *params, const double *v, int H, int W, double *G) {
  if (check_size(H, W)) return ORC_ERR_SHAPE;
  acts_t A;
  if (acts_alloc(&A, H, W)) return ORC_ERR_OOM;
  vgg_forward(params, v, &A);
  double *g = G;
  for (int s = 0; s < NSTYLE; s++) {
    int l = kStyleConv[s], c = kCout[l], h = A.h[l], w = A.w[l];
    gram_sum_rect(A.a[l], c, h, w, 0, h, 0, w, g);
    double np = (double)h * w;
    for (long k = 0; k < (long)c * c; k++) g[k] /= np;
    g += (long)c * c;
  }
  acts_free(&A);
  return ORC_OK;
}

/* spatial mean and std (population, std from diag(G) - mean^2) of the five style layers of v,
 * concatenated (64 + 128 + 256 + 512 + 512 = 1,472 values each) */
int orc_style_moments(const double *params, const double *v, int H, int W, double *mean_out,
                      double *std_out) {
  if (check_size(H, W)) return ORC_ERR_SHAPE;
  acts_t A;
  if (acts_alloc(&A, H, W)) return ORC_ERR_OOM;
  vgg_forward(params, v, &A);
  long o = 0;
  for (int s = 0; s < NSTYLE; s++) {
    int l = kStyleConv[s], c = kCout[l];
    long npix = (long)A.h[l] * A.w[l];
    double *G = (double *)malloc(sizeof(double) * (size_t)c * c);
    gram_sum_rect(A.a[l], c, A.h[l], A.w[l], 0, A.h[l], 0, A.w[l], G);
    for (long k = 0; k < (long)c * c; k++) G[k] /= (double)npix;
    for (int j = 0; j < c; j++) {
      double m = 0.0;
      for (long p = 0; p < npix; p++) m += A.a[l][(long)j * npix + p];
      mean_out[o + j] = m / (double)npix;
    }
    moment_terms(c, (double)npix, G, mean_out + o, mean_out + o, std_out + o, 0.0, 0.0,
                 std_out + o, NULL, NULL);
    free(G);
    o += c;
  }
  acts_free(&A);
  return ORC_OK;
}

/* content target V^{Lc}(u): 512 x floor(H/8) x floor(W/8) */
int orc_content_target(const double *params, const double *u, int H, int W, double *out) {
  return orc_features(params, u, H, W, CONTENT_CONV, out);
}

/* E(x) = lambda_c ||V^Lc(x) - V^Lc(u)||^2 + sum_L E~^L_style (Eq. 1-3, 5) and its gradient with
 * respect to x. E~^L_style = w_L ||G^L(x) - G^L(v)||_F^2 + w'_L ||mean - mu_L||^2 +
 * w''_L ||std - sigma_L||^2; w_mean / w_std may be NULL (plain Gram loss, Eq. 3), then
 * style_mean / style_std are unused. parts[0..4] = style terms per layer, parts[5] = content
 * term (may be NULL); grams_out receives G^L(x) (may be NULL); grad may be NULL (loss only). */
int orc_loss_grad_aug(const double *params, const double *x, int H, int W,
                      const double *content_t, const double *style_G, const double *style_mean,
                      const double *style_std, const double *w_style, const double *w_mean,
                      const double *w_std, double lambda_c, double *E_out, double *grad,
                      double *parts, double *grams_out) {
  if (check_size(H, W)) return ORC_ERR_SHAPE;
  acts_t A;
  if (acts_alloc(&A, H, W)) return ORC_ERR_OOM;
  vgg_forward(params, x, &A);
  double *fg[NCONV] = {0};
  double E = 0.0;
  const double *gref = style_G;
  double *gout = grams_out;
  long mo = 0;
  int rc = ORC_OK;
  const int aug = w_mean && w_std;
  for (int s = 0; s < NSTYLE; s++) {
    int l = kStyleConv[s], c = kCout[l], h = A.h[l], w = A.w[l];
    long npix = (long)h * w;
    double *G = (double *)malloc(sizeof(double) * (size_t)c * c);
    gram_sum_rect(A.a[l], c, h, w, 0, h, 0, w, G);
    for (long k = 0; k < (long)c * c; k++) G[k] /= (double)npix;
    double *alpha = NULL, *beta = NULL;
    double em = 0.0;
    if (aug) {
      double *mean = (double *)malloc(sizeof(double) * c);
      alpha = (double *)malloc(sizeof(double) * c);
      beta = (double *)malloc(sizeof(double) * c);
      for (int j = 0; j < c; j++) {
        double m = 0.0;
        for (long p = 0; p < npix; p++) m += A.a[l][(long)j * npix + p];
        mean[j] = m / (double)npix;
      }
      em = moment_terms(c, (double)npix, G, mean, style_mean + mo, style_std + mo, w_mean[s],
                        w_std[s], NULL, alpha, beta);
      free(mean);
    }
    if (grad) fg[l] = (double *)malloc(sizeof(double) * (size_t)c * npix);
    double e = gram_loss_grad_ab(A.a[l], c, npix, (double)npix, G, gref, w_style[s], beta, alpha,
                                 fg[l]) + em;
    free(alpha);
    free(beta);
    if (parts) parts[s] = e;
    E += e;
    if (gout) { memcpy(gout, G, sizeof(double) * (size_t)c * c); gout += (long)c * c; }
    free(G);
    gref += (long)c * c;
    mo += c;
  }
  {
    int l = CONTENT_CONV;
    long n = (long)kCout[l] * A.h[l] * A.w[l];
    double e = 0.0;
    if (grad) fg[l] = (double *)malloc(sizeof(double) * (size_t)n);
    for (long i = 0; i < n; i++) {
      double d = A.a[l][i] - content_t[i];
      e += d * d;
      if (grad) fg[l][i] = 2.0 * lambda_c * d;
    }
    e *= lambda_c;
    if (parts) parts[NSTYLE] = e;
    E += e;
  }
  *E_out = E;
  if (grad) rc = vgg_backward(params, &A, fg, grad);
  for (int l = 0; l < NCONV; l++) free(fg[l]);
  acts_free(&A);
  return rc;
}

/* the plain Gram loss (Eq. 1-3): orc_loss_grad_aug without the mean / std terms */
int orc_loss_grad(const double *params, const double *x, int H, int W, const double *content_t,
                  const double *style_G, const double *w_style, double lambda_c, double *E_out,
                  double *grad, double *parts, double *grams_out) {
  return orc_loss_grad_aug(params, x, H, W, content_t, style_G, NULL, NULL, w_style, NULL, NULL,
                           lambda_c, E_out, grad, parts, grams_out);
}

/* ------------------------------------------------------------------------------------------- */
/* Algorithm 1: blocks with margins, two passes                                                  */

/* Partition [0, L) into k intervals whose interior boundaries are multiples of 16, as even as
 * possible: b_i = 16 * round(i * L / (16 k)). Fails if an interval would be empty. */
static int plan_1d(int L, int k, int *b) {
  if (k < 1) return ORC_ERR_ARG;
  b[0] = 0;
  b[k] = L;
  for (int i = 1; i < k; i++) {
    double t = (double)i * L / (16.0 * k);
    b[i] = 16 * (int)floor(t + 0.5);
  }
  for (int i = 0; i < k; i++)
    if (b[i + 1] <= b[i]) return ORC_ERR_SHAPE;
  return ORC_OK;
}

/* copy x[:, y0:y1, x0:x1] into a 3 x (y1-y0) x (x1-x0) block */
static void extract_block(const double *x, int H, int W, int y0, int y1, int x0, int x1,
                          double *blk) {
  int h = y1 - y0, w = x1 - x0;
  (void)H;
  for (int c = 0; c < 3; c++)
    for (int y = 0; y < h; y++)
      memcpy(blk + ((long)c * h + y) * w, x + ((long)c * H + y0 + y) * W + x0,
             sizeof(double) * (size_t)w);
}

/* owned feature rows of a block at stride s: global rows j with s*j in [i0, i1) and j < n_glob,
 * returned as [j0, j1) in global indices */
static void owned_range(int i0, int i1, int s, int n_glob, int *j0, int *j1) {
  *j0 = (i0 + s - 1) / s;
  *j1 = imin((i1 + s - 1) / s, n_glob);
  if (*j1 < *j0) *j1 = *j0;
}

/* Algorithm 1 with a k_h x k_w partition, margin m1 in Step 1 and m2 in Step 2 (the paper uses
 * one margin for both). Step 1 adds each block's owned V V^T and channel sums; after it, mean and
 * std = (diag(G) - mean^2)^(1/2). Same outputs as orc_loss_grad_aug. */
int orc_loss_grad_tiled_aug(const double *params, const double *x, int H, int W,
                            const double *content_t, const double *style_G,
                            const double *style_mean, const double *style_std,
                            const double *w_style, const double *w_mean, const double *w_std,
                            double lambda_c, int k_h, int k_w, int m1, int m2, double *E_out,
                            double *grad, double *parts, double *grams_out) {
  const int aug = w_mean && w_std;
  if (check_size(H, W)) return ORC_ERR_SHAPE;
  /* margins are multiples of 16 so that every block's pooling grid is the image's */
  if (k_h < 1 || k_w < 1 || m1 < 0 || m2 < 0 || m1 % 16 || m2 % 16) return ORC_ERR_ARG;
  int *by = (int *)malloc(sizeof(int) * (k_h + 1)), *bx = (int *)malloc(sizeof(int) * (k_w + 1));
  if (plan_1d(H, k_h, by) || plan_1d(W, k_w, bx)) { free(by); free(bx); return ORC_ERR_SHAPE; }
  double *blk = (double *)malloc(sizeof(double) * 3 * (size_t)H * W);
  double *Gs[NSTYLE], *Ss[NSTYLE], *Al[NSTYLE], *Be[NSTYLE];
  long off[NSTYLE], moff[NSTYLE];
  long tot = 0, mtot = 0;
  for (int s = 0; s < NSTYLE; s++) {
    int c = kCout[kStyleConv[s]];
    Gs[s] = (double *)calloc((size_t)c * c, sizeof(double));
    Ss[s] = (double *)calloc((size_t)c, sizeof(double));
    Al[s] = (double *)calloc((size_t)c, sizeof(double));
    Be[s] = (double *)calloc((size_t)c, sizeof(double));
    off[s] = tot;
    moff[s] = mtot;
    tot += (long)c * c;
    mtot += c;
  }
  int rc = ORC_OK;

  /* Step 1: global style statistics of x, block by block (no graph kept) */
  for (int ty = 0; ty < k_h && rc == ORC_OK; ty++)
    for (int tx = 0; tx < k_w && rc == ORC_OK; tx++) {
      int iy0 = by[ty], iy1 = by[ty + 1], ix0 = bx[tx], ix1 = bx[tx + 1];
      int ey0 = imax(0, iy0 - m1), ey1 = imin(H, iy1 + m1);
      int ex0 = imax(0, ix0 - m1), ex1 = imin(W, ix1 + m1);
      int h = ey1 - ey0, w = ex1 - ex0;
      if (h < 16 || w < 16) { rc = ORC_ERR_SHAPE; break; }
      extract_block(x, H, W, ey0, ey1, ex0, ex1, blk);
      acts_t A;
      if (acts_alloc(&A, h, w)) { rc = ORC_ERR_OOM; break; }
      vgg_forward(params, blk, &A);
      for (int s = 0; s < NSTYLE; s++) {
        int l = kStyleConv[s], c = kCout[l], st = kStyleStride[s];
        int jy0, jy1, jx0, jx1;
        owned_range(iy0, iy1, st, H / st, &jy0, &jy1);
        owned_range(ix0, ix1, st, W / st, &jx0, &jx1);
        double *S = (double *)calloc((size_t)c * c, sizeof(double));
        const int ly0 = jy0 - ey0 / st, ly1 = jy1 - ey0 / st;
        const int lx0 = jx0 - ex0 / st, lx1 = jx1 - ex0 / st;
        gram_sum_rect(A.a[l], c, A.h[l], A.w[l], ly0, ly1, lx0, lx1, S);
        for (long k = 0; k < (long)c * c; k++) Gs[s][k] += S[k];
        for (int ch = 0; ch < c; ch++)
          for (int yy = ly0; yy < ly1; yy++)
            for (int xx = lx0; xx < lx1; xx++)
              Ss[s][ch] += A.a[l][((long)ch * A.h[l] + yy) * A.w[l] + xx];
        free(S);
      }
      acts_free(&A);
    }
  double E = 0.0;
  if (rc == ORC_OK) {
    for (int s = 0; s < NSTYLE; s++) {
      int c = kCout[kStyleConv[s]], st = kStyleStride[s];
      double np = (double)(H / st) * (double)(W / st);
      for (long k = 0; k < (long)c * c; k++) Gs[s][k] /= np;
      double e = gram_loss_grad(NULL, c, 0, np, Gs[s], style_G + off[s], w_style[s], NULL);
      if (aug) {
        for (int ch = 0; ch < c; ch++) Ss[s][ch] /= np;   /* channel sums -> mean */
        e += moment_terms(c, np, Gs[s], Ss[s], style_mean + moff[s], style_std + moff[s],
                          w_mean[s], w_std[s], NULL, Al[s], Be[s]);
      }
      if (parts) parts[s] = e;
      E += e;
      if (grams_out) memcpy(grams_out + off[s], Gs[s], sizeof(double) * (size_t)c * c);
    }
  }
  if (grad) memset(grad, 0, sizeof(double) * 3 * (size_t)H * W);

  /* Step 2: loss and gradient, block by block (forward recomputed with the graph) */
  double Ec = 0.0;
  int Hc = H / CONTENT_STRIDE, Wc = W / CONTENT_STRIDE;
  for (int ty = 0; ty < k_h && rc == ORC_OK; ty++)
    for (int tx = 0; tx < k_w && rc == ORC_OK; tx++) {
      int iy0 = by[ty], iy1 = by[ty + 1], ix0 = bx[tx], ix1 = bx[tx + 1];
      int ey0 = imax(0, iy0 - m2), ey1 = imin(H, iy1 + m2);
      int ex0 = imax(0, ix0 - m2), ex1 = imin(W, ix1 + m2);
      int h = ey1 - ey0, w = ex1 - ex0;
      if (h < 16 || w < 16) { rc = ORC_ERR_SHAPE; break; }
      extract_block(x, H, W, ey0, ey1, ex0, ex1, blk);
      acts_t A;
      if (acts_alloc(&A, h, w)) { rc = ORC_ERR_OOM; break; }
      vgg_forward(params, blk, &A);
      double *fg[NCONV] = {0};
      /* style feature gradients on the whole block from the global statistics (Table 1 row 2) */
      for (int s = 0; s < NSTYLE; s++) {
        int l = kStyleConv[s], c = kCout[l], st = kStyleStride[s];
        long npix = (long)A.h[l] * A.w[l];
        double np = (double)(H / st) * (double)(W / st);
        fg[l] = (double *)malloc(sizeof(double) * (size_t)c * npix + 8);
        gram_loss_grad_ab(A.a[l], c, npix, np, Gs[s], style_G + off[s], w_style[s],
                          aug ? Be[s] : NULL, aug ? Al[s] : NULL, fg[l]);
      }
      /* content: loss over the owned pixels, gradient on the whole block (Table 1 row 1) */
      {
        int l = CONTENT_CONV, c = kCout[l], hb = A.h[l], wb = A.w[l];
        long npix = (long)hb * wb;
        fg[l] = (double *)malloc(sizeof(double) * (size_t)c * npix + 8);
        int jy0, jy1, jx0, jx1;
        owned_range(iy0, iy1, CONTENT_STRIDE, Hc, &jy0, &jy1);
        owned_range(ix0, ix1, CONTENT_STRIDE, Wc, &jx0, &jx1);
        int oy = ey0 / CONTENT_STRIDE, ox = ex0 / CONTENT_STRIDE;
        for (int ch = 0; ch < c; ch++)
          for (int y = 0; y < hb; y++)
            for (int xx = 0; xx < wb; xx++) {
              long i = ((long)ch * hb + y) * wb + xx;
              double d = A.a[l][i] - content_t[((long)ch * Hc + oy + y) * Wc + ox + xx];
              fg[l][i] = 2.0 * lambda_c * d;
              int gy = oy + y, gx = ox + xx;
              if (gy >= jy0 && gy < jy1 && gx >= jx0 && gx < jx1) Ec += lambda_c * d * d;
            }
      }
      if (grad) {
        double *db = (double *)malloc(sizeof(double) * 3 * (size_t)h * w);
        rc = vgg_backward(params, &A, fg, db);
        /* keep the inner part of the block gradient */
        for (int c = 0; c < 3; c++)
          for (int y = iy0; y < iy1; y++)
            for (int xx = ix0; xx < ix1; xx++)
              grad[((long)c * H + y) * W + xx] = db[((long)c * h + y - ey0) * w + xx - ex0];
        free(db);
      }
      for (int l = 0; l < NCONV; l++) free(fg[l]);
      acts_free(&A);
    }
  if (parts) parts[NSTYLE] = Ec;
  *E_out = E + Ec;
  for (int s = 0; s < NSTYLE; s++) {
    free(Gs[s]);
    free(Ss[s]);
    free(Al[s]);
    free(Be[s]);
  }
  free(blk);
  free(by);
  free(bx);
  return rc;
}

int orc_loss_grad_tiled(const double *params, const double *x, int H, int W,
                        const double *content_t, const double *style_G, const double *w_style,
                        double lambda_c, int k_h, int k_w, int m1, int m2, double *E_out,
                        double *grad, double *parts, double *grams_out) {
  return orc_loss_grad_tiled_aug(params, x, H, W, content_t, style_G, NULL, NULL, w_style, NULL,
                                 NULL, lambda_c, k_h, k_w, m1, m2, E_out, grad, parts, grams_out);
}

/* ReLU1_1 features of x alone (3 x H x W -> 64 x H x W), rounded as stored in storage mode */
int orc_relu11(const double *params, const double *x, int H, int W, double *out) {
  if (H < 1 || W < 1) return ORC_ERR_SHAPE;
  const double *Wp[NCONV], *bp[NCONV];
  param_ptrs(params, Wp, bp);
  conv3x3_forward(x, 3, H, W, Wp[0], bp[0], 64, out, 0);
  relu_inplace(out, 64L * H * W);
  q_array(out, 64L * H * W);
  return ORC_OK;
}

/* Step 2 of Algorithm 1 for ONE block, given the global statistics: blk is the block extracted
 * with its margin (3 x h x w); G_glob holds G^L(x) of the whole image (np_glob[L] feature pixels)
 * and G_ref the style Grams. Feature gradients are formed on the whole block (Table 1 row 2) and
 * back-propagated; dblk receives dE/d(blk). The content term is left out (lambda_c = 0). The
 * caller keeps the inner part. */
int orc_block_style_grad(const double *params, const double *blk, int h, int w,
                         const double *G_glob, const double *G_ref, const double *np_glob,
                         const double *w_style, double *dblk) {
  if (check_size(h, w) && (h < 1 || w < 1)) return ORC_ERR_SHAPE;
  acts_t A;
  if (acts_alloc(&A, h, w)) return ORC_ERR_OOM;
  vgg_forward(params, blk, &A);
  double *fg[NCONV] = {0};
  long off = 0;
  for (int s = 0; s < NSTYLE; s++) {
    int l = kStyleConv[s], c = kCout[l];
    long npix = (long)A.h[l] * A.w[l];
    if (w_style[s] != 0.0 && npix > 0) {
      fg[l] = (double *)malloc(sizeof(double) * (size_t)c * npix + 8);
      gram_loss_grad(A.a[l], c, npix, np_glob[s], G_glob + off, G_ref + off, w_style[s], fg[l]);
    }
    off += (long)c * c;
  }
  int rc = vgg_backward(params, &A, fg, dblk);
  for (int l = 0; l < NCONV; l++) free(fg[l]);
  acts_free(&A);
  return rc;
}

/* the oracle's block partition, exposed for tests */
int orc_plan_1d(int L, int k, int *b) { return plan_1d(L, k, b); }
