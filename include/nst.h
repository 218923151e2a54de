/*
 * nst.h -- C ABI of libnst: the localized style-transfer loss and its image gradient on one GB300
 * (Galerne et al., "Scaling Painting Style Transfer", arXiv 2212.13459).
 *
 * Conventions for every call:
 *   - Images are float32, planar 3 x H x W (RGB, row-major, C-contiguous), in device memory unless
 *     the name ends in _host. The caller owns them; the library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Every device call
 *     is asynchronous on that stream unless stated; its inputs must stay valid until the stream
 *     reaches the work.
 *   - Argument errors are returned synchronously (NST_ERR_INVALID_ARG, NST_ERR_SHAPE,
 *     NST_ERR_STATE). Errors detected on the device (a bounded wait that ran out, a non-finite
 *     input) are latched in a device word; nst_sync_status() synchronizes the stream and returns
 *     it. No C++ exception crosses this boundary. nst_last_error() gives a message.
 *   - A context is bound to the device that was current at nst_create(); calls must come from a
 *     thread whose current device is that device. Calls on one context must not overlap.
 */
#ifndef NST_H
#define NST_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nst_ctx nst_ctx;
typedef struct nst_lbfgs nst_lbfgs;

typedef enum {
  NST_OK = 0,
  NST_ERR_INVALID_ARG = 1, /* null pointer, bad enum, negative size */
  NST_ERR_SHAPE = 2,       /* image smaller than 16 x 16, or a tile grid that does not fit */
  NST_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed (message in nst_last_error) */
  NST_ERR_OOM = 4,         /* device allocation failed */
  NST_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out (kernel returned early) */
  NST_ERR_NONFINITE = 6,   /* the image x held a NaN or Inf */
  NST_ERR_STATE = 7        /* call order violated (e.g. loss before targets) */
} nst_status;

enum { NST_PREC_FP32 = 0, NST_PREC_BF16 = 1 };
enum { NST_CONV_AUTO = 0, NST_CONV_SIMT = 1, NST_CONV_TC = 2 };
enum { NST_SCHED_AUTO = 0, NST_SCHED_TWO_PASS = 1 };

/* Run-time configuration.
 *   w_style[5]: w_L of the Gram loss at ReLU1_1..ReLU5_1 (Section 3.1, Eq. 3).
 *   lambda_c:   content weight (Section 3.1); the content loss is the unnormalised squared
 *               distance of ReLU4_2 features.
 *   tiles_h, tiles_w: the block partition of Section 4.1 given as a k_h x k_w grid; inner block
 *               boundaries lie on multiples of 16 px so every block shares the image's pooling grid.
 *   margin1, margin2: block margins in px (multiples of 16) for Step 1 and Step 2 of Algorithm 1.
 *               The paper uses 256 for both; 80 and 160 cover the ReLU5_1 receptive field
 *               (forward reach 70 px, gradient reach 155 px) and give the same result.
 *   precision:  NST_PREC_FP32 (FP32 storage, FP32 CUDA-core convolutions) or NST_PREC_BF16
 *               (BF16 storage, tcgen05 tensor-core convolutions with FP32 accumulation).
 *   conv_engine: NST_CONV_AUTO (tcgen05 for BF16, SIMT for FP32) or a forced engine (SIMT works
 *               for both precisions; TC needs BF16).
 *   max_batch_tiles: tiles processed per launch (0 = all tiles of the pass, within
 *               workspace_limit_bytes).
 *   workspace_limit_bytes: device workspace cap for activations of a tile batch (0 = 48 GiB).
 *   w_mean[5], w_std[5]: w'_L and w''_L of the augmented style loss (Section 3.2, Eq. 5):
 *               w'_L ||mean(V^L(x)) - mean(V^L(v))||^2 + w''_L ||std(V^L(x)) - std(V^L(v))||^2,
 *               population statistics over the image, std = (diag(G) - mean^2)^(1/2)
 *               (Algorithm 1, Step 1). 0 (the default) gives the plain Gram loss of Eq. 3.
 *   schedule:   NST_SCHED_TWO_PASS runs Algorithm 1 as printed: Step 1 forward with margin1,
 *               then every block's forward again (with margin2) before its backward.
 *               NST_SCHED_AUTO (the default) does the same unless every block of Step 2 fits in
 *               the workspace at once; then one forward pass with margin2 supplies both the
 *               statistics and the activations of the backward (resident; same E and dE/dx up
 *               to summation order, a third less work). */
typedef struct {
  float w_style[5];
  float lambda_c;
  int tiles_h, tiles_w;
  int margin1, margin2;
  int precision;
  int conv_engine;
  int max_batch_tiles;
  long long workspace_limit_bytes;
  float w_mean[5];
  float w_std[5];
  int schedule;
} nst_config;

/* Fill *cfg with the defaults: w_style = 0.2 each, lambda_c = 1e-3, 1 x 1 tiles, margins 80/160,
 * BF16, auto engine, auto batching. Host only. */
nst_status nst_config_default(nst_config *cfg);

/* Create a context on the current device. params_host: float32 host array of n_params values,
 * for conv l = conv1_1..conv5_1 in order: W_l[Cout][Cin][3][3] then b_l[Cout] (VGG-19 up to
 * ReLU5_1, Section 3.1; n_params = 12,944,960). The weights are copied; the caller keeps
 * ownership of params_host. */
nst_status nst_create(nst_ctx **out, const float *params_host, long long n_params,
                      const nst_config *cfg);
nst_status nst_destroy(nst_ctx *ctx);

/* Style statistics G^L(v), L in {ReLU_k_1}, of the style image v (3 x Hv x Wv, device), computed
 * block by block with Step 1 of Algorithm 1 (Require line of Algorithm 1). Stored in the context
 * (FP64). */
nst_status nst_style_targets(nst_ctx *ctx, const float *v_dev, int Hv, int Wv, void *stream);

/* Content target V^{ReLU4_2}(u) of the content image u (3 x H x W, device), computed block by
 * block (Require line of Algorithm 1). Stored in the context at the path's precision; fixes the
 * image size H x W for nst_loss_grad. */
nst_status nst_content_targets(nst_ctx *ctx, const float *u_dev, int H, int W, void *stream);

/* One evaluation of Algorithm 1: E(x) = E_content + sum_L w_L ||G^L(x) - G^L(v)||_F^2 (Eq. 1-3) and
 * grad = dE/dx, by two passes over the blocks. x_dev and grad_dev are 3 x H x W float32 device
 * arrays (H x W must match nst_content_targets); grad_dev is fully overwritten. loss_dev: one
 * double in device memory, or NULL. Requires both targets. */
nst_status nst_loss_grad(nst_ctx *ctx, const float *x_dev, int H, int W, float *grad_dev,
                         double *loss_dev, void *stream);

/* Same evaluation from host memory: copies x_host to the device, evaluates, returns the gradient
 * and the loss, and synchronizes the stream before returning. x_host should be page-locked for
 * full copy speed. A page-locked grad_host is written by the evaluation's last kernel directly
 * (no separate device-to-host copy); any other grad_host receives a copy. loss_host may be NULL. */
nst_status nst_loss_grad_host(nst_ctx *ctx, const float *x_host, int H, int W, float *grad_host,
                              double *loss_host, void *stream);

/* Statistics of the last completed nst_loss_grad (synchronizes the stream first):
 * parts_host[6] = the five Gram terms w_L ||G^L(x) - G^L(v)||^2 and the content term;
 * grams_host (may be NULL) = G^L(x) for the five style layers, concatenated row-major
 * (64^2 + 128^2 + 256^2 + 512^2 + 512^2 = 610,304 doubles). */
nst_status nst_get_stats(nst_ctx *ctx, double *parts_host, double *grams_host, void *stream);

/* The stored style Gram matrices G^L(v) (same layout as grams_host above). Synchronizes. */
nst_status nst_get_style_grams(nst_ctx *ctx, double *grams_host, void *stream);

/* The stored style moments mean(V^L(v)) and std(V^L(v)) of the five style layers,
 * concatenated (64 + 128 + 256 + 512 + 512 = 1,472 doubles each). Synchronizes. */
nst_status nst_get_style_moments(nst_ctx *ctx, double *mean_host, double *std_host,
                                 void *stream);

/* Per-kernel-class device time accumulated since the last nst_set_timing() call (CUDA events
 * around every launch while timing is enabled), in milliseconds, and the FLOPs the convolution
 * launches executed (2 * pixels * Cout * (9 Cin + K2) per launch, pixels = the output patches
 * the launch computed, partial patches and padding included):
 * out[0] = convolution ms, out[1] = convolution FLOPs, out[2] = Gram ms, out[3] = other ms,
 * out[4] = convolution launches, out[5] = all kernel launches (counted with timing on or off).
 * Synchronizes `stream`. */
nst_status nst_get_timing(nst_ctx *ctx, double *out6, void *stream);
/* Enable or disable per-launch event timing; either way the counters restart from zero. */
nst_status nst_set_timing(nst_ctx *ctx, int enable);

/* Change the schedule of an existing context (NST_SCHED_AUTO or NST_SCHED_TWO_PASS, see
 * nst_config); applies from the next nst_loss_grad. */
nst_status nst_set_schedule(nst_ctx *ctx, int schedule);

/* How the last nst_loss_grad ran (host only): *batches = block batches of Step 2 (each batch is
 * every block that fits in the workspace at once); *resident = 1 when all blocks fitted in one
 * batch, so one forward pass of every block (with the Step-2 margin) supplied both the Step-1
 * statistics and the activations Step 2 back-propagates through, instead of a Step-1 pass with
 * the smaller margin and a recomputed forward in Step 2 (Algorithm 1 as printed). Both give the
 * same E and dE/dx up to summation order. Either pointer may be NULL. */
nst_status nst_pass_info(nst_ctx *ctx, int *batches, int *resident);

/* Check of the failure path (no paper counterpart): one kernel whose bounded mbarrier wait can
 * never complete (the same wait the convolution kernels use, with a limit of `limit_cycles`
 * SM cycles, 1 .. 4e9) runs out, latches the timeout in ctx's status word and returns; the next
 * nst_sync_status then returns NST_ERR_TIMEOUT and clears it, and ctx stays usable. Nothing
 * faults or hangs. */
nst_status nst_check_timeout_path(nst_ctx *ctx, long long limit_cycles, void *stream);

/* Synchronize `stream` and return (then clear) the latched device status. */
nst_status nst_sync_status(nst_ctx *ctx, void *stream);

/* Message for the last error on ctx (or the last context-free error if ctx is NULL). */
const char *nst_last_error(nst_ctx *ctx);

/* The block partition used by the library (host only): rects_out receives tiles_h*tiles_w
 * entries of 8 ints {iy0, iy1, ix0, ix1, ey0, ey1, ex0, ex1} (inner and extended rectangles for
 * `margin`), row-major over the tile grid. */
nst_status nst_tile_plan(int H, int W, int tiles_h, int tiles_w, int margin, int *rects_out);

/* ---- L-BFGS (Section 3.1; history sizes of Section 5.1) --------------------------------------
 * The inverse-BFGS matrix of the m newest pairs (the matrix the two-loop recursion applies),
 * H0 = gamma I with gamma = s^T y / y^T y of the newest pair, pairs with y^T s <= 1e-10 skipped,
 * no line search: step 1 except min(1, 1/||g||_1) on the first iteration. Applied in its compact
 * form (two passes over the stored vectors per step). FP32 vectors, dot products summed in FP64
 * in a fixed order, all on the device (no host round trip). State (history 2 (m + 1) n floats)
 * is owned by the nst_lbfgs object, allocated at create. */
nst_status nst_lbfgs_create(nst_lbfgs **out, long long n, int m);
/* As nst_lbfgs_create, with flags. NST_LBFGS_HOST_HISTORY keeps the 2 (m + 1) history vectors in
 * page-locked host memory mapped into the device address space (on a Grace-Blackwell node the
 * step's kernels read them over NVLink-C2C): the GPU analogue of the paper's moving the L-BFGS
 * history to the CPU at the last scale to free device memory (Section 5.1). Same results. */
enum { NST_LBFGS_HOST_HISTORY = 1 };
nst_status nst_lbfgs_create_ex(nst_lbfgs **out, long long n, int m, int flags);
nst_status nst_lbfgs_destroy(nst_lbfgs *st);
/* One iteration: given x (device, n floats, updated in place) and g = grad E(x) (device), form
 * the new pair from the previous call, compute d = -H g and set x <- x + t d. */
nst_status nst_lbfgs_step(nst_lbfgs *st, float *x_dev, const float *g_dev, void *stream);
/* Number of pairs currently stored and iterations taken (host ints; synchronizes). */
nst_status nst_lbfgs_info(nst_lbfgs *st, int *pairs, long long *iters, void *stream);

/* ---- multiscale initialisation (Algorithm 2, "upscale current x by a factor 2") -------------
 * Bicubic (Keys a = -0.75, half-pixel centres, clamped borders) resampling of x_small
 * (3 x h x w, device) to x (3 x H x W, device). */
nst_status nst_upsample_init(const float *x_small_dev, int h, int w, float *x_dev, int H, int W,
                             void *stream);

/* ---- multiscale downscaling (Algorithm 2, "downscale u and v by a factor 2^(n-s)") ---------
 * Area averaging (adaptive average pooling) of x (3 x h x w, device) to out (3 x H x W, device),
 * H <= h, W <= w: output pixel (Y, X) is the mean of the input rows [floor(Y h / H),
 * ceil((Y+1) h / H)) and columns [floor(X w / W), ceil((X+1) w / W)); an integer factor gives
 * the box mean. */
nst_status nst_downscale(const float *x_dev, int h, int w, float *out_dev, int H, int W,
                         void *stream);

/* ---- single-layer convolution (unit-test entry of the convolution engines) -------------------
 * One 3x3 convolution layer of the trunk on NHWC tensors, as used inside nst_loss_grad:
 *   acc[b][y][x][n] = sum_{ky,kx,c} in[b][y+ky-1][x+kx-1][c] * w[n][ky*3+kx][c]      (taps = 9)
 *                   + sum_c in2[b][y][x][c] * w2[n][c]                               (k2 > 0)
 * with zero padding outside H x W. mode 0 (forward): out = relu(acc + bias[n]), and 0 outside the
 * valid region geom_dev[b] = {ey0, ex0, eh, ew} (eh/ew at this layer's resolution, level 0).
 * mode 1 (backward): out = acc * (mask > 0) (mask may be NULL: no gate), 0 outside the valid
 * region. dtype: NST_PREC_FP32 (float tensors) or NST_PREC_BF16 (bfloat16 tensors); engine:
 * NST_CONV_SIMT or NST_CONV_TC (BF16 only). taps is 9 or 0; cin, cout, k2 multiples of 64 (TC) or
 * 16 (SIMT). All pointers are device pointers owned by the caller. */
nst_status nst_conv3x3(int dtype, int engine, int B, int H, int W, int cin, int cout, int taps,
                       const void *in_dev, const void *w_dev, int k2, const void *in2_dev,
                       const void *w2_dev, const float *bias_dev, int mode, const void *mask_dev,
                       const int *geom_dev, void *out_dev, void *stream);

/* ---- single-layer Gram statistics (unit-test entry of the Gram engine) ------------------------
 * G = sum_p V_p V_p^T over the npix rows of V ([npix][C], row-major, NHWC features of one layer),
 * the un-normalised Gram matrix of Eq. 4 (divide by n_p for G^L). FP32 partial sums over pixel
 * chunks, reduced in FP64 in a fixed order (deterministic). dtype: NST_PREC_FP32 or
 * NST_PREC_BF16 elements; C a multiple of 64, 64 <= C <= 512; 1 <= npix < 2^31. G_dev: C*C
 * doubles in device memory, overwritten. Scratch for the partial sums (at most 1,216 blocks of
 * 64 x 64 floats, 19 MiB) is allocated stream-ordered and released on `stream`. Bad arguments
 * (including C outside 64..512 or not a multiple of 64) give NST_ERR_INVALID_ARG. */
nst_status nst_gram(int dtype, const void *V_dev, long long npix, int C, double *G_dev,
                    void *stream);

/* ---- Gram statistics without device allocation ----------------------------------------------
 * The paper has no counterpart: this is a library convenience. Same kernels and the same chunk
 * plan as nst_gram, so the result is bitwise identical to nst_gram's on the same input, for
 * callers that may not allocate device memory themselves (for example a plugin inside an
 * application whose own pool allocator owns the GPU, where cudaMalloc/cudaFree would
 * synchronize the device and bypass the pool). The chunk partial sums go to a fixed 19 MiB
 * array (1,216 blocks of 64 x 64 floats) inside libnst's device image instead of allocated
 * scratch; every GPU that loads the library keeps that array until the process exits. The call
 * allocates nothing.
 *   - dtype, V_dev, npix, G_dev as for nst_gram. C must be a multiple of 64, at least 64
 *     (otherwise NST_ERR_INVALID_ARG, as nst_gram); C > 512 is beyond the array's maximum and
 *     gives NST_ERR_SHAPE. Nothing is launched on either error; nst_last_error(NULL) says why.
 *   - A CUDA error still pending from earlier work when the call starts is returned as
 *     NST_ERR_CUDA (and cleared) before anything is launched.
 *   - The array's device address is looked up once per device and CUDA context, with that
 *     device current (again after cudaDeviceReset or when another context becomes current). The
 *     first call on each device (and context) does that look-up: make it before any stream
 *     capture.
 *   - All calls share the one array and it keeps the previous call's contents: calls whose work
 *     overlaps on the GPU (different streams, or different threads) race and corrupt each other;
 *     serialize them on one stream. */
nst_status nst_gram_noalloc(int dtype, const void *V_dev, long long npix, int C, double *G_dev,
                            void *stream);

/* Library version string. */
const char *nst_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NST_H */
