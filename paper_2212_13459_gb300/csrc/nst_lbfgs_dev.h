// nst_lbfgs_dev.h -- device-side state of the L-BFGS step (no host round trip per iteration).
#pragma once
#include "nst_internal.cuh"

namespace nst {

constexpr int kMaxHistory = 128;   // the paper uses 100 at the first scale and 10 afterwards
constexpr int kLbGroup = 4;        // history slots per group of the fused dot-product pass

struct LbfgsCtl {
  double gamma;              // H0 = gamma I: s^T y / y^T y of the newest stored pair (1 before)
  int count;                 // stored pairs
  int spare;                 // slot holding the last step s (the candidate pair)
  int order[kMaxHistory];    // slots of stored pairs, newest first; -1 = empty
  // written by the solve step for the combine step:
  // d = cg g + sum_i (cS[i] S[slot[i]] + cY[i] Y[slot[i]]), already multiplied by the step length
  int k;
  int slot[kMaxHistory];
  float cg;
  float cS[kMaxHistory], cY[kMaxHistory];
};

// the fused pass over the vectors: y = g - g_prev into the spare slot and, per stored pair and
// the candidate, the four dot products s.g, y.g, s.y_new, y.y_new (first: only ||g||_1)
void launch_lbfgs_dots(const float *g, const float *g_prev, const float *S, float *Y,
                       long long stride, long long n, const LbfgsCtl *c, int m, int first,
                       double *partials, cudaStream_t s);
// one CTA: fixed-order reductions, curvature test and history bookkeeping, the compact-form
// solve, coefficients of the step
void launch_lbfgs_solve(LbfgsCtl *c, const double *partials, int m, int first, double eps,
                        double *SY, double *YY, cudaStream_t s);
// the step: s = t d into the spare slot, x += s, g_prev = g
void launch_lbfgs_combine(float *x, float *S, const float *Y, long long stride, float *g_prev,
                          const float *g, long long n, const LbfgsCtl *c, cudaStream_t s);
int lbfgs_partials_count(int m);

}  // namespace nst
