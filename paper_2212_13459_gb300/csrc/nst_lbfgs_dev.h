// nst_lbfgs_dev.h -- device-side state of the L-BFGS step (no host round trip per iteration).
#pragma once
#include "nst_internal.cuh"

namespace nst {

constexpr int kMaxHistory = 128;   // the paper uses 100 at the first scale and 10 afterwards

// a vector given either directly (slot == null) or as slot *slot of a [slots][stride] array,
// resolved on the device; an empty slot (-1) makes the consuming kernel a no-op
struct VecRef {
  const float *base;
  const int *slot;
  long long stride;
};

struct LbfgsCtl {
  double ys, yy;     // y^T s and y^T y of the candidate pair
  double gamma;      // H0 = gamma I
  double t_first;    // min(1, 1/||g||_1) (first iteration)
  double beta;       // scratch of the second loop
  double one;        // 1.0 (step length of later iterations)
  int count;         // stored pairs
  int spare;         // slot holding the last step s (candidate pair)
  int order[kMaxHistory];  // slots of stored pairs, newest first; -1 = empty
};

void launch_dot_ref(const VecRef &a, const VecRef &b, long long n, double *partials, double *out,
                    const double *mul_base, const int *mul_slot, int abs_mode, cudaStream_t s);
void launch_axpy_ref(float *y, const VecRef &x, long long n, const double *c1, const double *c2,
                     float sign, cudaStream_t s);
void launch_sub_ref(const VecRef &out, const float *a, const float *b, long long n,
                    cudaStream_t s);
void launch_scale_dev(float *y, const float *x, long long n, const double *gamma, cudaStream_t s);
void launch_lbfgs_finish_ref(float *x, const VecRef &s_next, float *g_prev, const float *r,
                             const float *g, long long n, const double *t, cudaStream_t s);
void launch_lbfgs_accept(LbfgsCtl *c, double *rho, int m, double eps, cudaStream_t s);
int dot_partials_count();

}  // namespace nst
