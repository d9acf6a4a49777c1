// rBiCGStab device vectors and scalars. Internal to librk.
#pragma once
#include "rk_internal.h"

namespace rk {

struct BicgVecs {
  double* r;   // residual r_i (orthogonal to C)
  double* rt;  // shadow residual r~ = r_0
  double* p;   // search direction (preconditioned space)
  double* v;   // A M^{-1} p, projected onto C's complement
  double* s;   // s = r - alpha v
  double* t;   // A M^{-1} s, projected onto C's complement
  double* xt;  // x~: sum of alpha p + omega s (preconditioned space)
};

struct BicgScalars {
  double rho, alpha, omega, beta;
  double tolabs;   // tol * ||b||
  double rtnorm;   // ||r~||
  double s2;       // ||s||^2
  double upd;      // last updated residual norm
  double tmp[4];
  int it;          // iterations of this pass
  int matvecs;     // matrix-vector products of this pass
  int flag;        // 0 running, 1 converged (updated residual), 2 breakdown
  int stop;        // nonzero: the remaining kernels of the batch return
  int half;        // 1: converged at the half step (x~ += alpha p pending)
  int maxmv;       // cap on matrix-vector products of this pass (flag 3 when reached)
  int pad[2];
};

cudaError_t launch_bicg_foldcoef(const double* xi, int kc, double* coefv, cudaStream_t st);
cudaError_t launch_bicg_init(BicgScalars* s, const double* rho2, double tolabs, int maxmv, cudaStream_t st);
cudaError_t launch_bicg_p(const BicgVecs& v, BicgScalars* s, int64_t n, cudaStream_t st);
cudaError_t launch_bicg_alpha(BicgScalars* s, const double* dots, int kc, cudaStream_t st);
// C: kc columns (leading dimension ld), double-float (c_df) or FP64
cudaError_t launch_bicg_s(const BicgVecs& v, BicgScalars* s, int64_t n, int kc, const void* C, bool c_df, int64_t ld,
                          const double* eta1, double* xi, double* part, unsigned* counter, cudaStream_t st);
cudaError_t launch_bicg_half(const BicgVecs& v, BicgScalars* s, int64_t n, cudaStream_t st);
cudaError_t launch_bicg_t(const BicgVecs& v, BicgScalars* s, int64_t n, int kc, const void* C, bool c_df, int64_t ld,
                          const double* eta2, double* part, unsigned* counter, cudaStream_t st);
cudaError_t launch_bicg_r(const BicgVecs& v, BicgScalars* s, int64_t n, int kc, const double* eta1,
                          const double* eta2, double* xi, double* part, unsigned* counter, cudaStream_t st);

}  // namespace rk
