// Device-side state of one solve and the single-block kernels on the small
// Hessenberg / harmonic Ritz problems. Internal to librk.
#pragma once
#include "rk_internal.h"

namespace rk {

// Scalars and small arrays of a solve, in device memory. Sizes: m = Arnoldi
// steps per cycle, kmax = recycle capacity, nqmax = kmax + m + 2.
struct SolveState {
  double bnorm;      // ||b||
  double tolabs;     // tol * ||b||
  double est;        // |g_{j+1}| of the last Arnoldi step
  double rho2;       // ||r||^2 from the last residual / projection
  double nrm2[4];    // norms from fused reductions
  double bic[16];    // rBiCGStab scalars (see solver.cu)
  double scal[4];    // Arnoldi step: 1/alpha, 1/(alpha beta), h_jj/beta, beta
  int done;          // the current cycle stops (estimate met, happy breakdown)
  int jj;            // Arnoldi steps completed in the cycle
  int knew;          // recycle dimension after the last update
  int hr_status;     // 0 ok, else the harmonic Ritz solve failed (space kept)
  int bic_flag;      // rBiCGStab: 1 converged (||s|| or ||r||), 2 breakdown
  int bic_stop;      // rBiCGStab: skip further kernels this batch
  int upd_mode;      // Arnoldi update pass: 0 v_j and p_{j+1}, 1 v_j only, 2 none
  int nspmv;         // products A M^{-1} p taken in the current cycle
  int dev_err;       // nonzero: a bounded device wait gave up (kernel id)
  int wait_limit;    // > 0: polls before the Arnoldi inner products' copy producer gives up (test hook)
};

struct SmallBuffers {
  int m, kmax, nqmax;
  double* H;      // (m+1) x m, true Hessenberg, column-major
  double* R;      // (m+1) x m, Givens-rotated copy
  double* B;      // kmax x m, B = C^T A M^{-1} V
  double* g;      // m+1
  double* cs;     // m
  double* sn;     // m
  double* sv;     // m+2: column scales, v_l = sv[l] * q_l (stored q_l; 0 after a breakdown)
  double* hacc;   // nqmax: first-pass coefficients of the newest Hessenberg column
  double* dots;   // 2 nqmax + 8: reduced inner products
  double* coef;   // nqmax: coefficients handed to the update kernel
  double* y;      // m
  double* xcoef;  // nqmax: coefficients of the solution update
  double* gram;   // (kmax + m + 1) x kmax: [C V]^T M U
  double* QC;     // (kmax + m + 1) x kmax: C <- W_hat QC
  double* PU;     // (kmax + m) x kmax:     U <- W PU
  double* hrws;   // workspace of the harmonic Ritz solve (global fallback)
  double* tcws;   // digits of P for the tensor-core recycle update (dfgemm_tc_ws_bytes())
  size_t hrws_doubles;
};

cudaError_t launch_dcgs_coef(SolveState* s, SmallBuffers b, int kc, int j, int final_pass, cudaStream_t st);
cudaError_t launch_cycle_solve(SolveState* s, SmallBuffers b, int kc, cudaStream_t st);
// schur_f64: the Hessenberg reduction and the Francis iteration in FP64
// (else in double-float on the FP32 pipe)
cudaError_t launch_harmonic_ritz(SolveState* s, SmallBuffers b, int kc, int jj, int k, bool schur_f64,
                                 cudaStream_t st);
cudaError_t launch_set_scalar(SolveState* s, int which, cudaStream_t st);
cudaError_t launch_cycle_init(SolveState* s, SmallBuffers b, cudaStream_t st);
cudaError_t launch_set_tol(SolveState* s, double tol, cudaStream_t st);
// tolabs of the in-cycle stop test, set directly
cudaError_t launch_set_tolabs(SolveState* s, double tolabs, cudaStream_t st);
size_t harmonic_ritz_ws_doubles(int n);
cudaError_t launch_chol_rinv(int k, const double* G, double* Rinv, double* Rw, int* status, cudaStream_t st);

// Standalone harmonic Ritz selection on small matrices (for tests): G, F are
// (n+1) x n column-major device arrays; outputs QC ((n+1) x k), PU (n x k) and
// *knew (device int).
cudaError_t launch_harmonic_ritz_small(int n, const double* G, const double* F, int k, double* QC,
                                       double* PU, int* knew, double* ws, bool schur_f64, cudaStream_t st);

}  // namespace rk
