// Internal declarations of librk (CUDA, sm_103a). Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace rk {

constexpr int kNumSM = 152;          // GB300
constexpr int kRedThreads = 256;     // block size of the streaming reductions
constexpr int kMaxRedBlocks = 4 * kNumSM;

// Stencil tile: one thread per (x, y) column of a 32 x 8 tile, marching in z.
constexpr int kTX = 32;
constexpr int kTY = 8;

struct Dims {
  int nx, ny, nz;
  int px, py, pz;  // periodic flags
  int64_t n;
};

// Blocks of the deterministic grid reductions for a vector of length n: a
// function of n alone, so every reduction over n elements sums in one order.
inline int red_blocks(int64_t n) {
  int64_t b = (n + 4 * kRedThreads - 1) / (4 * kRedThreads);
  if (b < 1) b = 1;
  if (b > kMaxRedBlocks) b = kMaxRedBlocks;
  return (int)b;
}

// ---- stencil.cu
enum StencilMode { ST_PREC = 0, ST_PLAIN = 1, ST_RESID = 2 };
// y = A (dinv .* v) [ST_PREC], y = A v [ST_PLAIN], y = b - A v [ST_RESID].
// part (nullable): per-block partial sums of y^2, reduced by the last block into *nrm2.
cudaError_t launch_stencil(const Dims& d, int S, int mode, const double* coef, const double* dinv,
                           const double* v, const double* b, double* y, double* part,
                           unsigned* counter, double* nrm2, const int* skip_flag, cudaStream_t st);
int stencil_blocks(const Dims& d);

// ---- blas.cu
// out[q] = sum_i Q[q*ld + i] * w[i] (q < nq), then extra vectors e[0..ne) (w
// dotted with each), then (if self) sum w^2. Deterministic two-stage reduction.
struct DotsArgs {
  int64_t n;
  int nq;
  const double* Q;
  int64_t ld;
  const double* extra[3];
  int ne;
  int self;
  const double* w;
  double* part;       // red_blocks(n) * (nq + ne + self)
  unsigned* counter;
  double* out;        // nq + ne + self
  const int* skip_flag;  // nullable: when *skip_flag != 0 the kernel does nothing
};
cudaError_t launch_dots(const DotsArgs& a, cudaStream_t st);

// y[i] -= sum_q Q[q*ld + i] * c[q]; optional: y2 = second output (if non-null
// y is read from yin and written to y); nrm2 = ||y||^2 (deterministic).
struct UpdateArgs {
  int64_t n;
  int nq;
  const double* Q;
  int64_t ld;
  const double* c;    // device, nq
  const double* yin;  // nullable (then yin = y)
  double* y;
  double* part;
  unsigned* counter;
  double* nrm2;       // nullable
  const int* skip_flag;
};
cudaError_t launch_update(const UpdateArgs& a, cudaStream_t st);

// Row-tiled small GEMM, in place safe:
// out[c*ldo + i] = (accum ? out[c*ldo+i] : 0) + sum_q X_q[i] * P[q + c*np]
// where the input columns X are na columns of A (ld lda) followed by nb columns
// of Bm (ld ldb), the latter multiplied elementwise by bscale (nullable).
// nc output columns. P is device, np x nc column-major with np = na + nb.
struct GemmRowsArgs {
  int64_t n;
  int na, nb, nc;
  const double* A; int64_t lda;
  const double* Bm; int64_t ldb;
  const double* bscale;
  const double* P;      // device
  const int* dyn_nb;    // nullable: device int overriding nb (<= nb)
  const int* dyn_nc;    // nullable: device int overriding nc (<= nc)
  double* out; int64_t ldo;
  int accum;
  const int* skip_flag;
};
cudaError_t launch_gemm_rows(const GemmRowsArgs& a, cudaStream_t st);

// Gram block: out[q + l*nq] = sum_i Q_q[i] * d[i] * U_l[i], q < nq (Q = na
// columns of A then nb of Bm), l < nu. Deterministic.
struct GramArgs {
  int64_t n;
  int na, nb, nu;
  const double* A; int64_t lda;
  const double* Bm; int64_t ldb;
  const double* d;
  const double* U; int64_t ldu;
  double* part;
  unsigned* counter;
  double* out;
  const int* dyn_nb;
};
cudaError_t launch_gram(const GramArgs& a, cudaStream_t st);
int gram_blocks(int64_t n);

// Elementwise helpers for the BiCGStab recurrences (see solver.cu).
cudaError_t launch_copy(int64_t n, const double* src, double* dst, cudaStream_t st);
cudaError_t launch_fill(int64_t n, double val, double* dst, cudaStream_t st);

// Thread-local message returned by rk_last_error (solver.cu).
void set_last_error(const char* msg);

// ---- smalldense.cu : single-block kernels on the small Hessenberg problems.
struct ArnoldiState;  // defined in solver.cu / smalldense.cu shared header below

}  // namespace rk
