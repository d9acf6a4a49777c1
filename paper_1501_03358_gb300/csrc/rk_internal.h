// Internal declarations of librk (CUDA, sm_103a). Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <mutex>

namespace rk {

constexpr int kNumSM = 152;          // GB300
constexpr int kRedThreads = 256;     // block size of the streaming reductions
constexpr int kMaxRedBlocks = 4 * kNumSM;
// Completion counters of a problem: [0, kGroupCounters) for single-counter
// reductions, [kGroupCounters, kCounters) one per column group of the
// fused Arnoldi inner products.
constexpr int kGroupCounters = 64;
constexpr int kCounters = 1024;

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

// Per-device one-time set-up (the dynamic shared-memory opt-in of
// cudaFuncSetAttribute applies to the current device only): f runs once for
// each device on which a call site is reached, under a lock, and later calls
// on that device skip it; mask holds one bit per device (ordinals < 64).
std::mutex& setup_mutex();
template <typename F>
inline void once_per_device(std::atomic<uint64_t>& mask, F&& f) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  const uint64_t bit = 1ull << (dev & 63);
  if (mask.load(std::memory_order_acquire) & bit) return;
  std::lock_guard<std::mutex> lock(setup_mutex());
  if (mask.load(std::memory_order_acquire) & bit) return;
  f();
  mask.fetch_or(bit, std::memory_order_release);
}

// ---- stencil.cu
enum StencilMode { ST_PREC = 0, ST_PLAIN = 1, ST_RESID = 2, ST_LEFT = 3, ST_LRESID = 4, ST_JSWEEP = 5 };
// y = A (dinv .* v) [ST_PREC], y = A v [ST_PLAIN], y = b - A v [ST_RESID],
// y = dinv .* (A v) [ST_LEFT], y = dinv .* (b - A v) [ST_LRESID] (left
// preconditioning: the product, then one rounded multiplication),
// y = fma(kSdOmega, dinv .* (b - A v), v) [ST_JSWEEP: one damped point-Jacobi
// sweep from v for A y = b, the global sweep of the sub-domain preconditioner].
// part (nullable): per-block partial sums of y^2, reduced by the last block into *nrm2.
cudaError_t launch_stencil(const Dims& d, int S, int mode, const double* coef, const double* dinv,
                           const double* v, const double* b, double* y, double* part,
                           unsigned* counter, double* nrm2, const int* skip_flag, cudaStream_t st);
// The same products with a double-float input and/or output vector (the
// arithmetic stays FP64 in the same order; v = hi + lo on load, the result
// split into hi + lo on store).
// Mixed precision: A M^{-1} v with FP32 coefficients and 1/a_pp, FP32
// accumulation, double-float or FP64 input/output.
cudaError_t launch_stencil32(const Dims& d, int S, const float* coef32, const float* dinv32, const void* v,
                             bool v_df, void* y, bool y_df, const int* skip, cudaStream_t st);
// Double-float operator (RK_DF): bands and 1/a_pp as double-float copies
// (launch_round_df), v and y double-float (v_df / y_df) or FP64.
cudaError_t launch_round_df(int64_t n, const double* src, float2* dst, cudaStream_t st);
cudaError_t launch_stencil_dd(const Dims& d, int S, int mode, const float2* coefd, const float2* dinvd,
                              const void* v, bool v_df, void* y, bool y_df, const int* skip, cudaStream_t st);
cudaError_t launch_round_f32(int64_t n, const double* src, float* dst, cudaStream_t st);
// The FP32 operator in the modes ST_PREC, ST_PLAIN, ST_LEFT and ST_JSWEEP
// (y = fmaf(omega32, d32 .* (r32 - A32 v), v) with r32 FP32): v and y FP64
// (kind 0) or FP32 (kind 1); FP32 rounding of every step in band order.
cudaError_t launch_stencil32_ex(const Dims& d, int S, int mode, const float* coef32, const float* dinv32,
                                const void* v, int v_kind, void* y, int y_kind, const float* r32, const int* skip,
                                cudaStream_t st);
cudaError_t launch_stencil_df(const Dims& d, int S, int mode, const double* coef, const double* dinv,
                              const void* v, bool v_df, void* y, bool y_df, const int* skip_flag, cudaStream_t st);
int stencil_blocks(const Dims& d);
// The global damped sweep y = fma(kSdOmega, dinv .* (r - A z), z), y FP64 or
// double-float; part (nullable) as for launch_stencil.
cudaError_t launch_jsweep(const Dims& d, int S, const double* coef, const double* dinv, const double* z,
                          const double* r, void* y, bool y_df, double* part, unsigned* counter, double* nrm2,
                          const int* skip, cudaStream_t st);

// ---- subdomain.cu: the sub-domain Jacobi preconditioner of Sec. 2.1 (box of
// owned cells, overlap, local damped Jacobi sweeps from zero, relaxation)
constexpr int kSdBX = 16, kSdBY = 8, kSdBZ = 8;
constexpr int kSdOverlap = 1;
constexpr int kSdSweeps = 5;
constexpr double kSdOmega = 2.0 / 3.0;
int64_t subdomain_boxes(const Dims& d);
// z = the restricted local solutions for right-hand side r (every cell of z
// written); the global sweep is launch_jsweep(z, r).
cudaError_t launch_subdomain_local(const Dims& d, int S, const double* coef, const double* dinv, const double* r,
                                   double* z, const int* skip, cudaStream_t st);
// The double-float variant (RK_DF): bands and 1/a_pp from their double-float
// copies, r FP64 or double-float (r_df), z double-float.
// The FP32 variant (RK_MIXED): bands and 1/a_pp from their FP32 copies, r
// FP64 (rounded on load) or FP32 (r_f32), z FP32, every step in FP32 in the
// order of the FP64 kernel.
cudaError_t launch_subdomain_local32(const Dims& d, int S, const float* coef32, const float* dinv32, const void* r,
                                     bool r_f32, float* z, const int* skip, cudaStream_t st);
void subdomain_prepare();
cudaError_t launch_subdomain_local_dd(const Dims& d, int S, const float2* coefd, const float2* dinvd, const void* r,
                                      bool r_df, float2* z, const int* skip, cudaStream_t st);
// y = z + omega dinv (b - A z) in double-float (z, b double-float; y
// double-float or FP64)
cudaError_t launch_jsweep_dd(const Dims& d, int S, const float2* coefd, const float2* dinvd, const float2* z,
                             const float2* b, void* y, bool y_df, const int* skip, cudaStream_t st);
// x += v
cudaError_t launch_add(int64_t n, const double* v, double* x, cudaStream_t st);

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

// Blocks of the double-float Gram kernel for n rows (a function of n alone).
int gram_blocks(int64_t n);

// FP64 fma-rate probe: blocks x 256 threads x 8 chains x iters fma.
cudaError_t launch_fp64_probe(int blocks, int iters, cudaStream_t st);

// Elementwise helpers for the BiCGStab recurrences (see solver.cu).
cudaError_t launch_copy(int64_t n, const double* src, double* dst, cudaStream_t st);
cudaError_t launch_fill(int64_t n, double val, double* dst, cudaStream_t st);

// ---- dfblas.cu: the same roles over double-float (float2) columns.
struct DFDotsArgs {
  int64_t n;
  int nq;
  const float2* Q;     // nq DF columns, leading dimension ld
  int64_t ld;
  const double* extra[3];  // FP64 vectors dotted with w in FP64
  int ne;
  int self;            // append w^T w (DF)
  const void* w;       // double* or float2*
  double* part;        // red_blocks(n) * (nq + self + ne)
  unsigned* counter;
  double* out;         // [Q^T w (nq), w^T w (self), e^T w (ne)]
  const int* skip_flag;
};
cudaError_t launch_dfdots(const DFDotsArgs& a, bool w_is_df, cudaStream_t st);

struct DFUpdateArgs {
  int64_t n;
  int nq;
  const float2* Q;
  int64_t ld;
  const double* c;          // device, nq
  const void* yin;          // double* or float2*
  void* yout;               // double* or float2* (may alias yin)
  const double* scale_ptr;  // nullable
  int scale_rsqrt;          // scale = 1/sqrt(*scale_ptr)
  double* part;
  unsigned* counter;
  double* nrm2;             // nullable: ||y_out||^2
  const int* skip_flag;
};
cudaError_t launch_dfupdate(const DFUpdateArgs& a, bool in_df, bool out_df, cudaStream_t st);

// Fused inner products of one delayed-reorthogonalisation Arnoldi step:
// out = [Q^T p (nq), Q^T w (nq), p^T p, p^T w, w^T w] for the pending basis
// vector p and its product w = A M^{-1} p (both double-float columns).
struct DFDots2Args {
  int64_t n;
  int nq;
  const float2* Q;
  int64_t ld;
  const float2* p;
  const float2* w;
  double* part;       // dots2_blocks(n) * (2 nq + 3)
  unsigned* counter;  // one per column group (ceil(nq / 4) + 1 of them)
  double* out;        // 2 nq + 3
  const int* skip_flag;
  int* err;           // set nonzero if a bounded wait gives up
  const int* wait_limit;  // nullable; *wait_limit > 0: polls of the producer's stage-release waits
};
cudaError_t launch_dfdots2(const DFDots2Args& a, cudaStream_t st);
// one-time kernel attribute setup of the streaming kernels (idempotent)
void dfblas_prepare();
// x-extent of its grid (a function of n alone)
int dots2_blocks(int64_t n);

// The update of the same step, one pass over Q:
//   v      = (p - Q a) * scal[0]                      (final basis vector, into p)
//   p_next = (w - Q b) * scal[1] - v * scal[2]        (next pending vector, into w)
// *mode: 0 both, 1 v only, anything else: nothing.
struct DFUpdate2Args {
  int64_t n;
  int nq;
  const float2* Q;
  int64_t ld;
  const double* a;     // device, nq
  const double* b;     // device, nq
  const double* scal;  // device, 3
  float2* p;
  float2* w;
  const int* mode;
};
cudaError_t launch_dfupdate2(const DFUpdate2Args& a, cudaStream_t st);

struct DFGemmArgs {
  int64_t n;
  int na, nb, nc;
  const float2* A; int64_t lda;
  const float2* Bm; int64_t ldb;
  const double* bscale;  // nullable, multiplies the Bm columns
  const double* P;       // device, np x nc
  void* out; int64_t ldo;  // float2* (DF) or double*
  int accum;             // FP64 output only
};
cudaError_t launch_dfgemm_rows(const DFGemmArgs& a, bool out_df, cudaStream_t st);
// The same product on the tensor cores (digit-sliced, exact FP32
// accumulation; dftc.cu): DF output, 2 <= nc <= 32, na + nb <= 64. ws holds
// dfgemm_tc_ws_bytes() (16-byte aligned); err receives 3 if a bounded wait
// gave up. f64: A, Bm and out are FP64 columns (the pointers of a carry FP64
// data; the FP64 basis), the result rounded once in FP64.
size_t dfgemm_tc_ws_bytes();
bool dfgemm_tc_supported(const DFGemmArgs& a, bool out_df);
bool gemm_tc_f64_supported(int np, int nc, int accum);
cudaError_t launch_dfgemm_tc(const DFGemmArgs& a, void* ws, int* err, cudaStream_t st, bool f64 = false);
void dfgemm_tc_prepare();

struct DFGramArgs {
  int64_t n;
  int na, nb, nu;
  const float2* A; int64_t lda;
  const float2* Bm; int64_t ldb;
  const double* d;       // nullable
  const float2* U; int64_t ldu;
  double* part;
  unsigned* counter;
  double* out;
};
cudaError_t launch_dfgram(const DFGramArgs& a, cudaStream_t st);
cudaError_t launch_to_df(int64_t n, const double* src, float2* dst, const double* scale_ptr, int scale_rsqrt,
                         int ncols, int64_t lds, int64_t ldd, cudaStream_t st);
cudaError_t launch_from_df(int64_t n, const float2* src, double* dst, int ncols, int64_t lds, int64_t ldd,
                           cudaStream_t st);
cudaError_t launch_axpy_scaled(int64_t n, const double* s, const double* v, double* x, cudaStream_t st);

// ---- f64blas.cu: the same roles over FP64 columns (the RK_FP64 and RK_MIXED
// precisions store the basis, U and C in FP64 and project in FP64).
struct F64Dots2Args {
  int64_t n;
  int nq;
  const double* Q;
  int64_t ld;
  const double* p;
  const double* w;
  double* part;       // dots2_f64_rows(n) * (2 nq + 3)
  unsigned* counter;  // one per column group (ceil(nq / 8) + 1 of them)
  double* out;        // 2 nq + 3
  const int* skip_flag;
  int* err;           // set when a bounded wait of the tensor-core path gave up (may be NULL)
};
int dots2_f64_rows(int64_t n);
cudaError_t launch_dots2_f64(const F64Dots2Args& a, cudaStream_t st);
// ---- tcdots.cu: the same products on the tensor cores (exact digit
// products, FP64 accumulation); launch_dots2_f64 routes here when supported
bool dots2_tc_supported(const F64Dots2Args& a);
cudaError_t launch_dots2_tc(const F64Dots2Args& a, cudaStream_t st);

struct F64Update2Args {
  int64_t n;
  int nq;
  const double* Q;
  int64_t ld;
  const double* a;     // device, nq
  const double* b;     // device, nq
  const double* scal;  // device, 3
  double* p;
  double* w;
  const int* mode;
};
cudaError_t launch_update2_f64(const F64Update2Args& a, cudaStream_t st);

struct F64UpdateArgs {
  int64_t n;
  int nq;
  const double* Q;
  int64_t ld;
  const double* c;          // device, nq
  const double* yin;
  double* yout;             // may alias yin
  const double* scale_ptr;  // nullable
  int scale_rsqrt;
  double* part;
  unsigned* counter;
  double* nrm2;             // nullable: ||y_out||^2
  const int* skip_flag;
};
cudaError_t launch_update_f64(const F64UpdateArgs& a, cudaStream_t st);

struct F64GemmArgs {
  int64_t n;
  int na, nb, nc;
  const double* A; int64_t lda;
  const double* Bm; int64_t ldb;
  const double* bscale;  // nullable, multiplies the Bm columns
  const double* P;       // device, (na + nb) x nc
  double* out; int64_t ldo;
  int accum;
};
cudaError_t launch_gemm_rows_f64(const F64GemmArgs& a, cudaStream_t st);

struct F64GramArgs {
  int64_t n;
  int na, nb, nu;
  const double* A; int64_t lda;
  const double* Bm; int64_t ldb;
  const double* d;       // nullable
  const double* U; int64_t ldu;
  double* part;
  unsigned* counter;
  double* out;
};
cudaError_t launch_gram_f64(const F64GramArgs& a, cudaStream_t st);
cudaError_t launch_copy_scaled(int64_t n, const double* src, double* dst, const double* scale_ptr, int scale_rsqrt,
                               int ncols, int64_t lds, int64_t ldd, cudaStream_t st);
// change the storage of ncols columns (leading dimension ld) in place between
// FP64 and double-float
cudaError_t launch_convert_basis(int64_t n, int ncols, int64_t ld, void* base, bool to_df, cudaStream_t st);

// Thread-local message returned by rk_last_error (solver.cu).
void set_last_error(const char* msg);

// ---- smalldense.cu : single-block kernels on the small Hessenberg problems.
struct ArnoldiState;  // defined in solver.cu / smalldense.cu shared header below

}  // namespace rk
