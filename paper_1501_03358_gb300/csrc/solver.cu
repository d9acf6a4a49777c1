// Host driver and C ABI of librk: problems, recycle spaces, and the solvers
// of Sec. 2.2-2.4 (GMRES(m), rGCROT(m,k), rBiCGStab, hybrid) run as
// sequences of device kernels on the caller's stream.
//
// Device layout of a problem (N cells, ld = N rounded up to 32 doubles):
//   coef  S x ld     banded operator (copied from the caller)
//   dinv  ld         1 / a_pp (right point-Jacobi)
//   QB    (kmax + mcap + 1) x ld   columns [kmax - kc, kmax) hold C, columns
//                    kmax + j hold the Arnoldi vectors; so [C V_j] is one
//                    contiguous block for the block projections
//   Ub    kmax x ld  U, right-aligned the same way (A U = C)
//   bicg  7 x ld     rBiCGStab vectors
// The Arnoldi vectors are stored unnormalised (v_l = sv[l] q_l); the column
// scales are folded into the small coefficient vectors, never into a pass
// over N.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <map>
#include <algorithm>
#include <atomic>
#include <thread>

#include "rk.h"
#include "rk_internal.h"
#include "rk_solver.h"
#include "rk_bicg.h"
#include "rk_batch.h"
#include <chrono>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <sstream>

using namespace rk;

namespace {
thread_local std::string g_err = "no error";

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
}  // namespace

void rk::set_last_error(const char* msg) { g_err = msg; }
std::mutex& rk::setup_mutex() {
  static std::mutex mu;
  return mu;
}

namespace {

#define RK_CUDA(x)                                                                                \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess) return fail(RK_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define RK_TRY(x)              \
  do {                         \
    int r_ = (x);              \
    if (r_ != RK_OK) return r_; \
  } while (0)

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
}  // namespace

struct rk_context {
  rk_alloc_fn alloc = nullptr;
  rk_free_fn free_fn = nullptr;
  void* user = nullptr;
  int device = 0;
  double* part = nullptr;
  size_t part_n = 0;
  unsigned* counter = nullptr;
  int refs = 0;            // live problems created from this context
  bool destroyed = false;  // rk_context_destroy was called
};

namespace {

void context_free(rk_context* c);

void* dev_alloc(rk_context* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (size_t)round_up((int64_t)bytes, 256);
  if (c->alloc) return c->alloc(bytes, c->user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(rk_context* c, void* p) {
  if (!p) return;
  if (c->free_fn)
    c->free_fn(p, c->user);
  else if (cudaFree(p) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    if (std::getenv("RK_DEBUG")) std::fprintf(stderr, "librk: cudaFree failed: %s\n", cudaGetErrorName(e));
  }
}

template <typename T>
int alloc_into(rk_context* c, T** out, size_t count) {
  *out = (T*)dev_alloc(c, count * sizeof(T));
  if (!*out) return fail(RK_E_OOM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
  return RK_OK;
}

}  // namespace

// Opt-in per-kernel-class timing: CUDA events recorded on the solve's stream
// around every launch, reduced at the solve's synchronisation points.
enum ProfClass { PC_SPMV = 0, PC_RESID, PC_DOTS, PC_UPDATE, PC_GEMM, PC_GRAM, PC_SMALL, PC_BICG, PC_HRITZ, PC_SUBDOMAIN, PC_SUBDOMAIN_DF, PC_SUBDOMAIN32, PC_COUNT };
static const char* kProfNames[PC_COUNT] = {"spmv", "residual", "dots", "update", "gemm_rows", "gram", "small", "bicg", "harmonic_ritz", "subdomain_local",
                                             "subdomain_df", "subdomain32"};

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Pending { cudaEvent_t a, b; int cls; double bytes, fma; };
  std::vector<Pending> pending;
  double ms[PC_COUNT] = {0};
  double bytes[PC_COUNT] = {0};
  double fma[PC_COUNT] = {0};
  int64_t launches[PC_COUNT] = {0};
  cudaEvent_t get() {
    if (pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  void flush() {
    for (auto& q : pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) {
        ms[q.cls] += t;
        bytes[q.cls] += q.bytes;
        fma[q.cls] += q.fma;
        launches[q.cls] += 1;
      }
      pool.push_back(q.a);
      pool.push_back(q.b);
    }
    pending.clear();
  }
  void reset() {
    flush();
    for (int i = 0; i < PC_COUNT; ++i) ms[i] = bytes[i] = fma[i] = 0.0, launches[i] = 0;
  }
  ~Profiler() {
    for (auto& q : pending) { cudaEventDestroy(q.a); cudaEventDestroy(q.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct ProfScope {
  Profiler* pr;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  int cls;
  double bytes, fma;
  // b: algorithmic HBM bytes of the launch; f: its FP64 fused multiply-adds
  // (kernels on the FP64 pipe; 0 elsewhere)
  ProfScope(Profiler* p, int c, double b, cudaStream_t s, double f = 0.0) : pr(p), st(s), cls(c), bytes(b), fma(f) {
    if (pr->on) {
      a = pr->get();
      cudaEventRecord(a, st);
    }
  }
  ~ProfScope() {
    if (pr->on && a) {
      cudaEvent_t bev = pr->get();
      cudaEventRecord(bev, st);
      pr->pending.push_back({a, bev, cls, bytes, fma});
    }
  }
};

struct rk_problem {
  rk_context* ctx = nullptr;
  Profiler prof;
  // Captured Arnoldi cycles keyed by (recycle dim, steps, operator precision, keep v_steps);
  // valid while the buffers they reference are (cleared on reallocation).
  std::map<uint64_t, cudaGraphExec_t> graphs;
  cudaStream_t capture_stream = nullptr;  // capture only (graphs launch on the caller's stream)
  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
  Dims d{};
  int S = 7;
  int64_t n = 0, ld = 0;
  double* coef = nullptr;
  double* dinv = nullptr;
  double anorm_f = 0.0;  // ||A||_F
  int kmax = 0, mcap = 0, kdim = 0;
  float2* QB = nullptr;           // basis [C | V]: FP64 or double-float (bdf), 8 bytes per element
  float2* Ub = nullptr;           // U, in the same format
  bool bdf = false;               // the stored recycle space is double-float (RK_DF solves) rather than FP64
  double* rvec = nullptr;         // FP64 residual of the rGCROT cycle
  float* coef32 = nullptr;        // mixed precision: FP32 copy of the bands
  float* dinv32 = nullptr;        // mixed precision: FP32 1/a_pp
  float2* coefdf = nullptr;       // RK_DF: double-float copy of the bands
  float2* dinvdf = nullptr;       // RK_DF: double-float 1/a_pp
  double* sdw = nullptr;          // sub-domain preconditioner: 3 vectors (local result, operands)
  double* bicg = nullptr;
  // small
  double* small = nullptr;
  SmallBuffers sb{};
  SolveState* st = nullptr;       // device
  SolveState* st_h = nullptr;     // pinned host mirror
  BicgScalars* bs = nullptr;      // device
  BicgScalars* bs_h = nullptr;    // pinned host mirror
  double* eta = nullptr;          // eta1, eta2, xi, fold coefficients, k x k scratch
  double* part = nullptr;
  size_t part_n = 0;
  size_t small_n = 0, eta_n = 0;  // doubles held by small / eta
  unsigned* counter = nullptr;
  int* istat = nullptr;           // device ints for small kernels
  int solves = 0;
  int hyb_base = 0;  // first solve of the current rGCROT phase of RK_HYBRID
  int kside = 0;     // the stored recycle pair: 0 A U = C; 1 M^{-1} A U = C with point Jacobi;
                     // 2 M^{-1} A U = C with the sub-domain preconditioner
  double dinv_max = 0.0;  // max |1 / a_pp|

  float2* Vcol(int j) const { return QB + (int64_t)(kmax + j) * ld; }
  float2* Cblk(int kc) const { return QB + (int64_t)(kmax - kc) * ld; }
  float2* Ublk(int kc) const { return Ub + (int64_t)(kmax - kc) * ld; }
};

namespace {

size_t partials_needed(const rk_problem* p, int kmax, int mcap) {
  const int nq = 2 * (kmax + mcap + 1) + 6;
  size_t a = (size_t)red_blocks(p->n) * nq;
  size_t b = (size_t)gram_blocks(p->n) * (size_t)(kmax + mcap + 1) * (size_t)std::max(kmax, 1);
  size_t c = (size_t)stencil_blocks(p->d) + 4;
  size_t e = (size_t)red_blocks(p->n) * 4;
  return std::max(std::max(a, b), std::max(c, e));
}

void free_small(rk_problem* p) {
  dev_free(p->ctx, p->small);
  p->small = nullptr;
  p->small_n = 0;
  p->eta_n = 0;
  dev_free(p->ctx, p->eta);
  p->eta = nullptr;
  dev_free(p->ctx, p->part);
  p->part = nullptr;
}

// (Re)allocate the recycle/Arnoldi storage for capacity (kmax, mcap), keeping
// the stored recycle space. Transactional: every new buffer is allocated
// before the old ones are touched, so when the allocator returns NULL the
// problem keeps its previous buffers, capacity and recycle space unchanged
// (RK_E_OOM) and stays usable.
int ensure_capacity(rk_problem* p, int kneed, int mneed, cudaStream_t st) {
  if (kneed <= p->kmax && mneed <= p->mcap && p->QB && (p->kmax == 0 || p->Ub) && p->rvec && p->small && p->eta &&
      p->part)
    return RK_OK;
  const int kmax = std::max(kneed, p->kmax);
  const int mcap = std::max(mneed, p->mcap);
  if (kmax > 256) return fail(RK_E_INVALID, "recycle dimension above 256 is not supported");
  if (kmax + mcap + 1 > 512) return fail(RK_E_INVALID, "k + m above 511 is not supported");
  // sizes of the small buffers
  SmallBuffers b{};
  const int m = mcap, nq = kmax + mcap + 2;
  b.m = m;
  b.kmax = std::max(kmax, 1);
  b.nqmax = nq;
  const int nhr = kmax + mcap;
  b.hrws_doubles = harmonic_ritz_ws_doubles(std::max(nhr, 1));
  size_t total = 0;
  auto take = [&](size_t cnt) {
    size_t off = total;
    total += (size_t)round_up((int64_t)cnt, 32);
    return off;
  };
  const size_t oH = take((size_t)(m + 1) * m), oR = take((size_t)(m + 1) * m), oB = take((size_t)b.kmax * m),
               og = take(m + 1), ocs = take(m), osn = take(m), osv = take(m + 2), ohacc = take(nq),
               odots = take(2 * (size_t)nq + 8), ocoef = take(nq), oy = take(m), ox = take(nq),
               ogram = take((size_t)(kmax + m + 1) * b.kmax), oQC = take((size_t)(kmax + m + 1) * b.kmax),
               oPU = take((size_t)(kmax + m) * b.kmax), ows = take(b.hrws_doubles),
               otc = take((dfgemm_tc_ws_bytes() + 7) / 8);
  const size_t eta_n = (size_t)4 * (kmax + 4) + (size_t)kmax * kmax * 2 + 16;
  const size_t part_n = partials_needed(p, kmax, mcap);
  // allocate everything new first
  float2* QB = nullptr;
  float2* Ub = nullptr;
  double *rvec = nullptr, *small = nullptr, *eta = nullptr, *part = nullptr;
  int r = alloc_into(p->ctx, &QB, (size_t)(kmax + mcap + 1) * p->ld);
  if (r == RK_OK && kmax > 0) r = alloc_into(p->ctx, &Ub, (size_t)kmax * p->ld);
  if (r == RK_OK && !p->rvec) r = alloc_into(p->ctx, &rvec, (size_t)p->ld);
  if (r == RK_OK) r = alloc_into(p->ctx, &small, total);
  if (r == RK_OK) r = alloc_into(p->ctx, &eta, eta_n);
  if (r == RK_OK) r = alloc_into(p->ctx, &part, part_n);
  if (r != RK_OK) {
    dev_free(p->ctx, QB);
    dev_free(p->ctx, Ub);
    dev_free(p->ctx, rvec);
    dev_free(p->ctx, small);
    dev_free(p->ctx, eta);
    dev_free(p->ctx, part);
    return r;
  }
  p->drop_graphs();
  if (p->kdim > 0) {
    RK_CUDA(cudaMemcpyAsync(QB + (int64_t)(kmax - p->kdim) * p->ld, p->Cblk(p->kdim),
                            sizeof(float2) * p->ld * p->kdim, cudaMemcpyDeviceToDevice, st));
    RK_CUDA(cudaMemcpyAsync(Ub + (int64_t)(kmax - p->kdim) * p->ld, p->Ublk(p->kdim),
                            sizeof(float2) * p->ld * p->kdim, cudaMemcpyDeviceToDevice, st));
  }
  RK_CUDA(cudaStreamSynchronize(st));
  dev_free(p->ctx, p->QB);
  dev_free(p->ctx, p->Ub);
  p->QB = QB;
  p->Ub = Ub;
  p->kmax = kmax;
  p->mcap = mcap;
  if (rvec) p->rvec = rvec;
  free_small(p);
  p->small = small;
  p->small_n = total;
  b.H = small + oH;
  b.R = small + oR;
  b.B = small + oB;
  b.g = small + og;
  b.cs = small + ocs;
  b.sn = small + osn;
  b.sv = small + osv;
  b.hacc = small + ohacc;
  b.dots = small + odots;
  b.coef = small + ocoef;
  b.y = small + oy;
  b.xcoef = small + ox;
  b.gram = small + ogram;
  b.QC = small + oQC;
  b.PU = small + oPU;
  b.hrws = small + ows;
  b.tcws = small + otc;
  p->sb = b;
  RK_CUDA(cudaMemsetAsync(p->small, 0, total * sizeof(double), st));
  p->eta = eta;
  p->eta_n = eta_n;
  p->part = part;
  p->part_n = part_n;
  return RK_OK;
}

int sync_state(rk_problem* p, cudaStream_t st) {
  RK_CUDA(cudaMemcpyAsync(p->st_h, p->st, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
  RK_CUDA(cudaStreamSynchronize(st));
  p->prof.flush();
  if (p->st_h->dev_err != 0) {
    const int e = p->st_h->dev_err;
    RK_CUDA(cudaMemsetAsync(&p->st->dev_err, 0, sizeof(int), st));
    return fail(RK_E_DEVICE_TIMEOUT, "a bounded device wait gave up (code " + std::to_string(e) + ")");
  }
  return RK_OK;
}

// sum of squares of an FP64 device vector into st->nrm2[slot]
int norm2_into(rk_problem* p, const double* v, int slot, cudaStream_t st) {
  DotsArgs a{};
  a.n = p->n;
  a.nq = 0;
  a.Q = v;
  a.ld = p->ld;
  a.ne = 0;
  a.self = 1;
  a.w = v;
  a.part = p->part;
  a.counter = p->counter;
  a.out = &p->st->nrm2[slot];
  ProfScope ps(&p->prof, PC_DOTS, 8.0 * (double)p->n, st);
  RK_CUDA(launch_dots(a, st));
  return RK_OK;
}

// The stored basis, U and C are FP64 (RK_FP64, RK_MIXED) or double-float
// (RK_DF): p->bdf. Each helper below takes basis columns as untyped pointers
// and runs the kernel of the stored format; vectors named FP64 are FP64 in
// either case.

// out = [Q^T w (nq basis columns), then w^T w (self) or e^T w (extra, FP64)];
// w is a basis column (w_basis) or an FP64 vector
int bdots_launch(rk_problem* p, const void* Q, int nq, const void* w, bool w_basis, double* out, const int* skip,
                 cudaStream_t st, const double* extra0 = nullptr, int self = 0) {
  ProfScope ps(&p->prof, PC_DOTS, 8.0 * (nq + (extra0 ? 2 : 0) + 1) * (double)p->n, st,
               p->bdf ? 0.0 : (double)(nq + (extra0 ? 1 : 0) + self) * (double)p->n);
  if (!p->bdf) {
    DotsArgs a{};
    a.n = p->n;
    a.nq = nq;
    a.Q = (const double*)Q;
    a.ld = p->ld;
    a.extra[0] = extra0;
    a.ne = extra0 ? 1 : 0;
    a.self = self;
    a.w = (const double*)w;
    a.part = p->part;
    a.counter = p->counter;
    a.out = out;
    a.skip_flag = skip;
    RK_CUDA(launch_dots(a, st));
    return RK_OK;
  }
  DFDotsArgs a{};
  a.n = p->n;
  a.nq = nq;
  a.Q = (const float2*)Q;
  a.ld = p->ld;
  a.extra[0] = extra0;
  a.ne = extra0 ? 1 : 0;
  a.self = self;
  a.w = w;
  a.part = p->part;
  a.counter = p->counter;
  a.out = out;
  a.skip_flag = skip;
  RK_CUDA(launch_dfdots(a, w_basis, st));
  return RK_OK;
}

// y_out = (y_in - Q c) * scale, ||y_out||^2 -> nrm2 (y FP64)
int bupdate_launch(rk_problem* p, const void* Q, int nq, const double* c, const double* yin, double* yout,
                   double* nrm2, const int* skip, cudaStream_t st, const double* scale_ptr = nullptr,
                   int scale_rsqrt = 0) {
  ProfScope ps(&p->prof, PC_UPDATE, 8.0 * (nq + 2) * (double)p->n, st,
               p->bdf ? 0.0 : (double)(nq + (nrm2 ? 1 : 0)) * (double)p->n);
  if (!p->bdf) {
    F64UpdateArgs a{};
    a.n = p->n;
    a.nq = nq;
    a.Q = (const double*)Q;
    a.ld = p->ld;
    a.c = c;
    a.yin = yin;
    a.yout = yout;
    a.scale_ptr = scale_ptr;
    a.scale_rsqrt = scale_rsqrt;
    a.part = p->part;
    a.counter = p->counter;
    a.nrm2 = nrm2;
    a.skip_flag = skip;
    RK_CUDA(launch_update_f64(a, st));
    return RK_OK;
  }
  DFUpdateArgs a{};
  a.n = p->n;
  a.nq = nq;
  a.Q = (const float2*)Q;
  a.ld = p->ld;
  a.c = c;
  a.yin = yin;
  a.yout = yout;
  a.scale_ptr = scale_ptr;
  a.scale_rsqrt = scale_rsqrt;
  a.part = p->part;
  a.counter = p->counter;
  a.nrm2 = nrm2;
  a.skip_flag = skip;
  RK_CUDA(launch_dfupdate(a, false, false, st));
  return RK_OK;
}

// dots = [Q^T p, Q^T w, p^T p, p^T w, w^T w] of one Arnoldi step (basis columns)
int bdots2_launch(rk_problem* p, const void* Q, int nq, const void* pv, const void* w, double* out, const int* skip,
                  cudaStream_t st) {
  ProfScope ps(&p->prof, PC_DOTS, 8.0 * (nq + 2) * (double)p->n, st,
               p->bdf ? 0.0 : (double)(2 * nq + 3) * (double)p->n);
  if (!p->bdf) {
    F64Dots2Args a{};
    a.n = p->n;
    a.nq = nq;
    a.Q = (const double*)Q;
    a.ld = p->ld;
    a.p = (const double*)pv;
    a.w = (const double*)w;
    a.part = p->part;
    a.counter = p->counter + kGroupCounters;
    a.out = out;
    a.skip_flag = skip;
    a.err = &p->st->dev_err;
    RK_CUDA(launch_dots2_f64(a, st));
    return RK_OK;
  }
  DFDots2Args a{};
  a.n = p->n;
  a.nq = nq;
  a.Q = (const float2*)Q;
  a.ld = p->ld;
  a.p = (const float2*)pv;
  a.w = (const float2*)w;
  a.part = p->part;
  a.counter = p->counter + kGroupCounters;
  a.out = out;
  a.skip_flag = skip;
  a.err = &p->st->dev_err;
  a.wait_limit = &p->st->wait_limit;
  RK_CUDA(launch_dfdots2(a, st));
  return RK_OK;
}

// v = (p - Q a) s0 (in place), p_next = (w - Q b) s1 - v s2 (in place of w)
int bupdate2_launch(rk_problem* p, const void* Q, int nq, const double* ca, const double* cb, const double* scal,
                    void* pv, void* w, const int* mode, bool both, cudaStream_t st) {
  ProfScope ps(&p->prof, PC_UPDATE, 8.0 * (nq + (both ? 4 : 2)) * (double)p->n, st,
               p->bdf ? 0.0 : (double)(both ? 2 * nq + 1 : nq) * (double)p->n);
  if (!p->bdf) {
    F64Update2Args a{};
    a.n = p->n;
    a.nq = nq;
    a.Q = (const double*)Q;
    a.ld = p->ld;
    a.a = ca;
    a.b = cb;
    a.scal = scal;
    a.p = (double*)pv;
    a.w = (double*)w;
    a.mode = mode;
    RK_CUDA(launch_update2_f64(a, st));
    return RK_OK;
  }
  DFUpdate2Args a{};
  a.n = p->n;
  a.nq = nq;
  a.Q = (const float2*)Q;
  a.ld = p->ld;
  a.a = ca;
  a.b = cb;
  a.scal = scal;
  a.p = (float2*)pv;
  a.w = (float2*)w;
  a.mode = mode;
  RK_CUDA(launch_dfupdate2(a, st));
  return RK_OK;
}

// out (+)= [A cols | bscale .* B cols] P  (A, B basis columns; out basis
// columns (out_basis) or an FP64 vector)
int bgemm_launch(rk_problem* p, const void* A, int na, const void* Bm, int nb, const double* bscale, const double* P,
                 int nc, void* out, bool out_basis, int accum, cudaStream_t st) {
  const bool tc64 = !p->bdf && p->sb.tcws != nullptr && out_basis && gemm_tc_f64_supported(na + nb, nc, accum);
  ProfScope ps(&p->prof, PC_GEMM, 8.0 * (na + nb + nc * (accum ? 2 : 1) + (bscale ? 1 : 0)) * (double)p->n, st,
               p->bdf ? 0.0 : (tc64 ? (double)(nb + 7 * nc) : (double)(na + nb) * nc) * (double)p->n);
  if (!p->bdf) {
    F64GemmArgs a{};
    a.n = p->n;
    a.na = na;
    a.nb = nb;
    a.nc = nc;
    a.A = (const double*)A;
    a.lda = p->ld;
    a.Bm = (const double*)Bm;
    a.ldb = p->ld;
    a.bscale = bscale;
    a.P = P;
    a.out = (double*)out;
    a.ldo = p->ld;
    a.accum = accum;
    if (tc64) {
      // FP64 operands on the tensor cores: exact digit products, one rounding
      DFGemmArgs t{};
      t.n = p->n;
      t.na = na;
      t.nb = nb;
      t.nc = nc;
      t.A = (const float2*)A;
      t.lda = p->ld;
      t.Bm = (const float2*)Bm;
      t.ldb = p->ld;
      t.bscale = bscale;
      t.P = P;
      t.out = out;
      t.ldo = p->ld;
      t.accum = 0;
      RK_CUDA(launch_dfgemm_tc(t, p->sb.tcws, &p->st->dev_err, st, true));
      return RK_OK;
    }
    RK_CUDA(launch_gemm_rows_f64(a, st));
    return RK_OK;
  }
  DFGemmArgs a{};
  a.n = p->n;
  a.na = na;
  a.nb = nb;
  a.nc = nc;
  a.A = (const float2*)A;
  a.lda = p->ld;
  a.Bm = (const float2*)Bm;
  a.ldb = p->ld;
  a.bscale = bscale;
  a.P = P;
  a.out = out;
  a.ldo = p->ld;
  a.accum = accum;
  if (p->sb.tcws != nullptr && dfgemm_tc_supported(a, out_basis))
    RK_CUDA(launch_dfgemm_tc(a, p->sb.tcws, &p->st->dev_err, st));
  else
    RK_CUDA(launch_dfgemm_rows(a, out_basis, st));
  return RK_OK;
}

// out[q + l*(na+nb)] = [A B]_q^T diag(d) U_l (basis columns; d FP64, nullable)
int bgram_launch(rk_problem* p, const void* A, int na, const void* Bm, int nb, const double* d, const void* U, int nu,
                 double* out, cudaStream_t st) {
  ProfScope ps(&p->prof, PC_GRAM, 8.0 * (na + nb + nu + (d ? 1 : 0)) * (double)p->n, st,
               p->bdf ? 0.0 : (double)((na + nb) * nu + (d ? nu : 0)) * (double)p->n);
  if (!p->bdf) {
    F64GramArgs g{};
    g.n = p->n;
    g.na = na;
    g.nb = nb;
    g.nu = nu;
    g.A = (const double*)A;
    g.lda = p->ld;
    g.Bm = (const double*)Bm;
    g.ldb = p->ld;
    g.d = d;
    g.U = (const double*)U;
    g.ldu = p->ld;
    g.part = p->part;
    g.counter = p->counter;
    g.out = out;
    RK_CUDA(launch_gram_f64(g, st));
    return RK_OK;
  }
  DFGramArgs g{};
  g.n = p->n;
  g.na = na;
  g.nb = nb;
  g.nu = nu;
  g.A = (const float2*)A;
  g.lda = p->ld;
  g.Bm = (const float2*)Bm;
  g.ldb = p->ld;
  g.d = d;
  g.U = (const float2*)U;
  g.ldu = p->ld;
  g.part = p->part;
  g.counter = p->counter;
  g.out = out;
  RK_CUDA(launch_dfgram(g, st));
  return RK_OK;
}

// ncols FP64 columns (leading dimension lds) into basis columns (ldd),
// times scale (1, *scale_ptr or 1/sqrt(*scale_ptr))
int to_basis(rk_problem* p, const double* src, void* dst, const double* scale_ptr, int scale_rsqrt, int ncols,
             int64_t lds, int64_t ldd, cudaStream_t st) {
  if (p->bdf)
    RK_CUDA(launch_to_df(p->n, src, (float2*)dst, scale_ptr, scale_rsqrt, ncols, lds, ldd, st));
  else
    RK_CUDA(launch_copy_scaled(p->n, src, (double*)dst, scale_ptr, scale_rsqrt, ncols, lds, ldd, st));
  return RK_OK;
}

// basis columns into FP64 columns
int from_basis(const rk_problem* p, const void* src, double* dst, int ncols, int64_t lds, int64_t ldd,
               cudaStream_t st) {
  if (p->bdf)
    RK_CUDA(launch_from_df(p->n, (const float2*)src, dst, ncols, lds, ldd, st));
  else
    RK_CUDA(launch_copy_scaled(p->n, (const double*)src, dst, nullptr, 0, ncols, lds, ldd, st));
  return RK_OK;
}

// The storage of the recycle space for a solve of the given precision:
// RK_DF keeps the basis, U and C in double-float, the others in FP64; a
// stored space in the other format is converted in place.
int ensure_basis(rk_problem* p, bool want_df, cudaStream_t st) {
  if (p->bdf == want_df) return RK_OK;
  if (p->kdim > 0) {
    RK_CUDA(launch_convert_basis(p->n, p->kdim, p->ld, p->Cblk(p->kdim), want_df, st));
    RK_CUDA(launch_convert_basis(p->n, p->kdim, p->ld, p->Ublk(p->kdim), want_df, st));
  }
  p->bdf = want_df;
  return RK_OK;
}

// Structured-grid product on the solve stream, timed as one kernel class.
int stencil_launch(rk_problem* p, int mode, const double* v, const double* b, double* y, double* part,
                   unsigned* counter, double* nrm2, const int* skip, cudaStream_t st) {
  const bool resid = mode == ST_RESID;
  ProfScope ps(&p->prof, resid ? PC_RESID : PC_SPMV, 8.0 * (p->S + (resid ? 3 : 2)) * (double)p->n, st,
               (double)(p->S + (mode == ST_PLAIN ? 0 : 1)) * (double)p->n);
  RK_CUDA(launch_stencil(p->d, p->S, mode, p->coef, p->dinv, v, b, y, part, counter, nrm2, skip, st));
  return RK_OK;
}

int stencil_df_launch(rk_problem* p, int mode, const void* v, bool v_df, void* y, bool y_df, const int* skip,
                      cudaStream_t st) {
  ProfScope ps(&p->prof, PC_SPMV, 8.0 * (p->S + 2) * (double)p->n, st);
  RK_CUDA(launch_stencil_df(p->d, p->S, mode, p->coef, p->dinv, v, v_df, y, y_df, skip, st));
  return RK_OK;
}

// FP32 copy of the operator for the mixed-precision inner products (A11):
// coefficients and 1/a_pp rounded to nearest once.
int ensure_mixed(rk_problem* p, cudaStream_t st) {
  if (p->coef32 && p->dinv32) return RK_OK;
  float* c32 = nullptr;
  float* d32 = nullptr;
  int r = alloc_into(p->ctx, &c32, (size_t)p->S * p->n);
  if (r == RK_OK) r = alloc_into(p->ctx, &d32, (size_t)p->ld);
  if (r != RK_OK) {  // nothing installed: the problem is unchanged
    dev_free(p->ctx, c32);
    dev_free(p->ctx, d32);
    return r;
  }
  p->drop_graphs();
  dev_free(p->ctx, p->coef32);
  dev_free(p->ctx, p->dinv32);
  p->coef32 = c32;
  p->dinv32 = d32;
  RK_CUDA(launch_round_f32((int64_t)p->S * p->n, p->coef, p->coef32, st));
  RK_CUDA(launch_round_f32(p->n, p->dinv, p->dinv32, st));
  return RK_OK;
}

// Double-float copy of the operator for RK_DF: bands and 1/a_pp rounded to
// double-float once.
int ensure_dfop(rk_problem* p, cudaStream_t st) {
  if (p->coefdf && p->dinvdf) return RK_OK;
  float2* cdf = nullptr;
  float2* ddf = nullptr;
  int r = alloc_into(p->ctx, &cdf, (size_t)p->S * p->n);
  if (r == RK_OK) r = alloc_into(p->ctx, &ddf, (size_t)p->ld);
  if (r != RK_OK) {  // nothing installed: the problem is unchanged
    dev_free(p->ctx, cdf);
    dev_free(p->ctx, ddf);
    return r;
  }
  p->drop_graphs();
  dev_free(p->ctx, p->coefdf);
  dev_free(p->ctx, p->dinvdf);
  p->coefdf = cdf;
  p->dinvdf = ddf;
  RK_CUDA(launch_round_df((int64_t)p->S * p->n, p->coef, p->coefdf, st));
  RK_CUDA(launch_round_df(p->n, p->dinv, p->dinvdf, st));
  return RK_OK;
}

// Workspace of the sub-domain preconditioner (Sec. 2.1): three vectors of
// 8-byte words (FP64 or double-float).
int ensure_subdomain(rk_problem* p) {
  if (p->sdw) return RK_OK;
  p->drop_graphs();
  return alloc_into(p->ctx, &p->sdw, (size_t)3 * p->ld);
}

// y = M_df^{-1} r with the double-float variant of the sub-domain
// preconditioner (RK_DF): r FP64 (rounded to double-float into sdw[1]) or
// double-float; y double-float or FP64. r must not alias sdw[0].
int subdomain_df_launch(rk_problem* p, const void* r, bool r_df, void* y, bool y_df, const int* skip,
                        cudaStream_t st) {
  float2* z0 = (float2*)p->sdw;
  const float2* rd = (const float2*)r;
  if (!r_df) {
    float2* t = (float2*)(p->sdw + p->ld);
    RK_CUDA(launch_round_df(p->n, (const double*)r, t, st));
    rd = t;
  }
  {
    ProfScope ps(&p->prof, PC_SUBDOMAIN_DF, 8.0 * (p->S + 3) * (double)p->n, st);
    RK_CUDA(launch_subdomain_local_dd(p->d, p->S, p->coefdf, p->dinvdf, rd, true, z0, skip, st));
  }
  ProfScope ps(&p->prof, PC_SPMV, 8.0 * (p->S + 4) * (double)p->n, st);
  RK_CUDA(launch_jsweep_dd(p->d, p->S, p->coefdf, p->dinvdf, z0, rd, y, y_df, skip, st));
  return RK_OK;
}

// y = M^{-1} r with the sub-domain preconditioner (Sec. 2.1): the local
// sweeps of every box into sdw, then the global damped sweep into y (FP64 or
// double-float); with nrm2 set, ||y||^2 -> *nrm2. r must not alias sdw[0, ld).
int subdomain_launch(rk_problem* p, const double* r, void* y, bool y_df, double* nrm2, const int* skip,
                     cudaStream_t st) {
  {
    ProfScope ps(&p->prof, PC_SUBDOMAIN, 8.0 * (p->S + 3) * (double)p->n, st);
    RK_CUDA(launch_subdomain_local(p->d, p->S, p->coef, p->dinv, r, p->sdw, skip, st));
  }
  ProfScope ps(&p->prof, PC_SPMV, 8.0 * (p->S + 4) * (double)p->n, st);
  RK_CUDA(launch_jsweep(p->d, p->S, p->coef, p->dinv, p->sdw, r, y, y_df, nrm2 ? p->part : nullptr,
                        nrm2 ? p->counter : nullptr, nrm2, skip, st));
  return RK_OK;
}

// y = M32^{-1} r with the FP32 variant of the sub-domain preconditioner
// (RK_MIXED): r FP64 (rounded to FP32 into the scratch) or FP32 (r_f32,
// which must not lie in the first two FP32 vectors of the scratch); y FP64
// (y_kind 0) or FP32 (y_kind 1). Scratch: the preconditioner workspace as
// FP32 vectors [r32 | z32 | ...].
int subdomain32_launch(rk_problem* p, const void* r, bool r_f32, void* y, int y_kind, const int* skip,
                       cudaStream_t st) {
  float* f0 = reinterpret_cast<float*>(p->sdw);
  float* z32 = f0 + p->ld;
  const float* r32 = (const float*)r;
  if (!r_f32) {
    RK_CUDA(launch_round_f32(p->n, (const double*)r, f0, st));
    r32 = f0;
  }
  {
    ProfScope ps(&p->prof, PC_SUBDOMAIN32, 4.0 * (p->S + 3) * (double)p->n, st);
    RK_CUDA(launch_subdomain_local32(p->d, p->S, p->coef32, p->dinv32, r32, true, z32, skip, st));
  }
  ProfScope ps(&p->prof, PC_SPMV, 4.0 * (p->S + 4) * (double)p->n, st);
  RK_CUDA(launch_stencil32_ex(p->d, p->S, ST_JSWEEP, p->coef32, p->dinv32, z32, 1, y, y_kind, r32, skip, st));
  return RK_OK;
}

int ensure_operator(rk_problem* p, int precision, cudaStream_t st) {
  if (precision == RK_MIXED) return ensure_mixed(p, st);
  if (precision == RK_DF) return ensure_dfop(p, st);
  return RK_OK;
}

// A M^{-1} v of the recurrences: FP64 (bit-exact order), the FP32 operator
// (RK_MIXED) or the double-float operator (RK_DF)
int opapply_launch(rk_problem* p, int precision, const void* v, bool v_df, void* y, bool y_df, const int* skip,
                   cudaStream_t st, bool left = false, int pc = RK_PC_JACOBI) {
  if (precision == RK_MIXED && (left || pc == RK_PC_SUBDOMAIN)) {
    // the FP32 operator with the preconditioner from the left (point Jacobi
    // or the FP32 sub-domain sweeps), or the FP32 sub-domain preconditioner
    // from the right; FP64 vectors in and out (the mixed basis is FP64)
    if (v_df || y_df) return fail(RK_E_INVALID, "the FP32 products take FP64 vectors");
    float* f = reinterpret_cast<float*>(p->sdw);
    if (pc != RK_PC_SUBDOMAIN) {
      ProfScope ps(&p->prof, PC_SPMV, 8.0 * (0.5 * p->S + 2.5) * (double)p->n, st);
      RK_CUDA(launch_stencil32_ex(p->d, p->S, ST_LEFT, p->coef32, p->dinv32, v, 0, y, 0, nullptr, skip, st));
      return RK_OK;
    }
    float* t32 = f + 2 * p->ld;  // A32 v (left) or M32^{-1} v (right)
    if (left) {
      {
        ProfScope ps(&p->prof, PC_SPMV, 8.0 * (0.5 * p->S + 1.5) * (double)p->n, st);
        RK_CUDA(launch_stencil32_ex(p->d, p->S, ST_PLAIN, p->coef32, p->dinv32, v, 0, t32, 1, nullptr, skip, st));
      }
      return subdomain32_launch(p, t32, true, y, 0, skip, st);
    }
    RK_TRY(subdomain32_launch(p, v, false, t32, 1, skip, st));
    ProfScope ps(&p->prof, PC_SPMV, 8.0 * (0.5 * p->S + 1.5) * (double)p->n, st);
    RK_CUDA(launch_stencil32_ex(p->d, p->S, ST_PLAIN, p->coef32, p->dinv32, t32, 1, y, 0, nullptr, skip, st));
    return RK_OK;
  }
  if (pc == RK_PC_SUBDOMAIN && precision == RK_DF) {
    // the same products with the double-float operator and preconditioner
    float2* t = (float2*)(p->sdw + p->ld);
    if (left) {
      {
        ProfScope ps(&p->prof, PC_SPMV, 8.0 * (p->S + 2) * (double)p->n, st);
        RK_CUDA(launch_stencil_dd(p->d, p->S, ST_PLAIN, p->coefdf, p->dinvdf, v, v_df, t, true, skip, st));
      }
      return subdomain_df_launch(p, t, true, y, y_df, skip, st);
    }
    float2* z = (float2*)(p->sdw + 2 * p->ld);
    RK_TRY(subdomain_df_launch(p, v, v_df, z, true, skip, st));
    ProfScope ps(&p->prof, PC_SPMV, 8.0 * (p->S + 2) * (double)p->n, st);
    RK_CUDA(launch_stencil_dd(p->d, p->S, ST_PLAIN, p->coefdf, p->dinvdf, z, true, y, y_df, skip, st));
    return RK_OK;
  }
  if (pc == RK_PC_SUBDOMAIN) {
    // M^{-1} (A v) or A (M^{-1} v) with the sub-domain preconditioner (FP64)
    double* t = p->sdw + p->ld;
    if (left) {
      if (v_df)
        RK_TRY(stencil_df_launch(p, ST_PLAIN, v, true, t, false, skip, st));
      else
        RK_TRY(stencil_launch(p, ST_PLAIN, (const double*)v, nullptr, t, nullptr, nullptr, nullptr, skip, st));
      return subdomain_launch(p, t, y, y_df, nullptr, skip, st);
    }
    if (v_df || y_df) return fail(RK_E_INVALID, "right sub-domain product takes FP64 vectors");
    RK_TRY(subdomain_launch(p, (const double*)v, t, false, nullptr, skip, st));
    return stencil_launch(p, ST_PLAIN, t, nullptr, (double*)y, nullptr, nullptr, nullptr, skip, st);
  }
  const int mode = left ? ST_LEFT : ST_PREC;
  if (precision == RK_DF) {
    ProfScope ps(&p->prof, PC_SPMV, 8.0 * (p->S + 2) * (double)p->n, st);
    RK_CUDA(launch_stencil_dd(p->d, p->S, mode, p->coefdf, p->dinvdf, v, v_df, y, y_df, skip, st));
    return RK_OK;
  }
  if (precision != RK_MIXED) {
    if (!v_df && !y_df)
      return stencil_launch(p, mode, (const double*)v, nullptr, (double*)y, nullptr, nullptr, nullptr, skip, st);
    return stencil_df_launch(p, mode, v, v_df, y, y_df, skip, st);
  }
  ProfScope ps(&p->prof, PC_SPMV, 8.0 * (0.5 * p->S + 2.5) * (double)p->n, st);
  RK_CUDA(launch_stencil32(p->d, p->S, p->coef32, p->dinv32, v, v_df, y, y_df, skip, st));
  return RK_OK;
}

// C = orth(A U) in FP64 with U rescaled so that A U = C (CholQR2, as when C is formed from U)
// for the k stored columns.
int derive_c_from_u(rk_problem* p, int k, cudaStream_t st, bool left = false, int pc = RK_PC_JACOBI) {
  float2* Ud = p->Ublk(k);
  float2* Cd = p->Cblk(k);
  double* G = p->eta;
  double* Rinv = p->eta + (size_t)k * k;
  double* Rw = p->sb.hrws;
  if (left && pc == RK_PC_SUBDOMAIN) {
    RK_TRY(ensure_subdomain(p));
    for (int c = 0; c < k; ++c)
      RK_TRY(opapply_launch(p, RK_FP64, Ud + (int64_t)c * p->ld, p->bdf, Cd + (int64_t)c * p->ld, p->bdf, nullptr, st,
                            true, pc));
  } else {
    for (int c = 0; c < k; ++c) {
      if (p->bdf)
        RK_CUDA(launch_stencil_df(p->d, p->S, left ? ST_LEFT : ST_PLAIN, p->coef, p->dinv, Ud + (int64_t)c * p->ld,
                                  true, Cd + (int64_t)c * p->ld, true, nullptr, st));
      else
        RK_CUDA(launch_stencil(p->d, p->S, left ? ST_LEFT : ST_PLAIN, p->coef, p->dinv,
                               (const double*)(Ud + (int64_t)c * p->ld), nullptr, (double*)(Cd + (int64_t)c * p->ld),
                               nullptr, nullptr, nullptr, nullptr, st));
    }
  }
  for (int pass = 0; pass < 2; ++pass) {
    RK_TRY(bgram_launch(p, Cd, k, nullptr, 0, nullptr, Cd, k, G, st));
    RK_CUDA(launch_chol_rinv(k, G, Rinv, Rw, p->istat, st));
    int hs = 0;
    RK_CUDA(cudaMemcpyAsync(&hs, p->istat, sizeof(int), cudaMemcpyDeviceToHost, st));
    RK_CUDA(cudaStreamSynchronize(st));
    if (hs != 0) return fail(RK_E_INVALID, "A U is rank deficient (Cholesky of C~^T C~ failed)");
    RK_TRY(bgemm_launch(p, Cd, k, nullptr, 0, nullptr, Rinv, k, Cd, true, 0, st));
    RK_TRY(bgemm_launch(p, Ud, k, nullptr, 0, nullptr, Rinv, k, Ud, true, 0, st));
  }
  return RK_OK;
}

// The stored recycle pair for a solve on the given preconditioning side: the
// two sides' pairs span the same U with different C (A U versus M^{-1} A U,
// orthonormalised), so a switch re-derives C from U.
int ensure_side(rk_problem* p, bool left, int pc, cudaStream_t st) {
  const int want = left ? 1 + pc : 0;
  if (p->kdim > 0 && p->kside != want) RK_TRY(derive_c_from_u(p, p->kdim, st, left, pc));
  p->kside = want;
  return RK_OK;
}

// Projection onto C at the start of a cycle: xi = C^T r, r <- r - C xi, x <- x + U xi;
// ||r||^2 -> st->rho2 (r and x FP64).
int project_residual(rk_problem* p, int kc, double* r, double* x, cudaStream_t st) {
  if (kc == 0) return RK_OK;  // ||r||^2 already in st->rho2
  double* xi = p->eta;        // kc
  RK_TRY(bdots_launch(p, p->Cblk(kc), kc, r, false, xi, nullptr, st));
  RK_TRY(bupdate_launch(p, p->Cblk(kc), kc, xi, r, r, &p->st->rho2, nullptr, st));
  RK_TRY(bgemm_launch(p, p->Ublk(kc), kc, nullptr, 0, nullptr, xi, 1, x, false, 1, st));
  return RK_OK;
}

double model_words_cycle(int S, int kc, int jj, int m) {
  double w = 0.0;
  for (int j = 0; j < jj; ++j) w += S + 5 + 2.0 * (kc + j);
  w += (jj + kc + 3) + (S + 3);
  (void)m;
  return w;
}

// ---------------------------------------------------------------- GMRES / rGCROT
int solve_gcr(rk_problem* p, const double* b, double* x, const rk_solve_params& prm, rk_solve_info& info,
              bool recycle, bool update, cudaStream_t st) {
  const int m = prm.m;
  const int k = recycle ? prm.k : 0;
  const int maxmv = prm.max_matvec > 0 ? prm.max_matvec : 2000;
  const bool mixed = prm.precision == RK_MIXED;
  const int opk = prm.precision;
  const bool left = prm.precond_side == 1;  // Sec. 2.1: M^{-1} A for GMRES / rGCROT
  const int pc = prm.precond;
  const bool sd = pc == RK_PC_SUBDOMAIN;   // left only (checked by rk_solve)
  RK_TRY(ensure_capacity(p, std::max(k, p->kdim), m, st));
  RK_TRY(ensure_operator(p, opk, st));
  if (left) RK_TRY(ensure_subdomain(p));  // scratch for b - A x
  if (recycle) RK_TRY(ensure_side(p, left, pc, st));
  int kc = recycle ? p->kdim : 0;
  const double S = p->S;
  double words = 0.0;
  double* r = p->rvec;
  // ||b|| (left: also ||M^{-1} b||, the reference of the convergence test)
  RK_TRY(norm2_into(p, b, 0, st));
  { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_set_tol(p->st, prm.tol, st)); }
  RK_TRY(sync_state(p, st));
  const double bnorm_true = p->st_h->bnorm;
  if (!std::isfinite(bnorm_true)) return fail(RK_E_INVALID, "b contains NaN or Inf");
  if (left && bnorm_true != 0.0) {
    if (sd) {
      RK_TRY(subdomain_launch(p, b, r, false, nullptr, nullptr, st));
    } else {
      RK_CUDA(cudaMemsetAsync(r, 0, sizeof(double) * p->n, st));
      RK_CUDA(launch_axpy_scaled(p->n, p->dinv, b, r, st));
    }
    RK_TRY(norm2_into(p, r, 0, st));
    { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_set_tol(p->st, prm.tol, st)); }
    RK_TRY(sync_state(p, st));
  }
  const double bnorm = p->st_h->bnorm;
  const int resid_mode = left ? ST_LRESID : ST_RESID;
  if (bnorm_true == 0.0) {
    RK_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * p->n, st));
    RK_CUDA(cudaStreamSynchronize(st));
    info.status = RK_OK;
    info.recycle_dim = p->kdim;
    return RK_OK;
  }
  // stop test (Sec. 4: the L2 norm of the residual): ||b - A x|| <= tol ||b||.
  // The cycles work on their own residual (left: M^{-1}(b - A x)) with the
  // target tolp; with left preconditioning the true residual is checked
  // after every cycle and, when the preconditioned target is met but the
  // true residual is not, the target is scaled down by the observed shortfall.
  double tolp = prm.tol * bnorm;
  const double toltrue = prm.tol * bnorm_true;
  // r = b - A x (left: M^{-1}(b - A x)) in FP64 with ||r||^2 -> st->rho2
  auto residual = [&]() -> int {
    if (!sd) return stencil_launch(p, resid_mode, x, b, r, p->part, p->counter, &p->st->rho2, nullptr, st);
    double* t = p->sdw + p->ld;
    RK_TRY(stencil_launch(p, ST_RESID, x, b, t, nullptr, nullptr, nullptr, nullptr, st));
    return subdomain_launch(p, t, r, false, &p->st->rho2, nullptr, st);
  };
  // left: ||b - A x||^2 of the current x -> st->nrm2[1]
  auto true_norm = [&]() -> int {
    if (!left) return RK_OK;
    return stencil_launch(p, ST_RESID, x, b, p->sdw + p->ld, p->part, p->counter, &p->st->nrm2[1], nullptr, st);
  };
  double rho = 0.0, rt = 0.0;
  auto converged = [&]() -> bool {
    if (!left) return rho <= tolp;
    rt = std::sqrt(p->st_h->nrm2[1]);
    if (rt <= toltrue) return true;
    if (rho <= tolp) tolp = rho * (toltrue / rt);
    return false;
  };
  // initial residual; its projection onto C
  RK_TRY(residual());
  RK_TRY(project_residual(p, kc, r, x, st));
  RK_TRY(true_norm());
  words += (S + 3) + (kc ? 2.0 * kc + 3 : 0) + 1 + (left ? S + 3 : 0);
  RK_TRY(sync_state(p, st));
  rho = std::sqrt(p->st_h->rho2);
  int matvecs = 0, cycles = 0;
  double est = rho / bnorm;
  const int* done = &p->st->done;
  bool conv = converged();
  while (!conv && matvecs < maxmv) {
    if (left) { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_set_tolabs(p->st, tolp, st)); }
    const int steps = std::min(m, maxmv - matvecs);
    // one Arnoldi cycle (and the second pass of the last vector):
    // a fixed launch sequence whose kernels skip themselves once the device
    // flags say the cycle has stopped, so it is captured once per shape into
    // a CUDA graph and replayed (not while the per-kernel profiler runs)
    const bool keep_last = update && k > 0;
    auto cycle = [&](cudaStream_t st) -> int {
      // v_1 = r / rho, in the basis format
      RK_TRY(to_basis(p, r, p->Vcol(0), &p->st->rho2, 1, 1, p->ld, p->ld, st));
      { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_cycle_init(p->st, p->sb, st)); }
      // per step: one product, one fused inner-product pass and one update
      // pass per step (Gram-Schmidt against [C V_j] with the second pass of
      // each vector delayed to the next step)
      for (int j = 0; j < steps; ++j) {
        RK_TRY(opapply_launch(p, opk, p->Vcol(j), p->bdf, p->Vcol(j + 1), p->bdf, done, st, left, pc));
        const int nq = kc + j;
        RK_TRY(bdots2_launch(p, p->Cblk(kc), nq, p->Vcol(j), p->Vcol(j + 1), p->sb.dots, done, st));
        { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_dcgs_coef(p->st, p->sb, kc, j, 0, st)); }
        RK_TRY(bupdate2_launch(p, p->Cblk(kc), nq, p->sb.dots, p->sb.dots + nq, p->st->scal, p->Vcol(j),
                               p->Vcol(j + 1), &p->st->upd_mode, true, st));
      }
      // cycle end without convergence: second pass of the last vector
      // (completes column steps-1; v_steps is kept for the recycle update)
      const int nq = kc + steps;
      RK_TRY(bdots_launch(p, p->Cblk(kc), nq, p->Vcol(steps), true, p->sb.dots, done, st, nullptr, 1));
      { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_dcgs_coef(p->st, p->sb, kc, steps, 1, st)); }
      if (keep_last)
        RK_TRY(bupdate2_launch(p, p->Cblk(kc), nq, p->sb.dots, p->sb.dots, p->st->scal, p->Vcol(steps),
                               p->Vcol(steps), &p->st->upd_mode, false, st));
      return RK_OK;
    };
    if (p->prof.on) {
      RK_TRY(cycle(st));
    } else {
      const uint64_t key = ((uint64_t)kc << 32) | ((uint64_t)pc << 28) | ((uint64_t)steps << 4) | (left ? 8u : 0u) |
                           ((uint64_t)opk << 1) | (keep_last ? 1u : 0u);
      auto it = p->graphs.find(key);
      if (it == p->graphs.end()) {
        cudaGraph_t g = nullptr;
        if (!p->capture_stream) RK_CUDA(cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking));
        RK_CUDA(cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = cycle(p->capture_stream);
        const cudaError_t ce = cudaStreamEndCapture(p->capture_stream, &g);
        if (rc != RK_OK) {
          if (g) cudaGraphDestroy(g);
          return rc;
        }
        if (ce != cudaSuccess) return fail(RK_E_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(ce));
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return fail(RK_E_CUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(ie));
        it = p->graphs.emplace(key, ge).first;
      }
      RK_CUDA(cudaGraphLaunch(it->second, st));
    }
    RK_TRY(sync_state(p, st));
    const int jj = p->st_h->jj;
    if (jj == 0) break;
    est = p->st_h->est / bnorm;
    matvecs += p->st_h->nspmv;
    cycles += 1;
    // y, z = -B y, x <- x + M^{-1} V_j y + U z (left: x <- x + V_j y + U z)
    { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_cycle_solve(p->st, p->sb, kc, st)); }
    RK_TRY(bgemm_launch(p, p->Ublk(kc), kc, p->Vcol(0), jj, left ? nullptr : p->dinv, p->sb.xcoef, 1, x, false, 1,
                        st));
    words += model_words_cycle(p->S, kc, jj, m);
    // recycle update (harmonic Ritz)
    if (update && k > 0) {
      if (kc > 0) {
        // [C V_{j+1}]^T (M U), M = diag(A) = band 0 (left: F = W_hat^T W, no M)
        RK_TRY(bgram_launch(p, p->Cblk(kc), kc, p->Vcol(0), jj + 1, left ? nullptr : p->coef, p->Ublk(kc), kc,
                            p->sb.gram, st));
      }
      { ProfScope ps_(&p->prof, PC_HRITZ, 0.0, st); RK_CUDA(launch_harmonic_ritz(p->st, p->sb, kc, jj, k, !p->bdf, st)); }
      RK_TRY(sync_state(p, st));
      const int knew = p->st_h->knew;
      if (p->st_h->hr_status == 0 && knew > 0) {
        // C <- [C V_{j+1}] QC, U <- [U, M^{-1} V_j] PU (left: [U, V_j] PU), in place (row tiles)
        RK_TRY(bgemm_launch(p, p->Cblk(kc), kc, p->Vcol(0), jj + 1, nullptr, p->sb.QC, knew, p->Cblk(knew), true, 0,
                            st));
        RK_TRY(bgemm_launch(p, p->Ublk(kc), kc, p->Vcol(0), jj, left ? nullptr : p->dinv, p->sb.PU, knew,
                            p->Ublk(knew), true, 0, st));
        kc = knew;
        p->kdim = knew;
        words += 6.0 * kc + 3.0 * jj + 4;
      }
    }
    // true residual r = b - A x (left: M^{-1}(b - A x)); the next cycle projects it onto C
    RK_TRY(residual());
    RK_TRY(project_residual(p, kc, r, x, st));
    RK_TRY(true_norm());
    words += left ? S + 3 : 0;
    RK_TRY(sync_state(p, st));
    rho = std::sqrt(p->st_h->rho2);
    conv = converged();
  }
  if (mixed && update && p->kdim > 0) {
    // the FP32 operator leaves A U = C (left: M^{-1} A U = C) only to FP32
    // accuracy: re-derive C from U with the FP64 operator and preconditioner
    // so the space carried to the next solve keeps the pair exact
    RK_TRY(derive_c_from_u(p, p->kdim, st, left, pc));
  }
  info.matvecs = matvecs;
  info.cycles_or_iters = cycles;
  // left: ||b - A x|| of the returned x (the last check ran on it)
  info.relres_true = left ? rt / bnorm_true : rho / bnorm;
  info.relres_est = est;
  info.recycle_dim = p->kdim;
  info.model_bytes = 8.0 * words * (double)p->n;
  info.status = conv ? RK_OK : RK_E_NOT_CONVERGED;
  return info.status;
}

// ---------------------------------------------------------------- rBiCGStab
// One rBiCGStab solve (Algorithm 4) as a sequence of stages, so that the
// batched executor can run the iterations of many solves in shared launches
// while every other stage stays the single-problem code:
//   bicg_setup -> { bicg_pass_start -> iterations -> bicg_pass_end }* -> bicg_finish
struct BicgRun {
  rk_problem* p = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  rk_solve_params prm{};
  rk_solve_info* info = nullptr;
  int maxmv = 2000, opk = RK_FP64, pc = RK_PC_JACOBI, kc = 0;
  BicgVecs v{};
  double *eta1 = nullptr, *eta2 = nullptr, *xi = nullptr, *coefv = nullptr;
  double bnorm = 0.0, tolabs = 0.0, words = 0.0, rel = 0.0, upd = 0.0;
  int matvecs = 0, its = 0, restarts = 0, status = RK_E_NOT_CONVERGED;
  bool done = false;
};

int bicg_setup(BicgRun& R, rk_problem* p, const double* b, double* x, const rk_solve_params& prm,
               rk_solve_info& info, bool recycle, cudaStream_t st) {
  R.p = p;
  R.b = b;
  R.x = x;
  R.prm = prm;
  R.info = &info;
  R.maxmv = prm.max_matvec > 0 ? prm.max_matvec : 2000;
  R.opk = prm.precision;
  RK_TRY(ensure_capacity(p, p->kdim, std::max(p->mcap, 1), st));
  RK_TRY(ensure_operator(p, R.opk, st));
  if (!p->bicg) RK_TRY(alloc_into(p->ctx, &p->bicg, (size_t)7 * p->ld));
  if (recycle) RK_TRY(ensure_side(p, false, prm.precond, st));  // Sec. 2.1: BiCGStab is right-preconditioned
  R.pc = prm.precond;
  R.kc = recycle ? p->kdim : 0;
  BicgVecs& v = R.v;
  v.r = p->bicg;
  v.rt = p->bicg + p->ld;
  v.p = p->bicg + 2 * p->ld;
  v.v = p->bicg + 3 * p->ld;
  v.s = p->bicg + 4 * p->ld;
  v.t = p->bicg + 5 * p->ld;
  v.xt = p->bicg + 6 * p->ld;
  R.eta1 = p->eta;
  R.eta2 = p->eta + (p->kmax + 4);
  R.xi = p->eta + 2 * (p->kmax + 4);
  R.coefv = p->eta + 3 * (p->kmax + 4);
  RK_TRY(norm2_into(p, b, 0, st));
  { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_set_tol(p->st, prm.tol, st)); }
  RK_TRY(sync_state(p, st));
  R.bnorm = p->st_h->bnorm;
  if (!std::isfinite(R.bnorm)) return fail(RK_E_INVALID, "b contains NaN or Inf");
  if (R.bnorm == 0.0) {
    RK_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * p->n, st));
    RK_CUDA(cudaStreamSynchronize(st));
    info.status = RK_OK;
    info.recycle_dim = p->kdim;
    R.status = RK_OK;
    R.done = true;
    return RK_OK;
  }
  R.tolabs = prm.tol * R.bnorm;
  return RK_OK;
}

// r = b - A x; its projection: eta1 = C^T r, r -= C eta1, xi = -eta1; r~ = r,
// x~ = 0, the scalars of a new pass
int bicg_pass_start(BicgRun& R, cudaStream_t st) {
  rk_problem* p = R.p;
  const BicgVecs& v = R.v;
  const int kc = R.kc;
  RK_TRY(stencil_launch(p, ST_RESID, R.x, R.b, v.r, p->part, p->counter, &p->st->rho2, nullptr, st));
  if (kc) {
    RK_TRY(bdots_launch(p, p->Cblk(kc), kc, v.r, false, R.xi, nullptr, st));
    RK_TRY(bupdate_launch(p, p->Cblk(kc), kc, R.xi, v.r, v.r, &p->st->rho2, nullptr, st));
    // xi = -eta1 enters x at once (x <- x + U eta1); xi restarts from 0
    RK_TRY(bgemm_launch(p, p->Ublk(kc), kc, nullptr, 0, nullptr, R.xi, 1, R.x, false, 1, st));
    RK_CUDA(cudaMemsetAsync(R.xi, 0, sizeof(double) * kc, st));
  }
  { ProfScope ps_(&p->prof, PC_BICG, 24.0 * p->n, st); RK_CUDA(launch_copy(p->n, v.r, v.rt, st)); RK_CUDA(launch_fill(p->n, 0.0, v.xt, st)); }
  { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_bicg_init(p->bs, &p->st->rho2, R.tolabs, R.maxmv - R.matvecs, st)); }
  R.words += (p->S + 3) + 2.0 * kc + 4;
  return RK_OK;
}

// one iteration of Algorithm 4 on one problem (the kernels skip themselves
// once the scalars say the pass has stopped)
int bicg_iteration(BicgRun& R, cudaStream_t st) {
  rk_problem* p = R.p;
  const BicgVecs& v = R.v;
  const int kc = R.kc;
  { ProfScope ps_(&p->prof, PC_BICG, 32.0 * p->n, st, 2.0 * p->n); RK_CUDA(launch_bicg_p(v, p->bs, p->n, st)); }
  RK_TRY(opapply_launch(p, R.opk, v.p, false, v.v, false, &p->bs->stop, st, false, R.pc));
  RK_TRY(bdots_launch(p, p->Cblk(kc), kc, v.v, false, R.eta1, &p->bs->stop, st, v.rt));
  { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_bicg_alpha(p->bs, R.eta1, kc, st)); }
  { ProfScope ps_(&p->prof, PC_BICG, 8.0 * (kc + (kc ? 5 : 3)) * (double)p->n, st, (p->bdf ? 2.0 : kc + 2.0) * p->n); RK_CUDA(launch_bicg_s(v, p->bs, p->n, kc, p->Cblk(kc), p->bdf, p->ld, R.eta1, R.xi, p->part, p->counter, st)); }
  RK_TRY(opapply_launch(p, R.opk, v.s, false, v.t, false, &p->bs->stop, st, false, R.pc));
  if (kc) RK_TRY(bdots_launch(p, p->Cblk(kc), kc, v.t, false, R.eta2, &p->bs->stop, st));
  { ProfScope ps_(&p->prof, PC_BICG, 8.0 * (kc + (kc ? 3 : 2)) * (double)p->n, st, (p->bdf ? 2.0 : kc + 2.0) * p->n); RK_CUDA(launch_bicg_t(v, p->bs, p->n, kc, p->Cblk(kc), p->bdf, p->ld, R.eta2, p->part, p->counter, st)); }
  { ProfScope ps_(&p->prof, PC_BICG, 56.0 * p->n, st, 5.0 * p->n); RK_CUDA(launch_bicg_r(v, p->bs, p->n, kc, R.eta1, R.eta2, R.xi, p->part, p->counter, st)); }
  return RK_OK;
}

// after the pass stopped: the half step, the fold x <- x + M^{-1} x~ - U xi,
// the true residual b - A x in FP64 (residual replacement: the decision is
// taken on it, never on the recurrence's residual), and the decision
int bicg_pass_end(BicgRun& R, cudaStream_t st) {
  rk_problem* p = R.p;
  const BicgVecs& v = R.v;
  const int kc = R.kc;
  if (p->bs_h->half == 1) { ProfScope ps_(&p->prof, PC_BICG, 24.0 * p->n, st); RK_CUDA(launch_bicg_half(v, p->bs, p->n, st)); }
  R.matvecs += p->bs_h->matvecs;
  R.its += p->bs_h->it;
  R.upd = p->bs_h->upd;
  R.words += (double)p->bs_h->it * (2 * p->S + 4.0 * kc + 22);
  const int flag = p->bs_h->flag;
  if (R.pc == RK_PC_SUBDOMAIN) {
    RK_TRY(subdomain_launch(p, v.xt, p->sdw + p->ld, false, nullptr, nullptr, st));
    RK_CUDA(launch_add(p->n, p->sdw + p->ld, R.x, st));
  } else {
    RK_CUDA(launch_axpy_scaled(p->n, p->dinv, v.xt, R.x, st));
  }
  if (kc) {
    { ProfScope ps_(&p->prof, PC_SMALL, 0.0, st); RK_CUDA(launch_bicg_foldcoef(R.xi, kc, R.coefv, st)); }
    RK_TRY(bgemm_launch(p, p->Ublk(kc), kc, nullptr, 0, nullptr, R.coefv, 1, R.x, false, 1, st));
  }
  R.words += kc + 4;
  // true residual b - A x; above tol, Algorithm 4 restarts from the current x (residual replacement)
  RK_TRY(stencil_launch(p, ST_RESID, R.x, R.b, v.r, p->part, p->counter, &p->st->rho2, nullptr, st));
  RK_TRY(sync_state(p, st));
  R.rel = std::sqrt(p->st_h->rho2) / R.bnorm;
  if (R.rel <= R.prm.tol) {
    R.status = RK_OK;
    R.done = true;
  } else if (R.matvecs >= R.maxmv || flag == 3) {
    R.status = RK_E_NOT_CONVERGED;
    R.done = true;
  } else if (R.restarts >= 3) {
    R.status = flag == 2 ? RK_E_BREAKDOWN : RK_E_NOT_CONVERGED;
    R.done = true;
  } else {
    R.restarts += 1;
  }
  return RK_OK;
}

int bicg_finish(BicgRun& R) {
  rk_solve_info& info = *R.info;
  if (R.bnorm == 0.0) return RK_OK;
  info.matvecs = R.matvecs;
  info.cycles_or_iters = R.its;
  info.restarts = R.restarts;
  info.relres_true = R.rel;
  info.relres_est = R.upd / R.bnorm;
  info.recycle_dim = R.p->kdim;
  info.model_bytes = 8.0 * R.words * (double)R.p->n;
  info.status = R.status;
  return R.status;
}

// ---------------------------------------------------------------- rBiCGStab
int solve_bicg(rk_problem* p, const double* b, double* x, const rk_solve_params& prm, rk_solve_info& info,
               bool recycle, cudaStream_t st) {
  BicgRun R;
  RK_TRY(bicg_setup(R, p, b, x, prm, info, recycle, st));
  if (R.done) return RK_OK;
  const int NB = 8;
  while (!R.done) {
    RK_TRY(bicg_pass_start(R, st));
    bool running = true;
    while (running) {
      for (int it = 0; it < NB; ++it) RK_TRY(bicg_iteration(R, st));
      RK_CUDA(cudaMemcpyAsync(p->bs_h, p->bs, sizeof(BicgScalars), cudaMemcpyDeviceToHost, st));
      RK_CUDA(cudaStreamSynchronize(st));
      p->prof.flush();
      if (p->bs_h->stop) running = false;
    }
    RK_TRY(bicg_pass_end(R, st));
  }
  return bicg_finish(R);
}

void context_free(rk_context* c) {
  dev_free(c, c->part);
  dev_free(c, c->counter);
  delete c;
}

int check_grid(const rk_grid* g) {
  if (!g || g->nx <= 0 || g->ny <= 0 || g->nz <= 0) return fail(RK_E_INVALID, "grid extents must be positive");
  return RK_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* rk_last_error(void) { return g_err.c_str(); }

const char* rk_version(void) { return "rk 0.1 (sm_103a)"; }

int rk_context_create(rk_alloc_fn alloc, rk_free_fn free_fn, void* user, rk_context** out) {
  if (!out) return fail(RK_E_INVALID, "out is NULL");
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(RK_E_INVALID, "alloc and free must both be given");
  rk_context* c = new rk_context();
  c->alloc = alloc;
  c->free_fn = free_fn;
  c->user = user;
  RK_CUDA(cudaGetDevice(&c->device));
  c->counter = (unsigned*)dev_alloc(c, 64 * sizeof(unsigned));
  if (!c->counter) {
    delete c;
    return fail(RK_E_OOM, "counter allocation failed");
  }
  RK_CUDA(cudaMemset(c->counter, 0, 64 * sizeof(unsigned)));
  *out = c;
  return RK_OK;
}

void rk_context_destroy(rk_context* c) {
  if (!c) return;
  c->destroyed = true;
  if (c->refs == 0) context_free(c);
}

int rk_create_problem(rk_context* ctx, const rk_grid* grid, int32_t S, const double* coef, void* stream,
                      rk_problem** out) {
  if (!ctx || !out || !coef) return fail(RK_E_INVALID, "NULL argument");
  RK_TRY(check_grid(grid));
  if (S != 7 && S != 19) return fail(RK_E_INVALID, "S must be 7 or 19");
  cudaStream_t st = (cudaStream_t)stream;
  rk_problem* p = new rk_problem();
  p->ctx = ctx;
  ctx->refs += 1;
  p->S = S;
  p->d.nx = grid->nx;
  p->d.ny = grid->ny;
  p->d.nz = grid->nz;
  p->d.px = grid->periodic[0] ? 1 : 0;
  p->d.py = grid->periodic[1] ? 1 : 0;
  p->d.pz = grid->periodic[2] ? 1 : 0;
  p->n = (int64_t)grid->nx * grid->ny * grid->nz;
  p->d.n = p->n;
  p->ld = round_up(p->n, 32);
  auto cleanup = [&](int code) {
    rk_problem_destroy(p);
    return code;
  };
  int r;
  dfblas_prepare();
  dfgemm_tc_prepare();
  subdomain_prepare();
  if ((r = alloc_into(ctx, &p->coef, (size_t)S * p->n)) != RK_OK) return cleanup(r);
  if ((r = alloc_into(ctx, &p->dinv, (size_t)p->ld)) != RK_OK) return cleanup(r);
  if ((r = alloc_into(ctx, &p->counter, kCounters)) != RK_OK) return cleanup(r);
  if ((r = alloc_into(ctx, &p->st, 1)) != RK_OK) return cleanup(r);
  if ((r = alloc_into(ctx, &p->bs, 1)) != RK_OK) return cleanup(r);
  if ((r = alloc_into(ctx, &p->istat, 16)) != RK_OK) return cleanup(r);
  if (cudaMallocHost(&p->st_h, sizeof(SolveState)) != cudaSuccess ||
      cudaMallocHost(&p->bs_h, sizeof(BicgScalars)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(RK_E_OOM, "pinned host allocation failed"));
  }
  if (cudaMemcpyAsync(p->coef, coef, sizeof(double) * S * p->n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(p->counter, 0, kCounters * sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(p->st, 0, sizeof(SolveState), st) != cudaSuccess ||
      cudaMemsetAsync(p->bs, 0, sizeof(BicgScalars), st) != cudaSuccess)
    return cleanup(fail(RK_E_CUDA, "copying the coefficients failed"));
  // validation on the host copy (structural zeros, nonzero diagonal)
  {
    std::vector<double> h((size_t)S * p->n);
    if (cudaMemcpyAsync(h.data(), p->coef, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return cleanup(fail(RK_E_CUDA, "reading the coefficients back failed"));
    static const int OFF[19][3] = {{0, 0, 0},   {-1, 0, 0},  {1, 0, 0},   {0, -1, 0}, {0, 1, 0},
                                   {0, 0, -1},  {0, 0, 1},   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
                                   {1, 1, 0},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1}, {1, 0, 1},
                                   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {0, 1, 1}};
    double fro = 0.0;
    std::vector<double> dinv(p->ld, 0.0);
    for (int kk = 0; kk < grid->nz; ++kk)
      for (int j = 0; j < grid->ny; ++j)
        for (int i = 0; i < grid->nx; ++i) {
          const int64_t q = i + (int64_t)grid->nx * (j + (int64_t)grid->ny * kk);
          const double a0 = h[q];
          if (!(a0 != 0.0) || !std::isfinite(a0))
            return cleanup(fail(RK_E_INVALID, "zero or non-finite diagonal at cell " + std::to_string(q)));
          dinv[q] = 1.0 / a0;
          for (int s = 0; s < S; ++s) {
            const double c = h[(size_t)s * p->n + q];
            if (!std::isfinite(c)) return cleanup(fail(RK_E_INVALID, "non-finite coefficient"));
            fro += c * c;
            if (s == 0 || c == 0.0) continue;
            const int ii = i + OFF[s][0], jj = j + OFF[s][1], k2 = kk + OFF[s][2];
            const bool out_x = (ii < 0 || ii >= grid->nx) && !grid->periodic[0];
            const bool out_y = (jj < 0 || jj >= grid->ny) && !grid->periodic[1];
            const bool out_z = (k2 < 0 || k2 >= grid->nz) && !grid->periodic[2];
            if (out_x || out_y || out_z)
              return cleanup(fail(RK_E_INVALID, "band " + std::to_string(s) + " of cell " + std::to_string(q) +
                                                    " points out of a non-periodic face with a nonzero coefficient"));
          }
        }
    p->anorm_f = std::sqrt(fro);
    if (cudaMemcpyAsync(p->dinv, dinv.data(), sizeof(double) * p->ld, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return cleanup(fail(RK_E_CUDA, "uploading the preconditioner failed"));
  }
  *out = p;
  return RK_OK;
}

void rk_problem_destroy(rk_problem* p) {
  if (!p) return;
  p->drop_graphs();
  if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
  rk_context* c = p->ctx;
  dev_free(c, p->coef);
  dev_free(c, p->dinv);
  dev_free(c, p->QB);
  dev_free(c, p->Ub);
  dev_free(c, p->rvec);
  dev_free(c, p->coef32);
  dev_free(c, p->dinv32);
  dev_free(c, p->coefdf);
  dev_free(c, p->dinvdf);
  dev_free(c, p->sdw);
  dev_free(c, p->bicg);
  dev_free(c, p->small);
  dev_free(c, p->eta);
  dev_free(c, p->part);
  dev_free(c, p->counter);
  dev_free(c, p->st);
  dev_free(c, p->bs);
  dev_free(c, p->istat);
  if (p->st_h) cudaFreeHost(p->st_h);
  if (p->bs_h) cudaFreeHost(p->bs_h);
  delete p;
  c->refs -= 1;
  if (c->destroyed && c->refs == 0) context_free(c);
}

int rk_apply(const rk_problem* p, const double* v, double* y, int32_t precond, void* stream) {
  if (!p || !v || !y) return fail(RK_E_INVALID, "NULL argument");
  if (precond == 2) {
    rk_problem* pm = const_cast<rk_problem*>(p);
    RK_TRY(ensure_mixed(pm, (cudaStream_t)stream));
    RK_CUDA(launch_stencil32(p->d, p->S, p->coef32, p->dinv32, v, false, y, false, nullptr, (cudaStream_t)stream));
    RK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return RK_OK;
  }
  if (precond == 3) {
    rk_problem* pm = const_cast<rk_problem*>(p);
    RK_TRY(ensure_dfop(pm, (cudaStream_t)stream));
    RK_CUDA(launch_stencil_dd(p->d, p->S, ST_PREC, p->coefdf, p->dinvdf, v, false, y, false, nullptr,
                              (cudaStream_t)stream));
    RK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return RK_OK;
  }
  if (precond >= 5 && precond <= 8) {
    if (v == y) return fail(RK_E_INVALID, "y must not alias v");
    rk_problem* pm = const_cast<rk_problem*>(p);
    RK_TRY(ensure_subdomain(pm));
    if (precond >= 7) RK_TRY(ensure_dfop(pm, (cudaStream_t)stream));
    if (precond == 5)
      RK_TRY(subdomain_launch(pm, v, y, false, nullptr, nullptr, (cudaStream_t)stream));
    else if (precond == 6)
      RK_TRY(opapply_launch(pm, RK_FP64, v, false, y, false, nullptr, (cudaStream_t)stream, true, RK_PC_SUBDOMAIN));
    else if (precond == 7)
      RK_TRY(subdomain_df_launch(pm, v, false, y, false, nullptr, (cudaStream_t)stream));
    else
      RK_TRY(opapply_launch(pm, RK_DF, v, false, y, false, nullptr, (cudaStream_t)stream, true, RK_PC_SUBDOMAIN));
    RK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return RK_OK;
  }
  if (precond >= 9 && precond <= 11) {
    if (v == y) return fail(RK_E_INVALID, "y must not alias v");
    rk_problem* pm = const_cast<rk_problem*>(p);
    cudaStream_t st = (cudaStream_t)stream;
    RK_TRY(ensure_mixed(pm, st));
    RK_TRY(ensure_subdomain(pm));
    if (precond == 9)
      RK_TRY(subdomain32_launch(pm, v, false, y, 0, nullptr, st));
    else
      RK_TRY(opapply_launch(pm, RK_MIXED, v, false, y, false, nullptr, st, true,
                            precond == 10 ? RK_PC_SUBDOMAIN : RK_PC_JACOBI));
    RK_CUDA(cudaStreamSynchronize(st));
    return RK_OK;
  }
  if (precond < 0 || precond > 11) return fail(RK_E_INVALID, "precond must be 0..11");
  RK_CUDA(launch_stencil(p->d, p->S, precond == 4 ? ST_LEFT : (precond ? ST_PREC : ST_PLAIN), p->coef, p->dinv, v, nullptr, y, nullptr,
                         nullptr, nullptr, nullptr, (cudaStream_t)stream));
  RK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return RK_OK;
}

int rk_residual(const rk_problem* p, const double* b, const double* x, double* r, void* stream) {
  if (!p || !b || !x || !r) return fail(RK_E_INVALID, "NULL argument");
  RK_CUDA(launch_stencil(p->d, p->S, ST_RESID, p->coef, nullptr, x, b, r, nullptr, nullptr, nullptr, nullptr,
                         (cudaStream_t)stream));
  RK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return RK_OK;
}

int rk_dots(rk_context* ctx, int64_t n, int32_t nq, const double* Q, int64_t ld, const double* w, double* out,
            void* stream) {
  if (!ctx || !w || !out || (nq > 0 && !Q) || nq < 0 || n <= 0 || ld < n)
    return fail(RK_E_INVALID, "bad argument to rk_dots");
  const size_t need = (size_t)red_blocks(n) * (size_t)(nq + 1);
  if (need > ctx->part_n) {
    dev_free(ctx, ctx->part);
    ctx->part = (double*)dev_alloc(ctx, need * sizeof(double));
    ctx->part_n = ctx->part ? need : 0;
    if (!ctx->part) return fail(RK_E_OOM, "partials allocation failed");
  }
  DotsArgs a{};
  a.n = n;
  a.nq = nq;
  a.Q = Q;
  a.ld = ld;
  a.w = w;
  a.part = ctx->part;
  a.counter = ctx->counter;
  a.out = out;
  RK_CUDA(launch_dots(a, (cudaStream_t)stream));
  RK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return RK_OK;
}

int rk_row_gemm(rk_context* ctx, int64_t n, int32_t na, const double* A, int64_t lda, int32_t nb, const double* B,
                int64_t ldb, const double* s, const double* P, int32_t nc, double* out, int64_t ldo, int32_t engine,
                void* stream) {
  if (!ctx || n <= 0 || na < 0 || nb < 0 || na + nb < 1 || nc < 1 || !P || !out || ldo < n ||
      (na > 0 && (!A || lda < n)) || (nb > 0 && (!B || ldb < n)) || engine < 0 || engine > 3)
    return fail(RK_E_INVALID, "bad argument to rk_row_gemm");
  cudaStream_t st = (cudaStream_t)stream;
  if (engine == 3) {
    // the tensor-core product on FP64 operands as given (the RK_FP64 /
    // RK_MIXED recycle update)
    if (!gemm_tc_f64_supported(na + nb, nc, 0))
      return fail(RK_E_INVALID, "rk_row_gemm: the tensor-core engine needs 2 <= nc <= 32 and na + nb <= 64");
    void* ws = dev_alloc(ctx, dfgemm_tc_ws_bytes());
    int* err = (int*)dev_alloc(ctx, sizeof(int));
    int rc = RK_OK;
    if (!ws || !err) {
      rc = fail(RK_E_OOM, "rk_row_gemm: workspace allocation failed");
    } else {
      DFGemmArgs t{};
      t.n = n;
      t.na = na;
      t.nb = nb;
      t.nc = nc;
      t.A = (const float2*)A;
      t.lda = lda;
      t.Bm = (const float2*)B;
      t.ldb = ldb;
      t.bscale = s;
      t.P = P;
      t.out = out;
      t.ldo = ldo;
      t.accum = 0;
      cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
      if (e == cudaSuccess) e = launch_dfgemm_tc(t, ws, err, st, true);
      int herr = 0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess)
        rc = fail(RK_E_CUDA, std::string("rk_row_gemm: ") + cudaGetErrorString(e));
      else if (herr != 0)
        rc = fail(RK_E_DEVICE_TIMEOUT, "rk_row_gemm: a bounded device wait gave up");
    }
    cudaStreamSynchronize(st);
    dev_free(ctx, ws);
    dev_free(ctx, err);
    return rc;
  }
  if (engine == 2) {
    // the FP64 product of the RK_FP64 / RK_MIXED basis, on the operands as given
    F64GemmArgs g{};
    g.n = n;
    g.na = na;
    g.nb = nb;
    g.nc = nc;
    g.A = A;
    g.lda = lda;
    g.Bm = B;
    g.ldb = ldb;
    g.bscale = s;
    g.P = P;
    g.out = out;
    g.ldo = ldo;
    g.accum = 0;
    RK_CUDA(launch_gemm_rows_f64(g, st));
    RK_CUDA(cudaStreamSynchronize(st));
    return RK_OK;
  }
  DFGemmArgs a{};
  a.n = n;
  a.na = na;
  a.nb = nb;
  a.nc = nc;
  a.bscale = s;
  a.P = P;
  a.ldo = n;
  a.lda = n;
  a.ldb = n;
  a.accum = 0;
  if (engine == 1 && !dfgemm_tc_supported(a, true))
    return fail(RK_E_INVALID, "rk_row_gemm: the tensor-core engine needs 2 <= nc <= 32 and na + nb <= 64");
  // double-float copies of the operands, as the solver stores them
  const size_t cols = (size_t)na + nb + nc;
  float2* buf = (float2*)dev_alloc(ctx, cols * (size_t)n * sizeof(float2));
  void* ws = engine == 1 ? dev_alloc(ctx, dfgemm_tc_ws_bytes()) : nullptr;
  int* err = (int*)dev_alloc(ctx, sizeof(int));
  int rc = RK_OK;
  if (!buf || !err || (engine == 1 && !ws)) {
    rc = fail(RK_E_OOM, "rk_row_gemm: workspace allocation failed");
  } else {
    float2* Ad = buf;
    float2* Bd = buf + (size_t)na * n;
    float2* Od = Bd + (size_t)nb * n;
    a.A = Ad;
    a.Bm = Bd;
    a.out = Od;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess && na > 0) e = launch_to_df(n, A, Ad, nullptr, 0, na, lda, n, st);
    if (e == cudaSuccess && nb > 0) e = launch_to_df(n, B, Bd, nullptr, 0, nb, ldb, n, st);
    if (e == cudaSuccess) e = engine == 1 ? launch_dfgemm_tc(a, ws, err, st) : launch_dfgemm_rows(a, true, st);
    if (e == cudaSuccess) e = launch_from_df(n, Od, out, nc, n, ldo, st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
      rc = fail(RK_E_CUDA, std::string("rk_row_gemm: ") + cudaGetErrorString(e));
    else if (herr != 0)
      rc = fail(RK_E_DEVICE_TIMEOUT, "rk_row_gemm: a bounded device wait gave up");
  }
  cudaStreamSynchronize(st);
  dev_free(ctx, buf);
  dev_free(ctx, ws);
  dev_free(ctx, err);
  return rc;
}

int rk_arnoldi_dots(rk_context* ctx, int64_t n, int32_t nq, const double* Q, int64_t ld, const double* pv,
                    const double* w, double* out, int32_t precision, void* stream) {
  if (!ctx || n <= 0 || nq < 0 || nq > 128 || (nq > 0 && (!Q || ld < n)) || !pv || !w || !out ||
      (precision != RK_FP64 && precision != RK_DF))
    return fail(RK_E_INVALID, "bad argument to rk_arnoldi_dots");
  cudaStream_t st = (cudaStream_t)stream;
  const bool df = precision == RK_DF;
  const int ncols = 2 * nq + 3;
  const size_t nparts = (size_t)(df ? dots2_blocks(n) : dots2_f64_rows(n)) * ncols;
  const int ncnt = 64;
  const int64_t ldc = round_up(n, 32);  // column starts 256-byte aligned, as in the solver's basis
  double* part = (double*)dev_alloc(ctx, nparts * sizeof(double));
  unsigned* cnt = (unsigned*)dev_alloc(ctx, ncnt * sizeof(unsigned));
  float2* cp = df ? (float2*)dev_alloc(ctx, (size_t)(nq + 2) * ldc * sizeof(float2)) : nullptr;
  int* err = (int*)dev_alloc(ctx, sizeof(int));
  int rc = RK_OK;
  if (!part || !cnt || !err || (df && !cp)) {
    rc = fail(RK_E_OOM, "rk_arnoldi_dots: workspace allocation failed");
  } else {
    cudaError_t e = cudaMemsetAsync(cnt, 0, ncnt * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (df) {
      // the operands rounded to double-float, as RK_DF solves store them
      if (e == cudaSuccess && nq > 0) e = launch_to_df(n, Q, cp, nullptr, 0, nq, ld, ldc, st);
      if (e == cudaSuccess) e = launch_to_df(n, pv, cp + (int64_t)nq * ldc, nullptr, 0, 1, n, ldc, st);
      if (e == cudaSuccess) e = launch_to_df(n, w, cp + (int64_t)(nq + 1) * ldc, nullptr, 0, 1, n, ldc, st);
      DFDots2Args a{};
      a.n = n;
      a.nq = nq;
      a.Q = cp;
      a.ld = ldc;
      a.p = cp + (int64_t)nq * ldc;
      a.w = cp + (int64_t)(nq + 1) * ldc;
      a.part = part;
      a.counter = cnt;
      a.out = out;
      a.err = err;
      if (e == cudaSuccess) e = launch_dfdots2(a, st);
    } else {
      F64Dots2Args a{};
      a.n = n;
      a.nq = nq;
      a.Q = Q;
      a.ld = ld;
      a.p = pv;
      a.w = w;
      a.part = part;
      a.counter = cnt;
      a.out = out;
      a.err = err;
      if (e == cudaSuccess) e = launch_dots2_f64(a, st);
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
      rc = fail(RK_E_CUDA, std::string("rk_arnoldi_dots: ") + cudaGetErrorString(e));
    else if (herr != 0)
      rc = fail(RK_E_DEVICE_TIMEOUT, "rk_arnoldi_dots: a bounded device wait gave up");
  }
  cudaStreamSynchronize(st);
  dev_free(ctx, part);
  dev_free(ctx, cnt);
  dev_free(ctx, cp);
  dev_free(ctx, err);
  return rc;
}

int rk_set_recycle(rk_problem* p, const double* U, const double* C, int32_t k, void* stream) {
  if (!p) return fail(RK_E_INVALID, "NULL problem");
  cudaStream_t st = (cudaStream_t)stream;
  if (k < 0) return fail(RK_E_INVALID, "k < 0");
  if (k == 0) {
    p->kdim = 0;
    return RK_OK;
  }
  if (!U) return fail(RK_E_INVALID, "U is NULL");
  RK_TRY(ensure_capacity(p, k, std::max(p->mcap, 1), st));
  p->kdim = 0;  // replaced below; on any error the problem is left without a recycle space
  float2* Ud = p->Ublk(k);
  float2* Cd = p->Cblk(k);
  // the caller's FP64 N x k (leading dimension N) into the store (FP64, or
  // double-float after RK_DF solves)
  RK_TRY(to_basis(p, U, Ud, nullptr, 0, k, p->n, p->ld, st));
  double* G = p->eta;                     // k x k
  auto gram_cc = [&](float2* X) -> int { return bgram_launch(p, X, k, nullptr, 0, nullptr, X, k, G, st); };
  if (!C) {
    // forming C from U: C~ = A U; thin QR by CholQR2 (C~ = C R), U <- U R^{-1}
    RK_TRY(derive_c_from_u(p, k, st));
    p->kside = 0;
  } else {
    RK_TRY(to_basis(p, C, Cd, nullptr, 0, k, p->n, p->ld, st));
    // invariants: ||C^T C - I||_F and ||A U - C||_F
    RK_TRY(gram_cc(Cd));
    std::vector<double> hg((size_t)k * k);
    RK_CUDA(cudaMemcpyAsync(hg.data(), G, sizeof(double) * k * k, cudaMemcpyDeviceToHost, st));
    RK_CUDA(cudaStreamSynchronize(st));
    double e = 0.0;
    for (int a = 0; a < k; ++a)
      for (int c = 0; c < k; ++c) {
        const double t = hg[a + (size_t)c * k] - (a == c ? 1.0 : 0.0);
        e += t * t;
      }
    if (std::sqrt(e) > 1e-10) return fail(RK_E_RECYCLE_INVARIANT, "||C^T C - I||_F = " + std::to_string(std::sqrt(e)));
    double* tmp = p->rvec;
    double* onev = p->eta + (size_t)2 * k * k;
    const double one = 1.0;
    RK_CUDA(cudaMemcpyAsync(onev, &one, sizeof(double), cudaMemcpyHostToDevice, st));
    double eau = 0.0, un = 0.0;
    for (int c = 0; c < k; ++c) {
      if (p->bdf)
        RK_CUDA(launch_stencil_df(p->d, p->S, ST_PLAIN, p->coef, nullptr, Ud + (int64_t)c * p->ld, true, tmp, false,
                                  nullptr, st));
      else
        RK_CUDA(launch_stencil(p->d, p->S, ST_PLAIN, p->coef, nullptr, (const double*)(Ud + (int64_t)c * p->ld),
                               nullptr, tmp, nullptr, nullptr, nullptr, nullptr, st));
      // tmp <- A u_c - c_c, ||tmp||^2 ; ||u_c||^2
      RK_TRY(bupdate_launch(p, Cd + (int64_t)c * p->ld, 1, onev, tmp, tmp, &p->st->nrm2[2], nullptr, st));
      RK_TRY(bdots_launch(p, nullptr, 0, Ud + (int64_t)c * p->ld, true, &p->st->nrm2[3], nullptr, st, nullptr, 1));
      RK_TRY(sync_state(p, st));
      eau += p->st_h->nrm2[2];
      un += p->st_h->nrm2[3];
    }
    if (std::sqrt(eau) > 1e-10 * p->anorm_f * std::sqrt(un))
      return fail(RK_E_RECYCLE_INVARIANT, "||A U - C||_F too large: " + std::to_string(std::sqrt(eau)));
  }
  RK_CUDA(cudaStreamSynchronize(st));
  p->kdim = k;
  p->kside = 0;  // A U = C
  return RK_OK;
}

int rk_get_recycle(const rk_problem* p, double* U, double* C, int32_t* k, void* stream) {
  if (!p || !k) return fail(RK_E_INVALID, "NULL argument");
  if (*k < p->kdim) {
    *k = p->kdim;
    return fail(RK_E_INVALID, "capacity smaller than the recycle dimension");
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int kd = p->kdim;
  if (kd > 0) {
    if (U) RK_TRY(from_basis(p, p->Ublk(kd), U, kd, p->ld, p->n, st));
    if (C) RK_TRY(from_basis(p, p->Cblk(kd), C, kd, p->ld, p->n, st));
    RK_CUDA(cudaStreamSynchronize(st));
  }
  *k = kd;
  return RK_OK;
}

// The checks of a solve's parameters (RK_E_INVALID with a message).
int check_params(const rk_solve_params& prm) {
  if (!(prm.tol > 0.0)) return fail(RK_E_INVALID, "tol must be positive");
  if (prm.precision != RK_FP64 && prm.precision != RK_MIXED && prm.precision != RK_DF)
    return fail(RK_E_INVALID, "unknown precision");
  if (prm.k < 0) return fail(RK_E_INVALID, "k < 0");
  if (prm.hybrid_refresh < 0 || prm.hybrid_fallback < 0) return fail(RK_E_INVALID, "negative hybrid parameter");
  if (prm.precond_side != 0 && prm.precond_side != 1) return fail(RK_E_INVALID, "precond_side must be 0 or 1");
  if (prm.precond != RK_PC_JACOBI && prm.precond != RK_PC_SUBDOMAIN) return fail(RK_E_INVALID, "unknown precond");
  if (prm.precond == RK_PC_SUBDOMAIN && prm.mode != RK_RBICGSTAB && prm.precond_side != 1)
    return fail(RK_E_INVALID, "the sub-domain preconditioner is applied from the left in GMRES and rGCROT");
  if (prm.mode < RK_GMRES || prm.mode > RK_HYBRID) return fail(RK_E_INVALID, "unknown mode");
  return RK_OK;
}

// The solver a solve of this problem runs: RK_HYBRID resolves by the
// problem's solve counter (Sec. 2.4: rGCROT for the first hybrid_switch
// solves of a phase, then rBiCGStab with U, C frozen; every
// hybrid_refresh-th solve after the switch runs rGCROT to update the space).
int resolved_mode(const rk_problem* p, const rk_solve_params& prm) {
  if (prm.mode != RK_HYBRID) return prm.mode;
  const int t = p->solves - p->hyb_base;
  const bool refresh = prm.hybrid_refresh > 0 && t >= prm.hybrid_switch &&
                       (t - prm.hybrid_switch + 1) % prm.hybrid_refresh == 0;
  return (t < prm.hybrid_switch || refresh) ? RK_RGCROT : RK_RBICGSTAB;
}

int rk_solve(rk_problem* p, const double* b, double* x, const rk_solve_params* params, rk_solve_info* info,
             void* stream) {
  if (!p || !b || !x || !params) return fail(RK_E_INVALID, "NULL argument");
  rk_solve_params prm = *params;
  RK_TRY(check_params(prm));
  rk_solve_info loc{};
  rk_solve_info& inf = info ? *info : loc;
  std::memset(&inf, 0, sizeof(inf));
  cudaStream_t st = (cudaStream_t)stream;
  if (prm.precond == RK_PC_SUBDOMAIN) RK_TRY(ensure_subdomain(p));
  // the stored recycle space in the format of this solve's precision
  RK_TRY(ensure_basis(p, prm.precision == RK_DF, st));
  const bool hybrid = prm.mode == RK_HYBRID;
  int mode = resolved_mode(p, prm);
  inf.mode_used = mode;
  int rc;
  if (mode == RK_GMRES || mode == RK_RGCROT) {
    if (prm.m <= 0) return fail(RK_E_INVALID, "m must be positive");
    rc = solve_gcr(p, b, x, prm, inf, mode == RK_RGCROT, mode == RK_RGCROT && prm.update_recycle != 0, st);
  } else if (mode == RK_RBICGSTAB) {
    const int maxmv = prm.max_matvec > 0 ? prm.max_matvec : 2000;
    const bool fallback = hybrid && prm.hybrid_fallback > 0;
    rk_solve_params pb = prm;
    if (fallback && prm.hybrid_fallback < maxmv) pb.max_matvec = prm.hybrid_fallback;
    rc = solve_bicg(p, b, x, pb, inf, prm.k > 0, st);
    if (fallback && (rc == RK_E_NOT_CONVERGED || rc == RK_E_BREAKDOWN) && inf.matvecs < maxmv) {
      // Sec. 2.4 "switch back to rGCROT": finish from the current iterate
      // and start a new rGCROT phase with this solve
      if (prm.m <= 0) return fail(RK_E_INVALID, "m must be positive");
      rk_solve_info ig{};
      rk_solve_params pg = prm;
      pg.max_matvec = maxmv - inf.matvecs;
      const int rg = solve_gcr(p, b, x, pg, ig, true, prm.update_recycle != 0, st);
      ig.matvecs += inf.matvecs;
      ig.restarts += inf.restarts;
      ig.model_bytes += inf.model_bytes;
      ig.mode_used = RK_RGCROT;
      inf = ig;
      rc = rg;
      p->hyb_base = p->solves;
    }
  } else {
    return fail(RK_E_INVALID, "unknown mode");
  }
  if (rc == RK_OK || rc == RK_E_NOT_CONVERGED || rc == RK_E_BREAKDOWN) p->solves += 1;
  return rc;
}

int rk_profile_enable(rk_problem* p, int32_t on) {
  if (!p) return fail(RK_E_INVALID, "NULL problem");
  p->prof.reset();
  p->prof.on = on != 0;
  return RK_OK;
}

int rk_profile_read(rk_problem* p, rk_prof_entry* out, int32_t cap, int32_t* count) {
  if (!p || !count) return fail(RK_E_INVALID, "NULL argument");
  p->prof.flush();
  int nout = 0;
  for (int c = 0; c < PC_COUNT; ++c) {
    if (nout < cap && out) {
      std::memset(&out[nout], 0, sizeof(rk_prof_entry));
      std::strncpy(out[nout].name, kProfNames[c], sizeof(out[nout].name) - 1);
      out[nout].launches = p->prof.launches[c];
      out[nout].ms = p->prof.ms[c];
      out[nout].bytes = p->prof.bytes[c];
      out[nout].fma = p->prof.fma[c];
    }
    ++nout;
  }
  *count = nout;
  return RK_OK;
}

int rk_harmonic_ritz(rk_context* ctx, int32_t n, const double* G, const double* F, int32_t k, double* QC,
                     double* PU, int32_t* knew, int32_t precision, void* stream) {
  if (!ctx || !G || !F || !QC || !PU || !knew || n <= 0 || k <= 0 || k > n || n > 511 ||
      (precision != RK_FP64 && precision != RK_DF))
    return fail(RK_E_INVALID, "bad argument to rk_harmonic_ritz");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ws = harmonic_ritz_ws_doubles(n) + 8;
  if (ws > ctx->part_n) {
    dev_free(ctx, ctx->part);
    ctx->part = (double*)dev_alloc(ctx, ws * sizeof(double));
    ctx->part_n = ctx->part ? ws : 0;
    if (!ctx->part) return fail(RK_E_OOM, "workspace allocation failed");
  }
  int* dk = (int*)(ctx->counter + 32);
  RK_CUDA(launch_harmonic_ritz_small(n, G, F, k, QC, PU, dk, ctx->part, precision == RK_FP64, st));
  int h = 0;
  RK_CUDA(cudaMemcpyAsync(&h, dk, sizeof(int), cudaMemcpyDeviceToHost, st));
  RK_CUDA(cudaStreamSynchronize(st));
  if (h < 0) return fail(RK_E_BREAKDOWN, "harmonic Ritz eigen-solve failed (status " + std::to_string(-h) + ")");
  *knew = h;
  return RK_OK;
}

int rk_problem_stats(const rk_problem* p, int32_t* solves, int32_t* recycle_dim, int64_t* n) {
  if (!p) return fail(RK_E_INVALID, "NULL problem");
  if (solves) *solves = p->solves;
  if (recycle_dim) *recycle_dim = p->kdim;
  if (n) *n = p->n;
  return RK_OK;
}

int rk_fp64_fma_rate(double* fma_per_s, void* stream) {
  if (!fma_per_s) return fail(RK_E_INVALID, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = 4 * kNumSM, iters = 4096;
  const double fmas = (double)blocks * 256 * 8 * iters;
  cudaEvent_t e0, e1;
  RK_CUDA(cudaEventCreate(&e0));
  RK_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms the clocks up
    RK_CUDA(cudaEventRecord(e0, st));
    RK_CUDA(launch_fp64_probe(blocks, iters, st));
    RK_CUDA(cudaEventRecord(e1, st));
    RK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *fma_per_s = best > 0.f ? fmas / (best * 1e-3) : 0.0;
  return RK_OK;
}

int rk_problem_wait_limit(rk_problem* p, int32_t polls, void* stream) {
  if (!p || polls < 0) return fail(RK_E_INVALID, "bad argument to rk_problem_wait_limit");
  cudaStream_t st = (cudaStream_t)stream;
  RK_CUDA(cudaMemcpyAsync(&p->st->wait_limit, &polls, sizeof(int), cudaMemcpyHostToDevice, st));
  RK_CUDA(cudaStreamSynchronize(st));
  return RK_OK;
}

int rk_problem_reset(rk_problem* p) {
  if (!p) return fail(RK_E_INVALID, "NULL problem");
  p->kdim = 0;
  p->kside = 0;
  p->hyb_base = p->solves;
  return RK_OK;
}

int rk_problem_footprint(const rk_problem* p, const rk_solve_params* prm, int64_t* device_bytes) {
  if (!p || !prm || !device_bytes) return fail(RK_E_INVALID, "NULL argument");
  int64_t now = 0;
  RK_TRY(rk_problem_memory(p, &now));
  const size_t ld = (size_t)p->ld, n = (size_t)p->n, S = (size_t)p->S;
  // buffers a solve with these parameters makes that the problem lacks
  const bool gcr = prm->mode != RK_RBICGSTAB;
  const bool bicg = prm->mode == RK_RBICGSTAB || prm->mode == RK_HYBRID;
  const int kneed = std::max(std::max(prm->k, 0), p->kdim);
  const int kmax = std::max(kneed, p->kmax);
  const int mcap = std::max(gcr ? std::max(prm->m, 1) : 1, p->mcap);
  size_t add = 0;
  if (kmax > p->kmax || mcap > p->mcap || !p->QB) {
    // ensure_capacity: the new basis and small buffers replace the old ones
    // (both are held while the recycle space is copied over)
    size_t total = 0;
    auto take = [&](size_t cnt) { total += (size_t)round_up((int64_t)cnt, 32); };
    const int m = mcap, nq = kmax + mcap + 2, kk = std::max(kmax, 1);
    take((size_t)(m + 1) * m); take((size_t)(m + 1) * m); take((size_t)kk * m); take(m + 1); take(m); take(m);
    take(m + 2); take(nq); take(2 * (size_t)nq + 8); take(nq); take(m); take(nq);
    take((size_t)(kmax + m + 1) * kk); take((size_t)(kmax + m + 1) * kk); take((size_t)(kmax + m) * kk);
    take(harmonic_ritz_ws_doubles(std::max(kmax + mcap, 1))); take((dfgemm_tc_ws_bytes() + 7) / 8);
    add += 8 * (size_t)(kmax + mcap + 1) * ld + 8 * (size_t)kmax * ld + (p->rvec ? 0 : 8 * ld) +
           8 * (total + (size_t)4 * (kmax + 4) + (size_t)kmax * kmax * 2 + 16 + partials_needed(p, kmax, mcap));
  }
  if (prm->precision == RK_MIXED && !p->coef32) add += 4 * S * n + 4 * ld;
  if (prm->precision == RK_DF && !p->coefdf) add += 8 * S * n + 8 * ld;
  if ((prm->precond == RK_PC_SUBDOMAIN || prm->precond_side == 1) && !p->sdw) add += 8 * 3 * ld;
  if (bicg && !p->bicg) add += 8 * 7 * ld;
  *device_bytes = now + (int64_t)add;
  return RK_OK;
}

int rk_problem_memory(const rk_problem* p, int64_t* device_bytes) {
  if (!p || !device_bytes) return fail(RK_E_INVALID, "NULL argument");
  const size_t ld = (size_t)p->ld, n = (size_t)p->n, S = (size_t)p->S;
  size_t b = 8 * S * n + 8 * ld + sizeof(unsigned) * kCounters + sizeof(SolveState) + sizeof(BicgScalars) +
             16 * sizeof(int);
  if (p->QB) b += 8 * (size_t)(p->kmax + p->mcap + 1) * ld;
  if (p->Ub) b += 8 * (size_t)p->kmax * ld;
  if (p->rvec) b += 8 * ld;
  if (p->coef32) b += 4 * S * n;
  if (p->dinv32) b += 4 * ld;
  if (p->coefdf) b += 8 * S * n;
  if (p->dinvdf) b += 8 * ld;
  if (p->sdw) b += 8 * 3 * ld;
  if (p->bicg) b += 8 * 7 * ld;
  b += 8 * (p->small_n + p->eta_n + (p->part ? p->part_n : 0));
  *device_bytes = (int64_t)b;
  return RK_OK;
}

int rk_problem_release(rk_problem* p, void* stream) {
  if (!p) return fail(RK_E_INVALID, "NULL problem");
  RK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  p->drop_graphs();
  rk_context* c = p->ctx;
  dev_free(c, p->QB);
  dev_free(c, p->Ub);
  dev_free(c, p->rvec);
  dev_free(c, p->bicg);
  dev_free(c, p->coef32);
  dev_free(c, p->dinv32);
  dev_free(c, p->coefdf);
  dev_free(c, p->dinvdf);
  dev_free(c, p->sdw);
  p->sdw = nullptr;
  p->QB = nullptr;
  p->Ub = nullptr;
  p->rvec = nullptr;
  p->bicg = nullptr;
  p->coef32 = nullptr;
  p->dinv32 = nullptr;
  p->coefdf = nullptr;
  p->dinvdf = nullptr;
  free_small(p);
  p->part_n = 0;
  p->kmax = 0;
  p->mcap = 0;
  p->kdim = 0;
  return RK_OK;
}

// ====================================================== batched rBiCGStab phase
// The iterations of the rBiCGStab solves of a batch run as one launch per
// iteration phase over a work list of (problem, block) items (rk_batch.h);
// every other stage of those solves is the single-problem code, so each
// solve gives what it gives alone. The NB iterations between host checks are
// captured once per round into a CUDA graph and replayed.

namespace {

// Launch shapes of the batched phase, chosen per workload shape by timing
// candidates on the first replays (the results do not depend on them) and
// cached in memory and, when RK_TUNE_CACHE names a file, in that JSON file.
struct BatchShape {
  int bps;     // blocks per SM of the streaming kernels' persistent grid
  int sbps;    // blocks per SM of the stencil's persistent grid
  int zchunk;  // z planes per stencil tile
};
const BatchShape kShapes[] = {{4, 4, 8}, {2, 2, 8}, {8, 8, 8}, {4, 4, 4}, {4, 4, 16}, {8, 8, 16}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;  // shape key -> index into kShapes
bool g_tune_loaded = false;

const char* tune_path() { return std::getenv("RK_TUNE_CACHE"); }

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = tune_path();
  if (!path) return;
  std::ifstream f(path);
  if (!f) return;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string t = ss.str();
  // {"key": index, ...}: keys have no quotes or colons inside
  size_t pos = 0;
  while ((pos = t.find('"', pos)) != std::string::npos) {
    const size_t e = t.find('"', pos + 1);
    if (e == std::string::npos) break;
    const std::string key = t.substr(pos + 1, e - pos - 1);
    const size_t c = t.find(':', e);
    if (c == std::string::npos) break;
    const int v = std::atoi(t.c_str() + c + 1);
    if (v >= 0 && v < kNumShapes) g_tune[key] = v;
    pos = t.find_first_of(",}", c);
    if (pos == std::string::npos) break;
  }
}

void tune_save() {
  const char* path = tune_path();
  if (!path) return;
  std::ofstream f(path);
  if (!f) return;
  f << "{";
  bool first = true;
  for (auto& kv : g_tune) {
    f << (first ? "" : ", ") << "\"" << kv.first << "\": " << kv.second;
    first = false;
  }
  f << "}\n";
}

// the workload shape: problems, total cells (log2 bucket), bands, operator precision
std::string tune_key(const std::vector<BatchProb>& P) {
  int64_t cells = 0;
  int s19 = 0, f32 = 0;
  for (auto& q : P) {
    cells += q.d.n;
    s19 += q.S == 19;
    f32 += q.f32;
  }
  int lg = 0;
  while ((int64_t(1) << (lg + 1)) <= cells) ++lg;
  std::ostringstream k;
  k << "bicg-n" << P.size() << "-c" << lg << "-s" << (s19 * 2 >= (int)P.size() ? 19 : 7) << "-f" << (f32 ? 32 : 64);
  return k.str();
}

struct BatchDevice {
  rk_context* ctx = nullptr;
  BatchProb* P = nullptr;
  int2* red = nullptr;     // (problem, block) items of the streaming kernels
  int2* red2 = nullptr;    // the same for the problems with kc > 0 (the C^T t projection)
  int2* tiles[2] = {nullptr, nullptr};  // stencil tiles of the 7- and 19-band problems
  int nprob = 0, nred = 0, nred2 = 0, ntiles[2] = {0, 0};
  void release() {
    dev_free(ctx, P);
    dev_free(ctx, red);
    dev_free(ctx, red2);
    dev_free(ctx, tiles[0]);
    dev_free(ctx, tiles[1]);
    P = nullptr;
    red = red2 = tiles[0] = tiles[1] = nullptr;
  }
};

int upload(rk_context* ctx, const void* host, size_t bytes, void** dev, cudaStream_t st) {
  *dev = dev_alloc(ctx, bytes);
  if (!*dev) return fail(RK_E_OOM, "batched phase: device allocation failed");
  // an empty list has no host array (its device array is dev_alloc's minimum)
  if (bytes > 0) RK_CUDA(cudaMemcpyAsync(*dev, host, bytes, cudaMemcpyHostToDevice, st));
  return RK_OK;
}

// descriptors and work lists of the active runs for a tiling of zchunk planes
int batch_build(BatchDevice& D, std::vector<BatchProb>& P, int zchunk, cudaStream_t st) {
  std::vector<int2> red, red2, tl[2];
  for (int i = 0; i < (int)P.size(); ++i) {
    BatchProb& q = P[i];
    q.gx = (q.d.nx + kTX - 1) / kTX;
    q.gy = (q.d.ny + kTY - 1) / kTY;
    q.zchunk = std::min(zchunk, q.d.nz);
    q.gz = (q.d.nz + q.zchunk - 1) / q.zchunk;
    for (int b = 0; b < q.nblk; ++b) {
      red.push_back(make_int2(i, b));
      if (q.kc > 0) red2.push_back(make_int2(i, b));
    }
    const int nt = q.gx * q.gy * q.gz;
    for (int t = 0; t < nt; ++t) tl[q.S == 19].push_back(make_int2(i, t));
  }
  D.release();
  D.nprob = (int)P.size();
  D.nred = (int)red.size();
  D.nred2 = (int)red2.size();
  D.ntiles[0] = (int)tl[0].size();
  D.ntiles[1] = (int)tl[1].size();
  RK_TRY(upload(D.ctx, P.data(), sizeof(BatchProb) * P.size(), (void**)&D.P, st));
  RK_TRY(upload(D.ctx, red.data(), sizeof(int2) * red.size(), (void**)&D.red, st));
  RK_TRY(upload(D.ctx, red2.data(), sizeof(int2) * red2.size(), (void**)&D.red2, st));
  for (int s = 0; s < 2; ++s)
    RK_TRY(upload(D.ctx, tl[s].data(), sizeof(int2) * tl[s].size(), (void**)&D.tiles[s], st));
  RK_CUDA(cudaStreamSynchronize(st));
  return RK_OK;
}

// NB iterations of Algorithm 4 for every active problem, one launch per phase
cudaError_t batch_iterations(const BatchDevice& D, const BatchShape& sh, int NB, cudaStream_t st) {
  const int g = sh.bps * kNumSM, gs = sh.sbps * kNumSM;
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < NB && e == cudaSuccess; ++it) {
    e = launch_batch_bicg_p(D.P, D.red, D.nred, g, st);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s)
      e = launch_batch_stencil(D.P, D.tiles[s], D.ntiles[s], s ? 19 : 7, 0, gs, st);
    if (e == cudaSuccess) e = launch_batch_dots(D.P, D.red, D.nred, 0, g, st);
    if (e == cudaSuccess) e = launch_batch_bicg_alpha(D.P, D.nprob, st);
    if (e == cudaSuccess) e = launch_batch_bicg_s(D.P, D.red, D.nred, g, st);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s)
      e = launch_batch_stencil(D.P, D.tiles[s], D.ntiles[s], s ? 19 : 7, 1, gs, st);
    if (e == cudaSuccess) e = launch_batch_dots(D.P, D.red2, D.nred2, 1, g, st);
    if (e == cudaSuccess) e = launch_batch_bicg_t(D.P, D.red, D.nred, g, st);
    if (e == cudaSuccess) e = launch_batch_bicg_r(D.P, D.red, D.nred, g, st);
  }
  return e;
}

int batch_graph(const BatchDevice& D, const BatchShape& sh, int NB, cudaStream_t cap, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  RK_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  const cudaError_t e = batch_iterations(D, sh, NB, cap);
  const cudaError_t ce = cudaStreamEndCapture(cap, &g);
  if (e != cudaSuccess || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(RK_E_CUDA, std::string("batched phase capture: ") + cudaGetErrorString(e != cudaSuccess ? e : ce));
  }
  const cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return fail(RK_E_CUDA, std::string("batched phase instantiation: ") + cudaGetErrorString(ie));
  return RK_OK;
}

// The passes of the runs in R (set up by bicg_setup) with their iterations
// batched; on return every run is done (or *failed_at holds a failing run).
int run_bicg_batched(std::vector<BicgRun*>& R, rk_context* ctx, cudaStream_t st) {
  const int NB = 8;
  cudaStream_t cap = nullptr;
  RK_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  BatchDevice D;
  D.ctx = ctx;
  cudaGraphExec_t ge = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = RK_OK;
  auto cleanup = [&](int r) {
    if (ge) cudaGraphExecDestroy(ge);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    D.release();
    cudaStreamDestroy(cap);
    return r;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cleanup(fail(RK_E_CUDA, "batched phase: event creation failed"));
  while (rc == RK_OK) {
    std::vector<BicgRun*> act;
    for (auto* r : R)
      if (!r->done) act.push_back(r);
    if (act.empty()) break;
    for (auto* r : act)
      if ((rc = bicg_pass_start(*r, st)) != RK_OK) return cleanup(rc);
    std::vector<BatchProb> P(act.size());
    for (size_t i = 0; i < act.size(); ++i) {
      BicgRun& r = *act[i];
      rk_problem* p = r.p;
      BatchProb& q = P[i];
      q = BatchProb{};
      q.d = p->d;
      q.S = p->S;
      q.kc = r.kc;
      q.nblk = red_blocks(p->n);
      q.f32 = r.opk == RK_MIXED ? 1 : 0;
      q.ld = p->ld;
      q.coef = p->coef;
      q.dinv = p->dinv;
      q.coef32 = p->coef32;
      q.dinv32 = p->dinv32;
      q.v = r.v;
      q.bs = p->bs;
      q.C = reinterpret_cast<const double*>(p->Cblk(r.kc));
      q.eta1 = r.eta1;
      q.eta2 = r.eta2;
      q.xi = r.xi;
      q.part = p->part;
      q.counter = p->counter;
    }
    // the launch shape: cached, or tuned on this round's first replays
    const std::string key = tune_key(P);
    int shape = -1;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      tune_load();
      auto it = g_tune.find(key);
      if (it != g_tune.end()) shape = it->second;
    }
    const bool tuning = shape < 0;
    std::vector<float> times;
    int cur = -1;
    bool running = true;
    while (running) {
      const int want = tuning ? ((int)times.size() < kNumShapes ? (int)times.size() : shape) : shape;
      if (want != cur) {
        if (ge) {
          cudaGraphExecDestroy(ge);
          ge = nullptr;
        }
        if ((rc = batch_build(D, P, kShapes[want].zchunk, st)) != RK_OK) return cleanup(rc);
        if ((rc = batch_graph(D, kShapes[want], NB, cap, &ge)) != RK_OK) return cleanup(rc);
        cur = want;
      }
      const bool timed = tuning && (int)times.size() < kNumShapes;
      if (timed) RK_CUDA(cudaEventRecord(e0, st));
      RK_CUDA(cudaGraphLaunch(ge, st));
      if (timed) RK_CUDA(cudaEventRecord(e1, st));
      for (auto* r : act)
        RK_CUDA(cudaMemcpyAsync(r->p->bs_h, r->p->bs, sizeof(BicgScalars), cudaMemcpyDeviceToHost, st));
      RK_CUDA(cudaStreamSynchronize(st));
      running = false;
      for (auto* r : act)
        if (!r->p->bs_h->stop) running = true;
      if (timed) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        times.push_back(running ? ms : 1e30f);  // a replay in which every pass stopped is not comparable
        if ((int)times.size() == kNumShapes || !running) {
          shape = (int)(std::min_element(times.begin(), times.end()) - times.begin());
          if (times[shape] < 1e29f) {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune[key] = shape;
            tune_save();
          }
        }
      }
    }
    for (auto* r : act)
      if ((rc = bicg_pass_end(*r, st)) != RK_OK) return cleanup(rc);
  }
  return cleanup(rc);
}

}  // namespace

// the batch's teardown calls are not checked (nothing can be undone there);
// with RK_DEBUG set, a failing one is named on stderr
static void batch_dbg(cudaError_t e, const char* what) {
  if (e != cudaSuccess && std::getenv("RK_DEBUG")) std::fprintf(stderr, "librk: %s: %s\n", what, cudaGetErrorName(e));
}

int rk_solve_batch(rk_problem* const* problems, const double* const* b, double* const* x, int32_t n,
                   const rk_solve_params* params, rk_solve_info* infos, int32_t nthreads, void* stream) {
  if (n < 0) return fail(RK_E_INVALID, "n < 0");
  if (n == 0) return RK_OK;
  if (!problems || !b || !x || !params || !infos) return fail(RK_E_INVALID, "NULL argument");
  {
    std::vector<const rk_problem*> v(problems, problems + n);
    std::sort(v.begin(), v.end());
    for (int i = 0; i < n; ++i) {
      if (!v[i]) return fail(RK_E_INVALID, "NULL problem in the batch");
      if (i > 0 && v[i] == v[i - 1]) return fail(RK_E_INVALID, "a problem appears twice in the batch");
    }
  }
  const int T = std::max(1, std::min<int>(n, nthreads > 0 ? nthreads : 16));
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  RK_CUDA(cudaGetDevice(&dev));
  // the batch starts after the work already queued on `stream`
  cudaEvent_t start;
  RK_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  RK_CUDA(cudaEventRecord(start, st));
  std::vector<cudaStream_t> ws(T, nullptr);
  int rc_setup = RK_OK;
  for (int t = 0; t < T && rc_setup == RK_OK; ++t) {
    if (cudaStreamCreateWithFlags(&ws[t], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(ws[t], start, 0) != cudaSuccess)
      rc_setup = RK_E_CUDA;
  }
  std::vector<int> rc(n, RK_OK);
  std::vector<std::string> msg(n);
  // with RK_BATCHED_BICG=1, rBiCGStab solves (also the hybrid's after its
  // switch) with right point Jacobi and the FP64 basis run their iterations
  // in the batched phase launches; every other solve goes to the pool (by
  // default all of them: the pool was the faster executor on the measured
  // batches)
  const char* bb = std::getenv("RK_BATCHED_BICG");
  const bool batched_on = bb != nullptr && bb[0] == '1';
  std::vector<int> grp, rest;
  for (int i = 0; i < n; ++i) {
    const rk_solve_params& pr = params[i];
    const bool ok = batched_on && check_params(pr) == RK_OK && resolved_mode(problems[i], pr) == RK_RBICGSTAB &&
                    pr.precond == RK_PC_JACOBI && (pr.precision == RK_FP64 || pr.precision == RK_MIXED) &&
                    !(pr.mode == RK_HYBRID && pr.hybrid_fallback > 0) && !problems[i]->prof.on;
    (ok ? grp : rest).push_back(i);
  }
  // largest problems first (longest-processing-time order), so that the
  // batch does not end with one large solve running alone
  std::stable_sort(rest.begin(), rest.end(), [&](int a, int b2) { return problems[a]->n > problems[b2]->n; });
  if (rc_setup == RK_OK) {
    std::atomic<int> next{0};
    const int nrest = (int)rest.size();
    auto worker = [&](int t) {
      cudaSetDevice(dev);
      for (int q = next.fetch_add(1); q < nrest; q = next.fetch_add(1)) {
        const int i = rest[q];
        rc[i] = rk_solve(problems[i], b[i], x[i], &params[i], &infos[i], ws[t]);
        if (std::getenv("RK_DEBUG")) {
          const cudaError_t e = cudaPeekAtLastError();
          if (e != cudaSuccess)
            std::fprintf(stderr, "librk: after the solve of problem %d (worker %d): %s\n", i, t, cudaGetErrorName(e));
        }
        if (rc[i] != RK_OK) msg[i] = rk_last_error();
        infos[i].status = rc[i];
      }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) pool.emplace_back(worker, t);
    if (!grp.empty()) {
      // the batched group on stream ws[0] in this thread, beside the pool
      cudaStream_t gs = ws[0];
      std::vector<BicgRun> runs(grp.size());
      std::vector<BicgRun*> live;
      for (size_t g = 0; g < grp.size(); ++g) {
        const int i = grp[g];
        rk_problem* p = problems[i];
        rk_solve_info& inf = infos[i];
        std::memset(&inf, 0, sizeof(inf));
        inf.mode_used = RK_RBICGSTAB;
        int r = ensure_basis(p, false, gs);
        if (r == RK_OK) r = bicg_setup(runs[g], p, b[i], x[i], params[i], inf, params[i].k > 0, gs);
        if (r != RK_OK) {
          rc[i] = r;
          msg[i] = rk_last_error();
          runs[g].done = true;
          runs[g].status = r;
        } else if (!runs[g].done) {
          live.push_back(&runs[g]);
        }
      }
      int rb = run_bicg_batched(live, problems[grp[0]]->ctx, gs);
      for (size_t g = 0; g < grp.size(); ++g) {
        const int i = grp[g];
        if (rc[i] != RK_OK) {
          infos[i].status = rc[i];
          continue;
        }
        if (rb != RK_OK && !runs[g].done) {
          rc[i] = rb;
          msg[i] = rk_last_error();
          infos[i].status = rb;
          continue;
        }
        rc[i] = bicg_finish(runs[g]);
        if (rc[i] == RK_OK || rc[i] == RK_E_NOT_CONVERGED || rc[i] == RK_E_BREAKDOWN) problems[i]->solves += 1;
        if (rc[i] != RK_OK) msg[i] = "rBiCGStab solve status " + std::to_string(rc[i]);
        infos[i].status = rc[i];
      }
      if (T == 1) worker(0);  // one stream: the pool's share runs after the group
    } else {
      worker(0);
    }
    for (auto& th : pool) th.join();
    if (std::getenv("RK_DEBUG")) {
      const cudaError_t e = cudaPeekAtLastError();
      if (e != cudaSuccess) std::fprintf(stderr, "librk: before the batch teardown: %s\n", cudaGetErrorName(e));
    }
  }
  // work queued on `stream` afterwards runs after the whole batch
  for (int t = 0; t < T; ++t) {
    if (!ws[t]) continue;
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
      batch_dbg(cudaEventRecord(e, ws[t]), "cudaEventRecord(ws)");
      batch_dbg(cudaStreamWaitEvent(st, e, 0), "cudaStreamWaitEvent(caller)");
      batch_dbg(cudaEventDestroy(e), "cudaEventDestroy");
    }
    batch_dbg(cudaStreamDestroy(ws[t]), "cudaStreamDestroy(ws)");
  }
  batch_dbg(cudaEventDestroy(start), "cudaEventDestroy(start)");
  // every call above whose failure matters has been checked; drop what a
  // handled failure left in this thread's last-error slot, so that it is not
  // reported later against the caller's own next CUDA call
  {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && std::getenv("RK_DEBUG"))
      std::fprintf(stderr, "librk: rk_solve_batch cleared %s\n", cudaGetErrorName(e));
  }
  if (rc_setup != RK_OK) return fail(rc_setup, "creating the batch streams failed");
  for (int i = 0; i < n; ++i)
    if (rc[i] != RK_OK) return fail(rc[i], "problem " + std::to_string(i) + ": " + msg[i]);
  return RK_OK;
}


// Opaque recycle-space blob: 4 int64 (magic, n, k, side of the pair: 0
// A U = C, 1 M^{-1} A U = C with point Jacobi, 2 with the sub-domain
// preconditioner; plus 256 when the columns are double-float), then U and C
// as stored (k columns of n 8-byte elements each).
static const int64_t kRecycleMagic = 0x524b524543594331LL;  // "RKRECYC1"

int rk_recycle_bytes(const rk_problem* p, int64_t* bytes) {
  if (!p || !bytes) return fail(RK_E_INVALID, "NULL argument");
  *bytes = 32 + 2 * (int64_t)p->kdim * p->n * (int64_t)sizeof(float2);
  return RK_OK;
}

int rk_export_recycle(const rk_problem* p, void* buf, int64_t cap, void* stream) {
  if (!p || !buf) return fail(RK_E_INVALID, "NULL argument");
  int64_t need = 0;
  RK_TRY(rk_recycle_bytes(p, &need));
  if (cap < need) return fail(RK_E_INVALID, "export buffer too small");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t hdr[4] = {kRecycleMagic, p->n, p->kdim, p->kside + (p->bdf ? 256 : 0)};
  char* b = (char*)buf;
  RK_CUDA(cudaMemcpyAsync(b, hdr, sizeof(hdr), cudaMemcpyHostToDevice, st));
  const int k = p->kdim;
  if (k > 0) {
    const size_t col = sizeof(float2) * (size_t)p->n;
    RK_CUDA(cudaMemcpy2DAsync(b + 32, col, p->Ublk(k), sizeof(float2) * p->ld, col, k, cudaMemcpyDeviceToDevice, st));
    RK_CUDA(cudaMemcpy2DAsync(b + 32 + col * k, col, p->Cblk(k), sizeof(float2) * p->ld, col, k,
                              cudaMemcpyDeviceToDevice, st));
  }
  RK_CUDA(cudaStreamSynchronize(st));
  return RK_OK;
}

int rk_import_recycle(rk_problem* p, const void* buf, int64_t bytes, void* stream) {
  if (!p || !buf) return fail(RK_E_INVALID, "NULL argument");
  if (bytes < 32) return fail(RK_E_INVALID, "recycle blob too short");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t hdr[4];
  RK_CUDA(cudaMemcpyAsync(hdr, buf, sizeof(hdr), cudaMemcpyDeviceToHost, st));
  RK_CUDA(cudaStreamSynchronize(st));
  if (hdr[0] != kRecycleMagic) return fail(RK_E_INVALID, "not a recycle blob");
  if (hdr[1] != p->n) return fail(RK_E_INVALID, "recycle blob is for another problem size");
  const int64_t k = hdr[2];
  if (k < 0 || k > 256) return fail(RK_E_INVALID, "bad recycle dimension in blob");
  const int64_t side = hdr[3] & 255;
  const bool blob_df = (hdr[3] & 256) != 0;
  if (hdr[3] < 0 || hdr[3] > 511 || side > 2) return fail(RK_E_INVALID, "bad recycle side in blob");
  const size_t col = sizeof(float2) * (size_t)p->n;
  if (bytes < 32 + 2 * (int64_t)col * k) return fail(RK_E_INVALID, "recycle blob too short");
  p->kdim = 0;
  if (k == 0) return RK_OK;
  RK_TRY(ensure_capacity(p, (int)k, std::max(p->mcap, 1), st));
  const char* b = (const char*)buf;
  RK_CUDA(cudaMemcpy2DAsync(p->Ublk((int)k), sizeof(float2) * p->ld, b + 32, col, col, k, cudaMemcpyDeviceToDevice,
                            st));
  RK_CUDA(cudaMemcpy2DAsync(p->Cblk((int)k), sizeof(float2) * p->ld, b + 32 + col * k, col, col, k,
                            cudaMemcpyDeviceToDevice, st));
  RK_CUDA(cudaStreamSynchronize(st));
  p->kdim = (int)k;
  p->kside = (int)side;
  p->bdf = blob_df;
  return RK_OK;
}

}  // extern "C"
