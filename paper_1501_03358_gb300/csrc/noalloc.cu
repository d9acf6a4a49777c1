// rk_dots_noalloc: the block inner products of rk_dots with their reduction
// scratch in a fixed, statically allocated device array, for callers that
// cannot allocate device memory (see include/rk.h).
//
// The scratch (per-block partial sums and the last-block counter) lives in
// file-scope __device__ arrays: every GPU that loads the library holds them
// until the process exits. Host code never dereferences the symbols; it takes
// their device addresses once per device with cudaGetSymbolAddress.
#include <mutex>
#include <string>

#include "rk.h"
#include "rk_internal.h"

namespace {

constexpr int kNoAllocMaxCols = 64;
constexpr int kNoAllocPartDoubles = rk::kMaxRedBlocks * kNoAllocMaxCols;  // 38,912 doubles = 304 KiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_part[kNoAllocPartDoubles];
static __device__ __align__(256) unsigned g_noalloc_counter[64];

struct DevScratch {
  bool ready = false;
  double* part = nullptr;
  unsigned* counter = nullptr;
};

std::mutex g_mu;
DevScratch g_scratch[kMaxDevices];

int fail(int code, const std::string& msg) {
  rk::set_last_error(msg.c_str());
  return code;
}

int setup_device(int dev, DevScratch** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  DevScratch& s = g_scratch[dev];
  if (!s.ready) {
    void* p = nullptr;
    void* c = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_part);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&c, g_noalloc_counter);
    // the counter must start at zero; each launch leaves it at zero again
    if (e == cudaSuccess) e = cudaMemset(c, 0, sizeof(unsigned) * 64);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(RK_E_CUDA, std::string("no-alloc scratch set-up failed: ") + cudaGetErrorString(e));
    s.part = (double*)p;
    s.counter = (unsigned*)c;
    s.ready = true;
  }
  *out = &s;
  return RK_OK;
}

}  // namespace

extern "C" int rk_dots_noalloc(int64_t n, int32_t nq, const double* Q, int64_t ld, const double* w, double* out,
                               void* stream) {
  if (!w || !out || n <= 0 || nq < 0 || (nq > 0 && !Q) || ld < n)
    return fail(RK_E_INVALID, "bad argument to rk_dots_noalloc");
  if (nq > kNoAllocMaxCols)
    return fail(RK_E_INVALID, "rk_dots_noalloc: nq = " + std::to_string(nq) + " exceeds the fixed scratch limit of " +
                                  std::to_string(kNoAllocMaxCols) + " columns");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(RK_E_CUDA, "rk_dots_noalloc: no usable current device");
  DevScratch* s = nullptr;
  int rc = setup_device(dev, &s);
  if (rc != RK_OK) return rc;
  rk::DotsArgs a{};
  a.n = n;
  a.nq = nq;
  a.Q = Q;
  a.ld = ld;
  a.w = w;
  a.part = s->part;        // red_blocks(n) * nq <= kMaxRedBlocks * 64
  a.counter = s->counter;
  a.out = out;
  // the last-block counter must start at zero (every launch also leaves it
  // at zero); the partials need no clearing, each block writes its own slots
  e = cudaMemsetAsync(s->counter, 0, sizeof(unsigned), (cudaStream_t)stream);
  if (e == cudaSuccess) e = rk::launch_dots(a, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail(RK_E_CUDA, std::string("rk_dots_noalloc: ") + cudaGetErrorString(e));
  return RK_OK;
}
