// Streaming kernels over the double-float basis [C V] and U (float2 per
// element: hi, lo). Same roles as their FP64 counterparts — block inner
// products for the projections (Algorithms 3 and 4), the orthogonalisation
// update with its fused norm, the row-tiled solution and recycle updates
// (Algorithm 3) and the harmonic
// Ritz inner products — with every multiply-add in double-float arithmetic
// on the FP32 pipe (rk_df.cuh). Inner loops contain no FP64 instruction and
// no FP64<->FP32 conversion (both issue at the FP64 rate on GB300); per-thread
// and per-warp sums are double-float, the per-block partials FP64, and every
// reduction order is fixed by the launch shape.
#include <type_traits>

#include "rk_internal.h"
#include "rk_device.cuh"
#include "rk_df.cuh"
#include "rk_async.cuh"

namespace rk {

namespace {

constexpr int kDFCols = 16;
constexpr int kWarps = kRedThreads / 32;

template <typename T>
__device__ __forceinline__ float2 load_df(const T* p, int64_t i);
template <>
__device__ __forceinline__ float2 load_df<double>(const double* p, int64_t i) {
  const df v = df_from_double(__ldg(&p[i]));
  return make_float2(v.hi, v.lo);
}
template <>
__device__ __forceinline__ float2 load_df<float2>(const float2* p, int64_t i) {
  return __ldg(&p[i]);
}

// 8-byte asynchronous global -> shared copy (no register round trip), so a
// thread's tile loads are all in flight at once
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ float2 split2(double d) {
  const df v = df_from_double(d);
  return make_float2(v.hi, v.lo);
}

// Block reduction of per-thread DF values for ncol columns: warp xor trees in
// DF, then warp 0.. combines the 8 warp sums in DF and converts once.
// red: kWarps x kDFCols float2 in shared memory. Results to dst[c] (FP64).
__device__ __forceinline__ void block_df_reduce_cols(float2* vals, int ncol, float2 (*red)[kDFCols], double* dst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kDFCols; ++q) {
    if (q < ncol) {
      const float2 s = df_warp_sum(vals[q]);
      if (lane == 0) red[wid][q] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < ncol) {
    float2 s = red[0][threadIdx.x];
    for (int w = 1; w < kWarps; ++w) s = df_add(s, red[w][threadIdx.x]);
    dst[threadIdx.x] = df_to_double(s);
  }
  __syncthreads();
}

// out[q] = Q_q^T w (q < nq, DF columns), then (self) w^T w in DF, then w^T e_k
// for the FP64 extras e_k (FP64 arithmetic, used by rBiCGStab's r~).
// Grid: x = element chunks (red_blocks(n)), y = groups of kDotGroup columns
// (the last y slice takes the FP64 extras); each thread carries kDotGroup
// independent double-float chains, so registers stay low and occupancy high;
// w is re-read per group (from L2).
constexpr int kDotGroup = 4;

template <typename WT>
__global__ void __launch_bounds__(kRedThreads) k_dfdots(DFDotsArgs a) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  __shared__ float2 red[kWarps][kDFCols];
  __shared__ double redd[kWarps][4];
  __shared__ int lastflag;
  const WT* w = (const WT*)a.w;
  const int ndf = a.nq + a.self;  // DF columns; the self column is w itself
  const int ncols = ndf + a.ne;
  const int ngroups = (ndf + kDotGroup - 1) / kDotGroup;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((int)blockIdx.y < ngroups) {
    const int c0 = blockIdx.y * kDotGroup;
    const int nc = min(kDotGroup, ndf - c0);
    float sh[kDotGroup], sl[kDotGroup];
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) sh[q] = sl[q] = 0.f;
    const float2* base[kDotGroup];
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) {
      const int col = c0 + q;
      base[q] = (q < nc && col < a.nq) ? a.Q + (int64_t)col * a.ld : nullptr;
    }
    for (int64_t i = i0; i < a.n; i += stride) {
      const float2 wv = load_df<WT>(w, i);
      float2 v[kDotGroup];
#pragma unroll
      for (int q = 0; q < kDotGroup; ++q) v[q] = base[q] ? __ldg(&base[q][i]) : wv;
#pragma unroll
      for (int q = 0; q < kDotGroup; ++q)
        if (q < nc) df_mac(sh[q], sl[q], v[q].x, v[q].y, wv.x, wv.y);
    }
    float2 vals[kDFCols];
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) vals[q] = make_float2(sh[q], sl[q]);
    block_df_reduce_cols(vals, nc, red, a.part + (int64_t)blockIdx.x * ncols + c0);
  } else if (a.ne > 0) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t i = i0; i < a.n; i += stride) {
      double wi;
      if constexpr (std::is_same<WT, double>::value)
        wi = __ldg(&w[i]);
      else
        wi = df_to_double(__ldg(&w[i]));
#pragma unroll
      for (int e = 0; e < 3; ++e)
        if (e < a.ne) acc[e] = fma(__ldg(&a.extra[e][i]), wi, acc[e]);
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const double s = warp_sum(acc[e]);
      if (lane == 0) redd[wid][e] = s;
    }
    __syncthreads();
    if (threadIdx.x < a.ne) {
      double s = 0.0;
      for (int ww = 0; ww < kWarps; ++ww) s += redd[ww][threadIdx.x];
      a.part[(int64_t)blockIdx.x * ncols + ndf + threadIdx.x] = s;
    }
  }
  if (arrive_last(a.counter, &lastflag)) reduce_partials(a.part, gridDim.x, ncols, a.out);
}

// y_out = (y_in - sum_q Q_q c_q) * scale and ||y_out||^2.
// scale: 1; *scale_ptr; or 1/sqrt(*scale_ptr) when scale_rsqrt (1 if that
// value is not positive).
template <typename IT, typename OT>
__global__ void __launch_bounds__(kRedThreads) k_dfupdate(DFUpdateArgs a) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  extern __shared__ float2 cdf[];
  __shared__ float2 red[kWarps][kDFCols];
  __shared__ int lastflag;
  __shared__ float2 sc;
  for (int q = threadIdx.x; q < a.nq; q += blockDim.x) cdf[q] = split2(-a.c[q]);
  if (threadIdx.x == 0) {
    double s = 1.0;
    if (a.scale_ptr) {
      const double v = *a.scale_ptr;
      s = a.scale_rsqrt ? (v > 0.0 ? rsqrt(v) : 1.0) : v;
    }
    sc = split2(s);
  }
  __syncthreads();
  const float2 scale = sc;
  const bool scaled = a.scale_ptr != nullptr;
  const IT* yin = (const IT*)a.yin;
  OT* yout = (OT*)a.yout;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float nh = 0.f, nl = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const float2 y = load_df<IT>(yin, i);
    float sh = y.x, sl = y.y;  // accumulate y - sum Q c directly
    const float2* col = a.Q + i;
    int q = 0;
    for (; q + 4 <= a.nq; q += 4) {
      const float2 v0 = __ldg(col + (int64_t)(q + 0) * a.ld);
      const float2 v1 = __ldg(col + (int64_t)(q + 1) * a.ld);
      const float2 v2 = __ldg(col + (int64_t)(q + 2) * a.ld);
      const float2 v3 = __ldg(col + (int64_t)(q + 3) * a.ld);
      df_mac(sh, sl, v0.x, v0.y, cdf[q + 0].x, cdf[q + 0].y);
      df_mac(sh, sl, v1.x, v1.y, cdf[q + 1].x, cdf[q + 1].y);
      df_mac(sh, sl, v2.x, v2.y, cdf[q + 2].x, cdf[q + 2].y);
      df_mac(sh, sl, v3.x, v3.y, cdf[q + 3].x, cdf[q + 3].y);
    }
    for (; q < a.nq; ++q) {
      const float2 v = __ldg(col + (int64_t)q * a.ld);
      df_mac(sh, sl, v.x, v.y, cdf[q].x, cdf[q].y);
    }
    float2 r = make_float2(sh, sl);  // normalised by df_acc
    if (scaled) r = df_mul(r, scale);
    if constexpr (std::is_same<OT, float2>::value) {
      yout[i] = r;
    } else {
      yout[i] = df_to_double(r);
    }
    df_mac(nh, nl, r.x, r.y, r.x, r.y);
  }
  if (a.nrm2 == nullptr) return;
  float2 v[kDFCols];
  v[0] = make_float2(nh, nl);
  block_df_reduce_cols(v, 1, red, a.part + blockIdx.x);
  if (arrive_last(a.counter, &lastflag)) reduce_partials(a.part, gridDim.x, 1, a.nrm2);
}

// Delayed-reorthogonalisation inner products: [Q^T p, Q^T w, p^T p, p^T w,
// w^T w]. Grid: x = groups of kDotGroup columns of Q plus one slice for the
// three scalars, y = contiguous row ranges of rpb rows (dots2_blocks(n)).
// A block streams its vectors (p, w and its kDotGroup columns)
// through a kD2Stages-deep ring of shared-memory stages of kD2Rows rows,
// filled by bulk asynchronous copies: a producer warp refills a stage as soon
// as every consumer warp has released it ("empty" mbarrier) and the copies
// complete on the stage's "full" mbarrier, so the consumers never wait on a
// block-wide barrier and the loads in flight do not depend on registers. Each thread carries 2 x kDotGroup double-float chains that share
// every value of Q. Each column group has its own completion counter: the
// last row block of a group sums that group's partials (fixed order).
constexpr int kD2Rows = 512;   // rows per stage (2 per thread)
constexpr int kD2Stages = 3;
constexpr int kD2Vecs = 2 + kDotGroup;
constexpr size_t kD2Smem = (size_t)kD2Stages * kD2Vecs * kD2Rows * sizeof(float2);

// Block reduction of per-thread DF values for ncol columns among the first
// kRedThreads threads only (named barrier; the producer warp is absent).
__device__ __forceinline__ void consumer_df_reduce_cols(float2* vals, int ncol, float2 (*red)[kDFCols],
                                                        double* dst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kDFCols; ++q) {
    if (q < ncol) {
      const float2 s = df_warp_sum(vals[q]);
      if (lane == 0) red[wid][q] = s;
    }
  }
  named_sync(kRedThreads);
  if (threadIdx.x < ncol) {
    float2 s = red[0][threadIdx.x];
    for (int w = 1; w < kWarps; ++w) s = df_add(s, red[w][threadIdx.x]);
    dst[threadIdx.x] = df_to_double(s);
  }
  named_sync(kRedThreads);
}

constexpr int kD2Threads = kRedThreads + 32;  // 8 consumer warps + 1 producer warp

__global__ void __launch_bounds__(kD2Threads) k_dfdots2(DFDots2Args a, int64_t rpb) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  extern __shared__ __align__(128) float2 d2buf[];  // [stage][vector][row]
  __shared__ __align__(8) uint64_t full[kD2Stages];
  __shared__ __align__(8) uint64_t empty[kD2Stages];
  __shared__ float2 red[kWarps][kDFCols];
  __shared__ int lastflag;
  __shared__ int abort_at;  // first stage the producer did not issue (it gave up waiting)
  const int ncols = 2 * a.nq + 3;
  const int ngroups = (a.nq + kDotGroup - 1) / kDotGroup;
  const bool scal = (int)blockIdx.x >= ngroups;
  const int c0 = blockIdx.x * kDotGroup;
  const int nc = scal ? 0 : min(kDotGroup, a.nq - c0);
  const int nvec = 2 + nc;  // only this group's columns are copied
  const int64_t begin = (int64_t)blockIdx.y * rpb;
  const int64_t end = min(a.n, begin + rpb);
  const int nst = end > begin ? (int)((end - begin + kD2Rows - 1) / kD2Rows) : 0;
  const float2* src[kD2Vecs];
  src[0] = a.p;
  src[1] = a.w;
#pragma unroll
  for (int q = 0; q < kDotGroup; ++q) src[2 + q] = a.Q + (int64_t)(q < nc ? c0 + q : 0) * a.ld;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kD2Stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kWarps);
    }
    mbar_init_fence();
    abort_at = 0x7fffffff;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == kWarps) {
    // producer: refill a stage once every consumer warp has released it;
    // if that wait gives up, no copy is issued for stage s or later and the
    // consumers stop at stage s (every copy they wait for was issued)
    if (lane == 0) {
      const int lim = a.wait_limit != nullptr ? *a.wait_limit : 0;
      for (int s = 0; s < nst; ++s) {
        const int slot = s % kD2Stages;
        const unsigned par = (unsigned)((s / kD2Stages - 1) & 1);
        if (s >= kD2Stages &&
            !(lim > 0 ? mbar_wait_polls(&empty[slot], par, lim) : mbar_wait_bounded(&empty[slot], par))) {
          if (a.err) atomicExch(a.err, 2);
          abort_at = s;
          __threadfence_block();
          break;
        }
        const int64_t r0 = begin + (int64_t)s * kD2Rows;
        const int64_t rr = min((int64_t)kD2Rows, end - r0);
        const unsigned bytes = (unsigned)((rr & ~(int64_t)1) * sizeof(float2));
        mbar_arrive_expect_tx(&full[slot], bytes * nvec);
        if (bytes)
          for (int v = 0; v < nvec; ++v)
            bulk_g2s(d2buf + ((int64_t)slot * kD2Vecs + v) * kD2Rows, src[v] + r0, bytes, &full[slot]);
      }
    }
    return;
  }
  float ph[kDotGroup], pl[kDotGroup], wh[kDotGroup], wl[kDotGroup];
#pragma unroll
  for (int q = 0; q < kDotGroup; ++q) ph[q] = pl[q] = wh[q] = wl[q] = 0.f;
  float s0h = 0.f, s0l = 0.f, s1h = 0.f, s1l = 0.f, s2h = 0.f, s2l = 0.f;
  for (int s = 0; s < nst; ++s) {
    const int slot = s % kD2Stages;
    // wait for stage s, unless the producer gave up before issuing it
    bool got = false, stopped = false;
    for (int it = 0; it < kMbarPolls; ++it) {
      if (mbar_try_wait(&full[slot], (unsigned)((s / kD2Stages) & 1))) {
        got = true;
        break;
      }
      if (*(volatile int*)&abort_at <= s) {
        stopped = true;
        break;
      }
    }
    if (!got) {
      if (!stopped && a.err) atomicExch(a.err, 1);
      break;
    }
    const int64_t r0 = begin + (int64_t)s * kD2Rows;
    const int rr = (int)min((int64_t)kD2Rows, end - r0);
    const float2* sb = d2buf + (int64_t)slot * kD2Vecs * kD2Rows;
    if (rr == kD2Rows) {
      // full stage: two rows per thread, no conditions; lazy double-float
      // accumulation, renormalised once per stage
#pragma unroll
      for (int h = 0; h < kD2Rows / kRedThreads; ++h) {
        const int r = threadIdx.x + h * kRedThreads;
        const float2 pv = sb[r], wv = sb[kD2Rows + r];
        if (scal) {
          df_mac_lazy(s0h, s0l, pv.x, pv.y, pv.x, pv.y);
          df_mac_lazy(s1h, s1l, pv.x, pv.y, wv.x, wv.y);
          df_mac_lazy(s2h, s2l, wv.x, wv.y, wv.x, wv.y);
        } else {
#pragma unroll
          for (int q = 0; q < kDotGroup; ++q) {
            const float2 v = sb[(2 + q) * kD2Rows + r];
            df_mac_lazy(ph[q], pl[q], v.x, v.y, pv.x, pv.y);
            df_mac_lazy(wh[q], wl[q], v.x, v.y, wv.x, wv.y);
          }
        }
      }
      if (scal) {
        df_renorm(s0h, s0l);
        df_renorm(s1h, s1l);
        df_renorm(s2h, s2l);
      } else {
#pragma unroll
        for (int q = 0; q < kDotGroup; ++q) {
          df_renorm(ph[q], pl[q]);
          df_renorm(wh[q], wl[q]);
        }
      }
    } else {
      for (int r = threadIdx.x; r < rr; r += kRedThreads) {
        const bool direct = (r == rr - 1) && (rr & 1);
        const float2 pv = direct ? a.p[r0 + r] : sb[r];
        const float2 wv = direct ? a.w[r0 + r] : sb[kD2Rows + r];
        if (scal) {
          df_mac(s0h, s0l, pv.x, pv.y, pv.x, pv.y);
          df_mac(s1h, s1l, pv.x, pv.y, wv.x, wv.y);
          df_mac(s2h, s2l, wv.x, wv.y, wv.x, wv.y);
        } else {
#pragma unroll
          for (int q = 0; q < kDotGroup; ++q) {
            const float2 v = direct ? src[2 + q][r0 + r] : sb[(2 + q) * kD2Rows + r];
            df_mac(ph[q], pl[q], v.x, v.y, pv.x, pv.y);
            df_mac(wh[q], wl[q], v.x, v.y, wv.x, wv.y);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);  // this warp has read the stage
  }
  double* prow = a.part + (int64_t)blockIdx.y * ncols;
  float2 vals[kDFCols];
  int cA, nA, cB = 0, nB = 0;  // this group's partial columns
  if (!scal) {
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) vals[q] = make_float2(ph[q], pl[q]);
    consumer_df_reduce_cols(vals, nc, red, prow + c0);
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) vals[q] = make_float2(wh[q], wl[q]);
    consumer_df_reduce_cols(vals, nc, red, prow + a.nq + c0);
    cA = c0;
    nA = nc;
    cB = a.nq + c0;
    nB = nc;
  } else {
    vals[0] = make_float2(s0h, s0l);
    vals[1] = make_float2(s1h, s1l);
    vals[2] = make_float2(s2h, s2l);
    consumer_df_reduce_cols(vals, 3, red, prow + 2 * a.nq);
    cA = 2 * a.nq;
    nA = 3;
  }
  // the last row block of this group sums the group's partials
  __threadfence();
  named_sync(kRedThreads);
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(a.counter + blockIdx.x, 1u);
    lastflag = (t == gridDim.y - 1) ? 1 : 0;
  }
  named_sync(kRedThreads);
  if (lastflag) {
    __threadfence();
    if (threadIdx.x == 0) a.counter[blockIdx.x] = 0u;
    for (int t = wid; t < nA + nB; t += kWarps) {
      const int c = t < nA ? cA + t : cB + (t - nA);
      double sum = 0.0;
      for (int by = lane; by < (int)gridDim.y; by += 32) sum += __ldcg(&a.part[(int64_t)by * ncols + c]);
      sum = warp_sum(sum);
      if (lane == 0) a.out[c] = sum;
    }
  }
}

// v = (p - Q a) s0 into p; p_next = (w - Q b) s1 - v s2 into w (mode 0), or
// only v (mode 1). One read of Q feeds both double-float chains.
__global__ void __launch_bounds__(kRedThreads) k_dfupdate2(DFUpdate2Args a) {
  const int mode = *a.mode;
  if (mode != 0 && mode != 1) return;
  extern __shared__ float2 cab[];  // -a | -b, each padded to nq8 = round_up(nq, 8) with zeros
  __shared__ float2 sc[3];
  const int nq8 = (a.nq + 7) & ~7;
  for (int q = threadIdx.x; q < nq8; q += blockDim.x) {
    cab[q] = q < a.nq ? split2(-a.a[q]) : make_float2(0.f, 0.f);
    cab[nq8 + q] = (q < a.nq && mode == 0) ? split2(-a.b[q]) : make_float2(0.f, 0.f);
  }
  if (threadIdx.x < 3) sc[threadIdx.x] = split2(a.scal[threadIdx.x]);
  __syncthreads();
  const float2 s0 = sc[0], s1 = sc[1], s2 = sc[2];
  const float2* ca = cab;
  const float2* cb = cab + nq8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (mode == 1) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
      const float2 pv = a.p[i];
      float ah = pv.x, al = pv.y;
      const float2* col = a.Q + i;
      for (int q = 0; q < a.nq; ++q) {
        const float2 v = __ldg(col + (int64_t)q * a.ld);
        df_mac(ah, al, v.x, v.y, ca[q].x, ca[q].y);
      }
      a.p[i] = df_mul(make_float2(ah, al), s0);
    }
    return;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const float2 pv = a.p[i];
    const float2 wv = a.w[i];
    float ah = pv.x, al = pv.y, bh = wv.x, bl = wv.y;
    const float2* col = a.Q + i;
    // chunks of 8 columns, the last one predicated (no scalar tail: every
    // load of a row is issued before its multiply-adds)
    for (int q = 0; q < a.nq; q += 8) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = q + u < a.nq ? __ldg(col + (int64_t)(q + u) * a.ld) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        df_mac_lazy(ah, al, v[u].x, v[u].y, ca[q + u].x, ca[q + u].y);
        df_mac_lazy(bh, bl, v[u].x, v[u].y, cb[q + u].x, cb[q + u].y);
      }
      df_renorm(ah, al);
      df_renorm(bh, bl);
    }
    const float2 vf = df_mul(make_float2(ah, al), s0);
    const float2 pn = df_add(df_mul(make_float2(bh, bl), s1), df_neg(df_mul(vf, s2)));
    a.p[i] = vf;
    a.w[i] = pn;
  }
}

// Row-tiled X P (the solution and recycle updates of Algorithm 3)
// with X = [A (na DF cols), diag(bscale) Bm (nb DF cols)] and P (np x nc,
// FP64, column-major). P is held in shared memory as DF, transposed and
// zero-padded to ncg * CB columns. A block of ncg * tr threads takes a tile
// of tr rows; thread (g, r) computes row r for the CB output columns
// g*CB .. g*CB+CB-1, so one shared-memory load of X feeds CB independent
// double-float chains and the inner loop has no conditions. The row scale
// is applied once per output: acc = bscale_i * sum_{B} X P, then the A
// columns are added. out is DF (in place safe: a tile is read completely
// before it is written) or FP64 (optionally accumulated).
template <typename OT, int CB>
__global__ void __launch_bounds__(256) k_dfgemm2(DFGemmArgs a, int tr, int ncp) {
  extern __shared__ float2 xs[];  // X: np * tr | PT: np * ncp | SC: tr
  const int np = a.na + a.nb;
  float2* X = xs;
  float2* PT = xs + (int64_t)np * tr;
  float2* SC = PT + (int64_t)np * ncp;
  const int nthr = blockDim.x;
  for (int t = threadIdx.x; t < np * ncp; t += nthr) {
    const int q = t / ncp, c = t - q * ncp;
    PT[t] = c < a.nc ? split2(a.P[(int64_t)c * np + q]) : make_float2(0.f, 0.f);
  }
  const int g = threadIdx.x / tr, r = threadIdx.x - g * tr;
  const int c0 = g * CB;
  const int64_t ntiles = (a.n + tr - 1) / tr;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * tr;
    __syncthreads();  // previous tile fully consumed (and written, for in-place DF)
    for (int t = threadIdx.x; t < np * tr; t += nthr) {
      const int q = t / tr, rr = t - q * tr;
      const int64_t i = r0 + rr;
      const float2* src = q < a.na ? a.A + (int64_t)q * a.lda : a.Bm + (int64_t)(q - a.na) * a.ldb;
      if (i < a.n)
        cp_async8(&X[t], src + i);
      else
        X[t] = make_float2(0.f, 0.f);
    }
    if (a.bscale) {
      for (int rr = threadIdx.x; rr < tr; rr += nthr) {
        const int64_t i = r0 + rr;
        SC[rr] = i < a.n ? split2(__ldg(&a.bscale[i])) : make_float2(0.f, 0.f);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    float sh[CB], sl[CB];
#pragma unroll
    for (int u = 0; u < CB; ++u) sh[u] = sl[u] = 0.f;
    const float2* pt = PT + c0;
    // B columns first (they carry the row scale), then the scale, then A;
    // lazy double-float accumulation, renormalised every 8 terms
    auto run = [&](int q0, int q1) {
      for (int qb = q0; qb < q1; qb += 8) {
        const int qe = min(qb + 8, q1);
        for (int q = qb; q < qe; ++q) {
          const float2 xv = X[q * tr + r];
          const float2* pq = pt + (int64_t)q * ncp;
#pragma unroll
          for (int u = 0; u < CB; ++u) df_mac_lazy(sh[u], sl[u], xv.x, xv.y, pq[u].x, pq[u].y);
        }
#pragma unroll
        for (int u = 0; u < CB; ++u) df_renorm(sh[u], sl[u]);
      }
    };
    run(a.na, np);
    if (a.bscale && a.nb > 0) {
      const float2 sc = SC[r];
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const float2 v = df_mul(make_float2(sh[u], sl[u]), sc);
        sh[u] = v.x;
        sl[u] = v.y;
      }
    }
    run(0, a.na);
    const int64_t i = r0 + r;
    if (i < a.n) {
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const int c = c0 + u;
        if (c >= a.nc) break;
        if constexpr (std::is_same<OT, float2>::value) {
          ((float2*)a.out)[(int64_t)c * a.ldo + i] = make_float2(sh[u], sl[u]);
        } else {
          double* o = (double*)a.out + (int64_t)c * a.ldo + i;
          const double sv = (double)sh[u] + (double)sl[u];
          *o = a.accum ? *o + sv : sv;
        }
      }
    }
  }
}

// One output column (x updates): out_i (+)= sum_{q<na} A_q[i] p_q
// + bscale_i sum_{q>=na} B_q[i] p_q, streamed straight from global memory
// (each value is used once), coefficients in shared memory as DF.
template <typename OT>
__global__ void __launch_bounds__(kRedThreads) k_dfgemv(DFGemmArgs a) {
  extern __shared__ float2 pv[];
  const int np = a.na + a.nb;
  for (int q = threadIdx.x; q < np; q += blockDim.x) pv[q] = split2(a.P[q]);
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    float bh = 0.f, bl = 0.f, ah = 0.f, al = 0.f;
    int q = 0;
    for (; q + 4 <= a.nb; q += 4) {
      const float2 v0 = __ldg(a.Bm + (int64_t)(q + 0) * a.ldb + i);
      const float2 v1 = __ldg(a.Bm + (int64_t)(q + 1) * a.ldb + i);
      const float2 v2 = __ldg(a.Bm + (int64_t)(q + 2) * a.ldb + i);
      const float2 v3 = __ldg(a.Bm + (int64_t)(q + 3) * a.ldb + i);
      df_mac(bh, bl, v0.x, v0.y, pv[a.na + q + 0].x, pv[a.na + q + 0].y);
      df_mac(bh, bl, v1.x, v1.y, pv[a.na + q + 1].x, pv[a.na + q + 1].y);
      df_mac(bh, bl, v2.x, v2.y, pv[a.na + q + 2].x, pv[a.na + q + 2].y);
      df_mac(bh, bl, v3.x, v3.y, pv[a.na + q + 3].x, pv[a.na + q + 3].y);
    }
    for (; q < a.nb; ++q) {
      const float2 v = __ldg(a.Bm + (int64_t)q * a.ldb + i);
      df_mac(bh, bl, v.x, v.y, pv[a.na + q].x, pv[a.na + q].y);
    }
    q = 0;
    for (; q + 4 <= a.na; q += 4) {
      const float2 v0 = __ldg(a.A + (int64_t)(q + 0) * a.lda + i);
      const float2 v1 = __ldg(a.A + (int64_t)(q + 1) * a.lda + i);
      const float2 v2 = __ldg(a.A + (int64_t)(q + 2) * a.lda + i);
      const float2 v3 = __ldg(a.A + (int64_t)(q + 3) * a.lda + i);
      df_mac(ah, al, v0.x, v0.y, pv[q + 0].x, pv[q + 0].y);
      df_mac(ah, al, v1.x, v1.y, pv[q + 1].x, pv[q + 1].y);
      df_mac(ah, al, v2.x, v2.y, pv[q + 2].x, pv[q + 2].y);
      df_mac(ah, al, v3.x, v3.y, pv[q + 3].x, pv[q + 3].y);
    }
    for (; q < a.na; ++q) {
      const float2 v = __ldg(a.A + (int64_t)q * a.lda + i);
      df_mac(ah, al, v.x, v.y, pv[q].x, pv[q].y);
    }
    float2 bsum = make_float2(bh, bl);
    if (a.bscale && a.nb > 0) bsum = df_mul(bsum, split2(__ldg(&a.bscale[i])));
    const float2 r = df_add(make_float2(ah, al), bsum);
    if constexpr (std::is_same<OT, float2>::value) {
      ((float2*)a.out)[i] = r;
    } else {
      double* o = (double*)a.out + i;
      const double sv = df_to_double(r);
      *o = a.accum ? *o + sv : sv;
    }
  }
}

// Gram blocks out[q + l*np] = sum_i X_q[i] d[i] U_l[i] (the inner products
// of the harmonic Ritz problem of the recycle update). Each thread owns a 4 x 4 set of
// (q, l) pairs (strided by the number of sets) and a slice of the tile's rows (rows r = slice, slice + ns,
// ...); per row it reads 4 X and 4 Y values for 16 double-float
// multiply-adds. Tiles are row-major with odd strides (8-byte elements, so
// the row-by-row tile stores of a warp fall in distinct banks). The
// slices are summed in shared memory and each block writes its partials;
// a separate kernel reduces them over blocks in a fixed order.
constexpr int kGramTR = 64;
__global__ void __launch_bounds__(256) k_dfgram2(DFGramArgs a, int ob0, int nob, int ns, int sx, int sy) {
  extern __shared__ float2 gs2[];
  const int np = a.na + a.nb;
  const int nbq = (np + 3) / 4;
  float2* X = gs2;                          // kGramTR * sx
  float2* Y = X + (int64_t)kGramTR * sx;    // kGramTR * sy
  float2* D = Y + (int64_t)kGramTR * sy;    // kGramTR
  const int slice = threadIdx.x / nob, ob = threadIdx.x - slice * nob;
  const bool active = slice < ns;
  const int obg = ob0 + ob;
  const int nbl = (a.nu + 3) / 4;
  // the thread's pairs: q = qi + nbq*u, l = li + nbl*v (u, v < 4); adjacent
  // threads take adjacent q, so a warp's X reads are conflict-free
  const int qi = obg % nbq, li = obg / nbq;
  float sh[16], sl[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) sh[t] = sl[t] = 0.f;
  const int64_t ntiles = (a.n + kGramTR - 1) / kGramTR;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * kGramTR;
    __syncthreads();
    for (int t = threadIdx.x; t < np * kGramTR; t += blockDim.x) {
      const int q = t / kGramTR, r = t % kGramTR;
      const float2* src = q < a.na ? a.A + (int64_t)q * a.lda : a.Bm + (int64_t)(q - a.na) * a.ldb;
      const int64_t i = r0 + r;
      if (i < a.n)
        cp_async8(&X[r * sx + q], src + i);
      else
        X[r * sx + q] = make_float2(0.f, 0.f);
    }
    for (int t = threadIdx.x; t < a.nu * kGramTR; t += blockDim.x) {
      const int l = t / kGramTR, r = t % kGramTR;
      const int64_t i = r0 + r;
      if (i < a.n)
        cp_async8(&Y[r * sy + l], a.U + (int64_t)l * a.ldu + i);
      else
        Y[r * sy + l] = make_float2(0.f, 0.f);
    }
    for (int r = threadIdx.x; r < kGramTR; r += blockDim.x) {
      const int64_t i = r0 + r;
      D[r] = (a.d != nullptr && i < a.n) ? split2(__ldg(&a.d[i])) : make_float2(1.f, 0.f);
    }
    cp_async_wait_all();
    __syncthreads();
    if (a.d != nullptr) {
      for (int t = threadIdx.x; t < kGramTR * a.nu; t += blockDim.x) {
        const int r = t / a.nu, l = t - r * a.nu;
        Y[r * sy + l] = df_mul(Y[r * sy + l], D[r]);
      }
      __syncthreads();
    }
    if (active) {
      int cnt = 0;
      for (int r = slice; r < kGramTR; r += ns) {
        float2 xv[4], yv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          xv[u] = X[r * sx + qi + nbq * u];
          yv[u] = Y[r * sy + li + nbl * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            df_mac_lazy(sh[u * 4 + v], sl[u * 4 + v], xv[u].x, xv[u].y, yv[v].x, yv[v].y);
        if (++cnt == 8) {  // lazy accumulation, renormalised every 8 rows
          cnt = 0;
#pragma unroll
          for (int t = 0; t < 16; ++t) df_renorm(sh[t], sl[t]);
        }
      }
#pragma unroll
      for (int t = 0; t < 16; ++t) df_renorm(sh[t], sl[t]);
    }
  }
  // sum the slices: reuse the tile storage as [ns][nob][16] DF values
  __syncthreads();
  float2* red = gs2;
  if (active) {
#pragma unroll
    for (int t = 0; t < 16; ++t) red[((int64_t)slice * nob + ob) * 16 + t] = make_float2(sh[t], sl[t]);
  }
  __syncthreads();
  const int total = np * a.nu;
  for (int t = threadIdx.x; t < nob * 16; t += blockDim.x) {
    const int o = t / 16, e = t - o * 16;
    const int og = ob0 + o;
    const int q = og % nbq + nbq * (e / 4), l = og / nbq + ((a.nu + 3) / 4) * (e % 4);
    if (q >= np || l >= a.nu) continue;
    float2 s = red[(int64_t)o * 16 + e];
    for (int sl2 = 1; sl2 < ns; ++sl2) s = df_add(s, red[((int64_t)sl2 * nob + o) * 16 + e]);
    a.part[(int64_t)blockIdx.x * total + q + (int64_t)l * np] = df_to_double(s);
  }
}

// out[c] = sum_b part[b * ncols + c], one warp per column, fixed order.
__global__ void __launch_bounds__(256) k_reduce_cols(const double* __restrict__ part, int nblocks, int ncols,
                                                     double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ncols) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += part[(int64_t)b * ncols + c];
  s = warp_sum(s);
  if (lane == 0) out[c] = s;
}

__global__ void __launch_bounds__(kRedThreads) k_to_df(int64_t n, const double* __restrict__ src,
                                                       float2* __restrict__ dst, const double* scale_ptr,
                                                       int scale_rsqrt, int ncols, int64_t lds, int64_t ldd) {
  double scale = 1.0;
  if (scale_ptr) {
    const double v = *scale_ptr;
    scale = scale_rsqrt ? (v > 0.0 ? rsqrt(v) : 1.0) : v;
  }
  for (int c = 0; c < ncols; ++c)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      dst[c * ldd + i] = split2(__ldg(&src[c * lds + i]) * scale);
}

__global__ void __launch_bounds__(kRedThreads) k_from_df(int64_t n, const float2* __restrict__ src,
                                                         double* __restrict__ dst, int ncols, int64_t lds,
                                                         int64_t ldd) {
  for (int c = 0; c < ncols; ++c)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      dst[c * ldd + i] = df_to_double(__ldg(&src[c * lds + i]));
}

// x += dinv .* xt (FP64), the final M^{-1} x~ of Algorithm 4
__global__ void __launch_bounds__(kRedThreads) k_axpy_scaled(int64_t n, const double* __restrict__ s,
                                                             const double* __restrict__ v, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(__ldg(&s[i]), __ldg(&v[i]), x[i]);
}


}  // namespace

cudaError_t launch_dfdots(const DFDotsArgs& a, bool w_is_df, cudaStream_t st) {
  const int ndf = a.nq + a.self;
  const int groups = (ndf + kDotGroup - 1) / kDotGroup + (a.ne > 0 ? 1 : 0);
  if (groups == 0) return cudaSuccess;
  const dim3 grid(red_blocks(a.n), groups);
  if (w_is_df)
    k_dfdots<float2><<<grid, kRedThreads, 0, st>>>(a);
  else
    k_dfdots<double><<<grid, kRedThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dfupdate(const DFUpdateArgs& a, bool in_df, bool out_df, cudaStream_t st) {
  const size_t smem = (size_t)(a.nq > 0 ? a.nq : 1) * sizeof(float2);
  const int g = red_blocks(a.n);
  if (in_df && out_df)
    k_dfupdate<float2, float2><<<g, kRedThreads, smem, st>>>(a);
  else if (in_df)
    k_dfupdate<float2, double><<<g, kRedThreads, smem, st>>>(a);
  else if (out_df)
    k_dfupdate<double, float2><<<g, kRedThreads, smem, st>>>(a);
  else
    k_dfupdate<double, double><<<g, kRedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

int dots2_blocks(int64_t n) {
  int64_t b = (n + 16 * kD2Rows - 1) / (16 * kD2Rows);
  if (b < 1) b = 1;
  if (b > kNumSM) b = kNumSM;
  return (int)b;
}

// one-time attribute setup per device; also run when a problem is created,
// so that it never happens inside a graph capture
void dfblas_prepare() {
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_dfdots2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kD2Smem);
  });
}

cudaError_t launch_dfdots2(const DFDots2Args& a, cudaStream_t st) {
  dfblas_prepare();
  const int xb = dots2_blocks(a.n);
  const int64_t per = (a.n + xb - 1) / xb;
  const int64_t rpb = (per + kD2Rows - 1) / kD2Rows * kD2Rows;  // even: 16-byte aligned stages
  // x = column groups, y = row ranges: the groups of one row range are
  // adjacent in launch order, so p and w come from HBM once and from L2 for
  // the other groups
  const dim3 grid((a.nq + kDotGroup - 1) / kDotGroup + 1, xb);
  k_dfdots2<<<grid, kD2Threads, kD2Smem, st>>>(a, rpb);
  return cudaGetLastError();
}

cudaError_t launch_dfupdate2(const DFUpdate2Args& a, cudaStream_t st) {
  const size_t smem = (size_t)(a.nq > 0 ? 2 * ((a.nq + 7) & ~7) : 1) * sizeof(float2);
  k_dfupdate2<<<red_blocks(a.n), kRedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename OT, int CB>
static cudaError_t gemm2_go(const DFGemmArgs& a, int tr, int ncp, int threads, size_t smem, cudaStream_t st) {
  // one-time attribute setup per device
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_dfgemm2<OT, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  const int64_t ntiles = (a.n + tr - 1) / tr;
  const int64_t cap = (int64_t)kNumSM * 4;
  const int blocks = (int)(ntiles < cap ? ntiles : cap);
  k_dfgemm2<OT, CB><<<blocks, threads, smem, st>>>(a, tr, ncp);
  return cudaGetLastError();
}

// widths of the column groups that are compiled
constexpr int kGemmCB[] = {2, 4, 6, 8, 10, 12, 16};

template <typename OT>
static cudaError_t gemm2_pick(const DFGemmArgs& a, int cb, int tr, int ncp, int threads, size_t smem,
                              cudaStream_t st) {
  switch (cb) {
    case 2: return gemm2_go<OT, 2>(a, tr, ncp, threads, smem, st);
    case 4: return gemm2_go<OT, 4>(a, tr, ncp, threads, smem, st);
    case 6: return gemm2_go<OT, 6>(a, tr, ncp, threads, smem, st);
    case 8: return gemm2_go<OT, 8>(a, tr, ncp, threads, smem, st);
    case 10: return gemm2_go<OT, 10>(a, tr, ncp, threads, smem, st);
    case 12: return gemm2_go<OT, 12>(a, tr, ncp, threads, smem, st);
    default: return gemm2_go<OT, 16>(a, tr, ncp, threads, smem, st);
  }
}

cudaError_t launch_dfgemm_rows(const DFGemmArgs& a, bool out_df, cudaStream_t st) {
  const int np = a.na + a.nb;
  if (np == 0 || a.nc == 0) return cudaSuccess;
  if (a.nc == 1) {
    const size_t smem = (size_t)np * sizeof(float2);
    if (out_df)
      k_dfgemv<float2><<<red_blocks(a.n), kRedThreads, smem, st>>>(a);
    else
      k_dfgemv<double><<<red_blocks(a.n), kRedThreads, smem, st>>>(a);
    return cudaGetLastError();
  }
  // column groups: a power of two with at most 16 columns per group; the
  // group width rounded up to a compiled one (P padded with zero columns)
  int ncg = 1;
  while (ncg * 16 < a.nc) ncg *= 2;
  int cb = (a.nc + ncg - 1) / ncg;
  for (int w : kGemmCB)
    if (w >= cb) {
      cb = w;
      break;
    }
  const int ncp = ncg * cb;
  int tr = 256 / ncg;
  if (tr > 128) tr = 128;
  while (tr > 8 && ((size_t)np * tr + (size_t)np * ncp + tr) * sizeof(float2) > 200 * 1024) tr /= 2;
  const size_t smem = ((size_t)np * tr + (size_t)np * ncp + tr) * sizeof(float2);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const int threads = ncg * tr;
  return out_df ? gemm2_pick<float2>(a, cb, tr, ncp, threads, smem, st)
                : gemm2_pick<double>(a, cb, tr, ncp, threads, smem, st);
}

cudaError_t launch_dfgram(const DFGramArgs& a, cudaStream_t st) {
  const int np = a.na + a.nb;
  const int total = np * a.nu;
  if (total == 0) return cudaSuccess;
  const int nbq = (np + 3) / 4, nbl = (a.nu + 3) / 4;
  const int nblk = nbq * nbl;
  const int sx = ((np + 3) / 4) * 4 + 1, sy = ((a.nu + 3) / 4) * 4 + 1;
  const size_t tiles = ((size_t)kGramTR * (sx + sy) + kGramTR) * sizeof(float2);
  // one-time attribute setup per device
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_dfgram2, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  const int blocks = gram_blocks(a.n);
  for (int ob0 = 0; ob0 < nblk; ob0 += 256) {
    const int nob = nblk - ob0 < 256 ? nblk - ob0 : 256;
    int ns = 256 / nob;
    if (ns > 8) ns = 8;
    const size_t red = (size_t)ns * nob * 16 * sizeof(float2);
    const size_t smem = tiles > red ? tiles : red;
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    k_dfgram2<<<blocks, 256, smem, st>>>(a, ob0, nob, ns, sx, sy);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_reduce_cols<<<(total + 7) / 8, 256, 0, st>>>(a.part, blocks, total, a.out);
  return cudaGetLastError();
}

cudaError_t launch_to_df(int64_t n, const double* src, float2* dst, const double* scale_ptr, int scale_rsqrt,
                         int ncols, int64_t lds, int64_t ldd, cudaStream_t st) {
  k_to_df<<<red_blocks(n), kRedThreads, 0, st>>>(n, src, dst, scale_ptr, scale_rsqrt, ncols, lds, ldd);
  return cudaGetLastError();
}

cudaError_t launch_from_df(int64_t n, const float2* src, double* dst, int ncols, int64_t lds, int64_t ldd,
                           cudaStream_t st) {
  k_from_df<<<red_blocks(n), kRedThreads, 0, st>>>(n, src, dst, ncols, lds, ldd);
  return cudaGetLastError();
}

cudaError_t launch_axpy_scaled(int64_t n, const double* s, const double* v, double* x, cudaStream_t st) {
  k_axpy_scaled<<<red_blocks(n), kRedThreads, 0, st>>>(n, s, v, x);
  return cudaGetLastError();
}

}  // namespace rk
