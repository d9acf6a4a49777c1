// Streaming kernels over the double-float basis [C V] and U (float2 per
// element: hi, lo). Same roles as their FP64 counterparts — block inner
// products for the projections (Algorithm 3 lines 6a-9; Algorithm 4 lines
// 1c, 7a, 12a), the orthogonalisation update with its fused norm, the
// row-tiled solution and recycle updates (lines 13-13a, 14a) and the harmonic
// Ritz inner products — with every multiply-add in double-float arithmetic
// on the FP32 pipe (rk_df.cuh). Inner loops contain no FP64 instruction and
// no FP64<->FP32 conversion (both issue at the FP64 rate on GB300); per-thread
// and per-warp sums are double-float, the per-block partials FP64, and every
// reduction order is fixed by the launch shape.
#include <type_traits>

#include "rk_internal.h"
#include "rk_device.cuh"
#include "rk_df.cuh"

namespace rk {

namespace {

constexpr int kDFCols = 16;
constexpr int kOutPT = 4;  // output columns per thread in k_dfgemm_rows
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
// w^T w]. Grid: x = element chunks (red_blocks(n)), y = groups of kDotGroup
// columns of Q plus one slice for the three scalars. Each thread carries
// 2 x kDotGroup double-float chains that share every load of Q.
__global__ void __launch_bounds__(kRedThreads) k_dfdots2(DFDots2Args a) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  __shared__ float2 red[kWarps][kDFCols];
  __shared__ int lastflag;
  const int ncols = 2 * a.nq + 3;
  const int ngroups = (a.nq + kDotGroup - 1) / kDotGroup;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double* prow = a.part + (int64_t)blockIdx.x * ncols;
  float2 vals[kDFCols];
  if ((int)blockIdx.y < ngroups) {
    const int c0 = blockIdx.y * kDotGroup;
    const int nc = min(kDotGroup, a.nq - c0);
    float ph[kDotGroup], pl[kDotGroup], wh[kDotGroup], wl[kDotGroup];
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) ph[q] = pl[q] = wh[q] = wl[q] = 0.f;
    const float2* base[kDotGroup];
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) base[q] = a.Q + (int64_t)(q < nc ? c0 + q : c0) * a.ld;
    for (int64_t i = i0; i < a.n; i += stride) {
      const float2 pv = __ldg(&a.p[i]);
      const float2 wv = __ldg(&a.w[i]);
      float2 v[kDotGroup];
#pragma unroll
      for (int q = 0; q < kDotGroup; ++q) v[q] = __ldg(&base[q][i]);
#pragma unroll
      for (int q = 0; q < kDotGroup; ++q) {
        if (q < nc) {
          df_mac(ph[q], pl[q], v[q].x, v[q].y, pv.x, pv.y);
          df_mac(wh[q], wl[q], v[q].x, v[q].y, wv.x, wv.y);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) vals[q] = make_float2(ph[q], pl[q]);
    block_df_reduce_cols(vals, nc, red, prow + c0);
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) vals[q] = make_float2(wh[q], wl[q]);
    block_df_reduce_cols(vals, nc, red, prow + a.nq + c0);
  } else {
    float s0h = 0.f, s0l = 0.f, s1h = 0.f, s1l = 0.f, s2h = 0.f, s2l = 0.f;
    for (int64_t i = i0; i < a.n; i += stride) {
      const float2 pv = __ldg(&a.p[i]);
      const float2 wv = __ldg(&a.w[i]);
      df_mac(s0h, s0l, pv.x, pv.y, pv.x, pv.y);
      df_mac(s1h, s1l, pv.x, pv.y, wv.x, wv.y);
      df_mac(s2h, s2l, wv.x, wv.y, wv.x, wv.y);
    }
    vals[0] = make_float2(s0h, s0l);
    vals[1] = make_float2(s1h, s1l);
    vals[2] = make_float2(s2h, s2l);
    block_df_reduce_cols(vals, 3, red, prow + 2 * a.nq);
  }
  if (arrive_last(a.counter, &lastflag)) reduce_partials(a.part, gridDim.x, ncols, a.out);
}

// v = (p - Q a) s0 into p; p_next = (w - Q b) s1 - v s2 into w (mode 0), or
// only v (mode 1). One read of Q feeds both double-float chains.
__global__ void __launch_bounds__(kRedThreads) k_dfupdate2(DFUpdate2Args a) {
  const int mode = *a.mode;
  if (mode != 0 && mode != 1) return;
  extern __shared__ float2 cab[];  // -a (nq) | -b (nq)
  __shared__ float2 sc[3];
  for (int q = threadIdx.x; q < a.nq; q += blockDim.x) {
    cab[q] = split2(-a.a[q]);
    cab[a.nq + q] = split2(-a.b[q]);
  }
  if (threadIdx.x < 3) sc[threadIdx.x] = split2(a.scal[threadIdx.x]);
  __syncthreads();
  const float2 s0 = sc[0], s1 = sc[1], s2 = sc[2];
  const float2* ca = cab;
  const float2* cb = cab + a.nq;
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
    int q = 0;
    for (; q + 4 <= a.nq; q += 4) {
      const float2 v0 = __ldg(col + (int64_t)(q + 0) * a.ld);
      const float2 v1 = __ldg(col + (int64_t)(q + 1) * a.ld);
      const float2 v2 = __ldg(col + (int64_t)(q + 2) * a.ld);
      const float2 v3 = __ldg(col + (int64_t)(q + 3) * a.ld);
      df_mac(ah, al, v0.x, v0.y, ca[q + 0].x, ca[q + 0].y);
      df_mac(bh, bl, v0.x, v0.y, cb[q + 0].x, cb[q + 0].y);
      df_mac(ah, al, v1.x, v1.y, ca[q + 1].x, ca[q + 1].y);
      df_mac(bh, bl, v1.x, v1.y, cb[q + 1].x, cb[q + 1].y);
      df_mac(ah, al, v2.x, v2.y, ca[q + 2].x, ca[q + 2].y);
      df_mac(bh, bl, v2.x, v2.y, cb[q + 2].x, cb[q + 2].y);
      df_mac(ah, al, v3.x, v3.y, ca[q + 3].x, ca[q + 3].y);
      df_mac(bh, bl, v3.x, v3.y, cb[q + 3].x, cb[q + 3].y);
    }
    for (; q < a.nq; ++q) {
      const float2 v = __ldg(col + (int64_t)q * a.ld);
      df_mac(ah, al, v.x, v.y, ca[q].x, ca[q].y);
      df_mac(bh, bl, v.x, v.y, cb[q].x, cb[q].y);
    }
    const float2 vf = df_mul(make_float2(ah, al), s0);
    const float2 pn = df_add(df_mul(make_float2(bh, bl), s1), df_neg(df_mul(vf, s2)));
    a.p[i] = vf;
    a.w[i] = pn;
  }
}

// Row-tiled X P with X = [A (na DF cols), Bm (nb DF cols) .* bscale]; out is
// DF (in place safe per tile) or FP64 (optionally accumulated).
template <typename OT>
__global__ void __launch_bounds__(256) k_dfgemm_rows(DFGemmArgs a, int tr) {
  extern __shared__ float2 xs[];  // X: np * tr | P: np * nc | scale: tr
  const int np = a.na + a.nb;
  float2* X = xs;
  float2* P = xs + (int64_t)np * tr;
  float2* SC = P + (int64_t)np * a.nc;
  for (int t = threadIdx.x; t < np * a.nc; t += blockDim.x) P[t] = split2(a.P[t]);
  const int64_t ntiles = (a.n + tr - 1) / tr;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * tr;
    __syncthreads();
    if (a.bscale) {
      for (int r = threadIdx.x; r < tr; r += blockDim.x) {
        const int64_t i = r0 + r;
        SC[r] = i < a.n ? split2(__ldg(&a.bscale[i])) : make_float2(0.f, 0.f);
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < np * tr; t += blockDim.x) {
      const int q = t / tr, r = t - q * tr;
      const int64_t i = r0 + r;
      if (i < a.n) {
        const float2* src = q < a.na ? &a.A[(int64_t)q * a.lda + i] : &a.Bm[(int64_t)(q - a.na) * a.ldb + i];
        cp_async8(&X[t], src);
      } else {
        X[t] = make_float2(0.f, 0.f);
      }
    }
    cp_async_wait_all();
    if (a.bscale && a.nb > 0) {
      __syncthreads();
      for (int t = a.na * tr + threadIdx.x; t < np * tr; t += blockDim.x) X[t] = df_mul(X[t], SC[t % tr]);
    }
    __syncthreads();
    // each thread: one row, kOutPT output columns (independent chains that
    // share every X load)
    const int ncg = (a.nc + kOutPT - 1) / kOutPT;
    for (int t = threadIdx.x; t < ncg * tr; t += blockDim.x) {
      const int cg = t / tr, r = t - cg * tr;
      const int64_t i = r0 + r;
      if (i >= a.n) continue;
      const int c0 = cg * kOutPT;
      float sh[kOutPT], sl[kOutPT];
#pragma unroll
      for (int u = 0; u < kOutPT; ++u) sh[u] = sl[u] = 0.f;
      for (int q = 0; q < np; ++q) {
        const float2 xv = X[q * tr + r];
#pragma unroll
        for (int u = 0; u < kOutPT; ++u) {
          if (c0 + u < a.nc) {
            const float2 pv = P[(int64_t)(c0 + u) * np + q];
            df_mac(sh[u], sl[u], xv.x, xv.y, pv.x, pv.y);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kOutPT; ++u) {
        const int c = c0 + u;
        if (c >= a.nc) continue;
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

constexpr int kDFGramPPT = 8;

// out[q + l*np] = sum_i X_q[i] * (d[i] * U_l[i]), X = [A, Bm] DF, U DF.
__global__ void __launch_bounds__(256) k_dfgram(DFGramArgs a, int pair0, int npairs_pass, int tr) {
  extern __shared__ float2 gs[];
  __shared__ int lastflag;
  const int np = a.na + a.nb;
  float2* X = gs;                       // np * tr
  float2* Y = gs + (int64_t)np * tr;    // nu * tr
  float2* D = Y + (int64_t)a.nu * tr;   // tr
  float sh[kDFGramPPT], sl[kDFGramPPT];
  int qq[kDFGramPPT], ll[kDFGramPPT];
#pragma unroll
  for (int t = 0; t < kDFGramPPT; ++t) {
    sh[t] = sl[t] = 0.f;
    const int pr = pair0 + threadIdx.x + t * blockDim.x;
    qq[t] = pr % np;
    ll[t] = pr / np;
  }
  const int pend = pair0 + npairs_pass;
  const int64_t ntiles = (a.n + tr - 1) / tr;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * tr;
    __syncthreads();
    if (a.d != nullptr) {
      for (int r = threadIdx.x; r < tr; r += blockDim.x) {
        const int64_t i = r0 + r;
        D[r] = i < a.n ? split2(__ldg(&a.d[i])) : make_float2(0.f, 0.f);
      }
      __syncthreads();
    }
    // tiles stored row-major (X[r][q], Y[r][l]): in the product loop the
    // lanes of a warp read consecutive q (and mostly one l), so shared-memory
    // accesses are conflict-free; global reads stay coalesced along r
    for (int t = threadIdx.x; t < np * tr; t += blockDim.x) {
      const int q = t / tr, r = t - q * tr;
      const int64_t i = r0 + r;
      float2* dst = &X[r * np + q];
      if (i < a.n)
        cp_async8(dst, q < a.na ? &a.A[(int64_t)q * a.lda + i] : &a.Bm[(int64_t)(q - a.na) * a.ldb + i]);
      else
        *dst = make_float2(0.f, 0.f);
    }
    for (int t = threadIdx.x; t < a.nu * tr; t += blockDim.x) {
      const int l = t / tr, r = t - l * tr;
      const int64_t i = r0 + r;
      float2* dst = &Y[r * a.nu + l];
      if (i < a.n)
        cp_async8(dst, &a.U[(int64_t)l * a.ldu + i]);
      else
        *dst = make_float2(0.f, 0.f);
    }
    cp_async_wait_all();
    if (a.d != nullptr) {
      __syncthreads();
      for (int t = threadIdx.x; t < a.nu * tr; t += blockDim.x) Y[t] = df_mul(Y[t], D[t / a.nu]);
    }
    __syncthreads();
    // the thread's pairs advance together, row by row: kDFGramPPT
    // independent double-float chains per thread
    for (int r = 0; r < tr; ++r) {
#pragma unroll
      for (int t = 0; t < kDFGramPPT; ++t) {
        const int pr = pair0 + threadIdx.x + t * blockDim.x;
        if (pr < pend) {
          const float2 xv = X[r * np + qq[t]], yv = Y[r * a.nu + ll[t]];
          df_mac(sh[t], sl[t], xv.x, xv.y, yv.x, yv.y);
        }
      }
    }
  }
  const int total = np * a.nu;
#pragma unroll
  for (int t = 0; t < kDFGramPPT; ++t) {
    const int pr = pair0 + threadIdx.x + t * blockDim.x;
    if (pr < pend) a.part[(int64_t)blockIdx.x * total + pr] = (double)sh[t] + (double)sl[t];
  }
  if (arrive_last(a.counter, &lastflag)) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = pair0 + wid; c < pend; c += nw) {
      double s = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(&a.part[(int64_t)b * total + c]);
      s = warp_sum(s);
      if (lane == 0) a.out[c] = s;
    }
  }
}

// dst (DF) = src (FP64) * scale; scale = 1, *scale_ptr, or 1/sqrt(*scale_ptr)
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

// x += dinv .* xt (FP64), the M^{-1} x~ of Algorithm 4 line 17a
__global__ void __launch_bounds__(kRedThreads) k_axpy_scaled(int64_t n, const double* __restrict__ s,
                                                             const double* __restrict__ v, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(__ldg(&s[i]), __ldg(&v[i]), x[i]);
}

int dfgemm_tile_rows(int np) { return np <= 96 ? 64 : 32; }

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

cudaError_t launch_dfdots2(const DFDots2Args& a, cudaStream_t st) {
  const dim3 grid(red_blocks(a.n), (a.nq + kDotGroup - 1) / kDotGroup + 1);
  k_dfdots2<<<grid, kRedThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dfupdate2(const DFUpdate2Args& a, cudaStream_t st) {
  const size_t smem = (size_t)(a.nq > 0 ? 2 * a.nq : 1) * sizeof(float2);
  k_dfupdate2<<<red_blocks(a.n), kRedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dfgemm_rows(const DFGemmArgs& a, bool out_df, cudaStream_t st) {
  const int np = a.na + a.nb;
  if (np == 0 || a.nc == 0) return cudaSuccess;
  const int tr = dfgemm_tile_rows(np);
  const size_t smem = ((size_t)np * tr + (size_t)np * a.nc + tr) * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dfgemm_rows<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(k_dfgemm_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  const int64_t ntiles = (a.n + tr - 1) / tr;
  const int blocks = (int)(ntiles < 4 * kNumSM ? ntiles : 4 * kNumSM);
  if (out_df)
    k_dfgemm_rows<float2><<<blocks, 256, smem, st>>>(a, tr);
  else
    k_dfgemm_rows<double><<<blocks, 256, smem, st>>>(a, tr);
  return cudaGetLastError();
}

cudaError_t launch_dfgram(const DFGramArgs& a, cudaStream_t st) {
  const int np = a.na + a.nb;
  const int total = np * a.nu;
  if (total == 0) return cudaSuccess;
  const int tr = 32;
  const size_t smem = ((size_t)np * tr + (size_t)a.nu * tr + tr) * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dfgram, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  const int per_pass = 256 * kDFGramPPT;
  const int blocks = gram_blocks(a.n);
  for (int p0 = 0; p0 < total; p0 += per_pass) {
    const int npp = total - p0 < per_pass ? total - p0 : per_pass;
    k_dfgram<<<blocks, 256, smem, st>>>(a, p0, npp, tr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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
